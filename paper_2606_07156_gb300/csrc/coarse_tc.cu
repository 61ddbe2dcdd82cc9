// Cluster locating on the tensor cores (the low-precision fast path of CL,
// Section 2.1), with an exact re-rank so that the probed lists and their
// distances are the ones of the FP32 rule.
//
// 1. Operands: x^ = fl32(x - mu) with mu the centroids' mean (distances are
//    translation invariant, and centring shrinks the norms the rounding error
//    scales with). Each row is scaled by a power of two 2^e that puts its
//    largest magnitude in [2^(top-1), 2^top) (top = 14 for BF16 and FP16, 8
//    for FP8 E4M3, whose largest finite value is 448), rounded to the
//    operand format (nearest even) and zero-padded to Dp columns, a multiple
//    of one 128-byte K chunk. Per row, in FP32: xn = the sum of the squared
//    rounded values (unscaled), xd >= ||x~ - x^|| + 2^-23 ||x^|| (directed
//    rounding upward: the rounding error of the operand plus that of the
//    centring) and xs = 2^-e.
// 2. D~[q][l] = fl32(fl32(qn + cn) - fl32(2 dot)), dot = fl32(fl32(acc qs) cs)
//    and acc the tensor cores' FP32 product of the scaled rows: a persistent
//    kernel, one CTA per SM, walks 128 x 256 tiles. One thread loads 128-byte
//    K chunks of both operands with TMA (128-byte swizzle) into a 4-stage
//    ring; one issues tcgen05.mma (kind::f16 for BF16 / FP16, kind::f8f6f4
//    for E4M3) into one of two TMEM accumulators; four warps drain the other
//    accumulator (tcgen05.ld -> registers -> a padded shared-memory transpose
//    -> coalesced rows of D~), so that a tile's epilogue overlaps the next
//    tile's MMAs.
// 3. Error bound per pair: |D~ - D2| <= eps(D~, rows), D2 the FP32-rule
//    distance (derivation at rerank_bound). T = the nprobe-th smallest of the
//    upper bounds D~ + eps (rounded up by at most 255 units of its last place:
//    a radix select that stops at bins of 256); every list of the FP32
//    top-nprobe has D~ - eps <= T, so those candidates are re-ranked with the
//    FP32 rule itself (same operation order as coarse.cu) and the nprobe
//    smallest (D2, l) kept: identical output to the plain path. The re-rank
//    runs in three kernels: a select kernel per query (bounds, T, the
//    candidate list, up to kCap of them to the workspace as work items of 32),
//    a distance kernel whose warps walk every query's items, and a merge
//    kernel (one warp per query); indexes whose keys do not fit in shared
//    memory take a streaming kernel instead.
//
// Every mbarrier wait is bounded (by default about a second; the index option
// ANNS_OPT_WAIT_CYCLES sets the main loop's limit); on a timeout the kernel
// records ANNS_DEV_TIMEOUT in the index's device status word, tells its other
// roles to stop, waits (with the long limit) for the copies and MMAs it has
// issued, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "scan.cuh"

namespace anns {
namespace {

constexpr int kTM = 128;             // queries per tile = TMEM lanes
constexpr int kTN = 256;             // centroids per tile = FP32 TMEM columns per accumulator
constexpr int kKB = 128;             // K bytes per stage: one 128-byte swizzle row (4 MMAs of 32 bytes)
constexpr int kStages = 4;
constexpr int kGemmThreads = 192;    // warp 0: TMA, warp 1: MMA + TMEM owner, warps 2-5: epilogue
constexpr uint32_t kABytes = kTM * kKB;   // 16 KB
constexpr uint32_t kBBytes = kTN * kKB;   // 32 KB
constexpr uint32_t kStageBytes = kABytes + kBBytes;
constexpr int kEpiStride = 36;            // floats per staged epilogue row (16-byte aligned, no bank conflicts)
constexpr uint32_t kEpiBytes = 4 * 32 * kEpiStride * 4;
// alignment slack + ring + epilogue transposes + barriers; one CTA per SM (all 512 TMEM columns)
constexpr size_t kGemmSmem = 1024 + (size_t)kStages * kStageBytes + kEpiBytes + 256;
constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz: the default limit and the drain's

// Operand formats. Instruction descriptor (kind::f16 and kind::f8f6f4): D F32
// (bits 4-5 = 1), A format bits 7-9 and B format bits 10-12 (kind::f16: F16 0,
// BF16 1; kind::f8f6f4: E4M3 0), A and B K-major (bits 15, 16 = 0), N >> 3 at
// bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t idesc_of(uint32_t ab) {
  return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(kTN >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);
}

template <int F> struct TcFmt;
template <> struct TcFmt<ANNS_PREC_BF16> {
  using T = __nv_bfloat16;
  static constexpr int kElem = 2, kTop = 14;
  static constexpr uint32_t kIdesc = idesc_of(1);
  static constexpr CUtensorMapDataType kMap = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  __device__ static float round(float w, T& out) {
    out = __float2bfloat16_rn(w);
    return __bfloat162float(out);
  }
};
template <> struct TcFmt<ANNS_PREC_FP16> {
  using T = __half;
  static constexpr int kElem = 2, kTop = 14;
  static constexpr uint32_t kIdesc = idesc_of(0);
  static constexpr CUtensorMapDataType kMap = CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  __device__ static float round(float w, T& out) {
    out = __float2half_rn(w);
    return __half2float(out);
  }
};
template <> struct TcFmt<ANNS_PREC_FP8E4M3> {
  using T = __nv_fp8_storage_t;
  static constexpr int kElem = 1, kTop = 8;
  static constexpr uint32_t kIdesc = idesc_of(0);
  static constexpr CUtensorMapDataType kMap = CU_TENSOR_MAP_DATA_TYPE_UINT8;
  __device__ static float round(float w, T& out) {
    out = __nv_cvt_float_to_fp8(w, __NV_SATFINITE, __NV_E4M3);
    return __half2float(__half(__nv_cvt_fp8_to_halfraw(out, __NV_E4M3)));
  }
};

// Shared-memory matrix descriptor of a K-major operand written by TMA with the
// 128-byte swizzle: start address >> 4 (bits 0-13), leading offset unused for
// swizzled K-major (encoded 1), stride between 8-row groups 1024 bytes >> 4
// (bits 32-45), descriptor version 1 (46-47), base offset 0 (1024-byte
// aligned atoms), layout 128-byte swizzle (61-63 = 2). Within the 128-byte
// row, the k-th 32-byte group (one MMA's K) starts 32 k bytes further.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1u << 16) | ((uint64_t)(1024u >> 4) << 32) |
         (1ull << 46) | (2ull << 61);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// 2-D tiled TMA load of box (x, y) of the tensor map into shared memory,
// completing `bytes` on the mbarrier.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Wait, for at most `limit` clock cycles, for the phase of parity `parity` of
// the mbarrier to complete; false on timeout, or as soon as *abort is set
// (another role of the CTA gave up).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit = kWaitCycles,
                                          const volatile int* abort = nullptr) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (abort && *abort) return false;
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

template <int F>
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  if constexpr (F == ANNS_PREC_FP8E4M3) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(TcFmt<F>::kIdesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(TcFmt<F>::kIdesc), "r"(accumulate)
        : "memory");
  }
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
        "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
        "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// 2^e as an FP32 value, e in [-126, 127].
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

// One warp per row: x^ = fl32(x - mu), scaled by 2^e and rounded to the
// operand format (zero past dim). rows[0][row] = xn, rows[1][row] = xd,
// rows[2][row] = xs (layout in the file header).
template <int F>
__global__ void center_kernel(const float* __restrict__ X, int64_t n, int dim, int Dp, const float* __restrict__ mu,
                              typename TcFmt<F>::T* __restrict__ Xf, float* __restrict__ rows) {
  using Fm = TcFmt<F>;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const float* x = X + row * dim;
  float amax = 0.f;
  for (int d = lane; d < dim; d += 32) amax = fmaxf(amax, fabsf(sub_rn(x[d], mu[d])));
#pragma unroll
  for (int o = 16; o; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(kFull, amax, o));
  // e with amax 2^e in [2^(top-1), 2^top): top - 1 - floor(log2 amax), kept
  // where 2^e and 2^-e are normal FP32 values
  int e = 0;
  if (amax > 0.f && amax <= 3.4028235e38f) {
    const int ex = (int)((__float_as_uint(amax) >> 23) & 0xFFu) - 127;  // -127 for subnormal amax
    e = min(max(Fm::kTop - 1 - ex, -126), 126);
  }
  const float up = pow2f(e), down = pow2f(-e);
  float s = 0.f, h = 0.f, r = 0.f;
  for (int d = lane; d < Dp; d += 32) {
    const float v = d < dim ? sub_rn(x[d], mu[d]) : 0.f;
    typename Fm::T t;
    const float deq = mul_rn(Fm::round(mul_rn(v, up), t), down);
    Xf[row * Dp + d] = t;
    s = add_rn(s, mul_rn(deq, deq));
    h = __fmaf_ru(v, v, h);
    const float dv = sub_rn(deq, v);  // exact: the error of rounding v to fewer bits
    r = __fmaf_ru(dv, dv, r);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    s = add_rn(s, __shfl_xor_sync(kFull, s, o));
    h = __fadd_ru(h, __shfl_xor_sync(kFull, h, o));
    r = __fadd_ru(r, __shfl_xor_sync(kFull, r, o));
  }
  if (lane == 0) {
    rows[row] = s;
    rows[n + row] = __fadd_ru(__fsqrt_ru(r), __fmul_ru(1.1920929e-7f, __fsqrt_ru(h)));
    rows[2 * n + row] = down;
  }
}

// D~ for every 128 x 256 tile (tile t: query tile t / ntn, centroid tile
// t % ntn), persistent: CTA b takes tiles b, b + grid, ...
template <int F>
__global__ void __launch_bounds__(kGemmThreads, 1) coarse_tc_kernel(
    const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ CUtensorMap tmC,
    const float* __restrict__ qrows, const float* __restrict__ crows, int64_t nq, int64_t nlist, int nK,
    float* __restrict__ dt, int* __restrict__ status, long long wait_limit) {
  unsigned char* base = anns_dyn_smem + ((1024u - (smem_addr(anns_dyn_smem) & 1023u)) & 1023u);
  float* epi = (float*)(base + kStages * kStageBytes);
  uint64_t* bars = (uint64_t*)(base + kStages * kStageBytes + kEpiBytes);
  // full[S] | empty[S] | acc_full[2] | acc_empty[2] | drain, then the TMEM slot and the abort flag
  uint32_t* slot = (uint32_t*)(bars + 2 * kStages + 5);
  volatile int* abort_flag = (volatile int*)(slot + 1);
  const uint32_t ring = smem_addr(base);
  const uint32_t full0 = smem_addr(bars), empty0 = full0 + 8 * kStages, accf0 = full0 + 16 * kStages,
                 acce0 = accf0 + 16, drain = acce0 + 16;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ntn = (nlist + kTN - 1) / kTN, ntiles = ((nq + kTM - 1) / kTM) * ntn;

  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"((uint32_t)(2 * kTN))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(full0 + 8 * i, 1);
      mbar_init(empty0 + 8 * i, 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(accf0 + 8 * a, 1);
      mbar_init(acce0 + 8 * a, 4);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;

  bool ok = true;
  if (tid == 0) {
    // TMA producer: chunk g (running over this CTA's tiles) goes to stage g % S
    int64_t g = 0;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const int q0 = (int)((t / ntn) * kTM), l0 = (int)((t % ntn) * kTN);
      for (int k = 0; k < nK; ++k, ++g) {
        const int st = (int)(g % kStages);
        if (g >= kStages) ok = mbar_wait(empty0 + 8 * st, (uint32_t)((g / kStages - 1) & 1), wait_limit, abort_flag);
        if (!ok) break;
        const uint32_t a_dst = ring + st * kStageBytes, b_dst = a_dst + kABytes;
        mbar_expect_tx(full0 + 8 * st, kStageBytes);
        tma_load_2d(a_dst, &tmQ, k * kKB / TcFmt<F>::kElem, q0, full0 + 8 * st);
        tma_load_2d(b_dst, &tmC, k * kKB / TcFmt<F>::kElem, l0, full0 + 8 * st);
      }
    }
    if (!ok) {
      *abort_flag = 1;
      atomicExch(status, ANNS_DEV_TIMEOUT);
      // let the copies already issued land before the CTA exits (long limit):
      // stage st received ceil((g - st) / S) copies, the last completing the
      // phase of parity (count - 1) & 1, and no copy follows it
      for (int st = 0; st < kStages; ++st) {
        const int64_t count = g > st ? (g - st + kStages - 1) / kStages : 0;
        if (count > 0) mbar_wait(full0 + 8 * st, (uint32_t)((count - 1) & 1));
      }
    }
  } else if (tid == 32) {
    // MMA issuer: tile i of this CTA accumulates into TMEM columns (i & 1) * 256
    int64_t g = 0;
    int i = 0;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++i) {
      const int a = i & 1, use = i >> 1;
      if (use > 0) ok = mbar_wait(acce0 + 8 * a, (uint32_t)((use - 1) & 1), wait_limit, abort_flag);
      if (!ok) break;
      tc_fence_after();
      const uint32_t d = tmem + (uint32_t)(a * kTN);
      for (int k = 0; k < nK; ++k, ++g) {
        const int st = (int)(g % kStages);
        ok = mbar_wait(full0 + 8 * st, (uint32_t)((g / kStages) & 1), wait_limit, abort_flag);
        if (!ok) break;
        tc_fence_after();
        const uint32_t a_addr = ring + st * kStageBytes, b_addr = a_addr + kABytes;
#pragma unroll
        for (int ks = 0; ks < kKB / 32; ++ks)
          tc_mma<F>(d, smem_desc_sw128(a_addr + ks * 32), smem_desc_sw128(b_addr + ks * 32),
                    (k > 0 || ks > 0) ? 1u : 0u);
        tc_commit(empty0 + 8 * st);
      }
      if (!ok) break;
      tc_commit(accf0 + 8 * a);
    }
    if (!ok) {
      *abort_flag = 1;
      atomicExch(status, ANNS_DEV_TIMEOUT);
    }
    tc_commit(drain);  // arrives once every MMA issued above has completed
    mbar_wait(drain, 0);
  } else if (warp >= 2) {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows of the tile)
    const int lg = warp & 3;
    float* buf = epi + (warp - 2) * 32 * kEpiStride;
    int i = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int a = i & 1;
      // every lane waits; the warp goes on only together (tcgen05.ld is .sync.aligned)
      const bool got = mbar_wait(accf0 + 8 * a, (uint32_t)((i >> 1) & 1), wait_limit, abort_flag);
      if (!__all_sync(kFull, got)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const int64_t q0 = (t / ntn) * kTM + lg * 32, l0 = (t % ntn) * kTN;
      const int64_t qr = q0 + lane;  // this thread's row
      const float qn_r = qr < nq ? qrows[qr] : 0.f, qs_r = qr < nq ? qrows[2 * nq + qr] : 0.f;
      for (int c0 = 0; c0 < kTN; c0 += 32) {
        float v[32];
        tc_ld32(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(a * kTN + c0), v);
#pragma unroll
        for (int j = 0; j < 32; j += 4)
          *(float4*)(buf + lane * kEpiStride + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        __syncwarp();
        const int64_t l = l0 + c0 + lane;
        const bool lok = l < nlist;
        const float cn_l = lok ? crows[l] : 0.f, cs_l = lok ? crows[2 * nlist + l] : 0.f;
        for (int rr = 0; rr < 32; ++rr) {
          const float qn_b = __shfl_sync(kFull, qn_r, rr), qs_b = __shfl_sync(kFull, qs_r, rr);
          const float dot = mul_rn(mul_rn(buf[rr * kEpiStride + lane], qs_b), cs_l);
          if (lok && q0 + rr < nq) dt[(q0 + rr) * nlist + l] = sub_rn(add_rn(qn_b, cn_l), mul_rn(2.f, dot));
        }
        __syncwarp();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acce0 + 8 * a);
    }
    if (!ok && lane == 0) {
      *abort_flag = 1;
      atomicExch(status, ANNS_DEV_TIMEOUT);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * kTN))
                 : "memory");
}

// eps >= |D~ - D2| for a pair, D2 the FP32-rule distance. With x^ the centred
// FP32 vectors and x~ their rounded operands, delta = (q~ - c~) - (q - c) has
// ||delta|| <= dn = qd + cd (the rows' rounding errors plus the FP32
// centring, 2^-23 ||x^||). S = ||q~ - c~||^2 differs from D~ by the FP32
// evaluation error e_f <= (2 Dp + 8) 2^-24 (qn + cn) (norm sums, the FP32
// accumulator of the products, the final combination; kef carries the
// constant), from the exact distance by at most dn (2 sqrt(S) + dn), and the
// FP32 rule differs from the exact distance by at most (dim + 2) 2^-24 of it
// (kfp). Constants padded by 1 %.
// sqrt(sup) comes from rsqrtf (at most 2 ulp from 1 / sqrt), whose error the
// 1 % padding covers many times over.
__device__ __forceinline__ float rerank_bound(float dt, float qn, float qd, float cn, float cd, float kef,
                                              float kfp) {
  const float ef = kef * (qn + cn);
  const float dn = (qd + cd) * 1.01f;
  const float sup = fmaxf(dt, 0.f) + ef;
  const float rt = sup > 0.f ? sup * rsqrtf(sup) : 0.f;  // inf -> NaN -> the list is a candidate
  const float E = dn * (2.f * rt * 1.01f + dn);
  return (ef + E + kfp * (sup + E)) * 1.01f + 1e-30f;
}

// Order-preserving key of an upper bound (non-negative floats order like
// their bit patterns): negative values and -0 map to 0, NaN to +inf.
__device__ __forceinline__ uint32_t upper_key(float u) {
  return u > 0.f ? __float_as_uint(u) : (u <= 0.f ? 0u : 0x7F800000u);
}

struct RerankArgs {
  const float* Q;
  const float* C;
  const float* dt;
  const float* qrows;
  const float* crows;
  int64_t nq, nlist;
  int dim;
  float kef, kfp;
  int nprobe;
  const int32_t* npq;
  int32_t* probes;
  float* probe_d2;
  int* ncand;
};

constexpr int kRWarps = 8, kRThreads = kRWarps * 32;
constexpr int kRTile = 32 * 33;  // floats of one warp's staging tile (32 x 32 swizzled, or 32 rows of 33)

// FP32-rule distances of up to 32 candidates (lane i: candidate i; ids in
// cand[0..nc)), dim % 4 == 0. Each 32-dimension chunk of the 32 rows is loaded
// as 16-byte pieces (8 lanes per row segment, coalesced), one chunk ahead, and
// staged in the warp's tile with the 16-byte pieces XOR-swizzled by row, so
// that both the row-wise stores and the lane-per-row reads are free of bank
// conflicts; each lane accumulates its row in ascending dimension order.
__device__ __forceinline__ float batch_d2_v4(const float* __restrict__ C, const float* qs, int dim,
                                             const int32_t* cand, int nc, float* tile) {
  const int lane = threadIdx.x & 31, sub = lane >> 3, cc = lane & 7;
  int32_t rid[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = 4 * i + sub;
    rid[i] = cand[r < nc ? r : 0];
  }
  float4 buf[8];
  auto load = [&](int d0) {
    const int d = d0 + 4 * cc;
#pragma unroll
    for (int i = 0; i < 8; ++i)
      buf[i] = d < dim ? __ldg((const float4*)(C + (int64_t)rid[i] * dim + d)) : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  load(0);
  float acc = 0.f;
  for (int d0 = 0; d0 < dim; d0 += 32) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = 4 * i + sub;
      *(float4*)(tile + r * 32 + ((cc ^ (r & 7)) << 2)) = buf[i];
    }
    __syncwarp();
    if (d0 + 32 < dim) load(d0 + 32);
    const int nch = min(32, dim - d0) >> 2;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c < nch) {
        const float4 t = *(const float4*)(tile + lane * 32 + ((c ^ (lane & 7)) << 2));
        const float4 q = *(const float4*)(qs + d0 + 4 * c);
        float e = sub_rn(q.x, t.x);
        acc = add_rn(acc, mul_rn(e, e));
        e = sub_rn(q.y, t.y);
        acc = add_rn(acc, mul_rn(e, e));
        e = sub_rn(q.z, t.z);
        acc = add_rn(acc, mul_rn(e, e));
        e = sub_rn(q.w, t.w);
        acc = add_rn(acc, mul_rn(e, e));
      }
    }
    __syncwarp();
  }
  return acc;
}

// The same for any dim: row elements one at a time into a padded tile.
__device__ __forceinline__ float batch_d2_any(const float* __restrict__ C, const float* qs, int dim,
                                              const int32_t* cand, int nc, float* tile) {
  const int lane = threadIdx.x & 31;
  float acc = 0.f;
  for (int d0 = 0; d0 < dim; d0 += 32) {
    for (int r = 0; r < 32; ++r) {
      const int32_t lr = cand[r < nc ? r : 0];
      tile[r * 33 + lane] = d0 + lane < dim ? __ldg(C + (int64_t)lr * dim + d0 + lane) : 0.f;
    }
    __syncwarp();
    const int dd_end = min(32, dim - d0);
    for (int dd = 0; dd < dd_end; ++dd) {
      const float e = sub_rn(qs[d0 + dd], tile[lane * 33 + dd]);
      acc = add_rn(acc, mul_rn(e, e));
    }
    __syncwarp();
  }
  return acc;
}

// An upper bound, within 2^8 - 1 units of the last place, of the np-th
// smallest of keys[0..n) (1 <= np <= n), all in [kmin, kmax] <= +inf: radix
// levels of 8 bits over key - kmin, the first level's shift fitted to the
// range, each level counting only the keys inside the bin chosen before, until
// the bins are at most 2^8 keys wide; the top of the last bin chosen.
__device__ uint32_t block_select(const uint32_t* keys, int64_t n, int np, uint32_t kmin, uint32_t kmax, int* hist,
                                 uint32_t* sh) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int shift = 0;
  while (((kmax - kmin) >> shift) > 255u) ++shift;
  uint32_t lo = 0;                        // relative start of the current range
  uint32_t span_m1 = kmax - kmin;         // its length - 1 (keys <= 0x7F800000: no overflow)
  int need = np;
  for (;;) {
    for (int i = tid; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int64_t l = tid; l < n; l += blockDim.x) {
      const uint32_t rel = keys[l] - kmin - lo;   // wraps below lo: outside the range
      if (rel <= span_m1) atomicAdd(&hist[rel >> shift], 1);
    }
    __syncthreads();
    if (warp == 0) {
      int c[8], run = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) { c[i] = hist[lane * 8 + i]; run += c[i]; }
      int incl = run;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      const int excl = incl - run;
      int pick = -1, below = 0;
      if (excl < need && need <= incl) {
        int acc = excl;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          if (pick < 0 && acc + c[i] >= need) { pick = lane * 8 + i; below = acc; }
          acc += c[i];
        }
      }
      const unsigned who = __ballot_sync(kFull, pick >= 0);
      const int src = who ? __ffs(who) - 1 : 0;
      pick = __shfl_sync(kFull, pick, src);
      below = __shfl_sync(kFull, below, src);
      if (lane == 0) { sh[0] = who ? (uint32_t)pick : 255u; sh[1] = who ? (uint32_t)below : 0u; }
    }
    __syncthreads();
    lo += sh[0] << shift;
    need -= (int)sh[1];
    span_m1 = (1u << shift) - 1u;
    if (shift <= 8) break;
    shift = shift >= 16 ? shift - 8 : 8;
  }
  return min(kmin + lo + span_m1, 0x7F800000u);  // the last bin may reach past +inf's key
}

// Candidate lists of the split re-rank: up to kCap candidates per query in
// the workspace, their distances computed by rerank_dist_kernel (one warp per
// 32 candidates, over all queries at once) and merged by rerank_merge_kernel.
constexpr int kCap = 512;

struct RerankSplit {
  int32_t* cbuf;   // [nq][kCap] candidate lists
  float* cdist;    // [nq][kCap] their FP32-rule distances
  int2* items;     // [nq * kCap / 32] work items (query, batch)
  int* nitems;     // item count (zeroed before the select kernel)
};

// Writes the np <= 128 entries of a warp's list (padding -1 / +inf) as the
// query's probes.
template <int R>
__device__ __forceinline__ void write_probes(const RerankArgs& a, int64_t q, int np, const WarpTopK<R, int32_t>& top) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int e = r * 32 + lane;
    if (e < a.nprobe) {
      const bool ok = e < np && top.d[r] != INFINITY;
      a.probes[q * a.nprobe + e] = ok ? top.id[r] : -1;
      a.probe_d2[q * a.nprobe + e] = ok ? top.d[r] : INFINITY;
    }
  }
}

// One block per query, every list's upper key and lower bound held in shared
// memory.
// A: eps, the key of D~ + eps and the lower bound D~ - eps of every list, and
//    the keys' range.
// B: T >= the np-th smallest key, within 255 units of the last place
//    (block_select).
// C: the candidates, D~ - eps <= T, appended to a block-wide list.
// Then, with at most kCap candidates, the list goes to the workspace with one
// work item per 32 candidates; otherwise the block computes their FP32-rule
// distances itself, 32 per warp batch (batches dealt round-robin to the
// warps), each warp keeping its top-np by (D2, l), the warps' lists merged at
// the end. Queries with np = 0 get their padding here.
// Dynamic shared memory: qs [dim rounded up to 4] | keys [nlist rounded up to
// 4] (then the candidate list) | lower [nlist], whose space then holds the
// warps' staging tiles [8][1056].
template <int R, bool V4>
__global__ void __launch_bounds__(kRThreads, 3) rerank_select_kernel(RerankArgs a, RerankSplit sp) {
  __shared__ int hist[256];
  __shared__ uint32_t sh[2];
  __shared__ int total;
  __shared__ uint32_t kr[2][kRWarps];
  const int dq = (a.dim + 3) & ~3;
  const int64_t nl4 = (a.nlist + 3) & ~3;
  float* qs = (float*)anns_dyn_smem;
  uint32_t* keys = (uint32_t*)(qs + dq);
  float* lower = (float*)(keys + nl4);
  float* tiles = lower;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t q = blockIdx.x, nlist = a.nlist;
  const int np = a.npq ? min(max(a.npq[q], 0), a.nprobe) : a.nprobe;
  WarpTopK<R, int32_t> top;
  top.init();
  if (np == 0) {
    if (warp == 0) write_probes<R>(a, q, 0, top);
    if (threadIdx.x == 0 && a.ncand) a.ncand[q] = 0;
    return;
  }
  const float* row = a.dt + q * nlist;
  const float qn = a.qrows[q], qd = a.qrows[a.nq + q];
  if (threadIdx.x == 0) total = 0;
  // A: eight lists per thread per round, all their loads issued before any
  // use (D~ streams from HBM once)
  uint32_t kmin = 0xFFFFFFFFu, kmax = 0;
  for (int64_t b0 = threadIdx.x; b0 < nlist; b0 += 8 * kRThreads) {
    float d[8], cn[8], cd[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t l = b0 + j * kRThreads;
      const bool in = l < nlist;
      d[j] = in ? row[l] : 0.f;
      cn[j] = in ? a.crows[l] : 0.f;
      cd[j] = in ? a.crows[nlist + l] : 0.f;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t l = b0 + j * kRThreads;
      if (l < nlist) {
        const float b = rerank_bound(d[j], qn, qd, cn[j], cd[j], a.kef, a.kfp);
        const uint32_t k = upper_key(d[j] + b);
        keys[l] = k;
        lower[l] = d[j] - b;
        kmin = min(kmin, k);
        kmax = max(kmax, k);
      }
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    kmin = min(kmin, __shfl_xor_sync(kFull, kmin, o));
    kmax = max(kmax, __shfl_xor_sync(kFull, kmax, o));
  }
  if (lane == 0) { kr[0][warp] = kmin; kr[1][warp] = kmax; }
  __syncthreads();
  kmin = 0xFFFFFFFFu;
  kmax = 0;
  for (int w = 0; w < kRWarps; ++w) {
    kmin = min(kmin, kr[0][w]);
    kmax = max(kmax, kr[1][w]);
  }
  // B
  const float T = __uint_as_float(block_select(keys, nlist, np, kmin, kmax, hist, sh));
  __syncthreads();  // keys are free: they become the candidate list
  // C
  int32_t* cand = (int32_t*)keys;
  for (int64_t b0 = (int64_t)warp * 32; b0 < nlist; b0 += kRThreads) {
    const int64_t l = b0 + lane;
    const bool c = l < nlist && !(lower[l] > T);
    const unsigned m = __ballot_sync(kFull, c);
    if (m) {
      int at = 0;
      if (lane == 0) at = atomicAdd(&total, __popc(m));
      at = __shfl_sync(kFull, at, 0);
      if (c) cand[at + __popc(m & ((1u << lane) - 1u))] = (int32_t)l;
    }
  }
  __syncthreads();
  const int nc_all = total;
  if (threadIdx.x == 0 && a.ncand) a.ncand[q] = nc_all;
  if (nc_all <= kCap) {
    for (int i = threadIdx.x; i < nc_all; i += kRThreads) sp.cbuf[q * kCap + i] = cand[i];
    const int nb = (nc_all + 31) >> 5;
    if (threadIdx.x == 0) sh[0] = (uint32_t)atomicAdd(sp.nitems, nb);
    __syncthreads();
    if (threadIdx.x < nb) sp.items[sh[0] + threadIdx.x] = make_int2((int)q, threadIdx.x);
    return;
  }
  // D, in the block: the query itself and the staging tiles (over `lower`)
  for (int d = threadIdx.x; d < dq; d += kRThreads) qs[d] = d < a.dim ? a.Q[q * a.dim + d] : 0.f;
  __syncthreads();
  float thd = INFINITY;
  int32_t thi = INT32_MAX;
  float* tile = tiles + warp * kRTile;
  for (int b0 = warp * 32; b0 < nc_all; b0 += kRWarps * 32) {
    const int nc = min(32, nc_all - b0);
    const float d = V4 ? batch_d2_v4(a.C, qs, a.dim, cand + b0, nc, tile)
                       : batch_d2_any(a.C, qs, a.dim, cand + b0, nc, tile);
    top.offer(lane < nc, d, lane < nc ? cand[b0 + lane] : 0, np, thd, thi);
  }
  __syncthreads();  // tiles are free: they hold the warps' lists
  float* md = tiles;
  int32_t* mi = (int32_t*)(tiles + kRWarps * R * 32);
#pragma unroll
  for (int r = 0; r < R; ++r) { md[(warp * R + r) * 32 + lane] = top.d[r]; mi[(warp * R + r) * 32 + lane] = top.id[r]; }
  __syncthreads();
  if (warp == 0) {
    for (int w = 1; w < kRWarps; ++w)
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float v = md[(w * R + r) * 32 + lane];
        top.offer(v != INFINITY, v, mi[(w * R + r) * 32 + lane], np, thd, thi);
      }
    write_probes<R>(a, q, np, top);
  }
}

constexpr int kDWarps = 4;  // warps per block of the distance kernel

// FP32-rule distances of the work items' candidates, one warp per item (a
// query and 32 of its candidates), the warps walking the item list; the query
// is read from global memory (a broadcast load per 16 bytes).
template <bool V4>
__global__ void __launch_bounds__(kDWarps * 32) rerank_dist_kernel(RerankArgs a, RerankSplit sp) {
  __shared__ __align__(16) float tiles[kDWarps][kRTile];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = *sp.nitems;
  for (int it = blockIdx.x * kDWarps + warp; it < n; it += gridDim.x * kDWarps) {
    const int2 w = sp.items[it];
    const int64_t q = w.x;
    const int b0 = w.y * 32;
    const int nc = min(32, a.ncand[q] - b0);
    const int32_t* cand = sp.cbuf + q * kCap + b0;
    const float* qrow = a.Q + q * a.dim;
    const float d = V4 ? batch_d2_v4(a.C, qrow, a.dim, cand, nc, tiles[warp])
                       : batch_d2_any(a.C, qrow, a.dim, cand, nc, tiles[warp]);
    if (lane < nc) sp.cdist[q * kCap + b0 + lane] = d;
  }
}

// The top-np of each query's candidates by (D2, l), one warp per query
// (queries with np = 0 or more than kCap candidates were finished by the
// select kernel).
template <int R>
__global__ void __launch_bounds__(256) rerank_merge_kernel(RerankArgs a, RerankSplit sp) {
  const int64_t q = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (q >= a.nq) return;
  const int np = a.npq ? min(max(a.npq[q], 0), a.nprobe) : a.nprobe;
  const int nc = a.ncand[q];
  if (np == 0 || nc > kCap) return;
  WarpTopK<R, int32_t> top;
  top.init();
  float thd = INFINITY;
  int32_t thi = INT32_MAX;
  for (int b0 = 0; b0 < nc; b0 += 32) {
    const bool v = b0 + lane < nc;
    top.offer(v, v ? sp.cdist[q * kCap + b0 + lane] : 0.f, v ? sp.cbuf[q * kCap + b0 + lane] : 0, np, thd, thi);
  }
  write_probes<R>(a, q, np, top);
}

// The re-rank for index sizes whose keys do not fit in shared memory: the
// bounds are recomputed at each pass instead of held, and each warp scans its
// own lists (strided), queueing candidates in a per-warp buffer.
template <int R>
__global__ void __launch_bounds__(kRThreads) rerank_stream_kernel(RerankArgs a) {
  __shared__ float md[kRWarps][R * 32];
  __shared__ int32_t mi[kRWarps][R * 32];
  __shared__ float tile[kRWarps][32 * 33];
  __shared__ int32_t qbuf[kRWarps][64];
  __shared__ int hist[256];
  __shared__ uint32_t sh[2];
  __shared__ int total;
  __shared__ uint32_t kr[2][kRWarps];
  float* qs = (float*)anns_dyn_smem;  // [dim]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t q = blockIdx.x, nlist = a.nlist;
  const int np = a.npq ? min(max(a.npq[q], 0), a.nprobe) : a.nprobe;
  const float* row = a.dt + q * nlist;
  const float qn = a.qrows[q], qd = a.qrows[a.nq + q];
  for (int d = threadIdx.x; d < a.dim; d += kRThreads) qs[d] = a.Q[q * a.dim + d];
  if (threadIdx.x == 0) total = 0;
  auto bound = [&](int64_t l) { return rerank_bound(row[l], qn, qd, a.crows[l], a.crows[nlist + l], a.kef, a.kfp); };
  float T = INFINITY;
  if (np > 0) {
    uint32_t kmin = 0xFFFFFFFFu, kmax = 0;
    for (int64_t l = threadIdx.x; l < nlist; l += kRThreads) {
      const uint32_t k = upper_key(row[l] + bound(l));
      kmin = min(kmin, k);
      kmax = max(kmax, k);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      kmin = min(kmin, __shfl_xor_sync(kFull, kmin, o));
      kmax = max(kmax, __shfl_xor_sync(kFull, kmax, o));
    }
    if (lane == 0) { kr[0][warp] = kmin; kr[1][warp] = kmax; }
    for (int i = threadIdx.x; i < 256; i += kRThreads) hist[i] = 0;
    __syncthreads();
    kmin = 0xFFFFFFFFu;
    kmax = 0;
    for (int w = 0; w < kRWarps; ++w) {
      kmin = min(kmin, kr[0][w]);
      kmax = max(kmax, kr[1][w]);
    }
    // one level: T = the top of the 256-bin bin holding the np-th smallest key
    int shift = 0;
    while (((kmax - kmin) >> shift) > 255u) ++shift;
    for (int64_t l = threadIdx.x; l < nlist; l += kRThreads)
      atomicAdd(&hist[(upper_key(row[l] + bound(l)) - kmin) >> shift], 1);
    __syncthreads();
    if (warp == 0) {
      int c[8], run = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) { c[i] = hist[lane * 8 + i]; run += c[i]; }
      int incl = run;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      const int excl = incl - run;
      int pick = -1;
      if (excl < np && np <= incl) {
        int acc = excl;
        for (int i = 0; i < 8; ++i) {
          if (acc + c[i] >= np) { pick = lane * 8 + i; break; }
          acc += c[i];
        }
      }
      const unsigned who = __ballot_sync(kFull, pick >= 0);
      pick = __shfl_sync(kFull, pick, who ? __ffs(who) - 1 : 0);
      if (lane == 0) sh[0] = who ? (uint32_t)pick : 255u;
    }
    __syncthreads();
    const uint64_t top_key = (uint64_t)kmin + (((uint64_t)sh[0] + 1) << shift) - 1;
    T = __uint_as_float(top_key > 0x7F800000ull ? 0x7F800000u : (uint32_t)top_key);
  }
  WarpTopK<R, int32_t> top;
  top.init();
  float thd = INFINITY;
  int32_t thi = INT32_MAX;
  int nq_w = 0, seen = 0;
  for (int64_t b0 = (int64_t)warp * 32; np > 0 && b0 < nlist; b0 += kRThreads) {
    const int64_t l = b0 + lane;
    const bool cand = l < nlist && !(row[l] - bound(l) > T);
    const unsigned m = __ballot_sync(kFull, cand);
    if (cand) qbuf[warp][nq_w + __popc(m & ((1u << lane) - 1u))] = (int32_t)l;
    nq_w += __popc(m);
    __syncwarp();
    if (nq_w >= 32) {
      const float d = batch_d2_any(a.C, qs, a.dim, qbuf[warp], 32, tile[warp]);
      top.offer(true, d, qbuf[warp][lane], np, thd, thi);
      seen += 32;
      const int rest = nq_w - 32;
      const int32_t mv = lane < rest ? qbuf[warp][32 + lane] : 0;
      __syncwarp();
      if (lane < rest) qbuf[warp][lane] = mv;
      nq_w = rest;
      __syncwarp();
    }
  }
  if (nq_w > 0) {
    const float d = batch_d2_any(a.C, qs, a.dim, qbuf[warp], nq_w, tile[warp]);
    top.offer(lane < nq_w, d, lane < nq_w ? qbuf[warp][lane] : 0, np, thd, thi);
    seen += nq_w;
  }
  if (lane == 0 && seen) atomicAdd(&total, seen);
#pragma unroll
  for (int r = 0; r < R; ++r) { md[warp][r * 32 + lane] = top.d[r]; mi[warp][r * 32 + lane] = top.id[r]; }
  __syncthreads();
  if (warp == 0) {
    for (int w = 1; w < kRWarps && np > 0; ++w)
#pragma unroll
      for (int r = 0; r < R; ++r) top.offer(md[w][r * 32 + lane] != INFINITY, md[w][r * 32 + lane],
                                            mi[w][r * 32 + lane], np, thd, thi);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int e = r * 32 + lane;
      if (e < a.nprobe) {
        const bool ok = e < np && top.d[r] != INFINITY;
        a.probes[q * a.nprobe + e] = ok ? top.id[r] : -1;
        a.probe_d2[q * a.nprobe + e] = ok ? top.d[r] : INFINITY;
      }
    }
    if (lane == 0 && a.ncand) a.ncand[q] = total;
  }
}

constexpr int kFmts[3] = {ANNS_PREC_BF16, ANNS_PREC_FP16, ANNS_PREC_FP8E4M3};

int fmt_slot(int prec) { return prec == ANNS_PREC_BF16 ? 0 : prec == ANNS_PREC_FP16 ? 1 : 2; }
int fmt_elem(int prec) { return prec == ANNS_PREC_FP8E4M3 ? 1 : 2; }

// Dynamic shared memory of the select kernel for this index: qs | keys |
// lower (or the tiles).
size_t rerank_smem(const Index& ix) {
  const size_t nl4 = (size_t)((ix.nlist + 3) & ~3);
  return (size_t)((ix.dim + 3) & ~3) * 4 + nl4 * 4 + std::max(nl4 * 4, (size_t)kRWarps * kRTile * 4);
}
constexpr size_t kRerankSmemMax = 200 * 1024;  // beyond it: the streaming re-rank

template <int F>
cudaError_t launch_center(const float* X, int64_t n, int dim, int Dp, const float* mu, void* Xf, float* rows,
                          cudaStream_t s) {
  center_kernel<F><<<(unsigned)((n + 7) / 8), 256, 0, s>>>(X, n, dim, Dp, mu, (typename TcFmt<F>::T*)Xf, rows);
  note_launch();
  return cudaGetLastError();
}

cudaError_t center_any(int prec, const float* X, int64_t n, int dim, int Dp, const float* mu, void* Xf,
                       float* rows, cudaStream_t s) {
  switch (prec) {
    case ANNS_PREC_BF16: return launch_center<ANNS_PREC_BF16>(X, n, dim, Dp, mu, Xf, rows, s);
    case ANNS_PREC_FP16: return launch_center<ANNS_PREC_FP16>(X, n, dim, Dp, mu, Xf, rows, s);
    default: return launch_center<ANNS_PREC_FP8E4M3>(X, n, dim, Dp, mu, Xf, rows, s);
  }
}

}  // namespace

bool coarse_tc_format(int prec) {
  return prec == ANNS_PREC_BF16 || prec == ANNS_PREC_FP16 || prec == ANNS_PREC_FP8E4M3;
}

int coarse_tc_dp(const Index& ix, int prec) {
  const int per = kKB / fmt_elem(prec);
  return (int)((ix.dim + per - 1) / per * per);
}

// Centroid operands (once per index): mu, and per format the centred, scaled,
// rounded centroids and their rows (cn, cd, cs).
int prepare_coarse_tc(Index& ix, const std::vector<float>& cent) {
  std::vector<double> mu64(ix.dim, 0.0);
  for (int64_t l = 0; l < ix.nlist; ++l)
    for (int64_t d = 0; d < ix.dim; ++d) mu64[d] += cent[l * ix.dim + d];
  std::vector<float> mu(ix.dim);
  for (int64_t d = 0; d < ix.dim; ++d) mu[d] = (float)(mu64[d] / (double)ix.nlist);
  cudaError_t e = cudaMalloc(&ix.tc_mu, ix.dim * sizeof(float));
  for (int f = 0; f < 3 && e == cudaSuccess; ++f) {
    const int prec = kFmts[f];
    e = cudaMalloc(&ix.tc_c[f], (size_t)ix.nlist * coarse_tc_dp(ix, prec) * fmt_elem(prec));
    if (e == cudaSuccess) e = cudaMalloc(&ix.tc_crows[f], (size_t)ix.nlist * 3 * sizeof(float));
  }
  if (e == cudaSuccess) e = cudaMalloc(&ix.dev_status, 16);
  if (e == cudaSuccess) e = cudaMemcpy(ix.tc_mu, mu.data(), ix.dim * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(ix.dev_status, 0, 16);
  for (int f = 0; f < 3 && e == cudaSuccess; ++f)
    e = center_any(kFmts[f], ix.centroids, ix.nlist, (int)ix.dim, coarse_tc_dp(ix, kFmts[f]), ix.tc_mu, ix.tc_c[f],
                   ix.tc_crows[f], 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e == cudaSuccess ? ANNS_OK : cuda_fail(e, "coarse fast-path setup");
}

// Tensor map of a row-major operand [rows x Dp] (elements of `elem` bytes):
// boxes of 128 bytes x box_rows rows, 128-byte swizzle, zero fill past the
// last row. Built through the driver entry point (no link to the driver
// library).
static cudaError_t make_tmap(CUtensorMap* map, CUtensorMapDataType type, int elem, const void* base, int64_t rows,
                             int Dp, int box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult qr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr);
    if (e != cudaSuccess) return e;
    if (qr != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)Dp, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)Dp * elem};
  const cuuint32_t box[2] = {(cuuint32_t)(kKB / elem), (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(map, type, 2, const_cast<void*>(base), dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Workspace: the queries' operand [nq x Dp] (any format) | rows [3][nq] |
// candidate counts [nq] | item count | candidate lists [nq][kCap] | their
// distances [nq][kCap] | work items [nq * kCap / 32].
static size_t tc_operand_bytes(const Index& ix, int64_t nq) {
  size_t b = 0;
  for (int prec : kFmts) b = std::max(b, (size_t)nq * coarse_tc_dp(ix, prec) * fmt_elem(prec));
  return (b + 255) & ~size_t(255);
}

static size_t tc_small_bytes(int64_t nq) { return ((size_t)nq * 16 + 16 + 255) & ~size_t(255); }

size_t coarse_tc_workspace_bytes(const Index& ix, int64_t nq) {
  return tc_operand_bytes(ix, nq) + tc_small_bytes(nq) + (size_t)nq * kCap * 8 + (size_t)nq * (kCap / 32) * 8;
}

const int* coarse_tc_candidates(const Index& ix, const void* ws, int64_t nq) {
  return (const int*)((const char*)ws + tc_operand_bytes(ix, nq) + (size_t)nq * 12);
}

template <int F>
static cudaError_t launch_gemm(const Index& ix, void* Qf, const float* qrows, int64_t nq, float* dt, cudaStream_t s) {
  using Fm = TcFmt<F>;
  const int f = fmt_slot(F), Dp = coarse_tc_dp(ix, F);
  CUtensorMap tmQ, tmC;
  cudaError_t e = make_tmap(&tmQ, Fm::kMap, Fm::kElem, Qf, nq, Dp, kTM);
  if (e == cudaSuccess) e = make_tmap(&tmC, Fm::kMap, Fm::kElem, ix.tc_c[f], ix.nlist, Dp, kTN);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(coarse_tc_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem);
  int sms = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix.device);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = ((nq + kTM - 1) / kTM) * ((ix.nlist + kTN - 1) / kTN);
  const unsigned grid = (unsigned)std::min<int64_t>(ntiles, sms);
  coarse_tc_kernel<F><<<grid, kGemmThreads, kGemmSmem, s>>>(
      tmQ, tmC, qrows, ix.tc_crows[f], nq, ix.nlist, Dp * Fm::kElem / kKB, dt, ix.dev_status,
      ix.opt_wait_cycles > 0 ? ix.opt_wait_cycles : kWaitCycles);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_coarse_tc(const Index& ix, int prec, const float* Q, int64_t nq, int nprobe,
                             const int32_t* nprobe_per_q, void* ws, float* dt, int32_t* probes, float* probe_d2,
                             cudaStream_t s) {
  const int f = fmt_slot(prec), Dp = coarse_tc_dp(ix, prec);
  void* Qf = ws;
  float* qrows = (float*)((char*)ws + tc_operand_bytes(ix, nq));  // qn | qd | qs
  int* ncand = (int*)(qrows + 3 * nq);                               // then the item count
  cudaError_t e = center_any(prec, Q, nq, (int)ix.dim, Dp, ix.tc_mu, Qf, qrows, s);
  if (e != cudaSuccess) return e;
  switch (prec) {
    case ANNS_PREC_BF16: e = launch_gemm<ANNS_PREC_BF16>(ix, Qf, qrows, nq, dt, s); break;
    case ANNS_PREC_FP16: e = launch_gemm<ANNS_PREC_FP16>(ix, Qf, qrows, nq, dt, s); break;
    default: e = launch_gemm<ANNS_PREC_FP8E4M3>(ix, Qf, qrows, nq, dt, s); break;
  }
  if (e != cudaSuccess) return e;
  RerankArgs a{Q, ix.centroids, dt, qrows, ix.tc_crows[f], nq, ix.nlist, (int)ix.dim,
               (float)((2.0 * Dp + 8.0) * 5.9604644775390625e-8 * 1.01), (float)((ix.dim + 2) * 5.9604644775390625e-8),
               nprobe, nprobe_per_q, probes, probe_d2, ncand};
  char* after = (char*)ws + tc_operand_bytes(ix, nq) + tc_small_bytes(nq);
  RerankSplit sp{(int32_t*)after, (float*)(after + (size_t)nq * kCap * 4), (int2*)(after + (size_t)nq * kCap * 8),
                 (int*)(ncand + nq)};
  const int R = (nprobe + 31) / 32;
  const unsigned g = (unsigned)nq;
  const size_t smem = rerank_smem(ix);
  const bool v4 = ix.dim % 4 == 0, q16 = ((uintptr_t)Q & 15u) == 0;
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ix.device);
  if (e != cudaSuccess) return e;
  auto run = [&](auto kern, unsigned grid, unsigned threads, size_t sm, auto... args) {
    cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e2 != cudaSuccess) return e2;
    kern<<<grid, threads, sm, s>>>(args...);
    note_launch();
    return cudaGetLastError();
  };
  auto run_r = [&](auto r_tag) {
    constexpr int RR = decltype(r_tag)::value;
    if (smem > kRerankSmemMax) return run(rerank_stream_kernel<RR>, g, kRThreads, (size_t)ix.dim * 4, a);
    cudaError_t e2 = cudaMemsetAsync(sp.nitems, 0, sizeof(int), s);
    if (e2 == cudaSuccess)
      e2 = v4 ? run(rerank_select_kernel<RR, true>, g, kRThreads, smem, a, sp)
              : run(rerank_select_kernel<RR, false>, g, kRThreads, smem, a, sp);
    // the distance kernel's grid: every block resident at once (the warps
    // stride over the item list)
    auto dist = [&](auto kern) {
      int per_sm = 0;
      cudaError_t e3 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kDWarps * 32, 0);
      if (e3 != cudaSuccess) return e3;
      return run(kern, (unsigned)(sms * std::max(per_sm, 1)), kDWarps * 32, 0, a, sp);
    };
    if (e2 == cudaSuccess) e2 = v4 && q16 ? dist(rerank_dist_kernel<true>) : dist(rerank_dist_kernel<false>);
    if (e2 == cudaSuccess) e2 = run(rerank_merge_kernel<RR>, (unsigned)((nq + 7) / 8), 256, 0, a, sp);
    return e2;
  };
  switch (R) {
    case 1: e = run_r(std::integral_constant<int, 1>{}); break;
    case 2: e = run_r(std::integral_constant<int, 2>{}); break;
    case 3: e = run_r(std::integral_constant<int, 3>{}); break;
    default: e = run_r(std::integral_constant<int, 4>{}); break;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace anns
