// Cluster locating on the tensor cores (the BF16 fast path of CL, Section 2.1),
// with an exact re-rank so that the probed lists and their distances are the
// ones of the FP32 rule.
//
// 1. Operands: q^ = fl32(q - mu), c^ = fl32(c - mu) with mu the centroids'
//    mean (distances are translation invariant, and centring shrinks the
//    norms the rounding error scales with), rounded to BF16 (nearest even)
//    and zero-padded to Dp = dim rounded up to 64. Per row: qn = sum of the
//    squared BF16 values (FP32), qh >= ||q^||_2.
// 2. D~[q][l] = fl32(fl32(qn + cn) - fl32(2 <q~, c~>)): a 128 x 256 tile per
//    CTA, tcgen05.mma kind::f16 (BF16 x BF16, FP32 accumulator in TMEM). One
//    thread loads 64-wide K chunks of both operands with TMA (128-byte
//    swizzle) into a 4-stage ring (full barriers: TMA transaction bytes);
//    another issues the MMAs and releases each stage with tcgen05.commit
//    (empty barriers); a final commit hands the accumulator to all four
//    warps, which read it with tcgen05.ld, stage the tile in shared memory
//    and write it out row by row.
// 3. Error bound per pair: |D~ - D2| <= eps(D~, norms), D2 the FP32-rule
//    distance (derivation at rerank_bound). T >= the nprobe-th smallest of
//    D~ + eps; every list of the FP32 top-nprobe has D~ - eps <= T, so those
//    candidates are re-ranked with the FP32 rule itself (same operation order
//    as coarse.cu) and the nprobe smallest (D2, l) kept: identical output to
//    the plain path.
//
// Every mbarrier wait is bounded (by default about a second; the index option
// ANNS_OPT_WAIT_CYCLES sets the main loop's limit); on a timeout the kernel
// records ANNS_DEV_TIMEOUT in the index's device status word, waits (with the
// long limit) for the copies and MMAs it has issued, frees its TMEM and
// returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "scan.cuh"

namespace anns {
namespace {

constexpr int kTM = 128;             // queries per tile = TMEM lanes
constexpr int kTN = 256;             // centroids per tile = FP32 TMEM columns
constexpr int kKC = 64;              // K elements per stage (4 MMAs of K = 16; one 128-byte swizzle row)
constexpr int kStages = 4;
constexpr int kGemmThreads = 128;    // one warpgroup: warp w reads TMEM lanes 32w..32w+31
constexpr uint32_t kABytes = kTM * kKC * 2;   // 16 KB
constexpr uint32_t kBBytes = kTN * kKC * 2;   // 32 KB
constexpr uint32_t kStageBytes = kABytes + kBBytes;
// ring + barriers + 1 KB alignment slack; one CTA per SM (256 of 512 TMEM columns)
constexpr size_t kGemmSmem = (size_t)kStages * kStageBytes + 1024 + 256;
constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz: the default limit and the drain's

// Instruction descriptor, kind::f16: D F32 (bits 4-5 = 1), A BF16 (bits 7-9 =
// 1), B BF16 (bits 10-12 = 1), A and B K-major (bits 15, 16 = 0), N >> 3 at
// bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                            ((uint32_t)(kTM >> 4) << 24);

// Shared-memory matrix descriptor of a K-major operand written by TMA with the
// 128-byte swizzle: start address >> 4 (bits 0-13), leading offset unused for
// swizzled K-major (encoded 1), stride between 8-row groups 1024 bytes >> 4
// (bits 32-45), descriptor version 1 (46-47), base offset 0 (1024-byte
// aligned atoms), layout 128-byte swizzle (61-63 = 2). Within the 128-byte
// row, the k-th group of 16 elements starts 32 k bytes further.
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
// the mbarrier to complete; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit = kWaitCycles) {
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
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// One warp per row: x^ = fl32(x - mu) in BF16 (zero past dim); per row
// xn = FP32 sum of the squared BF16 values, xh >= ||x^||_2 and
// xe >= ||bf16(x^) - x^||_2 (both from FP64 sums, rounded up).
__global__ void center_bf16_kernel(const float* __restrict__ X, int64_t n, int dim, int Dp,
                                   const float* __restrict__ mu, __nv_bfloat16* __restrict__ Xb,
                                   float* __restrict__ xn, float* __restrict__ xh, float* __restrict__ xe) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  float s = 0.f;
  double h = 0.0, r = 0.0;
  for (int d = lane; d < Dp; d += 32) {
    float v = 0.f;
    if (d < dim) v = sub_rn(X[row * dim + d], mu[d]);
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    Xb[row * Dp + d] = b;
    const float bf = __bfloat162float(b);
    s = add_rn(s, mul_rn(bf, bf));
    h += (double)v * (double)v;
    const double dv = (double)bf - (double)v;
    r += dv * dv;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    s = add_rn(s, __shfl_xor_sync(kFull, s, o));
    h += __shfl_xor_sync(kFull, h, o);
    r += __shfl_xor_sync(kFull, r, o);
  }
  if (lane == 0) {
    xn[row] = s;
    xh[row] = __double2float_ru(sqrt(h) * (1.0 + 1e-12));
    xe[row] = __double2float_ru(sqrt(r) * (1.0 + 1e-12));
  }
}

// D~ for a 128 x 256 tile (grid: x over centroid tiles, y over query tiles).
__global__ void __launch_bounds__(kGemmThreads) coarse_tc_kernel(
    const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ CUtensorMap tmC, const float* __restrict__ qn,
    const float* __restrict__ cn, int64_t nq, int64_t nlist, int Dp, float* __restrict__ dt,
    int* __restrict__ status, long long wait_limit) {
  unsigned char* base = anns_dyn_smem + ((1024u - (smem_addr(anns_dyn_smem) & 1023u)) & 1023u);
  uint64_t* bars = (uint64_t*)(base + kStages * kStageBytes);  // full[S] | empty[S] | done
  uint32_t* slot = (uint32_t*)(bars + 2 * kStages + 1);
  const uint32_t ring = smem_addr(base);
  const uint32_t full0 = smem_addr(bars), empty0 = full0 + 8 * kStages, done = full0 + 16 * kStages;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int q0 = (int)(blockIdx.y * kTM), l0 = (int)(blockIdx.x * kTN);
  const int nK = Dp / kKC;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"((uint32_t)kTN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(full0 + 8 * i, 1);
      mbar_init(empty0 + 8 * i, 1);
    }
    mbar_init(done, 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;

  bool ok = true;
  int issued = 0;  // K chunks whose copies the producer has issued
  if (tid == 0) {
    // TMA producer
    for (int i = 0; i < nK && ok; ++i) {
      const int st = i % kStages;
      if (i >= kStages) ok = mbar_wait(empty0 + 8 * st, (uint32_t)((i / kStages - 1) & 1), wait_limit);
      if (!ok) break;
      const uint32_t a_dst = ring + st * kStageBytes, b_dst = a_dst + kABytes;
      mbar_expect_tx(full0 + 8 * st, kStageBytes);
      tma_load_2d(a_dst, &tmQ, i * kKC, q0, full0 + 8 * st);
      tma_load_2d(b_dst, &tmC, i * kKC, l0, full0 + 8 * st);
      issued = i + 1;
    }
  } else if (tid == 32) {
    // MMA issuer
    for (int i = 0; i < nK && ok; ++i) {
      const int st = i % kStages;
      ok = mbar_wait(full0 + 8 * st, (uint32_t)((i / kStages) & 1), wait_limit);
      if (!ok) break;
      tc_fence_after();
      const uint32_t a_addr = ring + st * kStageBytes, b_addr = a_addr + kABytes;
#pragma unroll
      for (int ks = 0; ks < kKC / 16; ++ks)
        tc_mma(tmem, smem_desc_sw128(a_addr + ks * 32), smem_desc_sw128(b_addr + ks * 32),
               (i > 0 || ks > 0) ? 1u : 0u);
      tc_commit(empty0 + 8 * st);
    }
    tc_commit(done);  // arrives when every MMA issued above has completed
  }
  // everyone: the accumulator is complete once `done` fires
  const bool done_ok = mbar_wait(done, 0, wait_limit);
  ok = __syncthreads_and(ok && done_ok);
  tc_fence_after();
  if (ok) {
    // TMEM -> registers -> shared tile [128][256] (the ring is free now) -> rows out
    float* tileS = (float*)base;
    const int r = warp * 32 + lane;
    for (int c0 = 0; c0 < kTN; c0 += 16) {
      float acc[16];
      tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, acc);
#pragma unroll
      for (int j = 0; j < 16; ++j) tileS[r * (kTN + 1) + c0 + j] = acc[j];
    }
    __syncthreads();
    for (int rr = warp; rr < kTM; rr += kGemmThreads / 32) {
      const int64_t q = (int64_t)q0 + rr;
      if (q >= nq) break;
      const float qv = qn[q];
      for (int c = lane; c < kTN; c += 32) {
        const int64_t l = (int64_t)l0 + c;
        if (l < nlist) dt[q * nlist + l] = sub_rn(add_rn(qv, cn[l]), mul_rn(2.f, tileS[rr * (kTN + 1) + c]));
      }
    }
  } else if (tid == 0) {
    atomicExch(status, ANNS_DEV_TIMEOUT);
  }
  if (!ok) {
    // let the copies and MMAs already issued finish before the CTA exits (long
    // limit): stage st received ceil((issued - st) / kStages) copies, the last
    // completing the phase of parity (count - 1) & 1, and no copy follows it
    if (tid == 0)
      for (int st = 0; st < kStages; ++st) {
        const int count = issued > st ? (issued - st + kStages - 1) / kStages : 0;
        if (count > 0) mbar_wait(full0 + 8 * st, (uint32_t)((count - 1) & 1));
      }
    if (tid == 32) mbar_wait(done, 0);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)kTN)
                 : "memory");
}

// eps >= |D~ - D2| for a pair, D2 the FP32-rule distance. With x^ the centred
// FP32 vectors and x~ their BF16 roundings, delta = (q~ - c~) - (q - c) has
// ||delta|| <= dn = qe + ce + 2^-23 (qh + ch) (the rows' BF16 rounding errors
// plus the FP32 centring). S = ||q~ - c~||^2 differs from D~ by the FP32
// evaluation error e_f <= (2 Dp + 8) 2^-24 (qn + cn) (norm sums, the FP32
// accumulator of the products, the final combination), from the exact
// distance by at most dn (2 sqrt(S) + dn), and the FP32 rule differs from the
// exact distance by at most (dim + 2) 2^-24 of it. Constants padded by 1 %.
struct RowNorms { float n, h, e; };
__device__ __forceinline__ float rerank_bound(float dt, RowNorms q, RowNorms c, int dim, int Dp) {
  const float ef = (float)(2 * Dp + 8) * 5.9604645e-8f * (q.n + c.n) * 1.01f;
  const float dn = (q.e + c.e + 1.1920929e-7f * (q.h + c.h)) * 1.01f;
  const float sup = fmaxf(dt, 0.f) + ef;
  const float E = dn * (2.f * sqrtf(sup) * 1.01f + dn);
  return (ef + E + (float)(dim + 2) * 5.9604645e-8f * (sup + E)) * 1.01f + 1e-30f;
}

constexpr int kRWarps = 8, kRThreads = kRWarps * 32;

// Distances (FP32 rule) of up to 32 candidates, one per lane: the warp loads
// the candidates' centroid rows 32 dimensions at a time into a transposed
// tile (coalesced row segments) and each lane accumulates its own row in
// ascending dimension order.
__device__ __forceinline__ float batch_d2(const float* __restrict__ C, const float* qs, int dim, int32_t lc, int nc,
                                          float (*tile)[33]) {
  const int lane = threadIdx.x & 31;
  float acc = 0.f;
  for (int d0 = 0; d0 < dim; d0 += 32) {
    for (int r = 0; r < 32; ++r) {
      const int32_t lr = __shfl_sync(kFull, lc, r);
      tile[r][lane] = (r < nc && d0 + lane < dim) ? __ldg(C + (int64_t)lr * dim + d0 + lane) : 0.f;
    }
    __syncwarp();
    const int dd_end = min(32, dim - d0);
    for (int dd = 0; dd < dd_end; ++dd) {
      const float e = sub_rn(qs[d0 + dd], tile[lane][dd]);
      acc = add_rn(acc, mul_rn(e, e));
    }
    __syncwarp();
  }
  return acc;
}

// One block per query.
// Pass 1: T >= the np-th smallest upper bound u = D~ + eps: the keys (bits of
//   u; non-negative floats order like their bit patterns) are counted into
//   256 bins of (key - kmin) >> shift, the shift fitting the query's key range;
//   T is the top of the bin holding the np-th value.
// Pass 2: each warp scans its lists (strided), queues the candidates with
//   D~ - eps <= T (ballot compaction into a per-warp buffer), computes their
//   FP32-rule distances 32 at a time and keeps its top-np by (D2, l); the
//   warps' lists are merged at the end. Writes nprobe entries (padding -1 /
//   +inf) and the number of candidates.
template <int R>
__global__ void __launch_bounds__(kRThreads) rerank_kernel(
    const float* __restrict__ Q, const float* __restrict__ C, const float* __restrict__ dt,
    const float* __restrict__ qrows, const float* __restrict__ crows, int64_t nq, int64_t nlist, int dim, int Dp,
    int nprobe, const int32_t* __restrict__ npq, int32_t* __restrict__ probes, float* __restrict__ probe_d2,
    int* __restrict__ ncand) {
  __shared__ float md[kRWarps][R * 32];
  __shared__ int32_t mi[kRWarps][R * 32];
  __shared__ float tile[kRWarps][32][33];
  __shared__ int32_t qbuf[kRWarps][64];
  __shared__ int hist[256];
  __shared__ uint32_t sel_bucket;
  __shared__ int total;
  float* qs = (float*)anns_dyn_smem;  // [dim]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t q = blockIdx.x;
  const int np = npq ? min(max(npq[q], 0), nprobe) : nprobe;
  const float* row = dt + q * nlist;
  const RowNorms qr = {qrows[q], qrows[nq + q], qrows[2 * nq + q]};
  for (int d = threadIdx.x; d < dim; d += kRThreads) qs[d] = Q[q * dim + d];
  if (threadIdx.x == 0) total = 0;
  auto upper_key = [&](int64_t l) {
    const RowNorms cr = {crows[l], crows[nlist + l], crows[2 * nlist + l]};
    return __float_as_uint(fmaxf(row[l] + rerank_bound(row[l], qr, cr, dim, Dp), 0.f));
  };
  // pass 1: the key range of the upper bounds, then one count of
  // (key - kmin) >> shift into 256 bins (the shift fits the range), and T = the
  // top of the bin holding the np-th smallest key
  float T = INFINITY;
  if (np > 0) {
    uint32_t kmin = 0xFFFFFFFFu, kmax = 0;
    for (int64_t l = threadIdx.x; l < nlist; l += kRThreads) {
      const uint32_t key = upper_key(l);
      kmin = min(kmin, key);
      kmax = max(kmax, key);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      kmin = min(kmin, __shfl_xor_sync(kFull, kmin, o));
      kmax = max(kmax, __shfl_xor_sync(kFull, kmax, o));
    }
    if (lane == 0) { qbuf[warp][0] = (int32_t)kmin; qbuf[warp][1] = (int32_t)kmax; }
    for (int i = threadIdx.x; i < 256; i += kRThreads) hist[i] = 0;
    __syncthreads();
    kmin = 0xFFFFFFFFu;
    kmax = 0;
    for (int w = 0; w < kRWarps; ++w) {
      kmin = min(kmin, (uint32_t)qbuf[w][0]);
      kmax = max(kmax, (uint32_t)qbuf[w][1]);
    }
    int shift = 0;
    while (((kmax - kmin) >> shift) > 255u) ++shift;
    for (int64_t l = threadIdx.x; l < nlist; l += kRThreads) atomicAdd(&hist[(upper_key(l) - kmin) >> shift], 1);
    __syncthreads();
    if (warp == 0) {
      // bin where the running count reaches np
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
      uint32_t pick = 0xFFFFFFFFu;
      if (excl < np && np <= incl) {
        int acc = excl;
        for (int i = 0; i < 8; ++i) {
          if (acc + c[i] >= np) { pick = (uint32_t)(lane * 8 + i); break; }
          acc += c[i];
        }
      }
      const unsigned who = __ballot_sync(kFull, pick != 0xFFFFFFFFu);
      pick = __shfl_sync(kFull, pick, who ? __ffs(who) - 1 : 0);
      if (lane == 0) sel_bucket = who ? pick : 255u;  // (every list counted: np <= nlist keys, so found)
    }
    __syncthreads();
    const uint64_t top_key = (uint64_t)kmin + (((uint64_t)sel_bucket + 1) << shift) - 1;
    T = __uint_as_float(top_key > 0x7F800000ull ? 0x7F800000u : (uint32_t)top_key);
    __syncthreads();  // qbuf is reused below
  }
  // pass 2
  WarpTopK<R, int32_t> top;
  top.init();
  float thd = INFINITY;
  int32_t thi = INT32_MAX;
  int nq_w = 0, seen = 0;
  for (int64_t b0 = (int64_t)warp * 32; np > 0 && b0 < nlist; b0 += kRThreads) {
    const int64_t l = b0 + lane;
    bool cand = false;
    if (l < nlist) {
      const RowNorms cr = {crows[l], crows[nlist + l], crows[2 * nlist + l]};
      cand = row[l] - rerank_bound(row[l], qr, cr, dim, Dp) <= T;
    }
    const unsigned m = __ballot_sync(kFull, cand);
    if (cand) qbuf[warp][nq_w + __popc(m & ((1u << lane) - 1u))] = (int32_t)l;
    nq_w += __popc(m);
    __syncwarp();
    if (nq_w >= 32) {
      const int32_t lc = qbuf[warp][lane];
      const float d = batch_d2(C, qs, dim, lc, 32, tile[warp]);
      top.offer(true, d, lc, np, thd, thi);
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
    const int32_t lc = lane < nq_w ? qbuf[warp][lane] : 0;
    const float d = batch_d2(C, qs, dim, lc, nq_w, tile[warp]);
    top.offer(lane < nq_w, d, lc, np, thd, thi);
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
      if (e < nprobe) {
        const bool ok = e < np && top.d[r] != INFINITY;
        probes[q * nprobe + e] = ok ? top.id[r] : -1;
        probe_d2[q * nprobe + e] = ok ? top.d[r] : INFINITY;
      }
    }
    if (lane == 0 && ncand) ncand[q] = total;
  }
}

}  // namespace

int coarse_tc_dp(const Index& ix) { return (int)((ix.dim + kKC - 1) / kKC * kKC); }

// Centroid operands (once per index): mu, BF16 centred centroids and norms.
int prepare_coarse_tc(Index& ix, const std::vector<float>& cent) {
  const int Dp = coarse_tc_dp(ix);
  std::vector<double> mu64(ix.dim, 0.0);
  for (int64_t l = 0; l < ix.nlist; ++l)
    for (int64_t d = 0; d < ix.dim; ++d) mu64[d] += cent[l * ix.dim + d];
  std::vector<float> mu(ix.dim);
  for (int64_t d = 0; d < ix.dim; ++d) mu[d] = (float)(mu64[d] / (double)ix.nlist);
  cudaError_t e = cudaMalloc(&ix.tc_mu, ix.dim * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&ix.tc_cb, (size_t)ix.nlist * Dp * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc(&ix.tc_cn, (size_t)ix.nlist * 3 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&ix.dev_status, 16);
  if (e == cudaSuccess) e = cudaMemcpy(ix.tc_mu, mu.data(), ix.dim * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(ix.dev_status, 0, 16);
  if (e != cudaSuccess) return cuda_fail(e, "coarse fast-path setup");
  center_bf16_kernel<<<(unsigned)((ix.nlist + 7) / 8), 256>>>(ix.centroids, ix.nlist, (int)ix.dim, Dp, ix.tc_mu,
                                                             (__nv_bfloat16*)ix.tc_cb, ix.tc_cn,
                                                             ix.tc_cn + ix.nlist, ix.tc_cn + 2 * ix.nlist);
  note_launch();
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e == cudaSuccess ? ANNS_OK : cuda_fail(e, "coarse fast-path setup");
}

// Tensor map of a row-major BF16 matrix [rows x Dp]: boxes of 64 columns x
// box_rows rows, 128-byte swizzle, zero fill past the last row. Built through
// the driver entry point (no link to the driver library).
static cudaError_t make_tmap(CUtensorMap* map, const void* base, int64_t rows, int Dp, int box_rows) {
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
  const cuuint64_t strides[1] = {(cuuint64_t)Dp * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kKC, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
                            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

size_t coarse_tc_workspace_bytes(const Index& ix, int64_t nq) {
  return (size_t)nq * coarse_tc_dp(ix) * 2 + (size_t)nq * 4 * 4 + 256;
}

cudaError_t launch_coarse_tc(const Index& ix, const float* Q, int64_t nq, int nprobe,
                             const int32_t* nprobe_per_q, void* ws, float* dt, int32_t* probes,
                             float* probe_d2, cudaStream_t s) {
  const int Dp = coarse_tc_dp(ix);
  __nv_bfloat16* Qb = (__nv_bfloat16*)ws;
  float* qrows = (float*)((char*)ws + (((size_t)nq * Dp * 2 + 255) & ~size_t(255)));  // qn | qh | qe
  int* ncand = (int*)(qrows + 3 * nq);
  center_bf16_kernel<<<(unsigned)((nq + 7) / 8), 256, 0, s>>>(Q, nq, (int)ix.dim, Dp, ix.tc_mu, Qb, qrows,
                                                              qrows + nq, qrows + 2 * nq); note_launch();
  CUtensorMap tmQ, tmC;
  cudaError_t e = make_tmap(&tmQ, Qb, nq, Dp, kTM);
  if (e == cudaSuccess) e = make_tmap(&tmC, ix.tc_cb, ix.nlist, Dp, kTN);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(coarse_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((ix.nlist + kTN - 1) / kTN), (unsigned)((nq + kTM - 1) / kTM));
  coarse_tc_kernel<<<grid, kGemmThreads, kGemmSmem, s>>>(tmQ, tmC, qrows, ix.tc_cn, nq, ix.nlist, Dp, dt,
                                                         ix.dev_status,
                                                         ix.opt_wait_cycles > 0 ? ix.opt_wait_cycles : kWaitCycles);
  note_launch();
  const int R = (nprobe + 31) / 32;
  const unsigned g = (unsigned)nq;
  const size_t qsm = (size_t)ix.dim * sizeof(float);
  auto run = [&](auto kern) {
    cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qsm);
    if (e2 != cudaSuccess) return e2;
    kern<<<g, kRThreads, qsm, s>>>(Q, ix.centroids, dt, qrows, ix.tc_cn, nq, ix.nlist, (int)ix.dim, Dp, nprobe,
                                   nprobe_per_q, probes, probe_d2, ncand); note_launch();
    return cudaGetLastError();
  };
  switch (R) {
    case 1: e = run(rerank_kernel<1>); break;
    case 2: e = run(rerank_kernel<2>); break;
    case 3: e = run(rerank_kernel<3>); break;
    default: e = run(rerank_kernel<4>); break;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace anns
