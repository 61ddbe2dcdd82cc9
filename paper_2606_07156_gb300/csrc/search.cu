// RC + LC + precision + DC + TS (Section 2.1) for one query per thread block;
// the general kernel (any M, dsub, k) and the one behind the pair-level taps.
//
// Per probed list l of query q, the block
//   1. forms the FP32 LUT shifted by ||r_m||^2, T'[m][c] = fl32(P_l - 2 Q_q),
//      from the list's table P_l and the query's table 2 Q_q (LC),
//   2. if the pair's precision is b bits, quantises T' with one shared step
//      Delta = range/(2^b-1) and per-sub-table biases into a uint8 (b <= 8) or
//      uint16 table in shared memory, the offset B32 = the exact sum of D2 and
//      the biases rounded once to FP32,
//   3. scans the list's packed codes tile by tile, one vector per lane,
//      summing LUT entries in ascending m — FP32 sums for the plain LUT
//      (distance fl32(D2 + sum)), exact int32 sums S for quantised LUTs
//      (distance fl32(fl32(Delta32 * S) + B32)) (DC),
//   4. offers each distance to a per-warp sorted top-k list (TS).
// The LUT never leaves shared memory. At the end the warps' lists are merged.
//
// A launch keeps only the tables its pairs need: every width (the FP32 T',
// staged, and a level table of up to 16 bits), FP32 pairs only (no level
// table), or 1..8-bit pairs only (no FP32 table: the levels are built in two
// passes from rows streamed through a cp.async ring). Fewer bytes of shared
// memory per block leave room for more blocks per SM; the split search runs
// its wide pairs in one launch and its 1..8-bit pairs in a second, which
// merges the first one's per-query top-k.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "scan.cuh"

namespace anns {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

struct PairScal {
  double delta64;
  float s32, delta32, B32, range;
  int L;
};

// Table widths a query-major launch serves: every width (the FP32 table T'
// and a level table of up to 2 bytes an entry), FP32 pairs only (no level
// table), or 1..8-bit pairs only (a 1-byte level table and no FP32 table:
// the levels are built in two passes from global memory).
enum : int { kModeFull = 0, kModeFp32 = 1, kModeNarrow = 2 };

// Offsets from a 256-byte aligned base inside the block's dynamic shared
// memory (256 bytes of slack are allocated for the alignment): the FP32 table
// T, the level table q (1 or 2 bytes an entry), row statistics and scales.
// A table the mode does not use takes no space.
// Rows of P_l and 2 Q_q a warp of a kModeNarrow block keeps in flight while
// it builds a table (cp.async ring in shared memory).
__host__ __device__ constexpr int ring_rows(int R) { return R == 1 ? 2 : 4; }

struct SmemLayout {
  size_t T = 0, q = 0, bias = 0, rowmax = 0, scal = 0, d2 = 0, plist = 0, md = 0, mi = 0, ring = 0, total = 0;
  static size_t al(size_t x) { return (x + 15) & ~size_t(15); }
  SmemLayout() = default;
  SmemLayout(int64_t Mp, int R, int mode = kModeFull) {
    size_t o = 0;   // the tables first, at multiples of 256 bytes
    T = o; o += mode == kModeNarrow ? 0 : al(Mp * kKsub * 4);
    q = o; o += mode == kModeFp32 ? 0 : al(Mp * kKsub * (mode == kModeNarrow ? 1 : 2));
    bias = o; o += al(Mp * 4);
    rowmax = o; o += al(Mp * 4);
    scal = o; o += al(sizeof(PairScal));
    d2 = o; o += 16;
    plist = o; o += al((size_t)ANNS_MAX_NPROBE * 16 + 16);  // + the count
    md = o; o += al((size_t)kWarps * R * 32 * 4);
    mi = o; o += al((size_t)kWarps * R * 32 * 8);
    ring = o; o += mode == kModeNarrow ? al((size_t)kWarps * ring_rows(R) * 2 * kKsub * 4) : 0;
    total = o + 256;
  }
};

__device__ __forceinline__ unsigned char* aligned_smem() {
  const uint32_t a = smem_addr(anns_dyn_smem);
  return anns_dyn_smem + ((256u - (a & 255u)) & 255u);
}

struct Smem {
  float* T; void* q; float* bias; float* rowmax; PairScal* sc; float* d2; float* md; int64_t* mi;
  float* ring;  // kModeNarrow: per warp, ring_rows(R) slots of [P row | 2 Q row]
  int4* plist; int* npairs;  // query-major kernel: the block's pairs (list, n_l, bits, D2 bits) and their count
  uint32_t T_addr, q_addr;  // shared-memory byte addresses of the two tables
  __device__ explicit Smem(const SmemLayout& L) {
    unsigned char* b = aligned_smem();
    T = (float*)(b + L.T); q = b + L.q; bias = (float*)(b + L.bias); rowmax = (float*)(b + L.rowmax);
    sc = (PairScal*)(b + L.scal); d2 = (float*)(b + L.d2); md = (float*)(b + L.md); mi = (int64_t*)(b + L.mi);
    plist = (int4*)(b + L.plist); npairs = (int*)(b + L.plist + (size_t)ANNS_MAX_NPROBE * 16);
    ring = (float*)(b + L.ring);
    T_addr = smem_addr(T);
    q_addr = smem_addr(q);
  }
};

// Round to nearest (ties to even) of y in [0, 2^22), read from the low bits of
// fl32(y + 1.5 * 2^23): the sum lies in [2^23, 2^24), where consecutive FP32
// values are 1 apart, so the IEEE addition itself rounds y to the nearest
// integer n and the result's bit pattern is 0x4B400000 + n.
__device__ __forceinline__ uint32_t rint_bits(float y) { return __float_as_uint(add_rn(y, 12582912.0f)); }

// Per-pair step Delta and offset B from the row statistics `bias`, `rowmax`
// (every warp derives the shared step; warp 0 also the offset B32, the exact
// sum of D2 and the row minima rounded once, and writes *out).
// The FP64 step delta64 (an FP64 division) is only computed for the taps.
// Returns s32.
template <bool WITH_D64>
__device__ __forceinline__ float pair_scale(int M, int b, const float* rowmax, PairScal* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float range = 0.f;
  for (int m = lane; m < M; m += 32) range = fmaxf(range, rowmax[m]);
  range = warp_max(range);
  const int L = (1 << b) - 1;
  // fl32 of the FP64 quotient equals the correctly rounded FP32 quotient
  const float s32 = range > 0.f ? __fdiv_rn((float)L, range) : 0.f;
  if (warp == 0 && lane == 0) {
    PairScal sc;
    sc.delta64 = WITH_D64 && range > 0.f ? __ddiv_rn((double)range, (double)L) : 0.0;
    sc.s32 = s32;
    sc.delta32 = range > 0.f ? __fdiv_rn(range, (float)L) : 0.f;
    sc.B32 = 0.f;  // pair_offset writes it
    sc.range = range;
    sc.L = L;
    *out = sc;
  }
  return s32;
}

// The pair's offset B32 (warp 0): the exact sum of D2 and the row minima,
// rounded once. Called once the levels are written, when the build's
// registers are free; the caller synchronises before the scan reads it.
__device__ __noinline__ void pair_offset(int M, float d2, const float* bias, PairScal* out) {
  const float B32 = warp_exact_sum(bias, M, d2, true);
  if ((threadIdx.x & 31) == 0) out->B32 = B32;
}

// Levels of 8 entries of one row: t = rint(fl32(fl32(T' - bias) * s32)).
// min(t, L) of the rule never binds: T' - bias <= range and s32 <= (L / range)
// (1 + 2^-24), so the product rounds to at most L + ulp(L) < L + 1/2.
__device__ __forceinline__ void quantise8(const float (&x)[8], float mn, float s32, uint32_t (&n)[8]) {
#pragma unroll
  for (int e = 0; e < 8; ++e) n[e] = rint_bits(mul_rn(sub_rn(x[e], mn), s32));
}

// Packs the 8 levels (low bits of n) of `lane` into table row `row`, 1 or 2
// bytes each, at the entries row_at() gives.
__device__ __forceinline__ void store_levels(int b, const uint32_t (&n)[8], void* row, int lane) {
  if (b <= 8) {
    uint8_t* r = (uint8_t*)row;
    *(uint32_t*)(r + row_at(lane, 0)) =
        __byte_perm(__byte_perm(n[0], n[1], 0x0040), __byte_perm(n[2], n[3], 0x0040), 0x5410);
    *(uint32_t*)(r + row_at(lane, 1)) =
        __byte_perm(__byte_perm(n[4], n[5], 0x0040), __byte_perm(n[6], n[7], 0x0040), 0x5410);
  } else {
    uint16_t* r = (uint16_t*)row;
    *(uint2*)(r + row_at(lane, 0)) = make_uint2(__byte_perm(n[0], n[1], 0x5410), __byte_perm(n[2], n[3], 0x5410));
    *(uint2*)(r + row_at(lane, 1)) = make_uint2(__byte_perm(n[4], n[5], 0x5410), __byte_perm(n[6], n[7], 0x5410));
  }
}

// Steps 1-2 for one pair, T' staged in shared memory (any Mp): all threads of
// the block take part. P and qt2 are the pair's list table and query table
// ([Mp * 256], rows M..Mp-1 zero). Warp w builds rows m = w, w + nwarps, ...;
// lane i owns the 8 entries row_at() gives, so each row's minimum and range come
// from warp shuffles during the build, and each warp quantises the rows it
// built (two block barriers for a b-bit pair, one for an FP32 pair). The FP32
// T' stays in shared memory for every pair (the LUT taps read it).
__device__ void build_lut(const float* __restrict__ P, const float* __restrict__ qt2, int M, int Mp,
                          int b, float d2, Smem& s) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int m = warp; m < Mp; m += nwarps) {
    float t[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (m >= M) {
      st_row8(s.T + m * kKsub, lane, t);
      continue;
    }
    float p[8], q[8];
    ldg_row8(P + m * kKsub, lane, p);
    ldg_row8(qt2 + m * kKsub, lane, q);
#pragma unroll
    for (int e = 0; e < 8; ++e) t[e] = sub_rn(p[e], q[e]);
    st_row8(s.T + m * kKsub, lane, t);
    if (b != 0) {
      float mn = t[0];
#pragma unroll
      for (int e = 1; e < 8; ++e) mn = fminf(mn, t[e]);
      mn = warp_min(mn);
      float mx = 0.f;
#pragma unroll
      for (int e = 0; e < 8; ++e) mx = fmaxf(mx, sub_rn(t[e], mn));
      mx = warp_max(mx);
      if (lane == 0) { s.bias[m] = mn; s.rowmax[m] = mx; }
    }
  }
  __syncthreads();
  if (b == 0) return;
  const float s32 = pair_scale<true>(M, b, s.rowmax, s.sc);
  const size_t esz = b <= 8 ? 1 : 2;
  for (int m = warp; m < Mp; m += nwarps) {
    float x[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float mn = 0.f;
    if (m < M) {
      mn = s.bias[m];
      const float* row = s.T + m * kKsub;
      const float4 u = *(const float4*)(row + row_at(lane, 0)), v = *(const float4*)(row + row_at(lane, 1));
      x[0] = u.x; x[1] = u.y; x[2] = u.z; x[3] = u.w; x[4] = v.x; x[5] = v.y; x[6] = v.z; x[7] = v.w;
    }
    uint32_t n[8];
    quantise8(x, mn, s32, n);
    store_levels(b, n, (uint8_t*)s.q + (size_t)m * kKsub * esz, lane);
  }
  if (warp == 0) pair_offset(M, d2, s.bias, s.sc);
  __syncthreads();
}

// Steps 1-2 with T' kept in registers (Mp == RPW * warps of the block): warp w
// owns rows w + r * nwarps, r < RPW. An FP32 pair stores T' into `T`; a
// quantised pair never writes T', each warp quantising its rows from
// registers into `lv` once the block-wide range is known (same values as
// build_lut, one block barrier fewer and no FP32 round trip through shared
// memory). One barrier between the row statistics and the scale; the caller
// synchronises before reading the tables.
template <int RPW>
__device__ __forceinline__ void build_lut_regs(const float* __restrict__ P, const float* __restrict__ qt2,
                                               int M, int b, float d2, float* T, void* lv, float* bias,
                                               float* rowmax, PairScal* sc) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  float t[RPW][8];
  float mn[RPW];
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    const int m = warp + r * nwarps;
    mn[r] = 0.f;
    if (m < M) {
      float p[8], q[8];
      ldg_row8(P + m * kKsub, lane, p);
      ldg_row8(qt2 + m * kKsub, lane, q);
#pragma unroll
      for (int e = 0; e < 8; ++e) t[r][e] = sub_rn(p[e], q[e]);
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) t[r][e] = 0.f;
    }
  }
  if (b == 0) {
#pragma unroll
    for (int r = 0; r < RPW; ++r) st_row8(T + (warp + r * nwarps) * kKsub, lane, t[r]);
    return;
  }
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    const int m = warp + r * nwarps;
    if (m < M) {
      float lo = t[r][0], hi = t[r][0];
#pragma unroll
      for (int e = 1; e < 8; ++e) { lo = fminf(lo, t[r][e]); hi = fmaxf(hi, t[r][e]); }
      mn[r] = warp_min(lo);
      // max over entries of fl32(t - mn) = fl32(max t - mn): rounding is monotone
      const float mx = sub_rn(warp_max(hi), mn[r]);
      if (lane == 0) { bias[m] = mn[r]; rowmax[m] = mx; }
    }
  }
  __syncthreads();
  const float s32 = pair_scale<false>(M, b, rowmax, sc);
  const size_t esz = b <= 8 ? 1 : 2;
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    uint32_t n[8];
    quantise8(t[r], mn[r], s32, n);
    store_levels(b, n, (uint8_t*)lv + (size_t)(warp + r * nwarps) * kKsub * esz, lane);
  }
  if (warp == 0) pair_offset(M, d2, bias, sc);
}

// 16-byte asynchronous copy global -> shared (no register staging), and the
// group bookkeeping: wait_group N returns once at most N of this thread's most
// recent groups are still in flight.
__device__ __forceinline__ void cp_async16(float* smem_dst, const float* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem_dst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Steps 1-2 for a 1..8-bit pair without an FP32 table (kModeNarrow), in two
// passes over the pair's rows of P_l and 2 Q_q: the row statistics from T'
// formed from the rows, then the levels from T' formed again (the same
// operations, so the same values as build_lut), written as bytes. Each warp
// streams its rows m = warp + nwarps i through a ring of RS slots in shared
// memory, RS rows in flight; a lane copies, and later reads, exactly the
// 16-byte pieces at row_at(lane, 0) and row_at(lane, 1), so the slots need no
// warp barrier. A pass starts with the rows 0..RS-1 requested (prime()) and
// ends with no copy in flight, which lets the search kernel request a pass's
// first rows before the work that precedes it, and run the statistics pass
// of the next pair right after each warp's share of the scan.
template <int RS>
struct NarrowBuild {
  const float* P;
  const float* qt2;
  float* slots;
  int nr, warp, lane;
  static constexpr int kWarpsPerBlock = kWarps;
  __device__ NarrowBuild(const float* __restrict__ P_, const float* __restrict__ qt2_, int M, const Smem& s)
      : P(P_), qt2(qt2_) {
    warp = threadIdx.x >> 5;
    lane = threadIdx.x & 31;
    slots = s.ring + (size_t)warp * RS * 2 * kKsub;
    nr = warp < M ? (M - warp + kWarpsPerBlock - 1) / kWarpsPerBlock : 0;  // rows m = warp + nwarps i < M
  }
  // Requests row index i into slot i % RS and commits one group per call
  // (empty beyond the warp's rows), so wait_group counts rows.
  __device__ __forceinline__ void issue(int i) const {
    if (i < nr) {
      const int m = warp + kWarpsPerBlock * i;
      float* d = slots + (i % RS) * 2 * kKsub;
      cp_async16(d + row_at(lane, 0), P + m * kKsub + row_at(lane, 0));
      cp_async16(d + row_at(lane, 1), P + m * kKsub + row_at(lane, 1));
      cp_async16(d + kKsub + row_at(lane, 0), qt2 + m * kKsub + row_at(lane, 0));
      cp_async16(d + kKsub + row_at(lane, 1), qt2 + m * kKsub + row_at(lane, 1));
    }
    cp_async_commit();
  }
  __device__ __forceinline__ void prime() const {
#pragma unroll
    for (int i = 0; i < RS; ++i) issue(i);
  }
  // T' of this lane's 8 entries of the row in slot i % RS (landed)
  __device__ __forceinline__ void row(int i, float (&t)[8]) const {
    const float* d = slots + (i % RS) * 2 * kKsub;
    const float4 p0 = *(const float4*)(d + row_at(lane, 0)), p1 = *(const float4*)(d + row_at(lane, 1));
    const float4 q0 = *(const float4*)(d + kKsub + row_at(lane, 0)), q1 = *(const float4*)(d + kKsub + row_at(lane, 1));
    t[0] = sub_rn(p0.x, q0.x); t[1] = sub_rn(p0.y, q0.y); t[2] = sub_rn(p0.z, q0.z); t[3] = sub_rn(p0.w, q0.w);
    t[4] = sub_rn(p1.x, q1.x); t[5] = sub_rn(p1.y, q1.y); t[6] = sub_rn(p1.z, q1.z); t[7] = sub_rn(p1.w, q1.w);
  }
  // Pass 1 (rows primed): the minimum and range of this warp's rows, taken
  // RS at a time (slot j holds row index i0 + j).
  __device__ void stats(Smem& s) const {
    for (int i0 = 0;; i0 += RS) {
#pragma unroll
      for (int j = 0; j < RS; ++j) {
        const int i = i0 + j;
        if (i >= nr) {
          cp_async_wait<0>();
          return;
        }
        cp_async_wait<RS - 1>();  // row i's group has landed
        float t[8];
        row(j, t);
        float lo = t[0], hi = t[0];
#pragma unroll
        for (int e = 1; e < 8; ++e) {
          lo = fminf(lo, t[e]);
          hi = fmaxf(hi, t[e]);
        }
        const int m = warp + kWarpsPerBlock * i;
        const float mn = warp_min(lo);
        // max over entries of fl32(t - mn) = fl32(max t - mn): rounding is monotone
        const float mx = sub_rn(warp_max(hi), mn);
        if (lane == 0) { s.bias[m] = mn; s.rowmax[m] = mx; }
        issue(i + RS);  // into the slot just read (this lane's own pieces)
      }
    }
  }
  // Pass 2 (rows primed, every row's statistics visible to the block): the
  // shared step, this warp's levels and zero padding rows, and (warp 0) the
  // offset. The caller synchronises before the scan reads them.
  __device__ void levels(int M, int Mp, int b, float d2, Smem& s) const {
    const float s32 = pair_scale<false>(M, b, s.rowmax, s.sc);
    for (int i0 = 0; i0 < nr; i0 += RS) {
#pragma unroll
      for (int j = 0; j < RS; ++j) {
        const int i = i0 + j;
        if (i >= nr) break;
        cp_async_wait<RS - 1>();
        float t[8];
        row(j, t);
        const int m = warp + kWarpsPerBlock * i;
        uint32_t n[8];
        quantise8(t, s.bias[m], s32, n);
        store_levels(b, n, (uint8_t*)s.q + (size_t)m * kKsub, lane);
        issue(i + RS);
      }
    }
    cp_async_wait<0>();
    for (int m = M + ((warp - M % kWarpsPerBlock + kWarpsPerBlock) % kWarpsPerBlock); m < Mp; m += kWarpsPerBlock) {
      const uint32_t z[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};  // padding rows: level 0
      store_levels(b, z, (uint8_t*)s.q + (size_t)m * kKsub, lane);
    }
    if (warp == 0) pair_offset(M, d2, s.bias, s.sc);
  }
};

template <int NCHUNK>
__device__ __forceinline__ void load_tile(const uint8_t* __restrict__ tile, int lane, uint4 (&w)[NCHUNK]) {
#pragma unroll
  for (int c = 0; c < NCHUNK; ++c)
    w[c] = __ldg(reinterpret_cast<const uint4*>(tile + c * kTileChunkBytes + lane * kChunkBytes));
}

__device__ __forceinline__ float dequant(int S, const PairScal& sc) {
  return add_rn(mul_rn(sc.delta32, __int2float_rn(S)), sc.B32);
}

// Distance of the vector whose code tile words are w, for a pair whose table
// was built with `b` bits (0 = FP32, at T_addr; else levels at q_addr) and
// coarse distance d2.
template <int NCHUNK>
__device__ __forceinline__ float pair_distance(int b, float d2, uint32_t T_addr, uint32_t q_addr,
                                               const PairScal& sc, const uint4 (&w)[NCHUNK],
                                               int* S_out = nullptr) {
  if (b == 0) return add_rn(d2, adc_f32<NCHUNK>(T_addr, w));
  const int S = b <= 8 ? adc_int<uint8_t, NCHUNK>(q_addr, w) : adc_int<uint16_t, NCHUNK>(q_addr, w);
  if (S_out) *S_out = S;
  return dequant(S, sc);
}

struct SearchArgs {
  const float* Q; const float* qt; int64_t nq, dim, nlist;
  const float* centroids; const float* ltab;
  const uint8_t* codes; const int64_t* ids;
  const int32_t* list_len; const int64_t* vec_off; const int64_t* tile_off;
  int M, Mp, nprobe, k;
  const int32_t* npq; const int32_t* kpq;
  const int32_t* probes; const float* probe_d2; const uint8_t* bits;
  const int32_t* order;
  // 1: leave out the pairs on 1..8-bit tables of rank >= 1 (the grouped
  // kernels take them); 2: of every rank (the narrow pass takes them)
  int skip_narrow;
  int ids32;  // every id fits in int32 (the 128-entry lists then hold 32-bit ids)
  int64_t* ids_out; float* dists_out;
  // kModeNarrow: the query's top-k over its other pairs ([nq * k], padding
  // +inf), which bounds the scan and joins the final merge; or null
  const float* part_d; const int64_t* part_i;
  SmemLayout lay;
};

// End of a query: the warps' lists are merged into warp 0, which writes the
// query's k results (padding id -1, distance +inf). Ends with a barrier.
template <int R, typename IdT>
__device__ __forceinline__ void merge_and_write(const SearchArgs& a, Smem& s, WarpTopK<R, IdT>& top,
                                                int64_t q, int kq, float& thd, IdT& thi) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (a.part_d && kq > 0) {
    // the top-k of the query's other pairs joins warp 0's list
    if (warp == 0)
      for (int e0 = 0; e0 < kq; e0 += 32) {
        const int e = e0 + lane;
        const float cd = e < kq ? a.part_d[q * a.k + e] : INFINITY;
        const IdT ci = e < kq ? (IdT)a.part_i[q * a.k + e] : IdMax<IdT>::v();
        top.offer(cd != INFINITY, cd, ci, kq, thd, thi);
      }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    s.md[(warp * R + r) * 32 + lane] = top.d[r];
    s.mi[(warp * R + r) * 32 + lane] = (int64_t)top.id[r];
  }
  __syncthreads();
  if (warp == 0) {
    for (int w2 = 1; w2 < kWarps && kq > 0; ++w2)
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float cd = s.md[(w2 * R + r) * 32 + lane];
        const IdT ci = (IdT)s.mi[(w2 * R + r) * 32 + lane];
        top.offer(cd != INFINITY, cd, ci, kq, thd, thi);
      }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int e = r * 32 + lane;
      if (e < a.k) {
        const bool ok = e < kq && top.d[r] != INFINITY;
        a.ids_out[q * a.k + e] = ok ? (int64_t)top.id[r] : -1;
        a.dists_out[q * a.k + e] = ok ? top.d[r] : INFINITY;
      }
    }
  }
  __syncthreads();
}

// Query-major search: one query per block at a time. Per pair the block builds
// the table (in registers for Mp <= 32, else staged in shared memory; in two
// passes from global memory for kModeNarrow), then every warp scans tiles of
// the list. Four blocks per SM for Mp <= 32 (two with the 128-entry lists of
// k > 32); without the FP32 table (kModeNarrow) three (two with the 128-entry
// lists, whose inserts need the registers); without the level table
// (kModeFp32) two up to Mp = 96, where two FP32 tables fit in shared memory
// (beyond it a second block cannot be resident, and the register cap would
// only cost spills).
template <int MODE, int NCHUNK, int R>
constexpr int qm_blocks() {
  return MODE == kModeNarrow ? (R == 1 ? (NCHUNK <= 2 ? 4 : 3) : 2)
                             : (NCHUNK <= 2 ? (R == 1 ? 4 : 2) : (MODE == kModeFp32 && NCHUNK <= 6 ? 2 : 1));
}

// IdT: the id type of the warps' lists (int32_t when every id of the index
// fits, for the 128-entry lists: fewer registers and shuffles per insert).
template <int NCHUNK, int R, int MODE, typename IdT = int64_t>
__global__ void __launch_bounds__(kThreads, qm_blocks<MODE, NCHUNK, R>()) search_kernel(const SearchArgs a) {
  Smem s(a.lay);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tstride = (int64_t)a.Mp * kKsub;
  for (int64_t qi = blockIdx.x; qi < a.nq; qi += gridDim.x) {
    const int64_t q = a.order ? (int64_t)a.order[qi] : qi;
    const int np = a.npq ? min(max(a.npq[q], 0), a.nprobe) : a.nprobe;
    const int kq = a.kpq ? min(max(a.kpq[q], 0), a.k) : a.k;
    WarpTopK<R, IdT> top;
    top.init();
    float thd = INFINITY;
    IdT thi = IdMax<IdT>::v();
    // 128-entry lists (k > 32): the block shares the smallest k-th distance
    // any warp holds (at least k vectors lie at or below it, so no farther
    // vector can enter the final top-k; equal distances are kept)
    float* blim = s.d2 + 1;
    if (R > 1 && threadIdx.x == 0) *blim = INFINITY;
    // the probe ranks this block scans, found by warp 0 in one parallel pass
    // (lane i reads rank 32 r + i) and kept in shared memory: the pairs'
    // metadata costs one round of loads per query instead of a dependent chain
    // of loads per rank
    if (warp == 0) {
      int base = 0;
      for (int j0 = 0; j0 < np && kq > 0; j0 += 32) {
        const int j = j0 + lane;
        int l = -1, n_l = 0, b = 0;
        float d2 = 0.f;
        if (j < np) {
          const int64_t i = q * a.nprobe + j;
          l = a.probes[i];
          b = a.bits[i];
          d2 = a.probe_d2[i];
          if (l >= 0) n_l = a.list_len[l];
        }
        const bool narrow = b >= 1 && b <= 8;
        const bool use = l >= 0 && n_l > 0 &&
                         (MODE == kModeNarrow ? narrow
                                              : !(narrow && (a.skip_narrow == 2 || (a.skip_narrow == 1 && j >= 1))));
        const unsigned m = __ballot_sync(kFull, use);
        if (use) s.plist[base + __popc(m & ((1u << lane) - 1u))] = make_int4(l, n_l, b, __float_as_int(d2));
        base += __popc(m);
      }
      if (lane == 0) *s.npairs = base;
    }
    __syncthreads();
    const int npairs = *s.npairs;
    // kModeNarrow: no vector beyond the k-th distance of the query's other
    // pairs can enter the final top-k (equal distances are kept: the id decides)
    const float bnd = MODE == kModeNarrow && a.part_d && kq > 0 ? a.part_d[q * a.k + kq - 1] : INFINITY;
    // kModeNarrow runs pair e as [barrier] levels of e, request of the rows
    // of e + 1 [barrier] scan of e, statistics of e + 1, second request of its
    // rows (iteration -1 takes the statistics of pair 0): two block barriers
    // a pair instead of three, the first rows of each pass requested before
    // the work that precedes it, and the warps that finish their tiles first
    // go on to the next statistics
    using Narrow = NarrowBuild<ring_rows(R)>;
    const float* qt2 = a.qt + q * tstride;
    if constexpr (MODE == kModeNarrow) {
      if (npairs > 0) Narrow(a.ltab + (size_t)s.plist[0].x * tstride, qt2, a.M, s).prime();
    }
    for (int e = MODE == kModeNarrow ? -1 : 0; e < npairs; ++e) {
      if (MODE == kModeNarrow && e < 0) {
        if (npairs > 0) {
          const Narrow nb(a.ltab + (size_t)s.plist[0].x * tstride, qt2, a.M, s);
          nb.stats(s);
          nb.prime();
        }
        continue;
      }
      const int4 pe = s.plist[e];
      const int l = pe.x, n_l = pe.y, b = pe.z;
      const float d2 = __int_as_float(pe.w);
      const int64_t tile0 = a.tile_off[l], vec0 = a.vec_off[l];  // requested before the table build
      if constexpr (MODE == kModeNarrow) {
        __syncthreads();  // every row's statistics of this pair are in; the previous scan is over
        Narrow(a.ltab + (size_t)l * tstride, qt2, a.M, s).levels(a.M, a.Mp, b, d2, s);
        if (e + 1 < npairs) Narrow(a.ltab + (size_t)s.plist[e + 1].x * tstride, qt2, a.M, s).prime();
        __syncthreads();
      } else if constexpr (NCHUNK <= 2) {
        build_lut_regs<NCHUNK * 16 / kWarps>(a.ltab + (size_t)l * tstride, qt2, a.M, b, d2,
                                             s.T, s.q, s.bias, s.rowmax, s.sc);
        __syncthreads();
      } else {
        build_lut(a.ltab + (size_t)l * tstride, qt2, a.M, a.Mp, b, d2, s);
      }
      const PairScal sc = *s.sc;
      const int ntile = (n_l + kTileVecs - 1) / kTileVecs;
      const uint8_t* tp = a.codes + ((size_t)tile0 * NCHUNK + 0) * kTileChunkBytes +
                          (size_t)warp * NCHUNK * kTileChunkBytes;
      const int64_t* idp = a.ids + vec0;
      for (int t = warp; t < ntile; t += kWarps, tp += (size_t)kWarps * NCHUNK * kTileChunkBytes) {
        uint4 w[NCHUNK];
        load_tile<NCHUNK>(tp, lane, w);
        const float d = pair_distance<NCHUNK>(b, d2, s.T_addr, s.q_addr, sc, w);
        const int v = t * kTileVecs + lane;
        const float lim = R > 1 ? *(volatile float*)blim : INFINITY;
        const bool pre = v < n_l && d <= thd && d <= bnd && d <= lim;
        if (__any_sync(kFull, pre)) {
          const IdT id = pre ? (IdT)__ldg(idp + v) : IdMax<IdT>::v();
          const float before = thd;
          top.offer(pre, d, id, kq, thd, thi);
          if (R > 1 && lane == 0 && thd < before && thd < lim) {
            // lower the shared limit (a retry lost to the cap only prunes less)
            int* w = (int*)blim;
            int old = *(volatile int*)w;
            for (int it = 0; it < 64 && thd < __int_as_float(old); ++it) {
              const int seen = atomicCAS(w, old, __float_as_int(thd));
              if (seen == old) break;
              old = seen;
            }
          }
        }
      }
      if constexpr (MODE == kModeNarrow) {
        if (e + 1 < npairs) {
          const Narrow nb(a.ltab + (size_t)s.plist[e + 1].x * tstride, qt2, a.M, s);
          nb.stats(s);  // writes only row statistics, which no scan reads
          nb.prime();
        }
      } else {
        __syncthreads();  // the next pair overwrites the LUT
      }
    }
    merge_and_write<R, IdT>(a, s, top, q, kq, thd, thi);
  }
}

// FP32-rule coarse distance of one (query, list) pair, computed by one thread
// (same operation order as the CL kernel).
__device__ float pair_d2(const float* qv, const float* cv, int dim) {
  float acc = 0.f;
  for (int d = 0; d < dim; ++d) {
    const float e = sub_rn(qv[d], cv[d]);
    acc = add_rn(acc, mul_rn(e, e));
  }
  return acc;
}

__device__ float block_pair_d2(const SearchArgs& a, int q, int l, Smem& s) {
  if (threadIdx.x == 0) *s.d2 = pair_d2(a.Q + (size_t)q * a.dim, a.centroids + (size_t)l * a.dim, (int)a.dim);
  __syncthreads();
  return *s.d2;
}

// One block per pair: LUT build + quantisation, written out (anns_compute_luts).
__global__ void __launch_bounds__(kThreads) luts_kernel(const SearchArgs a, const int32_t* pq,
                                                        const int32_t* pl, const uint8_t* pb,
                                                        int64_t npairs, float* T_out,
                                                        uint16_t* t_out, double* scale_out) {
  Smem s(a.lay);
  const int64_t tstride = (int64_t)a.Mp * kKsub;
  for (int64_t p = blockIdx.x; p < npairs; p += gridDim.x) {
    const int q = pq[p], l = pl[p], b = pb[p] <= 16 ? pb[p] : 0;
    if (q < 0 || q >= a.nq || l < 0 || l >= a.nlist) continue;  // out-of-range pair: skipped
    const float d2 = block_pair_d2(a, q, l, s);
    build_lut(a.ltab + (size_t)l * tstride, a.qt + (size_t)q * tstride, a.M, a.Mp, b, d2, s);
    const int nent = a.M * kKsub;
    for (int e = threadIdx.x; e < nent; e += blockDim.x) {
      if (T_out) T_out[p * nent + e] = s.T[e];
      if (t_out) t_out[p * nent + e] = b == 0 ? 0 : b <= 8 ? ((const uint8_t*)s.q)[e] : ((const uint16_t*)s.q)[e];
    }
    if (scale_out && threadIdx.x == 0) {
      scale_out[p * 4 + 0] = b ? s.sc->delta64 : 0.0;
      scale_out[p * 4 + 1] = b ? (double)s.sc->B32 : (double)d2;
      scale_out[p * 4 + 2] = b ? (double)s.sc->range : 0.0;
      scale_out[p * 4 + 3] = b ? (double)s.sc->s32 : 0.0;
    }
    __syncthreads();
  }
}

// One block per pair: every distance of the list (anns_scan_pairs).
template <int NCHUNK>
__global__ void __launch_bounds__(kThreads) scan_pairs_kernel(const SearchArgs a, const int32_t* pq,
                                                              const int32_t* pl, const uint8_t* pb,
                                                              int64_t npairs, const int64_t* off,
                                                              float* dist_out, int32_t* S_out) {
  Smem s(a.lay);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t tstride = (int64_t)a.Mp * kKsub;
  for (int64_t p = blockIdx.x; p < npairs; p += gridDim.x) {
    const int q = pq[p], l = pl[p], b = pb[p] <= 16 ? pb[p] : 0;
    if (q < 0 || q >= a.nq || l < 0 || l >= a.nlist) continue;  // out-of-range pair: skipped
    const float d2 = block_pair_d2(a, q, l, s);
    build_lut(a.ltab + (size_t)l * tstride, a.qt + (size_t)q * tstride, a.M, a.Mp, b, d2, s);
    const int n_l = a.list_len[l];
    const int ntile = (n_l + kTileVecs - 1) / kTileVecs;
    const uint8_t* base = a.codes + (size_t)a.tile_off[l] * NCHUNK * kTileChunkBytes;
    const PairScal sc = *s.sc;
    for (int t = warp; t < ntile; t += kWarps) {
      uint4 w[NCHUNK];
      load_tile<NCHUNK>(base + (size_t)t * NCHUNK * kTileChunkBytes, lane, w);
      const int v = t * kTileVecs + lane;
      int S = 0;
      const float d = pair_distance<NCHUNK>(b, d2, s.T_addr, s.q_addr, sc, w, &S);
      if (v < n_l) {
        dist_out[off[p] + v] = d;
        if (S_out) S_out[off[p] + v] = S;
      }
    }
    __syncthreads();
  }
}

SearchArgs make_args(const Index& ix, const float* Q, const float* qt, int R, int mode = kModeFull) {
  SearchArgs a{};
  a.Q = Q; a.qt = qt; a.dim = ix.dim; a.nlist = ix.nlist;
  a.centroids = ix.centroids; a.ltab = ix.ltab; a.codes = ix.codes; a.ids = ix.ids;
  a.list_len = ix.list_len; a.vec_off = ix.vec_off; a.tile_off = ix.tile_off;
  a.M = (int)ix.M; a.Mp = (int)ix.Mp;
  a.lay = SmemLayout(ix.Mp, R, mode);
  return a;
}

template <typename K>
cudaError_t prep(K kernel, size_t smem) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem > (size_t)optin) return cudaErrorInvalidValue;  // index too wide for one block
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename K>
cudaError_t launch_query_major(K kern, const SearchArgs& a, cudaStream_t s) {
  cudaError_t e = prep(kern, a.lay.total);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)std::min<int64_t>(a.nq, 1 << 30);
  kern<<<grid, kThreads, a.lay.total, s>>>(a); note_launch();
  return cudaGetLastError();
}

template <int NCHUNK, int R, typename IdT>
cudaError_t run_search_id(const SearchArgs& a, int mode, cudaStream_t s) {
  switch (mode) {
    case kModeFp32: return launch_query_major(search_kernel<NCHUNK, R, kModeFp32, IdT>, a, s);
    case kModeNarrow: return launch_query_major(search_kernel<NCHUNK, R, kModeNarrow, IdT>, a, s);
    default: return launch_query_major(search_kernel<NCHUNK, R, kModeFull, IdT>, a, s);
  }
}

template <int NCHUNK, int R>
cudaError_t run_search(const SearchArgs& a, int mode, cudaStream_t s) {
  if constexpr (R > 1) {
    if (a.ids32) return run_search_id<NCHUNK, R, int32_t>(a, mode, s);
  }
  return run_search_id<NCHUNK, R, int64_t>(a, mode, s);
}

template <int NCHUNK>
cudaError_t run_search_r(const SearchArgs& a, int R, int mode, cudaStream_t s) {
  return R == 1 ? run_search<NCHUNK, 1>(a, mode, s) : run_search<NCHUNK, 4>(a, mode, s);
}

template <int NCHUNK>
cudaError_t run_scan_pairs(const SearchArgs& a, const int32_t* pq, const int32_t* pl, const uint8_t* pb,
                           int64_t npairs, const int64_t* off, float* dist_out, int32_t* S_out,
                           cudaStream_t s) {
  auto kern = scan_pairs_kernel<NCHUNK>;
  cudaError_t e = prep(kern, a.lay.total);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)std::min<int64_t>(npairs, 1 << 30);
  kern<<<grid, kThreads, a.lay.total, s>>>(a, pq, pl, pb, npairs, off, dist_out, S_out); note_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_search(const Index& ix, const float* qt, int64_t nq, int nprobe,
                          const int32_t* nprobe_per_q, int k, const int32_t* k_per_q,
                          const int32_t* probes, const float* probe_d2, const uint8_t* bits,
                          const int32_t* order, int64_t* ids_out, float* dists_out, cudaStream_t s,
                          int skip_narrow, int tables, const float* part_d, const int64_t* part_i) {
  const int R = k <= 32 ? 1 : 4;
  const int mode = tables == QM_TABLES_FP32 ? kModeFp32 : tables == QM_TABLES_NARROW ? kModeNarrow : kModeFull;
  SearchArgs a = make_args(ix, nullptr, qt, R, mode);
  a.nq = nq; a.nprobe = nprobe; a.k = k; a.npq = nprobe_per_q; a.kpq = k_per_q;
  a.probes = probes; a.probe_d2 = probe_d2; a.bits = bits; a.order = order; a.skip_narrow = skip_narrow;
  a.ids32 = ix.ids32 ? 1 : 0;
  a.ids_out = ids_out; a.dists_out = dists_out;
  a.part_d = mode == kModeNarrow ? part_d : nullptr;
  a.part_i = mode == kModeNarrow ? part_i : nullptr;
  switch (ix.nchunk) {
    case 1: return run_search_r<1>(a, R, mode, s);
    case 2: return run_search_r<2>(a, R, mode, s);
    case 3: return run_search_r<3>(a, R, mode, s);
    case 4: return run_search_r<4>(a, R, mode, s);
    case 5: return run_search_r<5>(a, R, mode, s);
    case 6: return run_search_r<6>(a, R, mode, s);
    case 7: return run_search_r<7>(a, R, mode, s);
    default: return run_search_r<8>(a, R, mode, s);
  }
}

cudaError_t launch_compute_luts(const Index& ix, const float* Q, const float* qt, int64_t nq,
                                const int32_t* pq, const int32_t* pl, const uint8_t* pb,
                                int64_t npairs, float* T_out, uint16_t* t_out, double* scale_out,
                                cudaStream_t s) {
  SearchArgs a = make_args(ix, Q, qt, 1);
  a.nq = nq;
  cudaError_t e = prep(luts_kernel, a.lay.total);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)std::min<int64_t>(npairs, 1 << 30);
  luts_kernel<<<grid, kThreads, a.lay.total, s>>>(a, pq, pl, pb, npairs, T_out, t_out, scale_out); note_launch();
  return cudaGetLastError();
}

cudaError_t launch_scan_pairs(const Index& ix, const float* Q, const float* qt, int64_t nq,
                              const int32_t* pq, const int32_t* pl, const uint8_t* pb,
                              int64_t npairs, const int64_t* off, float* dist_out, int32_t* S_out,
                              cudaStream_t s) {
  SearchArgs a = make_args(ix, Q, qt, 1);
  a.nq = nq;
  switch (ix.nchunk) {
    case 1: return run_scan_pairs<1>(a, pq, pl, pb, npairs, off, dist_out, S_out, s);
    case 2: return run_scan_pairs<2>(a, pq, pl, pb, npairs, off, dist_out, S_out, s);
    case 3: return run_scan_pairs<3>(a, pq, pl, pb, npairs, off, dist_out, S_out, s);
    case 4: return run_scan_pairs<4>(a, pq, pl, pb, npairs, off, dist_out, S_out, s);
    case 5: return run_scan_pairs<5>(a, pq, pl, pb, npairs, off, dist_out, S_out, s);
    case 6: return run_scan_pairs<6>(a, pq, pl, pb, npairs, off, dist_out, S_out, s);
    case 7: return run_scan_pairs<7>(a, pq, pl, pb, npairs, off, dist_out, S_out, s);
    default: return run_scan_pairs<8>(a, pq, pl, pb, npairs, off, dist_out, S_out, s);
  }
}

}  // namespace anns
