// Persistent search kernel for indexes whose codebook fits in registers
// (M * 256 * dsub <= 16 warps * 32 lanes * 64 floats, i.e. dim <= 128).
//
// Same arithmetic as search.cu (RC, LC, quantiser, ADC, top-k of Section 2.1,
// FP32 rule with explicit rounding), organised for the SM:
//  - one 512-thread block per SM walks the queries (atomic counter);
//  - warp w owns codebook rows m = w, w+16, ...; lane i owns entries
//    c = i + 32e (e < 8) of those rows, and keeps y_{m,c} in registers for the
//    whole kernel, so building a LUT is pure FP32 ALU work: no codebook
//    traffic from L2 or shared memory;
//  - the pairs (probed lists) of a query run as a two-slot pipeline: while
//    the warps scan pair j from one shared-memory table, they build the table
//    of pair j+1 into the other. Row minima/maxima go through shared memory,
//    then each warp quantises its own rows, still held in registers.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace anns {
namespace {

constexpr int kNW = 16;                 // warps per block
constexpr int kThreadsP = kNW * 32;

struct PairScalP {
  float delta32, B32;
};

struct PairInfo {
  int l, n_l, b, ntile;
  int64_t tile0, vbase;
};

struct PArgs {
  const float* Q; int64_t nq, dim;
  const float* centroids; const float* codebooks;
  const uint8_t* codes; const int64_t* ids;
  const int32_t* list_len; const int64_t* vec_off; const int64_t* tile_off;
  int M, dsub, nprobe, k;
  const int32_t* npq; const int32_t* kpq;
  const int32_t* probes; const uint8_t* bits;
  int64_t* ids_out; float* dists_out;
  int* counter;
  size_t off_r, off_rowmin, off_rowmax, off_scal, off_info, off_md, off_mi, total;
};

constexpr int kTabSlots = 3, kInfoSlots = 4;

template <int NCHUNK>
__host__ __device__ constexpr size_t table_bytes() { return (size_t)NCHUNK * 16 * kKsub * 4; }

template <int NCHUNK, int R>
size_t layout(PArgs& a) {
  auto al = [](size_t x) { return (x + 15) & ~size_t(15); };
  size_t o = kTabSlots * table_bytes<NCHUNK>();   // table slots at offset 0
  a.off_r = o; o += al(2 * a.dim * 4);
  a.off_rowmin = o; o += al(2 * NCHUNK * 16 * 4);
  a.off_rowmax = o; o += al(2 * NCHUNK * 16 * 4);
  a.off_scal = o; o += al(2 * sizeof(PairScalP));
  a.off_info = o; o += al(kInfoSlots * sizeof(PairInfo));
  a.off_md = o; o += al((size_t)kNW * R * 32 * 4);
  a.off_mi = o; o += al((size_t)kNW * R * 32 * 8);
  a.total = o;
  return o;
}

__device__ __forceinline__ unsigned word_of(const uint4& v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// One block's state. Pair p (probe rank p of the current query) moves through
// the stages  load/store inputs (stage p-3) -> build rows (p-2) -> quantise
// (p-1) -> scan (p), one block barrier per stage, so three pairs are in
// flight. Slots: tables p%3, residuals / row statistics / scales p%2, list
// facts p%4 — each is rewritten only after the barrier that ends its last use.
template <int NCHUNK, int R, int NROW, int DSUB>
struct Pipe {
  static constexpr int Mp = NCHUNK * 16;
  const PArgs& a;
  unsigned char* sm;
  float2 y[NROW][4][DSUB];  // this thread's codebook entries, (c, c+32) paired
  float2 tq[NROW][4];       // LUT values of the pair between build and quantise
  uint4 pf[NCHUNK];         // prefetched code tile
  int warp, lane;

  __device__ Pipe(const PArgs& args, unsigned char* s) : a(args), sm(s) {
    warp = threadIdx.x >> 5;
    lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < NROW; ++i) {
      const int m = warp + kNW * i;
#pragma unroll
      for (int h = 0; h < 4; ++h)
#pragma unroll
        for (int j = 0; j < DSUB; ++j) {
          const size_t e0 = (size_t)(m * kKsub + lane + 64 * h), e1 = e0 + 32;
          y[i][h][j] = m < a.M ? make_float2(__ldg(a.codebooks + e0 * DSUB + j), __ldg(a.codebooks + e1 * DSUB + j))
                               : make_float2(0.f, 0.f);
        }
    }
  }

  __device__ unsigned char* table(int p) const { return sm + (p % kTabSlots) * table_bytes<NCHUNK>(); }
  __device__ float* resid(int p) const { return (float*)(sm + a.off_r) + (p & 1) * a.dim; }
  __device__ float* rowmin(int p) const { return (float*)(sm + a.off_rowmin) + (p & 1) * Mp; }
  __device__ float* rowmax(int p) const { return (float*)(sm + a.off_rowmax) + (p & 1) * Mp; }
  __device__ PairScalP* scal(int p) const { return (PairScalP*)(sm + a.off_scal) + (p & 1); }
  __device__ PairInfo* info(int p) const { return (PairInfo*)(sm + a.off_info) + (p % kInfoSlots); }

  // Inputs of pair p: q - c_l into resid(p), list facts into info(p). The
  // loads are issued first (load_inputs) and stored after the stage's other
  // work (store_inputs), so their latency overlaps that work.
  struct Staged { float qd, cd; int l, n_l, b; int64_t tile0, vbase; };
  __device__ void load_inputs(int64_t q, int p, Staged& st) const {
    st.l = a.probes[q * a.nprobe + p];
    const int d = threadIdx.x;
    st.qd = 0.f; st.cd = 0.f;
    if (st.l >= 0 && d < a.dim) {
      st.qd = a.Q[q * a.dim + d];
      st.cd = a.centroids[(size_t)st.l * a.dim + d];
    }
    if (threadIdx.x == 0) {
      st.n_l = st.l >= 0 ? a.list_len[st.l] : 0;
      st.b = a.bits[q * a.nprobe + p];
      st.tile0 = st.l >= 0 ? a.tile_off[st.l] : 0;
      st.vbase = st.l >= 0 ? a.vec_off[st.l] : 0;
    }
  }
  __device__ void store_inputs(int p, const Staged& st) const {
    if (threadIdx.x < a.dim && st.l >= 0) resid(p)[threadIdx.x] = sub_rn(st.qd, st.cd);
    if (threadIdx.x == 0) {
      PairInfo pi;
      pi.l = st.l; pi.n_l = st.n_l; pi.b = st.b;
      pi.ntile = (st.n_l + kTileVecs - 1) / kTileVecs;
      pi.tile0 = st.tile0; pi.vbase = st.vbase;
      *info(p) = pi;
    }
  }

  // T for this warp's rows of pair p (FP32 rule, two entries per packed
  // operation). Plain pairs write the FP32 table now; quantised pairs keep T
  // in registers and publish row min/range. Rows M..Mp-1 are zero rows, so the
  // scan needs no bound on m.
  __device__ void build_rows(int p) {
    const PairInfo pi = *info(p);
    if (pi.n_l == 0) return;
    const float* r = resid(p);
#pragma unroll
    for (int i = 0; i < NROW; ++i) {
      const int m = warp + kNW * i;
      if (m >= Mp) continue;
      if (m >= a.M) {   // padding row
        if (pi.b == 0) {
          float* T = (float*)table(p);
#pragma unroll
          for (int e = 0; e < 8; ++e) T[m * kKsub + lane + 32 * e] = 0.f;
        }
        continue;
      }
      float2 rv[DSUB];
#pragma unroll
      for (int j = 0; j < DSUB; ++j) { const float v = r[m * DSUB + j]; rv[j] = make_float2(v, v); }
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < DSUB; ++j) {
          const float x0 = sub_rn(rv[j].x, y[i][h][j].x), x1 = sub_rn(rv[j].y, y[i][h][j].y);
          acc.x = add_rn(acc.x, mul_rn(x0, x0));
          acc.y = add_rn(acc.y, mul_rn(x1, x1));
        }
        tq[i][h] = acc;
      }
      if (pi.b == 0) {
        float* T = (float*)table(p);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          T[m * kKsub + lane + 64 * h] = tq[i][h].x;
          T[m * kKsub + lane + 64 * h + 32] = tq[i][h].y;
        }
      } else {
        float mn = fminf(tq[i][0].x, tq[i][0].y);
#pragma unroll
        for (int h = 1; h < 4; ++h) mn = fminf(mn, fminf(tq[i][h].x, tq[i][h].y));
        mn = warp_min(mn);
        float mx = 0.f;
#pragma unroll
        for (int h = 0; h < 4; ++h) mx = fmaxf(mx, fmaxf(sub_rn(tq[i][h].x, mn), sub_rn(tq[i][h].y, mn)));
        mx = warp_max(mx);
        if (lane == 0) { rowmin(p)[m] = mn; rowmax(p)[m] = mx; }
      }
    }
  }

  // Quantises this warp's rows of pair p with the shared step from the
  // largest row range; warp 0 also forms Delta32 and B32 (B summed in FP64 in
  // the fixed 32-lane tree order).
  __device__ void quantise_rows(int p) {
    const PairInfo pi = *info(p);
    if (pi.n_l == 0 || pi.b == 0) return;
    float range = 0.f;
    for (int m = lane; m < a.M; m += 32) range = fmaxf(range, rowmax(p)[m]);
    range = warp_max(range);
    const int L = (1 << pi.b) - 1;
    const float s32 = range > 0.f ? __fdiv_rn((float)L, range) : 0.f;
    if (warp == 0) {
      double B = 0.0;
      for (int m = lane; m < a.M; m += 32) B = __dadd_rn(B, (double)rowmin(p)[m]);
#pragma unroll
      for (int o = 16; o; o >>= 1) B = __dadd_rn(B, __shfl_xor_sync(kFull, B, o));
      if (lane == 0) {
        PairScalP sc;
        sc.delta32 = range > 0.f ? __fdiv_rn(range, (float)L) : 0.f;
        sc.B32 = __double2float_rn(B);
        *scal(p) = sc;
      }
    }
#pragma unroll
    for (int i = 0; i < NROW; ++i) {
      const int m = warp + kNW * i;
      if (m >= Mp) continue;
      int t[8];
      if (m < a.M) {
        const float mn = rowmin(p)[m];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const float2 yq = make_float2(mul_rn(sub_rn(tq[i][h].x, mn), s32), mul_rn(sub_rn(tq[i][h].y, mn), s32));
          t[2 * h] = min(__float2int_rn(yq.x), L);
          t[2 * h + 1] = min(__float2int_rn(yq.y), L);
        }
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) t[e] = 0;   // padding row
      }
      if (pi.b <= 8) {
        uint8_t* t8 = table(p);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          t8[m * kKsub + lane + 64 * h] = (uint8_t)t[2 * h];
          t8[m * kKsub + lane + 64 * h + 32] = (uint8_t)t[2 * h + 1];
        }
      } else {
        uint16_t* t16 = (uint16_t*)table(p);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          t16[m * kKsub + lane + 64 * h] = (uint16_t)t[2 * h];
          t16[m * kKsub + lane + 64 * h + 32] = (uint16_t)t[2 * h + 1];
        }
      }
    }
  }

  __device__ __forceinline__ void load_tile(const PairInfo& pi, int t, uint4 (&w)[NCHUNK]) const {
    const uint8_t* tile = a.codes + ((size_t)(pi.tile0 + t) * NCHUNK) * kTileChunkBytes + lane * kChunkBytes;
#pragma unroll
    for (int c = 0; c < NCHUNK; ++c) w[c] = __ldg(reinterpret_cast<const uint4*>(tile + c * kTileChunkBytes));
  }

  // Issues the load of this warp's first tile of pair p into pf.
  __device__ void prefetch_first(int p) {
    const PairInfo pi = *info(p);
    if (warp < pi.ntile) load_tile(pi, warp, pf);
  }

  // Integer ADC over all Mp sub-tables (padding rows are zero): exact sum.
  template <typename LT>
  __device__ __forceinline__ int adc_int(unsigned base, const uint4 (&w)[NCHUNK]) const {
    int acc0 = 0, acc1 = 0;
#pragma unroll
    for (int c = 0; c < NCHUNK; ++c)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const unsigned x = word_of(w[c], i);
        const int m = c * 16 + i * 4;
        acc0 += (int)lut_at<LT, 0>(sm, base, x, m) + (int)lut_at<LT, 1>(sm, base, x, m + 1);
        acc1 += (int)lut_at<LT, 2>(sm, base, x, m + 2) + (int)lut_at<LT, 3>(sm, base, x, m + 3);
      }
    return acc0 + acc1;
  }

  // FP32 ADC: acc = fl32(acc + T[m][code_m]) for m ascending (padding rows add 0).
  __device__ __forceinline__ float adc_f32(unsigned base, const uint4 (&w)[NCHUNK]) const {
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < NCHUNK; ++c)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const unsigned x = word_of(w[c], i);
        const int m = c * 16 + i * 4;
        acc = add_rn(acc, lut_at<float, 0>(sm, base, x, m));
        acc = add_rn(acc, lut_at<float, 1>(sm, base, x, m + 1));
        acc = add_rn(acc, lut_at<float, 2>(sm, base, x, m + 2));
        acc = add_rn(acc, lut_at<float, 3>(sm, base, x, m + 3));
      }
    return acc;
  }

  // Scans this warp's tiles of pair p (the first one is already in pf) and
  // leaves the first tile of pair p+1 (if has_next) prefetched in pf.
  __device__ void scan(int p, bool has_next, int kq, WarpTopK<R, int64_t>& top, float& thd,
                       int64_t& thi) {
    const PairInfo pi = *info(p);
    const unsigned slot_bytes = (unsigned)((p % kTabSlots) * table_bytes<NCHUNK>());
    PairScalP sc{};
    if (pi.b) sc = *scal(p);
    if (warp >= pi.ntile) {
      if (has_next) prefetch_first(p + 1);
      return;
    }
    for (int t = warp; t < pi.ntile; t += kNW) {
      uint4 w[NCHUNK];
#pragma unroll
      for (int c = 0; c < NCHUNK; ++c) w[c] = pf[c];
      if (t + kNW < pi.ntile) load_tile(pi, t + kNW, pf);
      else if (has_next) prefetch_first(p + 1);
      float d;
      if (pi.b == 0) d = adc_f32(slot_bytes / 4, w);
      else if (pi.b <= 8) d = add_rn(mul_rn(sc.delta32, __int2float_rn(adc_int<uint8_t>(slot_bytes, w))), sc.B32);
      else d = add_rn(mul_rn(sc.delta32, __int2float_rn(adc_int<uint16_t>(slot_bytes / 2, w))), sc.B32);
      const int v = t * kTileVecs + lane;
      const bool pre = v < pi.n_l && d <= thd;
      const int64_t id = pre ? __ldg(a.ids + pi.vbase + v) : INT64_MAX;
      top.offer(pre, d, id, kq, thd, thi);
    }
  }
};

template <int NCHUNK, int R, int NROW, int DSUB>
__global__ void __launch_bounds__(kThreadsP, 1) search_persistent_kernel(const PArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int64_t next_q;
  using PipeT = Pipe<NCHUNK, R, NROW, DSUB>;
  PipeT P(a, smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* md = (float*)(smem + a.off_md);
  int64_t* mi = (int64_t*)(smem + a.off_mi);
  for (;;) {
    if (threadIdx.x == 0) next_q = atomicAdd(a.counter, 1);
    __syncthreads();
    const int64_t q = next_q;
    if (q >= a.nq) break;
    const int np = a.npq ? min(max(a.npq[q], 0), a.nprobe) : a.nprobe;
    const int kq = a.kpq ? min(max(a.kpq[q], 0), a.k) : a.k;
    WarpTopK<R, int64_t> top;
    top.init();
    float thd = INFINITY;
    int64_t thi = INT64_MAX;
    if (kq > 0) {
      for (int s = -3; s < np; ++s) {
        typename PipeT::Staged st;
        const bool stage_in = s + 3 < np;
        if (stage_in) P.load_inputs(q, s + 3, st);
        if (s >= 0) P.scan(s, s + 1 < np, kq, top, thd, thi);
        else if (s == -1) P.prefetch_first(0);
        if (s + 1 >= 0 && s + 1 < np) P.quantise_rows(s + 1);
        if (s + 2 >= 0 && s + 2 < np) P.build_rows(s + 2);
        if (stage_in) P.store_inputs(s + 3, st);
        __syncthreads();
      }
    }
    // merge the per-warp lists into warp 0 and write the query's results
#pragma unroll
    for (int r = 0; r < R; ++r) {
      md[(warp * R + r) * 32 + lane] = top.d[r];
      mi[(warp * R + r) * 32 + lane] = top.id[r];
    }
    __syncthreads();
    if (warp == 0) {
      for (int w2 = 1; w2 < kNW && kq > 0; ++w2)
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const float cd = md[(w2 * R + r) * 32 + lane];
          const int64_t ci = mi[(w2 * R + r) * 32 + lane];
          top.offer(cd != INFINITY, cd, ci, kq, thd, thi);
        }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int e = r * 32 + lane;
        if (e < a.k) {
          const bool ok = e < kq && top.d[r] != INFINITY;
          a.ids_out[q * a.k + e] = ok ? top.id[r] : -1;
          a.dists_out[q * a.k + e] = ok ? top.d[r] : INFINITY;
        }
      }
    }
    __syncthreads();
  }
}

template <int NCHUNK, int R, int NROW, int DSUB>
cudaError_t run(PArgs& a, cudaStream_t s) {
  const size_t smem = layout<NCHUNK, R>(a);
  auto kern = search_persistent_kernel<NCHUNK, R, NROW, DSUB>;
  int dev = 0, sms = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem > (size_t)optin) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(a.counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::min<int64_t>(sms, a.nq);
  kern<<<grid, kThreadsP, smem, s>>>(a);
  return cudaGetLastError();
}

template <int NCHUNK, int R>
cudaError_t run_shape(PArgs& a, cudaStream_t s) {
  // (rows per warp, dsub) combinations whose codebook share fits 64 registers
  const int nrow = (a.M + kNW - 1) / kNW;
  if (nrow == 1 && a.dsub == 8) return run<NCHUNK, R, 1, 8>(a, s);
  if (nrow == 1 && a.dsub == 4) return run<NCHUNK, R, 1, 4>(a, s);
  if (nrow == 2 && a.dsub == 4) return run<NCHUNK, R, 2, 4>(a, s);
  if (nrow == 2 && a.dsub == 2) return run<NCHUNK, R, 2, 2>(a, s);
  if (nrow == 3 && a.dsub == 2) return run<NCHUNK, R, 3, 2>(a, s);
  if (nrow <= 4 && a.dsub == 1) return run<NCHUNK, R, 4, 1>(a, s);
  return cudaErrorNotSupported;
}

}  // namespace

bool persistent_supported(const Index& ix) {
  if (ix.dim > kThreadsP) return false;
  const int nrow = (int)((ix.M + kNW - 1) / kNW);
  const int d = (int)ix.dsub;
  return (nrow == 1 && (d == 8 || d == 4)) || (nrow == 2 && (d == 4 || d == 2)) ||
         (nrow == 3 && d == 2) || (nrow <= 4 && d == 1);
}

cudaError_t launch_search_persistent(const Index& ix, const float* Q, int64_t nq, int nprobe,
                                     const int32_t* nprobe_per_q, int k, const int32_t* k_per_q,
                                     const int32_t* probes, const uint8_t* bits, int64_t* ids_out,
                                     float* dists_out, int* counter, cudaStream_t s) {
  PArgs a{};
  a.Q = Q; a.nq = nq; a.dim = ix.dim;
  a.centroids = ix.centroids; a.codebooks = ix.codebooks; a.codes = ix.codes; a.ids = ix.ids;
  a.list_len = ix.list_len; a.vec_off = ix.vec_off; a.tile_off = ix.tile_off;
  a.M = (int)ix.M; a.dsub = (int)ix.dsub; a.nprobe = nprobe; a.k = k;
  a.npq = nprobe_per_q; a.kpq = k_per_q; a.probes = probes; a.bits = bits;
  a.ids_out = ids_out; a.dists_out = dists_out; a.counter = counter;
  const bool r1 = k <= 32;
  switch (ix.nchunk) {
    case 1: return r1 ? run_shape<1, 1>(a, s) : run_shape<1, 4>(a, s);
    case 2: return r1 ? run_shape<2, 1>(a, s) : run_shape<2, 4>(a, s);
    case 3: return r1 ? run_shape<3, 1>(a, s) : run_shape<3, 4>(a, s);
    case 4: return r1 ? run_shape<4, 1>(a, s) : run_shape<4, 4>(a, s);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace anns
