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
  double delta64, B64;
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

template <int NCHUNK>
__host__ __device__ constexpr size_t table_bytes() { return (size_t)NCHUNK * 16 * kKsub * 4; }

template <int NCHUNK, int R>
size_t layout(PArgs& a) {
  auto al = [](size_t x) { return (x + 15) & ~size_t(15); };
  size_t o = 2 * table_bytes<NCHUNK>();   // two table slots at offset 0
  a.off_r = o; o += al(2 * a.dim * 4);
  a.off_rowmin = o; o += al(2 * NCHUNK * 16 * 4);
  a.off_rowmax = o; o += al(2 * NCHUNK * 16 * 4);
  a.off_scal = o; o += al(2 * sizeof(PairScalP));
  a.off_info = o; o += al(2 * sizeof(PairInfo));
  a.off_md = o; o += al((size_t)kNW * R * 32 * 4);
  a.off_mi = o; o += al((size_t)kNW * R * 32 * 8);
  a.total = o;
  return o;
}

__device__ __forceinline__ unsigned word_of(const uint4& v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// Steps of one pipeline stage, parameterised at compile time by the code
// width (NCHUNK 16-byte chunks), the top-k capacity R*32, the codebook rows
// per warp NROW and the sub-vector length DSUB.
template <int NCHUNK, int R, int NROW, int DSUB>
struct Pipe {
  static constexpr int Mp = NCHUNK * 16;
  const PArgs& a;
  unsigned char* sm;
  float y[NROW][8][DSUB];   // this thread's codebook entries
  float tq[NROW][8];        // LUT values of the pair being built
  int warp, lane;

  __device__ Pipe(const PArgs& args, unsigned char* s) : a(args), sm(s) {
    warp = threadIdx.x >> 5;
    lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < NROW; ++i) {
      const int m = warp + kNW * i;
#pragma unroll
      for (int e = 0; e < 8; ++e)
#pragma unroll
        for (int j = 0; j < DSUB; ++j)
          y[i][e][j] = m < a.M ? __ldg(a.codebooks + ((size_t)(m * kKsub + lane + 32 * e)) * DSUB + j) : 0.f;
    }
  }

  __device__ unsigned char* table(int slot) const { return sm + slot * table_bytes<NCHUNK>(); }
  __device__ float* resid(int slot) const { return (float*)(sm + a.off_r) + slot * a.dim; }
  __device__ float* rowmin(int slot) const { return (float*)(sm + a.off_rowmin) + slot * Mp; }
  __device__ float* rowmax(int slot) const { return (float*)(sm + a.off_rowmax) + slot * Mp; }
  __device__ PairScalP* scal(int slot) const { return (PairScalP*)(sm + a.off_scal) + slot; }
  __device__ PairInfo* info(int slot) const { return (PairInfo*)(sm + a.off_info) + slot; }

  // Residual r = fl32(q - c_l) and list facts of probe rank j into `slot`.
  __device__ void stage_pair(int64_t q, int j, int slot) {
    const int l = a.probes[q * a.nprobe + j];
    const float* qv = a.Q + q * a.dim;
    float* r = resid(slot);
    if (l >= 0) {
      const float* cv = a.centroids + (size_t)l * a.dim;
      for (int d = threadIdx.x; d < a.dim; d += kThreadsP) r[d] = sub_rn(qv[d], cv[d]);
    }
    if (threadIdx.x == 0) {
      PairInfo pi;
      pi.l = l;
      pi.n_l = l >= 0 ? a.list_len[l] : 0;
      pi.b = a.bits[q * a.nprobe + j];
      pi.ntile = (pi.n_l + kTileVecs - 1) / kTileVecs;
      pi.tile0 = l >= 0 ? a.tile_off[l] : 0;
      pi.vbase = l >= 0 ? a.vec_off[l] : 0;
      *info(slot) = pi;
    }
  }

  // Build step 1: T for this warp's rows; FP32 tables are written out, for
  // quantised pairs the row minimum and the row range go to shared memory.
  __device__ void build_rows(int slot) {
    const PairInfo pi = *info(slot);
    if (pi.n_l == 0) return;
    const float* r = resid(slot);
#pragma unroll
    for (int i = 0; i < NROW; ++i) {
      const int m = warp + kNW * i;
      if (m >= a.M) continue;
      float rv[DSUB];
#pragma unroll
      for (int j = 0; j < DSUB; ++j) rv[j] = r[m * DSUB + j];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        float acc = 0.f;
#pragma unroll
        for (int j = 0; j < DSUB; ++j) {
          const float x = sub_rn(rv[j], y[i][e][j]);
          acc = add_rn(acc, mul_rn(x, x));
        }
        tq[i][e] = acc;
      }
      if (pi.b == 0) {
        float* T = (float*)table(slot);
#pragma unroll
        for (int e = 0; e < 8; ++e) T[m * kKsub + lane + 32 * e] = tq[i][e];
      } else {
        float mn = tq[i][0];
#pragma unroll
        for (int e = 1; e < 8; ++e) mn = fminf(mn, tq[i][e]);
        mn = warp_min(mn);
        float mx = 0.f;
#pragma unroll
        for (int e = 0; e < 8; ++e) mx = fmaxf(mx, sub_rn(tq[i][e], mn));
        mx = warp_max(mx);
        if (lane == 0) { rowmin(slot)[m] = mn; rowmax(slot)[m] = mx; }
      }
    }
  }

  // Build step 2 (after a barrier): the shared step from the largest row
  // range, then this warp's rows quantised into the table; warp 0 also forms
  // the FP64 offset B = sum of the row minima, m ascending.
  __device__ void quantise_rows(int slot) {
    const PairInfo pi = *info(slot);
    if (pi.n_l == 0 || pi.b == 0) return;
    float range = 0.f;
    for (int m = lane; m < a.M; m += 32) range = fmaxf(range, rowmax(slot)[m]);
    range = warp_max(range);
    const int L = (1 << pi.b) - 1;
    const float s32 = range > 0.f ? __double2float_rn(__ddiv_rn((double)L, (double)range)) : 0.f;
    if (warp == 0 && lane == 0) {
      PairScalP sc;
      sc.delta64 = range > 0.f ? __ddiv_rn((double)range, (double)L) : 0.0;
      double B = 0.0;
      for (int m = 0; m < a.M; ++m) B = __dadd_rn(B, (double)rowmin(slot)[m]);
      sc.B64 = B;
      sc.delta32 = __double2float_rn(sc.delta64);
      sc.B32 = __double2float_rn(B);
      *scal(slot) = sc;
    }
#pragma unroll
    for (int i = 0; i < NROW; ++i) {
      const int m = warp + kNW * i;
      if (m >= a.M) continue;
      const float mn = rowmin(slot)[m];
      if (pi.b <= 8) {
        uint8_t* t8 = table(slot);
#pragma unroll
        for (int e = 0; e < 8; ++e)
          t8[m * kKsub + lane + 32 * e] = (uint8_t)min(__float2int_rn(mul_rn(sub_rn(tq[i][e], mn), s32)), L);
      } else {
        uint16_t* t16 = (uint16_t*)table(slot);
#pragma unroll
        for (int e = 0; e < 8; ++e)
          t16[m * kKsub + lane + 32 * e] = (uint16_t)min(__float2int_rn(mul_rn(sub_rn(tq[i][e], mn), s32)), L);
      }
    }
  }

  template <typename LT>
  __device__ __forceinline__ int adc_int(const LT* __restrict__ t, const uint4 (&w)[NCHUNK]) const {
    int acc = 0;
#pragma unroll
    for (int c = 0; c < NCHUNK; ++c)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const unsigned x = word_of(w[c], i);
#pragma unroll
        for (int bb = 0; bb < 4; ++bb) {
          const int m = c * 16 + i * 4 + bb;
          if (m < a.M) acc += (int)t[m * kKsub + ((x >> (8 * bb)) & 255u)];
        }
      }
    return acc;
  }

  __device__ __forceinline__ float adc_f32(const float* __restrict__ T, const uint4 (&w)[NCHUNK]) const {
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < NCHUNK; ++c)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const unsigned x = word_of(w[c], i);
#pragma unroll
        for (int bb = 0; bb < 4; ++bb) {
          const int m = c * 16 + i * 4 + bb;
          if (m < a.M) acc = add_rn(acc, T[m * kKsub + ((x >> (8 * bb)) & 255u)]);
        }
      }
    return acc;
  }

  // Scans tiles [t0, t1) of the pair in `slot`, offering distances to the warp list.
  __device__ void scan(int slot, int t0, int t1, int kq, WarpTopK<R, int64_t>& top, float& thd,
                       int64_t& thi) const {
    const PairInfo pi = *info(slot);
    if (pi.n_l == 0) return;
    const uint8_t* base = a.codes + (size_t)pi.tile0 * NCHUNK * kTileChunkBytes;
    const unsigned char* tab = table(slot);
    PairScalP sc{};
    if (pi.b) sc = *scal(slot);
    for (int t = t0 + warp; t < t1; t += kNW) {
      uint4 w[NCHUNK];
      const uint8_t* tile = base + (size_t)t * NCHUNK * kTileChunkBytes + lane * kChunkBytes;
#pragma unroll
      for (int c = 0; c < NCHUNK; ++c) w[c] = __ldg(reinterpret_cast<const uint4*>(tile + c * kTileChunkBytes));
      float d;
      if (pi.b == 0) d = adc_f32((const float*)tab, w);
      else if (pi.b <= 8) d = add_rn(mul_rn(sc.delta32, __int2float_rn(adc_int((const uint8_t*)tab, w))), sc.B32);
      else d = add_rn(mul_rn(sc.delta32, __int2float_rn(adc_int((const uint16_t*)tab, w))), sc.B32);
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
  Pipe<NCHUNK, R, NROW, DSUB> P(a, smem);
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
    if (kq > 0 && np > 0) {
      // prologue: pair 0 into slot 0
      P.stage_pair(q, 0, 0);
      __syncthreads();
      P.build_rows(0);
      __syncthreads();
      P.quantise_rows(0);
      if (np > 1) P.stage_pair(q, 1, 1);
      __syncthreads();
      for (int j = 0; j < np; ++j) {
        const int cur = j & 1, nxt = cur ^ 1;
        const bool more = j + 1 < np;
        const int nt = P.info(cur)->ntile;
        const int half = (nt + 1) / 2;
        // stage A: rows of pair j+1, first half of pair j's tiles
        if (more) P.build_rows(nxt);
        P.scan(cur, 0, half, kq, top, thd, thi);
        __syncthreads();
        // stage B: quantise pair j+1, second half of pair j's tiles
        if (more) P.quantise_rows(nxt);
        P.scan(cur, half, nt, kq, top, thd, thi);
        __syncthreads();
        if (j + 2 < np) P.stage_pair(q, j + 2, cur);
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
