// Persistent search kernel for indexes with Mp <= 64 and k <= 32.
//
// Same arithmetic as search.cu (decomposed FP32 LUT T' = P_l - 2 Q_q, the
// quantiser, ADC and top-k of Section 2.1, explicit rounding), organised for
// the SM:
//  - one 1024-thread block per SM walks the queries (atomic counter) and copies
//    each query's table 2 Q_q into shared memory once;
//  - warp w builds LUT rows m = w, w+32, ...; lane i owns entries
//    c = 8i .. 8i+7 of those rows, so list-table loads, query-table loads and
//    table stores are 16-byte vectors; values stay in registers between the
//    build and the table write, which lets the row minima/maxima cross the
//    block first;
//  - the probed lists of a query flow through a pipeline with one block
//    barrier per stage: in stage s the block issues the list-table loads of
//    pair s+2, scans pair s, writes the table of pair s+1, builds pair s+2 and
//    loads the inputs of pair s+3; every warp prefetches its first code tile
//    of the next stage's pair.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "scan.cuh"

namespace anns {
namespace {

constexpr int kNW = 32;                 // warps per block
constexpr int kThreadsP = kNW * 32;
constexpr int kInfoSlots = 4;

struct PairScalP {
  float delta32, B32;
};

struct PairInfo {
  int l, n_l, b, ntile;
  int64_t tile0, vbase;
  float d2;
};

struct PArgs {
  const float* qt; int64_t nq;
  const float* ltab; const float* probe_d2;
  const uint8_t* codes; const int64_t* ids;
  const int32_t* list_len; const int64_t* vec_off; const int64_t* tile_off;
  int M, dsub, nprobe, k;
  const int32_t* npq; const int32_t* kpq;
  const int32_t* probes; const uint8_t* bits;
  int64_t* ids_out; float* dists_out;
  int* counter;
  size_t off_qt, off_rowmin, off_rowmax, off_scal, off_info, off_md, off_mi, off_q, total;
};

template <int NCHUNK>
__host__ __device__ constexpr size_t table_bytes() { return (size_t)NCHUNK * 16 * kKsub * 4; }

template <int NCHUNK>
size_t layout(PArgs& a) {
  auto al = [](size_t x) { return (x + 15) & ~size_t(15); };
  size_t o = 2 * table_bytes<NCHUNK>();   // two table slots at offset 0
  a.off_qt = o; o += al((size_t)NCHUNK * 16 * kKsub * 4);
  a.off_rowmin = o; o += al(2 * NCHUNK * 16 * 4);
  a.off_rowmax = o; o += al(2 * NCHUNK * 16 * 4);
  a.off_scal = o; o += al(2 * sizeof(PairScalP));
  a.off_info = o; o += al(kInfoSlots * sizeof(PairInfo));
  a.off_md = o; o += al((size_t)kNW * 32 * 4);
  a.off_mi = o; o += al((size_t)kNW * 32 * 8);
  a.off_q = o; o += 16;
  a.total = o + 256;   // slack for the 256-byte alignment of the base
  return a.total;
}

// Pair p (probe rank p of the current query) moves through the stages
//   load inputs (stage p-3) -> build (p-2) -> write table (p-1) -> scan (p).
// Slots: tables, row statistics and scales p%2, list facts p%4; each is
// rewritten only after the barrier that ends its last use.
template <int NCHUNK, int NROW>
struct Pipe {
  static constexpr int Mp = NCHUNK * 16;
  const PArgs& a;
  float tq[NROW][8];        // LUT values between build and table write
  float pp[NROW][8];        // list-table values loaded for the next build
  uint4 pf[NCHUNK];         // prefetched code tile
  int warp, lane;

  __device__ explicit Pipe(const PArgs& args) : a(args) {
    warp = threadIdx.x >> 5;
    lane = threadIdx.x & 31;
    const uint32_t raw = smem_addr(anns_dyn_smem);
    const uint32_t pad = (256u - (raw & 255u)) & 255u;
    base = anns_dyn_smem + pad;
    base_addr = raw + pad;
  }

  unsigned char* base;       // 256-byte aligned start of the layout
  uint32_t base_addr;        // its shared-memory byte address

  __device__ unsigned char* sm() const { return base; }
  __device__ unsigned table_off(int p) const { return (unsigned)((p & 1) * table_bytes<NCHUNK>()); }
  __device__ float* qtab() const { return (float*)(sm() + a.off_qt); }
  __device__ float* rowmin(int p) const { return (float*)(sm() + a.off_rowmin) + (p & 1) * Mp; }
  __device__ float* rowmax(int p) const { return (float*)(sm() + a.off_rowmax) + (p & 1) * Mp; }
  __device__ PairScalP* scal(int p) const { return (PairScalP*)(sm() + a.off_scal) + (p & 1); }
  __device__ PairInfo* info(int p) const { return (PairInfo*)(sm() + a.off_info) + (p % kInfoSlots); }

  // Copies the query's table 2 Q_q into shared memory (callers barrier after).
  __device__ void load_query_table(int64_t q) const {
    const float4* src = (const float4*)(a.qt + q * (int64_t)Mp * kKsub);
    float4* dst = (float4*)qtab();
    for (int i = threadIdx.x; i < Mp * kKsub / 4; i += kThreadsP) dst[i] = __ldg(src + i);
  }

  // List facts of pair p (thread 0), stored at the end of the stage.
  struct Staged { int l, n_l, b; int64_t tile0, vbase; float d2; };
  __device__ void load_inputs(int64_t q, int p, Staged& st) const {
    if (threadIdx.x != 0) return;
    const int64_t row = q * a.nprobe + p;
    st.l = a.probes[row];
    st.n_l = 0; st.b = 0; st.tile0 = 0; st.vbase = 0; st.d2 = 0.f;
    if (st.l >= 0) {
      st.n_l = a.list_len[st.l];
      st.b = a.bits[row];
      st.d2 = a.probe_d2[row];
      st.tile0 = a.tile_off[st.l];
      st.vbase = a.vec_off[st.l];
    }
  }
  __device__ void store_inputs(int p, const Staged& st) const {
    if (threadIdx.x != 0) return;
    PairInfo pi;
    pi.l = st.l; pi.n_l = st.n_l; pi.b = st.b; pi.d2 = st.d2;
    pi.ntile = (st.n_l + kTileVecs - 1) / kTileVecs;
    pi.tile0 = st.tile0; pi.vbase = st.vbase;
    *info(p) = pi;
  }

  // Issues this warp's list-table loads for pair p (used by build(p)).
  __device__ void load_list_rows(int p) {
    const PairInfo pi = *info(p);
    if (pi.n_l == 0) return;
    const float* P = a.ltab + (size_t)pi.l * Mp * kKsub;
#pragma unroll
    for (int i = 0; i < NROW; ++i) {
      const int m = warp + kNW * i;
      if (m >= a.M) continue;
      const float4* src = (const float4*)(P + m * kKsub + lane * 8);
      const float4 u = __ldg(src), v = __ldg(src + 1);
      pp[i][0] = u.x; pp[i][1] = u.y; pp[i][2] = u.z; pp[i][3] = u.w;
      pp[i][4] = v.x; pp[i][5] = v.y; pp[i][6] = v.z; pp[i][7] = v.w;
    }
  }

  // T' = fl32(P_l - 2 Q_q) for this warp's rows of pair p; quantised pairs
  // also publish each row's minimum and range.
  __device__ void build(int p) {
    const PairInfo pi = *info(p);
    if (pi.n_l == 0) return;
#pragma unroll
    for (int i = 0; i < NROW; ++i) {
      const int m = warp + kNW * i;
      if (m >= a.M) continue;
      const float4* qs = (const float4*)(qtab() + m * kKsub + lane * 8);
      const float4 u = qs[0], v = qs[1];
      const float qv[8] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w};
#pragma unroll
      for (int e = 0; e < 8; ++e) tq[i][e] = sub_rn(pp[i][e], qv[e]);
      if (pi.b != 0) {
        float mn = tq[i][0];
#pragma unroll
        for (int e = 1; e < 8; ++e) mn = fminf(mn, tq[i][e]);
        mn = warp_min(mn);
        float mx = 0.f;
#pragma unroll
        for (int e = 0; e < 8; ++e) mx = fmaxf(mx, sub_rn(tq[i][e], mn));
        mx = warp_max(mx);
        if (lane == 0) { rowmin(p)[m] = mn; rowmax(p)[m] = mx; }
      }
    }
  }

  // Writes the table of pair p: FP32 values for plain pairs, else levels with
  // the shared step from the largest row range (warp 0 also forms Delta32 and
  // B32 = fl32(D2 + B), B summed in FP64 in the fixed 32-lane tree order).
  // Rows M..Mp-1 are zero rows, so the scan needs no bound on m.
  __device__ void write_table(int p) {
    const PairInfo pi = *info(p);
    if (pi.n_l == 0) return;
    unsigned char* tab = sm() + table_off(p);
    if (pi.b == 0) {
#pragma unroll
      for (int i = 0; i < NROW; ++i) {
        const int m = warp + kNW * i;
        if (m >= Mp) continue;
        float4* T = (float4*)((float*)tab + m * kKsub + lane * 8);
        const bool live = m < a.M;
        T[0] = live ? make_float4(tq[i][0], tq[i][1], tq[i][2], tq[i][3]) : make_float4(0.f, 0.f, 0.f, 0.f);
        T[1] = live ? make_float4(tq[i][4], tq[i][5], tq[i][6], tq[i][7]) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      return;
    }
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
        sc.B32 = __double2float_rn(__dadd_rn((double)pi.d2, B));
        *scal(p) = sc;
      }
    }
#pragma unroll
    for (int i = 0; i < NROW; ++i) {
      const int m = warp + kNW * i;
      if (m >= Mp) continue;
      unsigned t[8];
      if (m < a.M) {
        const float mn = rowmin(p)[m];
#pragma unroll
        for (int e = 0; e < 8; ++e) t[e] = (unsigned)min(__float2int_rn(mul_rn(sub_rn(tq[i][e], mn), s32)), L);
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) t[e] = 0u;
      }
      if (pi.b <= 8) {
        uint2 v;
        v.x = t[0] | (t[1] << 8) | (t[2] << 16) | (t[3] << 24);
        v.y = t[4] | (t[5] << 8) | (t[6] << 16) | (t[7] << 24);
        *(uint2*)(tab + m * kKsub + lane * 8) = v;
      } else {
        uint4 v;
        v.x = t[0] | (t[1] << 16); v.y = t[2] | (t[3] << 16);
        v.z = t[4] | (t[5] << 16); v.w = t[6] | (t[7] << 16);
        *(uint4*)((uint16_t*)tab + m * kKsub + lane * 8) = v;
      }
    }
  }

  __device__ __forceinline__ void load_tile(const PairInfo& pi, int t, uint4 (&w)[NCHUNK]) const {
    const uint8_t* tile = a.codes + ((size_t)(pi.tile0 + t) * NCHUNK) * kTileChunkBytes + lane * kChunkBytes;
#pragma unroll
    for (int c = 0; c < NCHUNK; ++c) w[c] = __ldg(reinterpret_cast<const uint4*>(tile + c * kTileChunkBytes));
  }

  __device__ void prefetch_first(int p) {
    const PairInfo pi = *info(p);
    if (warp < pi.ntile) load_tile(pi, warp, pf);
  }

  // Scans this warp's tiles of pair p (the first is already in pf) and
  // leaves the first tile of pair p+1 (if has_next) prefetched in pf.
  __device__ void scan(int p, bool has_next, int kq, WarpTopK<1, int64_t>& top, float& thd,
                       int64_t& thi) {
    const PairInfo pi = *info(p);
    const uint32_t tb = base_addr + table_off(p);
    PairScalP sc{};
    if (pi.b) sc = *scal(p);
    if (warp >= pi.ntile) {
      if (has_next) prefetch_first(p + 1);
      return;
    }
    const int64_t* idp = a.ids + pi.vbase;
    for (int t = warp; t < pi.ntile; t += kNW) {
      uint4 w[NCHUNK];
#pragma unroll
      for (int c = 0; c < NCHUNK; ++c) w[c] = pf[c];
      if (t + kNW < pi.ntile) load_tile(pi, t + kNW, pf);
      else if (has_next) prefetch_first(p + 1);
      float d;
      if (pi.b == 0) d = add_rn(pi.d2, adc_f32<NCHUNK>(tb, w));
      else if (pi.b <= 8) d = add_rn(mul_rn(sc.delta32, __int2float_rn(adc_int<uint8_t, NCHUNK>(tb, w))), sc.B32);
      else d = add_rn(mul_rn(sc.delta32, __int2float_rn(adc_int<uint16_t, NCHUNK>(tb, w))), sc.B32);
      const int v = t * kTileVecs + lane;
      const bool pre = v < pi.n_l && d <= thd;
      if (__any_sync(kFull, pre)) {
        const int64_t id = pre ? __ldg(idp + v) : INT64_MAX;
        top.offer(pre, d, id, kq, thd, thi);
      }
    }
  }
};

template <int NCHUNK, int NROW>
__global__ void __launch_bounds__(kThreadsP, 1) search_persistent_kernel(const PArgs a) {
  using PipeT = Pipe<NCHUNK, NROW>;
  PipeT P(a);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* sm = P.base;
  float* md = (float*)(sm + a.off_md);
  int64_t* mi = (int64_t*)(sm + a.off_mi);
  int64_t* next_q = (int64_t*)(sm + a.off_q);
  for (;;) {
    if (threadIdx.x == 0) *next_q = atomicAdd(a.counter, 1);
    __syncthreads();
    const int64_t q = *next_q;
    if (q >= a.nq) break;
    const int np = a.npq ? min(max(a.npq[q], 0), a.nprobe) : a.nprobe;
    const int kq = a.kpq ? min(max(a.kpq[q], 0), a.k) : a.k;
    WarpTopK<1, int64_t> top;
    top.init();
    float thd = INFINITY;
    int64_t thi = INT64_MAX;
    if (kq > 0 && np > 0) {
      P.load_query_table(q);
      for (int s = -3; s < np; ++s) {
        typename PipeT::Staged st;
        const bool stage_in = s + 3 < np;
        if (stage_in) P.load_inputs(q, s + 3, st);
        const bool do_build = s + 2 >= 0 && s + 2 < np;
        if (do_build) P.load_list_rows(s + 2);
        if (s >= 0) P.scan(s, s + 1 < np, kq, top, thd, thi);
        else if (s == -1) P.prefetch_first(0);
        if (s + 1 >= 0 && s + 1 < np) P.write_table(s + 1);
        if (do_build) P.build(s + 2);
        if (stage_in) P.store_inputs(s + 3, st);
        __syncthreads();
      }
    }
    // merge the per-warp lists into warp 0 and write the query's results
    md[warp * 32 + lane] = top.d[0];
    mi[warp * 32 + lane] = top.id[0];
    __syncthreads();
    if (warp == 0) {
      for (int w2 = 1; w2 < kNW && kq > 0; ++w2) {
        const float cd = md[w2 * 32 + lane];
        const int64_t ci = mi[w2 * 32 + lane];
        top.offer(cd != INFINITY, cd, ci, kq, thd, thi);
      }
      if (lane < a.k) {
        const bool ok = lane < kq && top.d[0] != INFINITY;
        a.ids_out[q * a.k + lane] = ok ? top.id[0] : -1;
        a.dists_out[q * a.k + lane] = ok ? top.d[0] : INFINITY;
      }
    }
    __syncthreads();
  }
}

template <int NCHUNK, int NROW>
cudaError_t run(PArgs& a, cudaStream_t s) {
  const size_t smem = layout<NCHUNK>(a);
  auto kern = search_persistent_kernel<NCHUNK, NROW>;
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

}  // namespace

bool persistent_supported(const Index& ix, int k) {
  if (k > 32 || ix.nchunk > 4) return false;
  PArgs a{};
  a.M = (int)ix.M;
  size_t need = 0;
  switch (ix.nchunk) {
    case 1: need = layout<1>(a); break;
    case 2: need = layout<2>(a); break;
    case 3: need = layout<3>(a); break;
    default: need = layout<4>(a); break;
  }
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return need <= (size_t)optin;
}

cudaError_t launch_search_persistent(const Index& ix, const float* qt, int64_t nq, int nprobe,
                                     const int32_t* nprobe_per_q, int k, const int32_t* k_per_q,
                                     const int32_t* probes, const float* probe_d2,
                                     const uint8_t* bits, int64_t* ids_out, float* dists_out,
                                     int* counter, cudaStream_t s) {
  PArgs a{};
  a.qt = qt; a.nq = nq; a.ltab = ix.ltab; a.probe_d2 = probe_d2;
  a.codes = ix.codes; a.ids = ix.ids;
  a.list_len = ix.list_len; a.vec_off = ix.vec_off; a.tile_off = ix.tile_off;
  a.M = (int)ix.M; a.dsub = (int)ix.dsub; a.nprobe = nprobe; a.k = k;
  a.npq = nprobe_per_q; a.kpq = k_per_q; a.probes = probes; a.bits = bits;
  a.ids_out = ids_out; a.dists_out = dists_out; a.counter = counter;
  const bool two = ix.M > kNW;   // rows per warp
  switch (ix.nchunk) {
    case 1: return run<1, 1>(a, s);
    case 2: return run<2, 1>(a, s);
    case 3: return two ? run<3, 2>(a, s) : run<3, 1>(a, s);
    case 4: return two ? run<4, 2>(a, s) : run<4, 1>(a, s);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace anns
