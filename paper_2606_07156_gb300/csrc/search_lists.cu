// List-major search: one warp per probed (query, list) pair, blocks grouped
// by list (DC of Section 2.1 with the queries of a list batched, as the DRM
// groups of Section 4.1 share a cluster buffer).
//
// A persistent grid takes work items — a list and a batch of up to NW pairs
// probing it — from an atomic counter, in descending list size (Section 4.3's
// greedy scheduling by estimated work). Each warp of the block owns one pair:
//   1. builds the pair's table in its own slice of shared memory, lane i
//      owning entries c = 8i..8i+7 of every row: T' = fl32(P_l - 2 Q_q)
//      (FP32 rule of search.cu); for b-bit pairs a first pass finds the row
//      minima and the range (warp shuffles, no block barrier), a second pass
//      writes the levels, and the offset B32 is the exact sum of D2 and the
//      row minima rounded once to FP32;
//   2. scans every code tile of the list (the block's warps read the same
//      tiles, so all but the first read hit L1), offering distances to its
//      sorted top-k list;
//   3. writes the pair's top-k to the partial results [q][rank][k].
// A merge kernel then takes each query's top-k over its probes (TS).
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "scan.cuh"

namespace anns {
namespace {

struct LArgs {
  const float* qt; const float* ltab; const float* probe_d2; const uint8_t* bits;
  const uint8_t* codes; const int64_t* ids;
  const int32_t* list_len; const int64_t* vec_off; const int64_t* tile_off;
  const int32_t* order; const int* cnt; const int* off; const int* ioff; const int32_t* pairs;
  int nlist, M, nprobe, k;
  const int32_t* kpq;
  float* part_d; int64_t* part_i;
  int* counter;
  uint32_t region;   // bytes of one warp's table slice (a multiple of 256)
};

// ldg_row8 for data read once per warp (a query's table): not kept in L1, so
// the list's code tiles and list table, shared by the block's warps, stay there.
__device__ __forceinline__ void ldg_row8_stream(const float* row, int lane, float (&v)[8]) {
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]) : "l"(row + row_at(lane, 0)));
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7]) : "l"(row + row_at(lane, 1)));
}

template <int NCHUNK>
struct PairTable {
  static constexpr int Mp = NCHUNK * 16;
  static constexpr int SLOTS = (Mp + 31) / 32;
  float delta32 = 0.f, B32 = 0.f;

  // Builds the table of pair (P row block, Q row block) at shared byte address
  // `tab` (generic pointer `tp`), for `b` bits (0 = FP32).
  __device__ void build(const float* __restrict__ P, const float* __restrict__ Qt, int M, int b, float d2,
                        unsigned char* tp, int lane) {
    if (b == 0) {
      for (int m = 0; m < Mp; ++m) {
        float t[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (m < M) {
          float p[8], q[8];
          ldg_row8(P + m * kKsub, lane, p);
          ldg_row8_stream(Qt + m * kKsub, lane, q);
#pragma unroll
          for (int e = 0; e < 8; ++e) t[e] = sub_rn(p[e], q[e]);
        }
        st_row8((float*)tp + m * kKsub, lane, t);
      }
      return;
    }
    // pass 1: row minima (lane m%32 keeps row m in slot m/32) and the range
    float rm[SLOTS];
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) rm[s] = 0.f;
    float range = 0.f;
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      for (int mm = 0; mm < 32; ++mm) {
        const int m = s * 32 + mm;
        if (m >= M) break;
        float p[8], q[8], t[8];
        ldg_row8(P + m * kKsub, lane, p);
        ldg_row8_stream(Qt + m * kKsub, lane, q);
#pragma unroll
        for (int e = 0; e < 8; ++e) t[e] = sub_rn(p[e], q[e]);
        float mn = t[0];
#pragma unroll
        for (int e = 1; e < 8; ++e) mn = fminf(mn, t[e]);
        mn = warp_min(mn);
        float mx = 0.f;
#pragma unroll
        for (int e = 0; e < 8; ++e) mx = fmaxf(mx, sub_rn(t[e], mn));
        range = fmaxf(range, warp_max(mx));
        if (lane == mm) rm[s] = mn;
      }
    }
    const int L = (1 << b) - 1;
    const float s32 = range > 0.f ? __fdiv_rn((float)L, range) : 0.f;
    delta32 = range > 0.f ? __fdiv_rn(range, (float)L) : 0.f;
    ExactSum B;
    xsum_init(B);
#pragma unroll
    for (int s = 0; s < SLOTS; ++s)
      if (s * 32 + lane < M) xsum_add(B, rm[s]);
    if (lane == 0) xsum_add(B, d2);
    xsum_warp(B);
    B32 = xsum_round(B);
    // pass 2: levels
#pragma unroll
    for (int s = 0; s < SLOTS; ++s) {
      for (int mm = 0; mm < 32; ++mm) {
        const int m = s * 32 + mm;
        if (m >= Mp) break;
        unsigned t[8];
        if (m < M) {
          const float mn = __shfl_sync(kFull, rm[s], mm);
          float p[8], q[8];
          ldg_row8(P + m * kKsub, lane, p);
          ldg_row8_stream(Qt + m * kKsub, lane, q);
#pragma unroll
          for (int e = 0; e < 8; ++e)
            t[e] = (unsigned)min(__float2int_rn(mul_rn(sub_rn(sub_rn(p[e], q[e]), mn), s32)), L);
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) t[e] = 0u;
        }
        if (b <= 8) {
          *(uint32_t*)(tp + m * kKsub + row_at(lane, 0)) = t[0] | (t[1] << 8) | (t[2] << 16) | (t[3] << 24);
          *(uint32_t*)(tp + m * kKsub + row_at(lane, 1)) = t[4] | (t[5] << 8) | (t[6] << 16) | (t[7] << 24);
        } else {
          uint16_t* r = (uint16_t*)tp + m * kKsub;
          *(uint2*)(r + row_at(lane, 0)) = make_uint2(t[0] | (t[1] << 16), t[2] | (t[3] << 16));
          *(uint2*)(r + row_at(lane, 1)) = make_uint2(t[4] | (t[5] << 16), t[6] | (t[7] << 16));
        }
      }
    }
  }
};

template <int NCHUNK>
__device__ __forceinline__ void load_tile(const uint8_t* __restrict__ tile, uint4 (&w)[NCHUNK]) {
#pragma unroll
  for (int c = 0; c < NCHUNK; ++c) w[c] = __ldg(reinterpret_cast<const uint4*>(tile + c * kTileChunkBytes));
}

// Wide codes (NCHUNK > 4) need more registers per thread: at most 16 warps.
constexpr int max_warps(int nchunk) { return nchunk <= 4 ? 32 : 16; }

template <int NCHUNK, int R>
__global__ void __launch_bounds__(max_warps(NCHUNK) * 32) list_kernel(const LArgs a) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t raw = smem_addr(anns_dyn_smem);
  const uint32_t pad = (256u - (raw & 255u)) & 255u;
  unsigned char* base = anns_dyn_smem + pad;
  int* item_sh = (int*)(base + (size_t)nw * a.region);
  unsigned char* tp = base + (size_t)warp * a.region;
  const uint32_t tab = raw + pad + warp * a.region;
  const int nitems = a.ioff[a.nlist];
  for (;;) {
    __syncthreads();  // the previous item's warps are done with item_sh
    if (threadIdx.x == 0) {
      const int it = atomicAdd(a.counter, 1);
      int r = 0;
      if (it < nitems) {  // size rank r: the last with ioff[r] <= it
        int lo = 0, hi = a.nlist - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (a.ioff[mid] <= it) lo = mid; else hi = mid - 1;
        }
        r = lo;
      }
      item_sh[0] = it;
      item_sh[1] = r;
    }
    __syncthreads();
    const int it = item_sh[0];
    if (it >= nitems) break;
    const int r = item_sh[1];
    const int l = a.order[r];
    const int pi = (it - a.ioff[r]) * nw + warp;
    if (pi >= a.cnt[l]) continue;
    const int pid = a.pairs[a.off[l] + pi];
    const int q = pid / a.nprobe;
    const int b = a.bits[pid];
    const float d2 = a.probe_d2[pid];
    const size_t tstride = (size_t)NCHUNK * 16 * kKsub;
    const int need = b == 0 ? 4 : b <= 8 ? 1 : 2;   // table bytes per entry
    const int kq = (need * tstride > a.region) ? 0 : (a.kpq ? min(max(a.kpq[q], 0), a.k) : a.k);
    PairTable<NCHUNK> T;
    if (kq > 0) T.build(a.ltab + (size_t)l * tstride, a.qt + (size_t)q * tstride, a.M, b, d2, tp, lane);
    __syncwarp();
    WarpTopK<R, int64_t> top;
    top.init();
    float thd = INFINITY;
    int64_t thi = INT64_MAX;
    const int n_l = a.list_len[l];
    const int ntile = (n_l + kTileVecs - 1) / kTileVecs;
    const uint8_t* t0 = a.codes + (size_t)a.tile_off[l] * NCHUNK * kTileChunkBytes + lane * kChunkBytes;
    const int64_t* idp = a.ids + a.vec_off[l];
    uint4 nxt[NCHUNK];
    if (kq > 0 && ntile > 0) load_tile<NCHUNK>(t0, nxt);
    for (int t = 0; kq > 0 && t < ntile; ++t) {
      uint4 w[NCHUNK];
#pragma unroll
      for (int c = 0; c < NCHUNK; ++c) w[c] = nxt[c];
      if (t + 1 < ntile) load_tile<NCHUNK>(t0 + (size_t)(t + 1) * NCHUNK * kTileChunkBytes, nxt);
      float d;
      if (b == 0) d = add_rn(d2, adc_f32<NCHUNK>(tab, w));
      else if (b <= 8) d = add_rn(mul_rn(T.delta32, __int2float_rn(adc_int<uint8_t, NCHUNK>(tab, w))), T.B32);
      else d = add_rn(mul_rn(T.delta32, __int2float_rn(adc_int<uint16_t, NCHUNK>(tab, w))), T.B32);
      const int v = t * kTileVecs + lane;
      const bool pre = v < n_l && d <= thd;
      if (__any_sync(kFull, pre)) {
        const int64_t id = pre ? __ldg(idp + v) : INT64_MAX;
        top.offer(pre, d, id, kq, thd, thi);
      }
    }
    float* pd = a.part_d + (size_t)pid * a.k;
    int64_t* pix = a.part_i + (size_t)pid * a.k;
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
      const int e = rr * 32 + lane;
      if (e < a.k) {
        const bool ok = e < kq && top.d[rr] != INFINITY;
        pd[e] = ok ? top.d[rr] : INFINITY;
        pix[e] = ok ? top.id[rr] : -1;
      }
    }
    __syncwarp();  // the table slice is rewritten by this warp's next pair
  }
}

// One warp per query: the k smallest (d, id) over the partial results of its probes.
template <int R>
__global__ void __launch_bounds__(256) merge_kernel(const float* __restrict__ part_d,
                                                    const int64_t* __restrict__ part_i,
                                                    const int32_t* __restrict__ probes,
                                                    const int32_t* __restrict__ npq,
                                                    const int32_t* __restrict__ kpq, int64_t nq,
                                                    int nprobe, int k, int64_t* __restrict__ ids_out,
                                                    float* __restrict__ dists_out) {
  const int64_t q = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (q >= nq) return;
  const int np = npq ? min(max(npq[q], 0), nprobe) : nprobe;
  const int kq = kpq ? min(max(kpq[q], 0), k) : k;
  WarpTopK<R, int64_t> top;
  top.init();
  float thd = INFINITY;
  int64_t thi = INT64_MAX;
  for (int j = 0; kq > 0 && j < np; ++j) {
    const int64_t pid = q * nprobe + j;
    if (probes[pid] < 0) continue;
    for (int e0 = 0; e0 < kq; e0 += 32) {
      const int e = e0 + lane;
      const bool in = e < kq;
      const float d = in ? part_d[pid * k + e] : INFINITY;
      const int64_t id = in ? part_i[pid * k + e] : -1;
      top.offer(in && id >= 0, d, id, kq, thd, thi);
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int e = r * 32 + lane;
    if (e < k) {
      const bool ok = e < kq && top.d[r] != INFINITY;
      ids_out[q * k + e] = ok ? top.id[r] : -1;
      dists_out[q * k + e] = ok ? top.d[r] : INFINITY;
    }
  }
}

template <int NCHUNK, int R>
cudaError_t run_lists(const LArgs& a, int nw, size_t smem, int sms, cudaStream_t s) {
  auto kern = list_kernel<NCHUNK, R>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<sms, nw * 32, smem, s>>>(a); note_launch();
  return cudaGetLastError();
}

template <int NCHUNK>
cudaError_t run_lists_r(const LArgs& a, int R, int nw, size_t smem, int sms, cudaStream_t s) {
  return R == 1 ? run_lists<NCHUNK, 1>(a, nw, smem, sms, s) : run_lists<NCHUNK, 4>(a, nw, smem, sms, s);
}

}  // namespace

int list_major_warps(const Index& ix, int table_bytes_per_entry) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t region = (size_t)ix.Mp * kKsub * table_bytes_per_entry;
  const size_t avail = (size_t)optin > 1024 ? (size_t)optin - 1024 : 0;
  return (int)std::min<size_t>(max_warps((int)ix.nchunk), avail / region);
}

cudaError_t launch_search_lists(const Index& ix, const float* qt, int64_t nq, int nprobe,
                                const int32_t* nprobe_per_q, int k, const int32_t* k_per_q,
                                const int32_t* probes, const float* probe_d2, const uint8_t* bits,
                                int table_bytes_per_entry, const ListWork& w, int64_t* ids_out,
                                float* dists_out, cudaStream_t s) {
  const int nw = list_major_warps(ix, table_bytes_per_entry);
  if (nw < 1) return cudaErrorInvalidValue;
  cudaError_t e = launch_invert(ix, probes, nprobe_per_q, nq, nprobe, nw, w, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(w.counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  LArgs a{};
  a.qt = qt; a.ltab = ix.ltab; a.probe_d2 = probe_d2; a.bits = bits;
  a.codes = ix.codes; a.ids = ix.ids; a.list_len = ix.list_len; a.vec_off = ix.vec_off;
  a.tile_off = ix.tile_off; a.order = ix.order; a.cnt = w.cnt; a.off = w.off; a.ioff = w.ioff;
  a.pairs = w.pairs; a.nlist = (int)ix.nlist; a.M = (int)ix.M; a.nprobe = nprobe; a.k = k;
  a.kpq = k_per_q; a.part_d = w.part_d; a.part_i = w.part_i; a.counter = w.counter;
  a.region = (uint32_t)(ix.Mp * kKsub * table_bytes_per_entry);
  const size_t smem = (size_t)nw * a.region + 16 + 256;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int R = k <= 32 ? 1 : 4;
  switch (ix.nchunk) {
    case 1: e = run_lists_r<1>(a, R, nw, smem, sms, s); break;
    case 2: e = run_lists_r<2>(a, R, nw, smem, sms, s); break;
    case 3: e = run_lists_r<3>(a, R, nw, smem, sms, s); break;
    case 4: e = run_lists_r<4>(a, R, nw, smem, sms, s); break;
    case 5: e = run_lists_r<5>(a, R, nw, smem, sms, s); break;
    case 6: e = run_lists_r<6>(a, R, nw, smem, sms, s); break;
    case 7: e = run_lists_r<7>(a, R, nw, smem, sms, s); break;
    default: e = run_lists_r<8>(a, R, nw, smem, sms, s); break;
  }
  if (e != cudaSuccess) return e;
  const unsigned gm = (unsigned)((nq + 7) / 8);
  if (R == 1) {
    merge_kernel<1><<<gm, 256, 0, s>>>(w.part_d, w.part_i, probes, nprobe_per_q, k_per_q, nq, nprobe, k, ids_out, dists_out); note_launch();
  } else {
    merge_kernel<4><<<gm, 256, 0, s>>>(w.part_d, w.part_i, probes, nprobe_per_q, k_per_q, nq, nprobe, k, ids_out, dists_out); note_launch();
  }
  return cudaGetLastError();
}

}  // namespace anns
