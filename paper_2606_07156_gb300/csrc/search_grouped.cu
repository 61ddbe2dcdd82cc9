// Grouped search of the narrow pairs (tables of 1..8 bits). The pairs probing
// a list are taken four at a time, and their four byte tables are interleaved
// into one table of 32-bit words: entry c of row m holds the levels of the four
// queries in bytes 0..3. One shared-memory gather per (vector, sub-space) then
// serves four queries, and two 32-bit accumulators hold the four integer sums
// as 16-bit lanes (bytes 0 and 2, bytes 1 and 3; a sum of at most 128 levels
// of 255 stays below 2^16). The list's code tiles and list table are read once
// per group instead of once per pair. For table gathers this is how a
// narrower table becomes throughput (the gain the paper expects of lower
// precision, Sections 1, 2.2): 8-bit levels pack four queries per gather,
// where FP32 entries pack one.
//
// Each query's rank-0 pair and its wide pairs (FP32, 12 and 16 bits) go
// through the query-major kernel first; the k-th distance found there bounds
// the query's final k-th distance and prunes the grouped pairs' candidates. A
// merge then takes each query's top-k over both (TS). Results equal the other
// kernels' bit for bit: every table, integer sum and distance follows the same
// rules (search.cu).
//
// Per group (one block of 8 warps, persistent grid, groups taken from an
// atomic counter by (query chunk, descending list size); the last warp fetches
// the next group's item while the block scans the current one):
//   1. row statistics: for each (slot, row) the warps form T' = P_l - 2 Q_q
//      and its row minimum and range;
//   2. per slot: the shared step, its reciprocal scale and the offset (the
//      exact sum of D2 and the row minima, rounded once, as elsewhere);
//   3. levels: each warp recomputes T' for its rows of all four slots,
//      quantises and interleaves the four levels of each entry;
//   4. scan: warps take code tiles; per vector the four sums and one
//      integer test of all four against the block's limits; the few vectors
//      that pass get their distances and enter the warp's top-k lists (in
//      shared memory); the warps' lists are merged per slot and written to
//      the pairs' partial results.
#include <algorithm>
#include <utility>

#include "common.cuh"
#include "internal.h"
#include "scan.cuh"

namespace anns {
namespace {

constexpr int kGThreads = 256, kGWarps = kGThreads / 32, kSlots = 4;

struct GArgs {
  const float* qt; const float* ltab; const float* probe_d2; const uint8_t* bits;
  const uint8_t* codes; const int64_t* ids;
  const int32_t* list_len; const int64_t* vec_off; const int64_t* tile_off;
  const int32_t* order; const int* cnt; const int* off; const int* ioff; const int32_t* pairs;
  const int* gtab;  // bucket of each group
  int nlist, nb, M, Mp, nprobe, k;  // nb: (query chunk, list) buckets
  const int32_t* kpq;
  float* part_d; int64_t* part_i;
  const float* qm_d;  // [nq * k] query-major results (rank 0 and wide pairs): the bound
  int* counter;
};

// Per slot: the scale, the step and offset of the distances, the bound from
// the query-major pairs, the slot's k and its pair.
struct SlotScal { float s32, delta32, B32, bound; int kq, pid, pad0, pad1; };

// One group's work item: its list, number of pairs and per slot the pair, its
// query, table width, D2, k and bound (the query's k-th distance over its
// query-major pairs). Fetched by one warp while the block scans the previous
// group, so that the block never waits on this chain of dependent loads.
template <int S>
struct GItemT {
  int it, l, ns, n_l;
  int pid[S], q[S], bits[S], kq[S];
  float d2[S], bound[S];
  long long tile0, vec0;  // the list's first code tile and first id
};
using GItem = GItemT<4>;

// Bytes of the block's shared memory (256-aligned offsets).
struct GLayout {
  size_t tab, bias, rowmax, scal, item, lim, md, mi, total;
  __host__ __device__ GLayout(int Mp, int R, int S = kSlots) {
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t o = 0;
    tab = o; o += al((size_t)Mp * kKsub * 4);
    bias = o; o += al((size_t)S * Mp * 4);
    rowmax = o; o += al((size_t)S * Mp * 4);
    scal = o; o += al(sizeof(SlotScal) * S);
    item = o; o += al(2 * (S == kSlots ? sizeof(GItemT<kSlots>) : sizeof(GItemT<8>)));  // double buffer
    lim = o; o += al(4 * 4);
    md = o; o += al((size_t)S * kGWarps * R * 32 * 4);
    mi = o; o += al((size_t)S * kGWarps * R * 32 * 8);
    total = o + 256;
  }
};

// Packed word of sub-space K for the vector whose codes are w.
template <int K, int NCHUNK>
__device__ __forceinline__ void packed_acc(uint32_t base, const uint4 (&w)[NCHUNK], uint32_t& a02, uint32_t& a13) {
  const uint32_t x = code_word<K & ~3, NCHUNK>(w);
  const uint32_t code = __byte_perm(x, 0u, 0x4440u + (K & 3));
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1+%2];" : "=r"(v) : "r"(base + code * 4u), "n"(K * 1024));
  a02 += __byte_perm(v, 0u, 0x4240u);  // bytes 0 and 2 as 16-bit lanes
  a13 += __byte_perm(v, 0u, 0x4341u);  // bytes 1 and 3
}
template <int NCHUNK, int... K>
__device__ __forceinline__ void adc_packed_seq(uint32_t base, const uint4 (&w)[NCHUNK], uint32_t& a02, uint32_t& a13,
                                               std::integer_sequence<int, K...>) {
  (packed_acc<K, NCHUNK>(base, w, a02, a13), ...);
}

template <int NCHUNK>
__device__ __forceinline__ void load_codes(const uint8_t* __restrict__ tile, uint4 (&w)[NCHUNK]) {
#pragma unroll
  for (int c = 0; c < NCHUNK; ++c) w[c] = __ldg(reinterpret_cast<const uint4*>(tile + c * kTileChunkBytes));
}

__device__ __forceinline__ uint32_t rint_bits_g(float y) { return __float_as_uint(add_rn(y, 12582912.0f)); }

// Largest integer sum S in [0, 0x7FFF] whose distance fl32(fl32(delta * S) + B)
// is <= x, or -1 when none is (whole warp, uniform arguments). The distance
// never falls as S rises (both roundings are monotone), so d(S) <= x exactly
// when S <= smax_warp(x). Each round tests 32 evenly spaced candidates of the
// remaining interval [lo, hi] (d(lo) <= x); the passing ones form a prefix, so
// their count places the answer in one gap: three rounds for 2^15 values.
__device__ __forceinline__ int smax_warp(float x, float delta, float B) {
  const int lane = threadIdx.x & 31;
  int lo = -1, hi = 0x7FFF;
  while (lo < hi) {
    const int step = (hi - lo + 31) >> 5;  // 32 * step >= hi - lo: the candidates reach hi
    const int c = lo + (lane + 1) * step;
    const bool ok = c <= hi && add_rn(mul_rn(delta, __int2float_rn(c)), B) <= x;
    const int t = __popc(__ballot_sync(kFull, ok));
    const int nhi = min(hi, lo + (t + 1) * step - 1);
    lo = t > 0 ? lo + t * step : lo;
    hi = nhi;
  }
  return lo;
}

// Lowers a slot's 16-bit lane (word `reg`, half `half`) of the block's packed
// limits to v (if lower). A retry lost to the cap leaves a larger limit, which
// only prunes less.
__device__ __forceinline__ void lim_min_at(uint32_t* lim, int reg, int half, uint32_t v) {
  uint32_t* w = lim + reg;
  const int sh = half * 16;
  uint32_t old = *(volatile uint32_t*)w;
  for (int it = 0; it < 256; ++it) {
    if (((old >> sh) & 0xFFFFu) <= v) return;
    const uint32_t seen = atomicCAS(w, old, (old & ~(0xFFFFu << sh)) | (v << sh));
    if (seen == old) return;
    old = seen;
  }
}

// Byte tables: slots 0 and 2 share limit word 0, slots 1 and 3 word 1.
__device__ __forceinline__ void lim_min(uint32_t* lim, int s, uint32_t v) { lim_min_at(lim, s & 1, s >> 1, v); }

// A slot's offset (whole warp): the exact sum of D2 and the slot's row
// minima, rounded once (kept out of line: its accumulator does not add to the
// scan's register pressure).
__device__ __forceinline__ float slot_offset(const float* bias_s, int M, float d2, bool present) {
  return warp_exact_sum(bias_s, present ? M : 0, d2, true);
}

// The next group from the work queue (whole warp; lanes 0..S-1 take the slots).
template <int S = kSlots>
__device__ __forceinline__ void fetch_group(const GArgs& a, int ngroups, GItemT<S>* out, int lane) {
  int it = 0;
  if (lane == 0) it = atomicAdd(a.counter, 1);
  it = __shfl_sync(kFull, it, 0);
  if (it >= ngroups) {
    if (lane == 0) out->it = it;
    return;
  }
  const int b = a.gtab[it];
  const int l = a.order[b % a.nlist];
  const int key = (b / a.nlist) * a.nlist + l;
  const int i = it - a.ioff[b];
  const int ns = min(S, a.cnt[key] - S * i);
  if (lane < S) {
    const int p = lane < ns ? a.pairs[a.off[key] + S * i + lane] : -1;
    int qs = 0, bs = 8, kq = 0;
    float d2 = 0.f, bound = INFINITY;
    if (p >= 0) {
      qs = p / a.nprobe;
      bs = a.bits[p];
      d2 = a.probe_d2[p];
      kq = a.kpq ? min(max(a.kpq[qs], 0), a.k) : a.k;
      if (kq > 0) bound = a.qm_d[(size_t)qs * a.k + kq - 1];
    }
    out->pid[lane] = p; out->q[lane] = qs; out->bits[lane] = bs; out->kq[lane] = kq;
    out->d2[lane] = d2; out->bound[lane] = bound;
  }
  if (lane == 0) {
    out->it = it; out->l = l; out->ns = ns; out->n_l = a.list_len[l];
    out->tile0 = a.tile_off[l];
    out->vec0 = a.vec_off[l];
  }
}

// R: the warps' top-k lists hold R * 32 entries (k <= 32 R).
template <int NCHUNK, int R>
__global__ void __launch_bounds__(kGThreads, NCHUNK <= 2 ? 4 : (NCHUNK <= 4 ? 3 : (NCHUNK <= 6 ? 2 : 1)))
    packed_kernel(const GArgs a) {
  constexpr int Mp = NCHUNK * 16;
  const GLayout L(Mp, R);
  const uint32_t raw = smem_addr(anns_dyn_smem);
  const uint32_t pad = (256u - (raw & 255u)) & 255u;
  unsigned char* base = anns_dyn_smem + pad;
  uint32_t* tab = (uint32_t*)(base + L.tab);
  float* bias = (float*)(base + L.bias);
  float* rowmax = (float*)(base + L.rowmax);
  SlotScal* scal = (SlotScal*)(base + L.scal);
  GItem* items = (GItem*)(base + L.item);
  uint32_t* lim = (uint32_t*)(base + L.lim);  // 0x8000 + Smax per slot, 16-bit lanes (see the scan)
  float* md = (float*)(base + L.md);
  int64_t* mi = (int64_t*)(base + L.mi);
  const uint32_t tab_addr = raw + pad + (uint32_t)L.tab;
  const uint32_t lim_addr = raw + pad + (uint32_t)L.lim;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ngroups = a.ioff[a.nb];
  const size_t tstride = (size_t)Mp * kKsub;
  int cur = 0;
  if (warp == kGWarps - 1) fetch_group(a, ngroups, items, lane);
  for (;;) {
    __syncthreads();  // the previous group is done with the shared tables; items[cur] is complete
    if (threadIdx.x < 2) lim[threadIdx.x] = 0xFFFFFFFFu;  // every sum passes until the seeds
    const GItem& G = items[cur];
    if (G.it >= ngroups) break;
    const int l = G.l, ns = G.ns;
    int q[kSlots];
#pragma unroll
    for (int s = 0; s < kSlots; ++s) q[s] = G.q[s];
    const float* P = a.ltab + (size_t)l * tstride;
    // 1. row statistics: warp w takes rows m = w, w + 8, ...; the list-table
    //    row is loaded once for the group's slots, the query-table rows two
    //    slots at a time (an absent pair of slots reads nothing), and the
    //    reductions run side by side
    for (int m = warp; m < a.M; m += kGWarps) {
      float p[8], lo_v[kSlots], hi_v[kSlots];
      ldg_row8(P + m * kKsub, lane, p);
#pragma unroll
      for (int s0 = 0; s0 < kSlots; s0 += 2) {
        if (s0 >= ns) {  // absent slots (the group's uniform count): nothing to read
          lo_v[s0] = hi_v[s0] = lo_v[s0 + 1] = hi_v[s0 + 1] = 0.f;
          continue;
        }
        float qq[2][8];
#pragma unroll
        for (int u = 0; u < 2; ++u) ldg_row8(a.qt + (size_t)q[s0 + u] * tstride + m * kKsub, lane, qq[u]);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int s = s0 + u;
          lo_v[s] = hi_v[s] = sub_rn(p[0], qq[u][0]);
#pragma unroll
          for (int e = 1; e < 8; ++e) {
            const float tv = sub_rn(p[e], qq[u][e]);
            lo_v[s] = fminf(lo_v[s], tv);
            hi_v[s] = fmaxf(hi_v[s], tv);
          }
        }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1)
#pragma unroll
        for (int s = 0; s < kSlots; ++s) {
          lo_v[s] = fminf(lo_v[s], __shfl_xor_sync(kFull, lo_v[s], o));
          hi_v[s] = fmaxf(hi_v[s], __shfl_xor_sync(kFull, hi_v[s], o));
        }
#pragma unroll
      for (int s = 0; s < kSlots; ++s)
        // max over entries of fl32(t - mn) = fl32(max t - mn): rounding is monotone
        if (lane == 0 && s < ns) { bias[s * Mp + m] = lo_v[s]; rowmax[s * Mp + m] = sub_rn(hi_v[s], lo_v[s]); }
    }
    __syncthreads();
    // 2. per slot: step, scale and offset; the slot's k and its bound, the
    //    k-th distance of its query over the query-major pairs (rank 0 and
    //    the wide pairs), which seeds the scan's limit (no better candidate
    //    list holds a vector farther than that; equal distances are kept)
    if (warp < kSlots) {
      const int s = warp;
      float range = 0.f;
      const int p = G.pid[s], bs = G.bits[s];
      const float d2 = G.d2[s];
      if (s < ns) {
        for (int m = lane; m < a.M; m += 32) range = fmaxf(range, rowmax[s * Mp + m]);
        range = warp_max(range);
      }
      const float B32 = slot_offset(bias + s * Mp, a.M, d2, s < ns);
      // every lane forms the same values (range and B are warp-uniform)
      const int Lv = (1 << bs) - 1;
      SlotScal sc;
      sc.s32 = range > 0.f ? __fdiv_rn((float)Lv, range) : 0.f;
      sc.delta32 = range > 0.f ? __fdiv_rn(range, (float)Lv) : 0.f;
      sc.B32 = B32;
      sc.kq = s < ns ? G.kq[s] : 0;
      sc.bound = sc.kq > 0 ? G.bound[s] : INFINITY;
      sc.pid = p;
      sc.pad0 = sc.pad1 = 0;
      const int seed = sc.kq == 0 ? -1 : (sc.bound == INFINITY ? 0x7FFF : smax_warp(sc.bound, sc.delta32, sc.B32));
      if (lane == 0) {
        scal[s] = sc;
        lim_min(lim, s, (uint32_t)(0x8000 + seed));
      }
    }
    // the warps' top-k lists start empty
#pragma unroll
    for (int s = 0; s < kSlots; ++s)
#pragma unroll
      for (int r = 0; r < R; ++r) {
        md[(s * kGWarps + warp) * R * 32 + r * 32 + lane] = INFINITY;
        mi[(s * kGWarps + warp) * R * 32 + r * 32 + lane] = INT64_MAX;
      }
    __syncthreads();
    // 3. interleaved levels, row by row
    float s32[kSlots];
#pragma unroll
    for (int s = 0; s < kSlots; ++s) s32[s] = s < ns ? scal[s].s32 : 0.f;
    for (int m = warp; m < Mp; m += kGWarps) {
      // byte s of entry e's word holds slot s's level (absent slots and the
      // padding rows m >= M hold 0)
      uint32_t wv[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) wv[e] = 0u;
      if (m < a.M) {
        float p[8];
        ldg_row8(P + m * kKsub, lane, p);
#pragma unroll
        for (int s = 0; s < kSlots; ++s) {
          if (s < ns) {
            float qq[8];
            ldg_row8(a.qt + (size_t)q[s] * tstride + m * kKsub, lane, qq);
            const float mn = bias[s * Mp + m];
            // levels t = rint(fl32(fl32(T' - bias) * s32)) <= L, in the low byte
#pragma unroll
            for (int e = 0; e < 8; ++e)
              wv[e] = __byte_perm(wv[e], rint_bits_g(mul_rn(sub_rn(sub_rn(p[e], qq[e]), mn), s32[s])),
                                  0x3210u ^ (0x4u << (4 * s)) ^ ((uint32_t)s << (4 * s)));
          }
        }
      }
      *(uint4*)(tab + m * kKsub + row_at(lane, 0)) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
      *(uint4*)(tab + m * kKsub + row_at(lane, 1)) = make_uint4(wv[4], wv[5], wv[6], wv[7]);
    }
    __syncthreads();
    // 4. scan. The test per vector is on the integer sums: lim holds
    //    0x8000 + Smax per slot as 16-bit lanes laid out like the sums (slots
    //    0 and 2 in lim[0], 1 and 3 in lim[1]), where Smax is the largest sum
    //    whose distance is <= the smallest k-th distance any warp of the block
    //    holds (or the bound). Sums stay <= 128 * 255 < 0x8000, so lane - S
    //    borrows nothing and keeps bit 15 set exactly when S <= Smax. The
    //    warps' lists live in shared memory (md, mi) and are touched only for
    //    the vectors that pass.
    const int n_l = G.n_l;
    const int ntile = (n_l + kTileVecs - 1) / kTileVecs;
    const size_t tile_bytes = (size_t)NCHUNK * kTileChunkBytes;
    const uint8_t* tp = a.codes + (size_t)G.tile0 * tile_bytes + (size_t)warp * tile_bytes + lane * kChunkBytes;
    const int64_t* idp = a.ids + G.vec0;
    // the next group's item, fetched while the block scans this one
    if (warp == kGWarps - 1) fetch_group(a, ngroups, items + (cur ^ 1), lane);
    uint4 w[NCHUNK];
    if (warp < ntile) load_codes<NCHUNK>(tp, w);
    for (int t = warp; t < ntile; t += kGWarps) {
      uint4 wn[NCHUNK];
      const bool more = t + kGWarps < ntile;
      if (more) load_codes<NCHUNK>(tp + kGWarps * tile_bytes, wn);
      uint32_t a02 = 0u, a13 = 0u;
      adc_packed_seq<NCHUNK>(tab_addr, w, a02, a13, std::make_integer_sequence<int, NCHUNK * 16>{});
      uint32_t l02, l13;
      asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(l02), "=r"(l13) : "r"(lim_addr));
      const uint32_t p02 = (l02 - a02) & 0x80008000u, p13 = (l13 - a13) & 0x80008000u;
      const int v = t * kTileVecs + lane;
      const bool any = v < n_l && (p02 | p13) != 0u;
      if (__any_sync(kFull, any)) {
        const int64_t id = any ? __ldg(idp + v) : INT64_MAX;
#pragma unroll
        for (int s = 0; s < kSlots; ++s) {
          const uint32_t acc = (s & 1) ? a13 : a02, pm = (s & 1) ? p13 : p02;
          const bool ok = any && ((pm >> ((s >> 1) * 16 + 15)) & 1u);
          if (__any_sync(kFull, ok)) {
            const SlotScal sc = scal[s];
            float* ld = md + (s * kGWarps + warp) * R * 32;
            int64_t* li = mi + (s * kGWarps + warp) * R * 32;
            WarpTopK<R, int64_t> top;
#pragma unroll
            for (int r = 0; r < R; ++r) { top.d[r] = ld[r * 32 + lane]; top.id[r] = li[r * 32 + lane]; }
            // the warp's k-th entry, at most the bound (ties kept: the id decides)
            float thd = ld[sc.kq - 1];
            int64_t thi = li[sc.kq - 1];
            if (sc.bound < thd) { thd = sc.bound; thi = INT64_MAX; }
            const float d = add_rn(mul_rn(sc.delta32, __int2float_rn((int)((acc >> ((s >> 1) * 16)) & 0xFFFFu))),
                                   sc.B32);
            top.offer(ok, d, id, sc.kq, thd, thi);
            if (sc.bound < thd) thd = sc.bound;
#pragma unroll
            for (int r = 0; r < R; ++r) { ld[r * 32 + lane] = top.d[r]; li[r * 32 + lane] = top.id[r]; }
            if (thd != INFINITY) {
              const int sm = smax_warp(thd, sc.delta32, sc.B32);
              if (lane == 0) lim_min(lim, s, (uint32_t)(0x8000 + sm));
            }
            __syncwarp();
          }
        }
      }
      if (more) {
#pragma unroll
        for (int c = 0; c < NCHUNK; ++c) w[c] = wn[c];
      }
      tp += kGWarps * tile_bytes;
    }
    __syncthreads();
    // merge the warps' lists per slot; warp s writes slot s
    if (warp < ns) {
      const int s = warp;
      const SlotScal sc = scal[s];
      WarpTopK<R, int64_t> m;
      m.init();
      float th = INFINITY;
      int64_t ti = INT64_MAX;
      for (int w2 = 0; w2 < kGWarps && sc.kq > 0; ++w2)
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const float cd = md[(s * kGWarps + w2) * R * 32 + r * 32 + lane];
          const int64_t ci = mi[(s * kGWarps + w2) * R * 32 + r * 32 + lane];
          m.offer(cd != INFINITY, cd, ci, sc.kq, th, ti);
        }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int e = r * 32 + lane;
        if (e < a.k) {
          const bool ok = e < sc.kq && m.d[r] != INFINITY;
          a.part_d[(size_t)sc.pid * a.k + e] = ok ? m.d[r] : INFINITY;
          a.part_i[(size_t)sc.pid * a.k + e] = ok ? m.id[r] : -1;
        }
      }
    }
    cur ^= 1;
  }
}

// ---- 4-bit tables, eight queries per word ----------------------------------
//
// The pairs on tables of at most 4 bits are taken eight at a time: entry c of
// row m holds the eight queries' levels as nibbles (slot s in bits 4s..4s+3),
// so one shared-memory gather per (vector, sub-space) serves eight queries.
// The nibbles add up as byte lanes for the 16 sub-spaces of a code chunk
// (16 * 15 = 240 < 256), slots 0, 2, 4, 6 in one register and 1, 3, 5, 7 in
// another, and then widen into 16-bit lanes of four registers: W0 = (slot 0,
// slot 4), W1 = (2, 6), W2 = (1, 5), W3 = (3, 7); a sum of at most 128 levels
// of 15 stays below 2^15. Everything else (build, scale, offset, limits,
// top-k) is the 8-bit kernel's, with eight slots; the warps keep 32-entry
// lists (k <= 32).
constexpr int kNSlots = 8;
using NItem = GItemT<kNSlots>;

// Register and half of slot s's 16-bit sum lane (and limit lane).
__device__ __forceinline__ int nib_reg(int s) { return 2 * (s & 1) + ((s >> 1) & 1); }
__device__ __forceinline__ int nib_half(int s) { return s >> 2; }

template <int K, int NCHUNK>
__device__ __forceinline__ void nibble_acc(uint32_t base, const uint4 (&w)[NCHUNK], uint32_t& lo, uint32_t& hi) {
  const uint32_t x = code_word<K & ~3, NCHUNK>(w);
  const uint32_t code = __byte_perm(x, 0u, 0x4440u + (K & 3));
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1+%2];" : "=r"(v) : "r"(base + code * 4u), "n"(K * 1024));
  lo += v & 0x0F0F0F0Fu;          // slots 0, 2, 4, 6 as byte lanes
  hi += (v >> 4) & 0x0F0F0F0Fu;   // slots 1, 3, 5, 7
}
template <int NCHUNK, int C, int... J>
__device__ __forceinline__ void nibble_chunk(uint32_t base, const uint4 (&w)[NCHUNK], uint32_t (&W)[4],
                                             std::integer_sequence<int, J...>) {
  uint32_t lo = 0u, hi = 0u;
  (nibble_acc<C * 16 + J, NCHUNK>(base, w, lo, hi), ...);
  W[0] += __byte_perm(lo, 0u, 0x4240u);
  W[1] += __byte_perm(lo, 0u, 0x4341u);
  W[2] += __byte_perm(hi, 0u, 0x4240u);
  W[3] += __byte_perm(hi, 0u, 0x4341u);
}
template <int NCHUNK, int... C>
__device__ __forceinline__ void adc_nibble_seq(uint32_t base, const uint4 (&w)[NCHUNK], uint32_t (&W)[4],
                                               std::integer_sequence<int, C...>) {
  (nibble_chunk<NCHUNK, C>(base, w, W, std::make_integer_sequence<int, 16>{}), ...);
}

// Shared memory of the nibble kernel: the row statistics (bias, rowmax) live
// in the space of the warps' top-k lists, which start only after the levels
// are written (three blocks per SM at 48 sub-spaces).
struct NLayout {
  size_t tab, scal, item, lim, md, mi, bias, rowmax, total;
  __host__ __device__ explicit NLayout(int Mp) {
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t o = 0;
    tab = o; o += al((size_t)Mp * kKsub * 4);
    scal = o; o += al(sizeof(SlotScal) * kNSlots);
    item = o; o += al(2 * sizeof(GItemT<kNSlots>));
    lim = o; o += al(4 * 4);
    md = o;
    const size_t lists = al((size_t)kNSlots * kGWarps * 32 * 4) + al((size_t)kNSlots * kGWarps * 32 * 8);
    const size_t stats = 2 * al((size_t)kNSlots * Mp * 4);
    mi = md + al((size_t)kNSlots * kGWarps * 32 * 4);
    bias = md;
    rowmax = md + al((size_t)kNSlots * Mp * 4);
    o += lists > stats ? lists : stats;
    total = o + 256;
  }
};

template <int NCHUNK>
__global__ void __launch_bounds__(kGThreads, NCHUNK <= 4 ? 3 : 1) nibble_kernel(const GArgs a) {
  constexpr int Mp = NCHUNK * 16;
  const NLayout L(Mp);
  const uint32_t raw = smem_addr(anns_dyn_smem);
  const uint32_t pad = (256u - (raw & 255u)) & 255u;
  unsigned char* base = anns_dyn_smem + pad;
  uint32_t* tab = (uint32_t*)(base + L.tab);
  float* bias = (float*)(base + L.bias);
  float* rowmax = (float*)(base + L.rowmax);
  SlotScal* scal = (SlotScal*)(base + L.scal);
  NItem* items = (NItem*)(base + L.item);
  uint32_t* lim = (uint32_t*)(base + L.lim);  // 0x8000 + Smax per slot in the lanes of W0..W3
  float* md = (float*)(base + L.md);
  int64_t* mi = (int64_t*)(base + L.mi);
  const uint32_t tab_addr = raw + pad + (uint32_t)L.tab;
  const uint32_t lim_addr = raw + pad + (uint32_t)L.lim;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ngroups = a.ioff[a.nb];
  const size_t tstride = (size_t)Mp * kKsub;
  int cur = 0;
  if (warp == kGWarps - 1) fetch_group<kNSlots>(a, ngroups, items, lane);
  for (;;) {
    __syncthreads();  // the previous group is done with the shared tables; items[cur] is complete
    if (threadIdx.x < 4) lim[threadIdx.x] = 0xFFFFFFFFu;  // every sum passes until the seeds
    const NItem& G = items[cur];
    if (G.it >= ngroups) break;
    const int l = G.l, ns = G.ns;
    int q[kNSlots];
#pragma unroll
    for (int s = 0; s < kNSlots; ++s) q[s] = G.q[s];
    const float* P = a.ltab + (size_t)l * tstride;
    // 1. row statistics of the eight slots (the list-table row loaded once)
    for (int m = warp; m < a.M; m += kGWarps) {
      float p[8], lo_v[kNSlots], hi_v[kNSlots];
      ldg_row8(P + m * kKsub, lane, p);
#pragma unroll
      for (int s0 = 0; s0 < kNSlots; s0 += 2) {
        if (s0 >= ns) {  // absent slots (the group's uniform count): nothing to read
          lo_v[s0] = hi_v[s0] = lo_v[s0 + 1] = hi_v[s0 + 1] = 0.f;
          continue;
        }
        float qq[2][8];
#pragma unroll
        for (int u = 0; u < 2; ++u) ldg_row8(a.qt + (size_t)q[s0 + u] * tstride + m * kKsub, lane, qq[u]);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int s = s0 + u;
          lo_v[s] = hi_v[s] = sub_rn(p[0], qq[u][0]);
#pragma unroll
          for (int e = 1; e < 8; ++e) {
            const float tv = sub_rn(p[e], qq[u][e]);
            lo_v[s] = fminf(lo_v[s], tv);
            hi_v[s] = fmaxf(hi_v[s], tv);
          }
        }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1)
#pragma unroll
        for (int s = 0; s < kNSlots; ++s) {
          lo_v[s] = fminf(lo_v[s], __shfl_xor_sync(kFull, lo_v[s], o));
          hi_v[s] = fmaxf(hi_v[s], __shfl_xor_sync(kFull, hi_v[s], o));
        }
#pragma unroll
      for (int s = 0; s < kNSlots; ++s)
        if (lane == 0 && s < ns) { bias[s * Mp + m] = lo_v[s]; rowmax[s * Mp + m] = sub_rn(hi_v[s], lo_v[s]); }
    }
    __syncthreads();
    // 2. per slot (warp s): step, scale, offset (exact sum), k, bound and the limit seed
    {
      const int s = warp;
      float range = 0.f;
      const int p = G.pid[s], bs = G.bits[s];
      const float d2 = G.d2[s];
      if (s < ns) {
        for (int m = lane; m < a.M; m += 32) range = fmaxf(range, rowmax[s * Mp + m]);
        range = warp_max(range);
      }
      const float B32 = slot_offset(bias + s * Mp, a.M, d2, s < ns);
      const int Lv = (1 << bs) - 1;
      SlotScal sc;
      sc.s32 = range > 0.f ? __fdiv_rn((float)Lv, range) : 0.f;
      sc.delta32 = range > 0.f ? __fdiv_rn(range, (float)Lv) : 0.f;
      sc.B32 = B32;
      sc.kq = s < ns ? G.kq[s] : 0;
      sc.bound = sc.kq > 0 ? G.bound[s] : INFINITY;
      sc.pid = p;
      sc.pad0 = sc.pad1 = 0;
      const int seed = sc.kq == 0 ? -1 : (sc.bound == INFINITY ? 0x7FFF : smax_warp(sc.bound, sc.delta32, sc.B32));
      if (lane == 0) {
        scal[s] = sc;
        lim_min_at(lim, nib_reg(s), nib_half(s), (uint32_t)(0x8000 + seed));
      }
    }
    __syncthreads();
    // 3. interleaved levels: nibble s of entry e's word = slot s's level (<= 15)
    float s32[kNSlots];
#pragma unroll
    for (int s = 0; s < kNSlots; ++s) s32[s] = s < ns ? scal[s].s32 : 0.f;
    for (int m = warp; m < Mp; m += kGWarps) {
      uint32_t wv[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) wv[e] = 0u;
      if (m < a.M) {
        float p[8];
        ldg_row8(P + m * kKsub, lane, p);
#pragma unroll
        for (int s = 0; s < kNSlots; ++s) {
          if (s < ns) {
            float qq[8];
            ldg_row8(a.qt + (size_t)q[s] * tstride + m * kKsub, lane, qq);
            const float mn = bias[s * Mp + m];
#pragma unroll
            for (int e = 0; e < 8; ++e)
              wv[e] |= (rint_bits_g(mul_rn(sub_rn(sub_rn(p[e], qq[e]), mn), s32[s])) & 0xFu) << (4 * s);
          }
        }
      }
      *(uint4*)(tab + m * kKsub + row_at(lane, 0)) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
      *(uint4*)(tab + m * kKsub + row_at(lane, 1)) = make_uint4(wv[4], wv[5], wv[6], wv[7]);
    }
    __syncthreads();
    // the warps' top-k lists start empty (over the row statistics, no longer needed)
#pragma unroll
    for (int s = 0; s < kNSlots; ++s) {
      md[(s * kGWarps + warp) * 32 + lane] = INFINITY;
      mi[(s * kGWarps + warp) * 32 + lane] = INT64_MAX;
    }
    __syncthreads();
    // 4. scan: four 32-bit sum registers hold the eight slots' 16-bit lanes;
    //    lim holds 0x8000 + Smax in the same lanes (one integer test per lane)
    const int n_l = G.n_l;
    const int ntile = (n_l + kTileVecs - 1) / kTileVecs;
    const size_t tile_bytes = (size_t)NCHUNK * kTileChunkBytes;
    const uint8_t* tp = a.codes + (size_t)G.tile0 * tile_bytes + (size_t)warp * tile_bytes + lane * kChunkBytes;
    const int64_t* idp = a.ids + G.vec0;
    if (warp == kGWarps - 1) fetch_group<kNSlots>(a, ngroups, items + (cur ^ 1), lane);
    uint4 w[NCHUNK];
    if (warp < ntile) load_codes<NCHUNK>(tp, w);
    for (int t = warp; t < ntile; t += kGWarps) {
      uint4 wn[NCHUNK];
      const bool more = t + kGWarps < ntile;
      if (more) load_codes<NCHUNK>(tp + kGWarps * tile_bytes, wn);
      uint32_t W[4] = {0u, 0u, 0u, 0u};
      adc_nibble_seq<NCHUNK>(tab_addr, w, W, std::make_integer_sequence<int, NCHUNK>{});
      uint32_t lv[4];
      asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                   : "=r"(lv[0]), "=r"(lv[1]), "=r"(lv[2]), "=r"(lv[3]) : "r"(lim_addr));
      uint32_t pass[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) pass[r] = (lv[r] - W[r]) & 0x80008000u;
      const int v = t * kTileVecs + lane;
      const bool any = v < n_l && (pass[0] | pass[1] | pass[2] | pass[3]) != 0u;
      if (__any_sync(kFull, any)) {
        const int64_t id = any ? __ldg(idp + v) : INT64_MAX;
#pragma unroll
        for (int s = 0; s < kNSlots; ++s) {
          const int rg = nib_reg(s), hf = nib_half(s);
          const bool ok = any && ((pass[rg] >> (hf * 16 + 15)) & 1u);
          if (__any_sync(kFull, ok)) {
            const SlotScal sc = scal[s];
            float* ld = md + (s * kGWarps + warp) * 32;
            int64_t* li = mi + (s * kGWarps + warp) * 32;
            WarpTopK<1, int64_t> top;
            top.d[0] = ld[lane];
            top.id[0] = li[lane];
            float thd = ld[sc.kq - 1];
            int64_t thi = li[sc.kq - 1];
            if (sc.bound < thd) { thd = sc.bound; thi = INT64_MAX; }
            const float d = add_rn(mul_rn(sc.delta32, __int2float_rn((int)((W[rg] >> (hf * 16)) & 0xFFFFu))),
                                   sc.B32);
            top.offer(ok, d, id, sc.kq, thd, thi);
            if (sc.bound < thd) thd = sc.bound;
            ld[lane] = top.d[0];
            li[lane] = top.id[0];
            if (thd != INFINITY) {
              const int sm = smax_warp(thd, sc.delta32, sc.B32);
              if (lane == 0) lim_min_at(lim, rg, hf, (uint32_t)(0x8000 + sm));
            }
            __syncwarp();
          }
        }
      }
      if (more) {
#pragma unroll
        for (int c = 0; c < NCHUNK; ++c) w[c] = wn[c];
      }
      tp += kGWarps * tile_bytes;
    }
    __syncthreads();
    // merge the warps' lists per slot; warp s writes slot s
    if (warp < ns) {
      const int s = warp;
      const SlotScal sc = scal[s];
      WarpTopK<1, int64_t> m;
      m.init();
      float th = INFINITY;
      int64_t ti = INT64_MAX;
      for (int w2 = 0; w2 < kGWarps && sc.kq > 0; ++w2) {
        const float cd = md[(s * kGWarps + w2) * 32 + lane];
        const int64_t ci = mi[(s * kGWarps + w2) * 32 + lane];
        m.offer(cd != INFINITY, cd, ci, sc.kq, th, ti);
      }
      if (lane < a.k) {
        const bool ok = lane < sc.kq && m.d[0] != INFINITY;
        a.part_d[(size_t)sc.pid * a.k + lane] = ok ? m.d[0] : INFINITY;
        a.part_i[(size_t)sc.pid * a.k + lane] = ok ? m.id[0] : -1;
      }
    }
    cur ^= 1;
  }
}

// One warp per query: the k smallest (d, id) over the query-major partial
// top-k (wide pairs) and the partial top-k of the query's narrow pairs.
template <int R>
__global__ void __launch_bounds__(256) merge_grouped_kernel(
    const float* __restrict__ qm_d, const int64_t* __restrict__ qm_i, const float* __restrict__ part_d,
    const int64_t* __restrict__ part_i, const int32_t* __restrict__ probes, const uint8_t* __restrict__ bits,
    const int32_t* __restrict__ npq, const int32_t* __restrict__ kpq, int64_t nq, int nprobe, int k,
    int64_t* __restrict__ ids_out, float* __restrict__ dists_out) {
  const int64_t q = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (q >= nq) return;
  const int np = npq ? min(max(npq[q], 0), nprobe) : nprobe;
  const int kq = kpq ? min(max(kpq[q], 0), k) : k;
  WarpTopK<R, int64_t> top;
  top.init();
  float thd = INFINITY;
  int64_t thi = INT64_MAX;
  if (kq > 0)
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int e = r * 32 + lane;
      const bool in = e < kq;
      const float d = in ? qm_d[q * k + e] : INFINITY;
      const int64_t id = in ? qm_i[q * k + e] : -1;
      top.offer(in && id >= 0, d, id, kq, thd, thi);
    }
  for (int j = 0; kq > 0 && j < np; ++j) {
    const int64_t pid = q * nprobe + j;
    const int b = bits[pid];
    if (j == 0 || probes[pid] < 0 || b < 1 || b > 8) continue;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int e = r * 32 + lane;
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

inline int grouped_R(int k) { return k <= 32 ? 1 : 4; }

template <int NCHUNK, int R>
cudaError_t run_packed_r(const GArgs& a, cudaStream_t s) {
  auto kern = packed_kernel<NCHUNK, R>;
  const GLayout L(NCHUNK * 16, R);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGThreads, L.total);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  kern<<<sms * per_sm, kGThreads, L.total, s>>>(a); note_launch();
  return cudaGetLastError();
}

template <int NCHUNK>
cudaError_t run_packed(const GArgs& a, cudaStream_t s) {
  return grouped_R(a.k) == 1 ? run_packed_r<NCHUNK, 1>(a, s) : run_packed_r<NCHUNK, 4>(a, s);
}

template <int NCHUNK>
cudaError_t run_nibble(const GArgs& a, cudaStream_t s) {
  auto kern = nibble_kernel<NCHUNK>;
  const NLayout L(NCHUNK * 16);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGThreads, L.total);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  kern<<<sms * per_sm, kGThreads, L.total, s>>>(a); note_launch();
  return cudaGetLastError();
}

// The 4-bit pairs take the nibble kernel when the warps' lists are 32 wide
// (k <= 32), the option is on and its shared memory fits.
bool nibble_used(const Index& ix, int k) {
  if (!ix.opt_nibble || grouped_R(k) != 1) return false;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return NLayout((int)ix.Mp).total <= (size_t)optin;
}

}  // namespace

bool grouped_supported(const Index& ix, int k) {
  if (k > 128) return false;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return GLayout((int)ix.Mp, grouped_R(k)).total <= (size_t)optin;
}

size_t grouped_workspace_bytes(int64_t nq, int k) { return (size_t)nq * k * 12 + 256; }

int64_t grouped_qchunk(const Index& ix, int64_t nq) {
  if (ix.opt_qchunk > 0) return std::min<int64_t>(ix.opt_qchunk, std::max<int64_t>(nq, 1));
  int dev = 0, l2 = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
  const int64_t qt_bytes = ix.Mp * kKsub * 4;  // one query's tables
  const int64_t shared = ix.nlist * qt_bytes + ix.ntiles * ix.nchunk * kTileChunkBytes;  // list tables + codes
  if (nq <= 0 || l2 <= 0 || shared > l2 / 2) return std::max<int64_t>(nq, 1);
  // half of L2 for the current chunk's query tables (measured on the SIFT-shaped
  // workload: a quarter and an eighth are slower)
  return std::min<int64_t>(nq, std::max<int64_t>(256, (l2 / 2) / qt_bytes));
}

cudaError_t launch_search_grouped(const Index& ix, const float* qt, int64_t nq, int nprobe,
                                  const int32_t* nprobe_per_q, int k, const int32_t* k_per_q,
                                  const int32_t* probes, const float* probe_d2, const uint8_t* bits,
                                  const ListWork& w, void* qm_ws, int64_t* ids_out, float* dists_out,
                                  cudaStream_t s, cudaEvent_t after_qm, cudaEvent_t after_packed,
                                  cudaEvent_t after_nibble, const int32_t* qm_order) {
  // narrow pairs regrouped by list, largest lists first: the pairs on tables
  // of 5..8 bits in groups of four, those of 1..4 bits in groups of eight
  // (or all 1..8-bit pairs in groups of four without the nibble kernel)
  const bool nib = nibble_used(ix, k);
  ListWork w4 = w;
  w4.cnt = w.cnt4; w4.off = w.off4; w4.ioff = w.ioff4; w4.fill = w.fill4; w4.pairs = w.pairs4;
  w4.gtab = w.gtab4; w4.counter = w.counter4;
  cudaError_t e = launch_invert(ix, probes, nprobe_per_q, nq, nprobe, kSlots, w, s, bits, nib ? 5 : 1, 8);
  if (e != cudaSuccess) return e;
  if (nib) {
    e = launch_invert(ix, probes, nprobe_per_q, nq, nprobe, kNSlots, w4, s, bits, 1, 4);
    if (e != cudaSuccess) return e;
  }
  e = cudaMemsetAsync(w.counter, 0, 16 * sizeof(int), s);  // both queues' counters
  if (e != cudaSuccess) return e;
  // rank 0 and the wide pairs, query-major, into a partial top-k per query
  float* qm_d = (float*)qm_ws;
  int64_t* qm_i = (int64_t*)((char*)qm_ws + (((size_t)nq * k * 4 + 255) & ~size_t(255)));
  e = launch_search(ix, qt, nq, nprobe, nprobe_per_q, k, k_per_q, probes, probe_d2, bits, qm_order, qm_i, qm_d, s,
                    true);
  if (e != cudaSuccess) return e;
  if (after_qm) cudaEventRecord(after_qm, s);
  GArgs a{};
  a.qt = qt; a.ltab = ix.ltab; a.probe_d2 = probe_d2; a.bits = bits;
  a.codes = ix.codes; a.ids = ix.ids; a.list_len = ix.list_len; a.vec_off = ix.vec_off;
  a.tile_off = ix.tile_off; a.order = ix.order; a.cnt = w.cnt; a.off = w.off; a.ioff = w.ioff;
  a.pairs = w.pairs; a.gtab = w.gtab; a.nlist = (int)ix.nlist; a.nb = w.nbuckets;
  a.M = (int)ix.M; a.Mp = (int)ix.Mp; a.nprobe = nprobe; a.k = k;
  a.kpq = k_per_q; a.part_d = w.part_d; a.part_i = w.part_i; a.counter = w.counter; a.qm_d = qm_d;
  switch (ix.nchunk) {
    case 1: e = run_packed<1>(a, s); break;
    case 2: e = run_packed<2>(a, s); break;
    case 3: e = run_packed<3>(a, s); break;
    case 4: e = run_packed<4>(a, s); break;
    case 5: e = run_packed<5>(a, s); break;
    case 6: e = run_packed<6>(a, s); break;
    case 7: e = run_packed<7>(a, s); break;
    default: e = run_packed<8>(a, s); break;
  }
  if (e != cudaSuccess) return e;
  if (after_packed) cudaEventRecord(after_packed, s);
  if (nib) {
    GArgs b = a;
    b.cnt = w4.cnt; b.off = w4.off; b.ioff = w4.ioff; b.pairs = w4.pairs; b.gtab = w4.gtab; b.counter = w4.counter;
    switch (ix.nchunk) {
      case 1: e = run_nibble<1>(b, s); break;
      case 2: e = run_nibble<2>(b, s); break;
      case 3: e = run_nibble<3>(b, s); break;
      case 4: e = run_nibble<4>(b, s); break;
      case 5: e = run_nibble<5>(b, s); break;
      case 6: e = run_nibble<6>(b, s); break;
      case 7: e = run_nibble<7>(b, s); break;
      default: e = run_nibble<8>(b, s); break;
    }
    if (e != cudaSuccess) return e;
  }
  if (after_nibble) cudaEventRecord(after_nibble, s);
  if (grouped_R(k) == 1)
    merge_grouped_kernel<1><<<(unsigned)((nq + 7) / 8), 256, 0, s>>>(qm_d, qm_i, w.part_d, w.part_i, probes, bits,
                                                                   nprobe_per_q, k_per_q, nq, nprobe, k, ids_out,
                                                                   dists_out);
  else
    merge_grouped_kernel<4><<<(unsigned)((nq + 7) / 8), 256, 0, s>>>(qm_d, qm_i, w.part_d, w.part_i, probes, bits,
                                                                   nprobe_per_q, k_per_q, nq, nprobe, k, ids_out,
                                                                   dists_out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace anns
