// Device helpers shared by the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>
#include <cmath>

// The block's dynamic shared memory; every kernel carves its own layout from it.
extern __shared__ __align__(16) unsigned char anns_dyn_smem[];

namespace anns {

constexpr unsigned kFull = 0xffffffffu;

template <typename T> struct IdMax;
template <> struct IdMax<int32_t> { static __device__ __forceinline__ int32_t v() { return INT32_MAX; } };
template <> struct IdMax<int64_t> { static __device__ __forceinline__ int64_t v() { return INT64_MAX; } };

// Strict order on (distance, id): the tie rule of the top-k selection.
template <typename DT, typename IdT>
__device__ __forceinline__ bool key_less(DT d1, IdT i1, DT d2, IdT i2) {
  return d1 < d2 || (d1 == d2 && i1 < i2);
}

// Largest value of a distance type: the empty entry of a top-k list.
template <typename DT> struct DMax;
template <> struct DMax<float> { static __device__ __forceinline__ float v() { return INFINITY; } };
template <> struct DMax<uint32_t> { static __device__ __forceinline__ uint32_t v() { return 0xFFFFFFFFu; } };

// A warp-wide sorted list of the R*32 smallest (distance, id) keys seen so far
// (the priority queue of the TSM, Section 4.1, initialised to the maximum).
// Entry e = r*32 + lane lives in register slot r of lane `lane`; entries are
// ascending in e. All methods must be called by the whole warp with
// warp-uniform arguments. DT is the distance type (FP32, or exact integer
// distances).
template <int R, typename IdT, typename DT = float>
struct WarpTopK {
  DT d[R];
  IdT id[R];

  __device__ __forceinline__ void init() {
#pragma unroll
    for (int r = 0; r < R; ++r) { d[r] = DMax<DT>::v(); id[r] = IdMax<IdT>::v(); }
  }

  // Entry e (warp-uniform e < R*32), broadcast to all lanes.
  __device__ __forceinline__ void get(int e, DT& od, IdT& oid) const {
    DT vd = d[0];
    IdT vi = id[0];
#pragma unroll
    for (int r = 1; r < R; ++r) if ((e >> 5) == r) { vd = d[r]; vi = id[r]; }
    od = __shfl_sync(kFull, vd, e & 31);
    oid = __shfl_sync(kFull, vi, e & 31);
  }

  // Inserts (cd, cid) in order; the last entry falls off.
  __device__ __forceinline__ void insert(DT cd, IdT cid) {
    const int lane = threadIdx.x & 31;
    int pos = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) pos += __popc(__ballot_sync(kFull, key_less(d[r], id[r], cd, cid)));
#pragma unroll
    for (int r = R - 1; r >= 0; --r) {
      DT ud = __shfl_up_sync(kFull, d[r], 1);
      IdT ui = __shfl_up_sync(kFull, id[r], 1);
      if (r > 0) {
        DT cdd = __shfl_sync(kFull, d[r - 1], 31);
        IdT cii = __shfl_sync(kFull, id[r - 1], 31);
        if (lane == 0) { ud = cdd; ui = cii; }
      }
      const int g = r * 32 + lane;
      if (g == pos) { d[r] = cd; id[r] = cid; }
      else if (g > pos) { d[r] = ud; id[r] = ui; }
    }
  }

  // Offers one candidate per lane (valid lanes only); keeps the k smallest.
  // thd/thi hold entry k-1 on entry and are updated.
  __device__ __forceinline__ void offer(bool valid, DT cd, IdT cid, int k, DT& thd, IdT& thi) {
    unsigned mask = __ballot_sync(kFull, valid && key_less(cd, cid, thd, thi));
    while (mask) {
      const int src = __ffs(mask) - 1;
      mask &= mask - 1;
      const DT bd = __shfl_sync(kFull, cd, src);
      const IdT bi = __shfl_sync(kFull, cid, src);
      if (key_less(bd, bi, thd, thi)) {
        insert(bd, bi);
        get(k - 1, thd, thi);
      }
    }
  }
};

// Explicitly rounded FP32 operations (no contraction into FMA): the library
// follows the oracle's FP32 rules operation by operation.
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }


// ---- exact sum of FP32 values, rounded once --------------------------------
// Every finite FP32 value is an integer multiple of 2^-149 of magnitude below
// 2^277 * 2^-149, so a sum of them is N * 2^-149 with an integer N. N is held
// as nine base-2^32 digits, each in a 64-bit accumulator whose carries are
// propagated only once, at the end (a digit receives at most two 32-bit
// pieces per value, so fewer than 2^31 values fit). A sum with |N| >= 2^287
// is beyond the FP32 range and rounds to infinity. Integer addition is
// associative, so lanes may add their values in any order and combine by any
// reduction tree: the rounded result is the exact sum's nearest FP32 value
// (ties to even), whatever the order. Non-finite values are summed apart in
// FP32 and, if any occurs, are the result (IEEE inf/NaN propagation).
struct ExactSum {
  long long d[9];
  float nonfinite;
  bool any_nonfinite;
};

__device__ __forceinline__ void xsum_init(ExactSum& a) {
#pragma unroll
  for (int k = 0; k < 9; ++k) a.d[k] = 0;
  a.nonfinite = 0.f;
  a.any_nonfinite = false;
}

__device__ __forceinline__ void xsum_add(ExactSum& a, float v) {
  const uint32_t u = __float_as_uint(v);
  const uint32_t e = (u >> 23) & 0xffu;
  if (e == 0xffu) {
    a.nonfinite = __fadd_rn(a.nonfinite, v);
    a.any_nonfinite = true;
    return;
  }
  // v = sig * 2^(p - 149): sig carries the hidden bit of a normal value, and a
  // subnormal (e = 0) has the position of e = 1 without it
  const uint32_t sig = e ? ((u & 0x7fffffu) | 0x800000u) : (u & 0x7fffffu);
  const int p = e ? (int)e - 1 : 0;
  const unsigned long long w = (unsigned long long)sig << (p & 31);
  const long long lo = (long long)(w & 0xffffffffull), hi = (long long)(w >> 32);
  const int i = p >> 5;  // 0..7: the low piece goes to digit i, the high one to i + 1
  const bool neg = (u >> 31) != 0u;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const long long c = (k == i ? lo : 0ll) + (k == i + 1 ? hi : 0ll);
    a.d[k] += neg ? -c : c;
  }
}

// Sum over the warp's lanes (butterfly; every lane ends with the total).
__device__ __forceinline__ void xsum_warp(ExactSum& a) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
#pragma unroll
    for (int k = 0; k < 9; ++k) a.d[k] += __shfl_xor_sync(0xffffffffu, a.d[k], o);
    a.nonfinite = __fadd_rn(a.nonfinite, __shfl_xor_sync(0xffffffffu, a.nonfinite, o));
    a.any_nonfinite = __any_sync(0xffffffffu, a.any_nonfinite);
  }
}

// The accumulated exact sum rounded to the nearest FP32 value, ties to even.
__device__ __forceinline__ float xsum_round(const ExactSum& a) {
  if (a.any_nonfinite) return a.nonfinite;
  // carry propagation: N = c * 2^288 + sum_k g[k] 2^(32k), c in {0, -1}
  uint32_t g[9];
  long long c = 0;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const long long t = a.d[k] + c;
    g[k] = (uint32_t)(t & 0xffffffffll);
    c = t >> 32;  // arithmetic shift: the floor of t / 2^32
  }
  // |N| >= 2^288 (a carry beyond the top digit): the value exceeds 2^139, far
  // past the largest FP32 value, so it rounds to infinity of its sign
  if (c > 0) return INFINITY;
  if (c < -1) return -INFINITY;
  const bool neg = c < 0;
  if (neg) {  // |N| = two's complement of the 288-bit pattern
    unsigned long long carry = 1;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const unsigned long long t = (unsigned long long)(~g[k]) + carry;
      g[k] = (uint32_t)t;
      carry = t >> 32;
    }
  }
  int h = -1;  // the highest non-zero digit
#pragma unroll
  for (int k = 0; k < 9; ++k)
    if (g[k] != 0u) h = k;
  if (h < 0) return 0.f;
  uint32_t t0 = 0u, t1 = 0u, t2 = 0u;
  bool sticky = false;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    if (k == h) t0 = g[k];
    if (k == h - 1) t1 = g[k];
    if (k == h - 2) t2 = g[k];
    if (k < h - 2 && g[k] != 0u) sticky = true;
  }
  const int lz = __clz(t0);
  const int top = 32 * h + 31 - lz;  // bit index of the leading one of |N|
  uint32_t bits;
  if (top < 24) {
    // |N| < 2^24: exact in FP32, and N * 2^-149 has the bit pattern N (a
    // subnormal below 2^23; exponent field 1 from 2^23 on)
    bits = t0;
  } else {
    unsigned long long W = ((unsigned long long)t0 << 32) | t1;  // digits h, h-1
    uint32_t rest = t2;
    if (lz) {
      W = (W << lz) | (t2 >> (32 - lz));
      rest = t2 << lz;
    }
    // W holds bits top .. top-63 of |N|, leading one at bit 63
    uint32_t mant = (uint32_t)(W >> 40);
    const bool half = ((W >> 39) & 1ull) != 0ull;
    sticky = sticky || rest != 0u || (W & ((1ull << 39) - 1ull)) != 0ull;
    int E = top - 22;  // mant * 2^(top - 23 - 149) = 1.f * 2^(E - 127)
    if (half && (sticky || (mant & 1u))) {
      ++mant;
      if (mant == (1u << 24)) { mant >>= 1; ++E; }
    }
    bits = E >= 255 ? 0x7f800000u : (((uint32_t)E << 23) | (mant & 0x7fffffu));
  }
  return __uint_as_float(bits | (neg ? 0x80000000u : 0u));
}

// The exact sum of v[0..n) (lanes striding) and, if with_extra, `extra`
// (added by lane 0), rounded once to FP32; every lane gets the result. Fast
// path: when the nonzero values' lowest set-bit positions (LSB weights
// 2^(p-149), p = max(exponent field, 1) - 1) span at most 21 positions, any
// partial sum of up to 256 of them is a multiple of the smallest weight below
// 2^(21 + 24 + 8) of it, so every FP64 addition is exact and one FP64 -> FP32
// conversion is the single rounding; otherwise (or with a non-finite value)
// the fixed-point accumulator above.
__device__ __forceinline__ float warp_exact_sum(const float* v, int n, float extra, bool with_extra) {
  const int lane = threadIdx.x & 31;
  int pmin = 0x7fffffff, pmax = -1;
  bool odd = false;
  auto look = [&](float x) {
    const uint32_t u = __float_as_uint(x);
    const int e = (int)((u >> 23) & 0xffu);
    if (e == 0xff) { odd = true; return; }
    if ((u & 0x7fffffffu) == 0u) return;
    const int p = e ? e - 1 : 0;
    pmin = min(pmin, p);
    pmax = max(pmax, p);
  };
  for (int i = lane; i < n; i += 32) look(v[i]);
  if (with_extra && lane == 0) look(extra);
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    pmin = min(pmin, __shfl_xor_sync(0xffffffffu, pmin, o));
    pmax = max(pmax, __shfl_xor_sync(0xffffffffu, pmax, o));
  }
  odd = __any_sync(0xffffffffu, odd);
  if (!odd && n < 256 && (pmax < 0 || pmax - pmin <= 21)) {
    double acc = 0.0;
    for (int i = lane; i < n; i += 32) acc = __dadd_rn(acc, (double)v[i]);
    if (with_extra && lane == 0) acc = __dadd_rn(acc, (double)extra);
#pragma unroll
    for (int o = 16; o; o >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
    return __double2float_rn(acc);
  }
  ExactSum B;
  xsum_init(B);
  for (int i = lane; i < n; i += 32) xsum_add(B, v[i]);
  if (with_extra && lane == 0) xsum_add(B, extra);
  xsum_warp(B);
  return xsum_round(B);
}

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// The 8 entries of a 256-entry table row that lane i of a warp handles:
// 4i..4i+3 (half 0) and 128+4i..128+4i+3 (half 1). Each of the warp's two
// 16-byte accesses then covers 512 contiguous bytes: whole sectors from
// global memory, no bank conflicts in shared memory.
__device__ __forceinline__ int row_at(int lane, int h) { return h * 128 + lane * 4; }

// Entries of row `row` (256 floats) for `lane` in the order above.
__device__ __forceinline__ void ldg_row8(const float* __restrict__ row, int lane, float (&v)[8]) {
  const float4 a = __ldg((const float4*)(row + row_at(lane, 0)));
  const float4 b = __ldg((const float4*)(row + row_at(lane, 1)));
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// Writes 8 floats of row `row` (shared or global) for `lane`, same order.
__device__ __forceinline__ void st_row8(float* row, int lane, const float (&v)[8]) {
  *(float4*)(row + row_at(lane, 0)) = make_float4(v[0], v[1], v[2], v[3]);
  *(float4*)(row + row_at(lane, 1)) = make_float4(v[4], v[5], v[6], v[7]);
}

}  // namespace anns
