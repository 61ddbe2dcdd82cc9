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
template <typename IdT>
__device__ __forceinline__ bool key_less(float d1, IdT i1, float d2, IdT i2) {
  return d1 < d2 || (d1 == d2 && i1 < i2);
}

// A warp-wide sorted list of the R*32 smallest (distance, id) keys seen so far
// (the priority queue of the TSM, Section 4.1, initialised to the maximum).
// Entry e = r*32 + lane lives in register slot r of lane `lane`; entries are
// ascending in e. All methods must be called by the whole warp with
// warp-uniform arguments.
template <int R, typename IdT>
struct WarpTopK {
  float d[R];
  IdT id[R];

  __device__ __forceinline__ void init() {
#pragma unroll
    for (int r = 0; r < R; ++r) { d[r] = INFINITY; id[r] = IdMax<IdT>::v(); }
  }

  // Entry e (warp-uniform e < R*32), broadcast to all lanes.
  __device__ __forceinline__ void get(int e, float& od, IdT& oid) const {
    float vd = d[0];
    IdT vi = id[0];
#pragma unroll
    for (int r = 1; r < R; ++r) if ((e >> 5) == r) { vd = d[r]; vi = id[r]; }
    od = __shfl_sync(kFull, vd, e & 31);
    oid = __shfl_sync(kFull, vi, e & 31);
  }

  // Inserts (cd, cid) in order; the last entry falls off.
  __device__ __forceinline__ void insert(float cd, IdT cid) {
    const int lane = threadIdx.x & 31;
    int pos = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) pos += __popc(__ballot_sync(kFull, key_less(d[r], id[r], cd, cid)));
#pragma unroll
    for (int r = R - 1; r >= 0; --r) {
      float ud = __shfl_up_sync(kFull, d[r], 1);
      IdT ui = __shfl_up_sync(kFull, id[r], 1);
      if (r > 0) {
        float cdd = __shfl_sync(kFull, d[r - 1], 31);
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
  __device__ __forceinline__ void offer(bool valid, float cd, IdT cid, int k, float& thd, IdT& thi) {
    unsigned mask = __ballot_sync(kFull, valid && key_less(cd, cid, thd, thi));
    while (mask) {
      const int src = __ffs(mask) - 1;
      mask &= mask - 1;
      const float bd = __shfl_sync(kFull, cd, src);
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
