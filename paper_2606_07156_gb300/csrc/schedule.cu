// Greedy load scheduling of the query-major search (the analogue of the
// load-scheduling module of Section 4.3, applied to whole queries): queries
// are dispatched longest first, so that the expensive ones do not form the
// tail of a batch with uneven nprobe or skewed list sizes.
//
// The estimated cost of query q is, over the pairs the query-major kernel
// scans (all of them, or in the grouped search only rank 0 and the pairs on
// FP32, 12- or 16-bit tables), the sum of n_l * g(b) + kBuild: the list's
// lookups weighted by the width's gather cost g (3 for a 32-bit FP32 or
// 16-bit entry, 2 for a byte entry: the shared-memory wavefronts a random
// warp gather takes, measured on this GPU) plus the LUT build counted as
// kBuild such lookups (a build writes 256 entries per sub-space, each a few
// times the work of one lookup). The factor M is common to all queries and
// left out. Queries are bucketed by the leading 12 bits
// of the FP32 cost (exponent and 3 mantissa bits, i.e. within 12.5 %) and
// ordered by bucket, most expensive first, by a counting sort. The order
// within a bucket is unspecified; the results of a query do not depend on
// when it runs.
#include "common.cuh"
#include "internal.h"

namespace anns {
namespace {

constexpr int kBuckets = 4096;
constexpr int kBuild = 1536;

__device__ __forceinline__ int gather_cost(int b) { return (b >= 1 && b <= 8) ? 2 : 3; }

__global__ void cost_key_kernel(const int32_t* __restrict__ probes, const int32_t* __restrict__ npq,
                                const int32_t* __restrict__ list_len, const uint8_t* __restrict__ bits,
                                int skip_narrow, int64_t nq, int nprobe, int* __restrict__ key,
                                int* __restrict__ hist) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const int np = npq ? min(max(npq[q], 0), nprobe) : nprobe;
  int64_t cost = 0;
  for (int j = 0; j < np; ++j) {
    const int l = probes[q * nprobe + j];
    const int b = bits ? bits[q * nprobe + j] : 0;
    if (l < 0 || (skip_narrow && j >= 1 && b >= 1 && b <= 8)) continue;
    cost += (int64_t)list_len[l] * gather_cost(b) + kBuild;
  }
  // bucket from the leading bits of the FP32 cost; descending cost = ascending bucket
  const int lead = (int)(__float_as_uint((float)cost) >> 20);  // cost >= 0: sign bit 0
  const int b = kBuckets - 1 - min(lead, kBuckets - 1);
  key[q] = b;
  atomicAdd(hist + b, 1);
}

// One block: exclusive prefix of the bucket counts; resets the cursors.
__global__ void __launch_bounds__(1024) bucket_offsets_kernel(const int* __restrict__ hist,
                                                              int* __restrict__ off,
                                                              int* __restrict__ cursor) {
  __shared__ int part[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int base = 0; base < kBuckets; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int v = hist[i];
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) part[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int p = lane < (int)(blockDim.x / 32) ? part[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, p, o);
        if (lane >= o) p += y;
      }
      part[lane] = p;
    }
    __syncthreads();
    off[i] = carry + (warp ? part[warp - 1] : 0) + x - v;
    cursor[i] = 0;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += part[31];
    __syncthreads();
  }
}

__global__ void bucket_scatter_kernel(const int* __restrict__ key, const int* __restrict__ off,
                                      int* __restrict__ cursor, int64_t nq, int32_t* __restrict__ order) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const int b = key[q];
  order[off[b] + atomicAdd(cursor + b, 1)] = (int32_t)q;
}

}  // namespace

// Workspace: bucket counts | offsets | cursors | keys [nq] | order [nq].
size_t lpt_workspace_bytes(int64_t nq) { return (size_t)(3 * kBuckets + 2 * nq) * sizeof(int); }
int32_t* lpt_order_ptr(void* ws, int64_t nq) { return (int32_t*)ws + 3 * kBuckets + nq; }

cudaError_t launch_lpt_order(const Index& ix, const int32_t* probes, const int32_t* npq, int64_t nq,
                             int nprobe, void* ws, cudaStream_t s, const uint8_t* bits, bool skip_narrow) {
  int* hist = (int*)ws;
  int* off = hist + kBuckets;
  int* cursor = off + kBuckets;
  int* key = cursor + kBuckets;
  int32_t* order_out = lpt_order_ptr(ws, nq);
  cudaError_t e = cudaMemsetAsync(hist, 0, kBuckets * sizeof(int), s);
  if (e != cudaSuccess) return e;
  const unsigned g = (unsigned)((nq + 255) / 256);
  cost_key_kernel<<<g, 256, 0, s>>>(probes, npq, ix.list_len, bits, skip_narrow ? 1 : 0, nq, nprobe, key, hist);
  note_launch();
  bucket_offsets_kernel<<<1, 1024, 0, s>>>(hist, off, cursor); note_launch();
  bucket_scatter_kernel<<<g, 256, 0, s>>>(key, off, cursor, nq, order_out); note_launch();
  return cudaGetLastError();
}

}  // namespace anns
