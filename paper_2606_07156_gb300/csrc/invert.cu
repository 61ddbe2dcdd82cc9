// List-major work for the scan (DC of Section 2.1, grouped by list): the
// probed (query, rank) pairs are regrouped by list, and each list's pairs are
// cut into batches of `batch` pairs — the work items of the list-major
// kernel. Items are ordered by list size, largest first (a greedy
// longest-processing-time order, the analogue of the load scheduling of
// Section 4.3), through the index's size ranking.
//
//   count:   cnt[l]  = number of valid pairs probing list l (with narrow_bits:
//            only the pairs the grouped kernel packs: 1..8-bit tables, rank >= 1)
//   offsets: off[l]  = exclusive prefix of cnt over lists;
//            ioff[r] = exclusive prefix of ceil(cnt[order[r]] / batch) over
//                      size ranks r (ioff[nlist] = number of items)
//   scatter: pairs[off[l] + i] = q * nprobe + j for the pairs of list l (the
//            order within a list is unspecified; results do not depend on it)
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace anns {
namespace {

// Pair i takes part: probed (rank below the query's nprobe, list >= 0) and,
// with `bits`, one the grouped kernel packs: a table of 1..8 bits and probe
// rank >= 1 (rank 0 goes through the query-major kernel, whose result bounds
// the query's k-th distance for the grouped pairs).
__device__ __forceinline__ bool pair_selected(const int32_t* probes, const int32_t* npq, const uint8_t* bits,
                                              int64_t i, int nprobe) {
  const int64_t q = i / nprobe;
  const int j = (int)(i % nprobe);
  const int np = npq ? min(max(npq[q], 0), nprobe) : nprobe;
  if (j >= np || probes[i] < 0) return false;
  if (!bits) return true;
  const int b = bits[i];
  return j >= 1 && b >= 1 && b <= 8;
}

__global__ void count_kernel(const int32_t* __restrict__ probes, const int32_t* __restrict__ npq,
                             const uint8_t* __restrict__ bits, int64_t nq, int nprobe, int* __restrict__ cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq * nprobe) return;
  if (pair_selected(probes, npq, bits, i, nprobe)) atomicAdd(cnt + probes[i], 1);
}

// One block: exclusive scans over lists (pair offsets) and over size ranks
// (item offsets). Also resets the scatter cursors.
__global__ void __launch_bounds__(1024) offsets_kernel(const int* __restrict__ cnt,
                                                       const int32_t* __restrict__ order, int nlist,
                                                       int batch, int* __restrict__ off,
                                                       int* __restrict__ ioff, int* __restrict__ fill) {
  __shared__ int part[32];
  __shared__ int carry[2];
  if (threadIdx.x == 0) { carry[0] = 0; carry[1] = 0; }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int base = 0; base < nlist; base += blockDim.x) {
    const int l = base + threadIdx.x;
    const int v0 = l < nlist ? cnt[l] : 0;
    const int v1 = l < nlist ? (cnt[order[l]] + batch - 1) / batch : 0;
    for (int which = 0; which < 2; ++which) {
      const int v = which ? v1 : v0;
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
      const int excl = carry[which] + (warp ? part[warp - 1] : 0) + x - v;
      if (l < nlist) {
        if (which) ioff[l] = excl;
        else { off[l] = excl; fill[l] = 0; }
      }
      __syncthreads();
      if (threadIdx.x == blockDim.x - 1) carry[which] = excl + v;
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) { off[nlist] = carry[0]; ioff[nlist] = carry[1]; }
}

__global__ void scatter_kernel(const int32_t* __restrict__ probes, const int32_t* __restrict__ npq,
                               const uint8_t* __restrict__ bits, int64_t nq, int nprobe,
                               const int* __restrict__ off, int* __restrict__ fill, int32_t* __restrict__ pairs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq * nprobe) return;
  if (!pair_selected(probes, npq, bits, i, nprobe)) return;
  const int l = probes[i];
  pairs[off[l] + atomicAdd(fill + l, 1)] = (int32_t)i;
}

}  // namespace

cudaError_t launch_invert(const Index& ix, const int32_t* probes, const int32_t* npq, int64_t nq,
                          int nprobe, int batch, int* cnt, int* off, int* ioff, int* fill,
                          int32_t* pairs, cudaStream_t s, const uint8_t* narrow_bits) {
  const int64_t n = nq * nprobe;
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int) * ix.nlist, s);
  if (e != cudaSuccess) return e;
  const unsigned g = (unsigned)((n + 255) / 256);
  count_kernel<<<g, 256, 0, s>>>(probes, npq, narrow_bits, nq, nprobe, cnt); note_launch();
  offsets_kernel<<<1, 1024, 0, s>>>(cnt, ix.order, (int)ix.nlist, batch, off, ioff, fill); note_launch();
  scatter_kernel<<<g, 256, 0, s>>>(probes, npq, narrow_bits, nq, nprobe, off, fill, pairs); note_launch();
  return cudaGetLastError();
}

}  // namespace anns
