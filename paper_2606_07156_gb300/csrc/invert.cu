// List-major work for the scan (DC of Section 2.1, grouped by list): the
// probed (query, rank) pairs are regrouped by list, and each list's pairs are
// cut into batches of `batch` pairs — the work items of the list-major
// kernel. Items are ordered by list size, largest first (a greedy
// longest-processing-time order, the analogue of the load scheduling of
// Section 4.3), through the index's size ranking.
//
// The grouped kernel can split the queries into chunks of qchunk: a bucket is
// then a (chunk c, list l) pair, key c * nlist + l, and the items run chunk by
// chunk, so that only one chunk's query tables are in use at a time.
//
//   count:   cnt[key] = number of valid pairs of the bucket (with narrow_bits:
//            only the pairs a grouped kernel packs: rank >= 1 on tables of
//            blo..bhi bits, 1..8 or the 1..4 and 5..8 classes)
//   offsets: off[key] = exclusive prefix of cnt over keys;
//            ioff[c * nlist + r] = exclusive prefix of
//                      ceil(cnt[c * nlist + order[r]] / batch) over chunks and
//                      size ranks r (ioff[nbuckets] = number of items)
//   scatter: pairs[off[key] + i] = q * nprobe + j for the pairs of the bucket
//            (the order within a bucket is unspecified; results do not depend
//            on it)
//   groups:  (grouped kernel) gtab[g] = the (chunk, size rank) index of group g
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
                                              int64_t i, int nprobe, int blo, int bhi) {
  const int64_t q = i / nprobe;
  const int j = (int)(i % nprobe);
  const int np = npq ? min(max(npq[q], 0), nprobe) : nprobe;
  if (j >= np || probes[i] < 0) return false;
  if (!bits) return true;
  const int b = bits[i];
  return j >= 1 && b >= blo && b <= bhi;
}

__device__ __forceinline__ int bucket_of(const int32_t* probes, int64_t i, int nprobe, int64_t qchunk, int nlist) {
  return (int)((i / nprobe) / qchunk) * nlist + probes[i];
}

__global__ void count_kernel(const int32_t* __restrict__ probes, const int32_t* __restrict__ npq,
                             const uint8_t* __restrict__ bits, int blo, int bhi, int64_t nq, int nprobe,
                             int64_t qchunk, int nlist, int* __restrict__ cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq * nprobe) return;
  if (pair_selected(probes, npq, bits, i, nprobe, blo, bhi))
    atomicAdd(cnt + bucket_of(probes, i, nprobe, qchunk, nlist), 1);
}

// One block: exclusive scans over bucket keys (pair offsets) and over
// (chunk, size rank) (item offsets). Also resets the scatter cursors.
__global__ void __launch_bounds__(1024) offsets_kernel(const int* __restrict__ cnt,
                                                       const int32_t* __restrict__ order, int nlist, int nb,
                                                       int batch, int* __restrict__ off,
                                                       int* __restrict__ ioff, int* __restrict__ fill) {
  __shared__ int part[32];
  __shared__ int carry[2];
  if (threadIdx.x == 0) { carry[0] = 0; carry[1] = 0; }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int base = 0; base < nb; base += blockDim.x) {
    const int l = base + threadIdx.x;
    const int v0 = l < nb ? cnt[l] : 0;
    const int v1 = l < nb ? (cnt[(l / nlist) * nlist + order[l % nlist]] + batch - 1) / batch : 0;
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
      if (l < nb) {
        if (which) ioff[l] = excl;
        else { off[l] = excl; fill[l] = 0; }
      }
      __syncthreads();
      if (threadIdx.x == blockDim.x - 1) carry[which] = excl + v;
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) { off[nb] = carry[0]; ioff[nb] = carry[1]; }
}

__global__ void scatter_kernel(const int32_t* __restrict__ probes, const int32_t* __restrict__ npq,
                               const uint8_t* __restrict__ bits, int blo, int bhi, int64_t nq, int nprobe,
                               int64_t qchunk, int nlist, const int* __restrict__ off, int* __restrict__ fill,
                               int32_t* __restrict__ pairs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq * nprobe) return;
  if (!pair_selected(probes, npq, bits, i, nprobe, blo, bhi)) return;
  const int b = bucket_of(probes, i, nprobe, qchunk, nlist);
  pairs[off[b] + atomicAdd(fill + b, 1)] = (int32_t)i;
}

// gtab[g] = the bucket index (chunk * nlist + size rank) of group g.
__global__ void group_table_kernel(const int* __restrict__ ioff, int nb, int* __restrict__ gtab) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  for (int g = ioff[b]; g < ioff[b + 1]; ++g) gtab[g] = b;
}

}  // namespace

cudaError_t launch_invert(const Index& ix, const int32_t* probes, const int32_t* npq, int64_t nq,
                          int nprobe, int batch, const ListWork& w, cudaStream_t s, const uint8_t* narrow_bits,
                          int blo, int bhi) {
  const int64_t n = nq * nprobe;
  const int nlist = (int)ix.nlist;
  cudaError_t e = cudaMemsetAsync(w.cnt, 0, sizeof(int) * w.nbuckets, s);
  if (e != cudaSuccess) return e;
  const unsigned g = (unsigned)((n + 255) / 256);
  count_kernel<<<g, 256, 0, s>>>(probes, npq, narrow_bits, blo, bhi, nq, nprobe, w.qchunk, nlist, w.cnt);
  note_launch();
  offsets_kernel<<<1, 1024, 0, s>>>(w.cnt, ix.order, nlist, w.nbuckets, batch, w.off, w.ioff, w.fill); note_launch();
  scatter_kernel<<<g, 256, 0, s>>>(probes, npq, narrow_bits, blo, bhi, nq, nprobe, w.qchunk, nlist, w.off, w.fill,
                                   w.pairs);
  note_launch();
  if (narrow_bits) {  // the grouped kernel looks its groups up in a table
    group_table_kernel<<<(unsigned)((w.nbuckets + 255) / 256), 256, 0, s>>>(w.ioff, w.nbuckets, w.gtab);
    note_launch();
  }
  return cudaGetLastError();
}

}  // namespace anns
