// Cluster locating (CL, Section 2.1): squared L2 distance from every query to
// every centroid, then the nprobe nearest lists per query, ties by list id.
//
// Distances follow the FP32 rule exactly: acc = 0; for d ascending:
// e = fl32(q_d - c_d); acc = fl32(acc + fl32(e*e)) — no FMA contraction.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace anns {
namespace {

constexpr int kTQ = 64, kTL = 64, kDK = 32;

// 64 queries x 64 centroids per block; 16x16 threads each own a 4x4 block of
// outputs. The dimension loop is strictly ascending, as the rule requires.
__global__ void __launch_bounds__(256) coarse_d2_kernel(const float* __restrict__ Q,
                                                        const float* __restrict__ C, int64_t nq,
                                                        int64_t nlist, int64_t dim,
                                                        float* __restrict__ d2) {
  __shared__ float Qs[kDK][kTQ + 1];
  __shared__ float Cs[kDK][kTL + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t l0 = (int64_t)blockIdx.x * kTL;
  for (int64_t q0 = (int64_t)blockIdx.y * kTQ; q0 < nq; q0 += (int64_t)gridDim.y * kTQ) {
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

  for (int64_t d0 = 0; d0 < dim; d0 += kDK) {
#pragma unroll
    for (int it = 0; it < (kTQ * kDK) / 256; ++it) {
      const int idx = threadIdx.x + it * 256;
      const int row = idx / kDK, col = idx % kDK;
      const int64_t q = q0 + row, l = l0 + row, d = d0 + col;
      Qs[col][row] = (q < nq && d < dim) ? Q[q * dim + d] : 0.f;
      Cs[col][row] = (l < nlist && d < dim) ? C[l * dim + d] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int dd = 0; dd < kDK; ++dd) {
      float qv[4], cv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) qv[i] = Qs[dd][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) cv[j] = Cs[dd][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float e = sub_rn(qv[i], cv[j]);
          acc[i][j] = add_rn(acc[i][j], mul_rn(e, e));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t q = q0 + ty * 4 + i;
    if (q >= nq) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t l = l0 + tx * 4 + j;
      if (l < nlist) d2[q * nlist + l] = acc[i][j];
    }
  }
  }
}

// One warp per query: the nprobe_q smallest (D2, list id). D2 >= 0, so the
// float bits order like the values. One counting pass over a 256-bin
// histogram (per warp, in shared memory) of (key - kmin) >> shift, the shift
// chosen so that the row's key range fits, finds the bucket of the np-th
// smallest key; its upper end T bounds the np-th value, and only the lists
// with D2 bits <= T are offered to the sorted warp list (about np of them
// instead of every list), which orders them by (D2, id) as before.
template <int R>
__global__ void __launch_bounds__(256) coarse_select_kernel(const float* __restrict__ d2,
                                                            int64_t nq, int64_t nlist, int nprobe,
                                                            const int32_t* __restrict__ npq,
                                                            int32_t* __restrict__ probes,
                                                            float* __restrict__ probe_d2) {
  __shared__ int hist_all[8][256];
  const int64_t q = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  int* hist = hist_all[threadIdx.x >> 5];
  if (q >= nq) return;
  int np = nprobe;
  if (npq) np = min(max(npq[q], 0), nprobe);
  WarpTopK<R, int32_t> top;
  top.init();
  if (np > 0) {
    const float* row = d2 + q * nlist;
    uint32_t tkey = 0xFFFFFFFFu;
    if (nlist > np) {
      uint32_t kmin = 0xFFFFFFFFu, kmax = 0;
      for (int64_t l = lane; l < nlist; l += 32) {
        const uint32_t key = __float_as_uint(row[l]);
        kmin = min(kmin, key);
        kmax = max(kmax, key);
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        kmin = min(kmin, __shfl_xor_sync(kFull, kmin, o));
        kmax = max(kmax, __shfl_xor_sync(kFull, kmax, o));
      }
      int shift = 0;
      while (((kmax - kmin) >> shift) > 255u) ++shift;
#pragma unroll
      for (int i = 0; i < 8; ++i) hist[lane * 8 + i] = 0;
      __syncwarp();
      for (int64_t l = lane; l < nlist; l += 32)
        atomicAdd(&hist[(__float_as_uint(row[l]) - kmin) >> shift], 1);
      __syncwarp();
      // the bucket where the running count reaches np
      int c[8], run = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) { c[i] = hist[lane * 8 + i]; run += c[i]; }
      int incl = run;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      const int excl = incl - run;
      uint32_t pick = 0xFFFFFFFFu;
      if (excl < np && np <= incl) {
        int acc = excl;
        for (int i = 0; i < 8; ++i) {
          if (acc + c[i] >= np) { pick = (uint32_t)(lane * 8 + i); break; }
          acc += c[i];
        }
      }
      const unsigned who = __ballot_sync(kFull, pick != 0xFFFFFFFFu);
      __syncwarp();
      if (who) {  // always, as nlist > np keys were counted
        pick = __shfl_sync(kFull, pick, __ffs(who) - 1);
        const uint64_t top_key = (uint64_t)kmin + (((uint64_t)pick + 1) << shift) - 1;
        tkey = top_key > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)top_key;
      }
    }
    float thd = INFINITY;
    int32_t thi = INT32_MAX;
    for (int64_t base = 0; base < nlist; base += 32) {
      const int64_t l = base + lane;
      const bool valid = l < nlist;
      const float v = valid ? row[l] : INFINITY;
      const bool cand = valid && __float_as_uint(v) <= tkey;
      if (__any_sync(kFull, cand)) top.offer(cand, v, (int32_t)l, np, thd, thi);
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int e = r * 32 + lane;
    if (e < nprobe) {
      const bool ok = e < np && top.d[r] != INFINITY;
      probes[q * nprobe + e] = ok ? top.id[r] : -1;
      probe_d2[q * nprobe + e] = ok ? top.d[r] : INFINITY;
    }
  }
}

}  // namespace

cudaError_t launch_coarse(const Index& ix, const float* Q, int64_t nq, int nprobe,
                          const int32_t* nprobe_per_q, float* d2, int32_t* probes,
                          float* probe_d2, cudaStream_t s, cudaEvent_t between) {
  dim3 g1((unsigned)((ix.nlist + kTL - 1) / kTL), (unsigned)std::min<int64_t>((nq + kTQ - 1) / kTQ, 65535));
  coarse_d2_kernel<<<g1, 256, 0, s>>>(Q, ix.centroids, nq, ix.nlist, ix.dim, d2); note_launch();
  if (between) cudaEventRecord(between, s);
  const unsigned g2 = (unsigned)((nq + 7) / 8);
  const int R = (nprobe + 31) / 32;
  switch (R) {
    case 1: coarse_select_kernel<1><<<g2, 256, 0, s>>>(d2, nq, ix.nlist, nprobe, nprobe_per_q, probes, probe_d2); break;
    case 2: coarse_select_kernel<2><<<g2, 256, 0, s>>>(d2, nq, ix.nlist, nprobe, nprobe_per_q, probes, probe_d2); break;
    case 3: coarse_select_kernel<3><<<g2, 256, 0, s>>>(d2, nq, ix.nlist, nprobe, nprobe_per_q, probes, probe_d2); break;
    default: coarse_select_kernel<4><<<g2, 256, 0, s>>>(d2, nq, ix.nlist, nprobe, nprobe_per_q, probes, probe_d2); break;
  }
  note_launch();
  return cudaGetLastError();
}

}  // namespace anns
