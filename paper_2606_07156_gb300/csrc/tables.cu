// Per-query tables of the decomposed LUT (Section 2.1 LC): for every query
// q, sub-space m and codebook entry c, 2 Q_q[m][c] = 2 <q_m, y_mc> with the
// inner product accumulated in FP32, j ascending, one rounding per operation
// (acc = fl32(acc + fl32(q_j * y_j))), then doubled (exact). Rows M..Mp-1 are
// zero. A pair's FP32 LUT is then T' = fl32(P_l - 2 Q_q).
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace anns {
namespace {

// One thread per (query, m, c); consecutive threads take consecutive c, so
// codebook reads are coalesced and the query sub-vector is a broadcast.
__global__ void __launch_bounds__(256) query_table_kernel(const float* __restrict__ Q,
                                                          const float* __restrict__ books,
                                                          int64_t nq, int dim, int M, int Mp,
                                                          int dsub, float* __restrict__ qt) {
  const int64_t per_q = (int64_t)Mp * kKsub;
  const int64_t total = nq * per_q;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = i / per_q;
    const int e = (int)(i % per_q);
    const int m = e >> 8;
    float acc = 0.f;
    if (m < M) {
      const float* qv = Q + q * dim + m * dsub;
      const float* y = books + (size_t)e * dsub;
      for (int j = 0; j < dsub; ++j) acc = add_rn(acc, mul_rn(__ldg(qv + j), __ldg(y + j)));
    }
    qt[i] = mul_rn(2.f, acc);
  }
}

}  // namespace

cudaError_t launch_query_tables(const Index& ix, const float* Q, int64_t nq, float* qt, cudaStream_t s) {
  const int64_t total = nq * ix.Mp * kKsub;
  if (total == 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t grid = std::min<int64_t>((total + 255) / 256, (int64_t)sms * 16);
  query_table_kernel<<<(unsigned)grid, 256, 0, s>>>(Q, ix.codebooks, nq, (int)ix.dim, (int)ix.M,
                                                    (int)ix.Mp, (int)ix.dsub, qt); note_launch();
  return cudaGetLastError();
}

}  // namespace anns
