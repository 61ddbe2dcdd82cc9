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

// One block per query (grid-stride), thread c computes entry c of every row m
// and stores it coalesced. The query sub-vector is a broadcast; the codebook
// (M x 256 x dsub floats, L1/L2 resident) is read with 16-byte loads when dsub
// is a multiple of 4. The products and sums keep the order of the rule above.
__global__ void __launch_bounds__(256) query_table_kernel(const float* __restrict__ Q,
                                                          const float* __restrict__ books,
                                                          int64_t nq, int dim, int M, int Mp,
                                                          int dsub, float* __restrict__ qt) {
  const int c = threadIdx.x;
  for (int64_t q = blockIdx.x; q < nq; q += gridDim.x) {
    const float* qv = Q + q * dim;
    float* out = qt + q * (int64_t)Mp * kKsub;
    for (int m = 0; m < Mp; ++m) {
      float acc = 0.f;
      if (m < M) {
        const float* x = qv + m * dsub;
        const float* y = books + ((size_t)m * kKsub + c) * dsub;
        if ((dsub & 3) == 0) {
          for (int j = 0; j < dsub; j += 4) {
            const float4 yy = __ldg(reinterpret_cast<const float4*>(y + j));
            acc = add_rn(acc, mul_rn(__ldg(x + j), yy.x));
            acc = add_rn(acc, mul_rn(__ldg(x + j + 1), yy.y));
            acc = add_rn(acc, mul_rn(__ldg(x + j + 2), yy.z));
            acc = add_rn(acc, mul_rn(__ldg(x + j + 3), yy.w));
          }
        } else {
          for (int j = 0; j < dsub; ++j) acc = add_rn(acc, mul_rn(__ldg(x + j), __ldg(y + j)));
        }
      }
      out[m * kKsub + c] = mul_rn(2.f, acc);
    }
  }
}

}  // namespace

cudaError_t launch_query_tables(const Index& ix, const float* Q, int64_t nq, float* qt, cudaStream_t s) {
  if (nq == 0) return cudaSuccess;
  static_assert(kKsub == 256, "one thread per codebook entry");
  const int64_t grid = std::min<int64_t>(nq, (int64_t)1 << 30);
  query_table_kernel<<<(unsigned)grid, 256, 0, s>>>(Q, ix.codebooks, nq, (int)ix.dim, (int)ix.M,
                                                    (int)ix.Mp, (int)ix.dsub, qt); note_launch();
  return cudaGetLastError();
}

}  // namespace anns
