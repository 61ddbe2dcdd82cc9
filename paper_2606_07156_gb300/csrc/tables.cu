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
// is a multiple of 4 and 8-byte loads when it is 2. Four rows at a time, their
// loads issued before their arithmetic. The products and sums keep the order
// of the rule above.
template <int DS>  // dsub when fixed at compile time (2, 4, 8), else 0
__global__ void __launch_bounds__(256) query_table_kernel(const float* __restrict__ Q,
                                                          const float* __restrict__ books,
                                                          int64_t nq, int dim, int M, int Mp,
                                                          int dsub, float* __restrict__ qt) {
  const int c = threadIdx.x;
  for (int64_t q = blockIdx.x; q < nq; q += gridDim.x) {
    const float* qv = Q + q * dim;
    float* out = qt + q * (int64_t)Mp * kKsub;
    if constexpr (DS > 0) {
      for (int m0 = 0; m0 < Mp; m0 += 4) {
        float y[4][DS], x[4][DS];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int m = m0 + u;
          if (m < M) {
            const float* yr = books + ((size_t)m * kKsub + c) * DS;
#pragma unroll
            for (int j = 0; j < DS; j += (DS == 2 ? 2 : 4)) {
              if constexpr (DS == 2) {
                const float2 v = __ldg(reinterpret_cast<const float2*>(yr + j));
                y[u][j] = v.x; y[u][j + 1] = v.y;
              } else {
                const float4 v = __ldg(reinterpret_cast<const float4*>(yr + j));
                y[u][j] = v.x; y[u][j + 1] = v.y; y[u][j + 2] = v.z; y[u][j + 3] = v.w;
              }
            }
#pragma unroll
            for (int j = 0; j < DS; ++j) x[u][j] = __ldg(qv + m * DS + j);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int m = m0 + u;
          float acc = 0.f;
          if (m < M) {
#pragma unroll
            for (int j = 0; j < DS; ++j) acc = add_rn(acc, mul_rn(x[u][j], y[u][j]));
          }
          if (m < Mp) out[m * kKsub + c] = mul_rn(2.f, acc);
        }
      }
    } else {
      for (int m = 0; m < Mp; ++m) {
        float acc = 0.f;
        if (m < M) {
          const float* x = qv + m * dsub;
          const float* y = books + ((size_t)m * kKsub + c) * dsub;
          for (int j = 0; j < dsub; ++j) acc = add_rn(acc, mul_rn(__ldg(x + j), __ldg(y + j)));
        }
        out[m * kKsub + c] = mul_rn(2.f, acc);
      }
    }
  }
}

}  // namespace

cudaError_t launch_query_tables(const Index& ix, const float* Q, int64_t nq, float* qt, cudaStream_t s) {
  if (nq == 0) return cudaSuccess;
  static_assert(kKsub == 256, "one thread per codebook entry");
  const int64_t grid = std::min<int64_t>(nq, (int64_t)1 << 30);
  const unsigned g = (unsigned)grid;
  const int dim = (int)ix.dim, M = (int)ix.M, Mp = (int)ix.Mp, ds = (int)ix.dsub;
  switch (ds) {
    case 2: query_table_kernel<2><<<g, 256, 0, s>>>(Q, ix.codebooks, nq, dim, M, Mp, ds, qt); break;
    case 4: query_table_kernel<4><<<g, 256, 0, s>>>(Q, ix.codebooks, nq, dim, M, Mp, ds, qt); break;
    case 8: query_table_kernel<8><<<g, 256, 0, s>>>(Q, ix.codebooks, nq, dim, M, Mp, ds, qt); break;
    default: query_table_kernel<0><<<g, 256, 0, s>>>(Q, ix.codebooks, nq, dim, M, Mp, ds, qt);
  }
  note_launch();
  return cudaGetLastError();
}

}  // namespace anns
