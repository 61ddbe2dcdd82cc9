// The paper's sub-space precision granularity in CL and LC (Sections 3.2,
// 3.3, 4.2; swept in Section 5.3, Fig. 13): the dimensions are cut into
// slices and, inside each slice, the vectors (centroid slices in CL, the 256
// codebook entries of each PQ sub-space in LC) into sub-spaces with a centre,
// a size and a covering radius. Per (query, slice, sub-space), Eq. 2 with the
// query distance measured beyond the nearest sub-space chooses how many of
// the uint8 operands' most significant bits enter the partial distance
// (2, 4, 6 or 8). The rules are stated with anns_build_subspaces and
// anns_search_subspace in anns_amp.h; all distances here are exact integers.
//
//   subspace_cl_kernel (one block per query): the query's slices against
//     every sub-space centre (FP32 rule), the bits of every (slice,
//     sub-space), then D2_int of every list (truncated uint8 operands), the
//     nprobe smallest (D2_int, l) per warp and merged, and finally the probes
//     re-ordered by their FP32-rule coarse distance.
//   subspace_lc_kernel (one block per query, its probes in turn): the pair's
//     residual in the codebook's uint8 map, per sub-space m the bits of every
//     entry group, the integer table T_int[m][c] in shared memory, then the
//     list's code tiles scanned into exact integer sums and a (sum, id) top-k.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace anns {

// Installed partitions (host view); device arrays in one allocation.
struct Subspaces {
  int S = 0, w = 0, K = 0, Klc = 0;
  float cl_lo = 0.f, cl_inv = 1.f, lc_lo = 0.f, lc_inv = 1.f;
  void* dev = nullptr;
  float *cl_cent = nullptr, *cl_rad = nullptr, *lc_cent = nullptr, *lc_rad = nullptr;
  int32_t* cl_assign = nullptr;   // [S * nlist]
  uint8_t *c8 = nullptr, *lc_assign = nullptr, *y8 = nullptr;   // [nlist * D], [M * 256], [M * 256 * dsub]
  std::vector<int64_t> cl_size, lc_size;
  void* ws = nullptr;
  size_t ws_cap = 0;
};

namespace {

constexpr int kThreads = 256, kWarps = 8;

__device__ __forceinline__ int to_u8(float x, float lo, float inv) {
  const float y = rintf(mul_rn(sub_rn(x, lo), inv));  // half to even
  return y <= 0.f ? 0 : (y >= 255.f ? 255 : (int)y);
}

// Eq. 2 at the sub-space level: bits 2/4/6 when g reaches th2/th4/th6 (in
// that order), else 8; g = -inf for a zero radius.
__device__ __forceinline__ int bits_of(float dk, float dk1, float rk1, float rk, const float* th) {
  float g = -INFINITY;
  if (rk > 0.f) g = __fdiv_rn(sub_rn(sub_rn(sub_rn(dk, dk1), mul_rn(3.f, rk1)), rk), rk);
  return g >= th[0] ? 2 : (g >= th[1] ? 4 : (g >= th[2] ? 6 : 8));
}

__device__ __forceinline__ int sq_trunc(int a, int b, int t) {
  const int e = ((a >> t) - (b >> t)) << t;
  return e * e;
}

// Smallest (distance bits, index) key of the block: the nearest centre, ties
// to the lower index (distances are non-negative).
__device__ __forceinline__ unsigned long long key_of(float D, int k) {
  return ((unsigned long long)__float_as_uint(D) << 32) | (unsigned)k;
}

struct ClArgs {
  const float* Q; const float* C; int64_t nq, nlist; int dim, nprobe;
  int S, w, K;
  float lo, inv, th[3];
  const float* cent; const float* rad; const int32_t* assign; const uint8_t* c8;
  int32_t* probes; float* probe_d2; unsigned long long* low;
};

template <int R>
__global__ void __launch_bounds__(kThreads) subspace_cl_kernel(const ClArgs a) {
  unsigned char* sm = anns_dyn_smem;
  float* qf = (float*)sm;                                   // [dim]
  int* q8 = (int*)(sm + 4 * a.dim);                         // [dim]
  float* dk = (float*)(sm + 8 * a.dim);                     // [K]
  uint8_t* bits = (uint8_t*)(sm + 8 * a.dim + 4 * a.K);     // [S * K]
  uint32_t* md = (uint32_t*)(sm + ((8 * a.dim + 4 * a.K + a.S * a.K + 15) & ~15));  // [kWarps * R * 32]
  int32_t* mi = (int32_t*)(md + kWarps * R * 32);
  __shared__ unsigned long long best;
  __shared__ unsigned long long low_blk;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t q = blockIdx.x; q < a.nq; q += gridDim.x) {
    for (int d = threadIdx.x; d < a.dim; d += kThreads) {
      qf[d] = a.Q[q * a.dim + d];
      q8[d] = to_u8(qf[d], a.lo, a.inv);
    }
    if (threadIdx.x == 0) low_blk = 0ull;
    __syncthreads();
    // bits of every (slice, sub-space)
    for (int s = 0; s < a.S; ++s) {
      if (threadIdx.x == 0) best = ~0ull;
      __syncthreads();
      unsigned long long mine = ~0ull;
      for (int k = threadIdx.x; k < a.K; k += kThreads) {
        const float* c = a.cent + ((int64_t)s * a.K + k) * a.w;
        float acc = 0.f;
        for (int j = 0; j < a.w; ++j) {
          const float e = sub_rn(qf[s * a.w + j], c[j]);
          acc = add_rn(acc, mul_rn(e, e));
        }
        dk[k] = __fsqrt_rn(acc);
        const unsigned long long key = key_of(acc, k);
        mine = key < mine ? key : mine;
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(kFull, mine, o);
        mine = y < mine ? y : mine;
      }
      if (lane == 0) atomicMin(&best, mine);
      __syncthreads();
      const int k1 = (int)(best & 0xFFFFFFFFull);
      const float d1 = dk[k1], r1 = a.rad[(int64_t)s * a.K + k1];
      for (int k = threadIdx.x; k < a.K; k += kThreads)
        bits[s * a.K + k] = (uint8_t)bits_of(dk[k], d1, r1, a.rad[(int64_t)s * a.K + k], a.th);
      __syncthreads();
    }
    // integer distance of every list; each warp keeps its nprobe smallest (D2_int, l)
    WarpTopK<R, int32_t, uint32_t> top;
    top.init();
    uint32_t thd = 0xFFFFFFFFu;
    int32_t thi = INT32_MAX;
    unsigned long long low = 0;
    for (int64_t l0 = (int64_t)warp * 32; l0 < a.nlist; l0 += kThreads) {
      const int64_t l = l0 + lane;
      uint32_t D2 = 0;
      if (l < a.nlist) {
        const uint8_t* c = a.c8 + l * a.dim;
        for (int s = 0; s < a.S; ++s) {
          const int b = bits[s * a.K + a.assign[(int64_t)s * a.nlist + l]];
          low += b < 8;
          const int t = 8 - b;
          for (int j = s * a.w; j < (s + 1) * a.w; ++j) D2 += (uint32_t)sq_trunc(q8[j], c[j], t);
        }
      }
      top.offer(l < a.nlist, D2, (int32_t)l, a.nprobe, thd, thi);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) low += __shfl_xor_sync(kFull, low, o);
    if (lane == 0) atomicAdd(&low_blk, low);
#pragma unroll
    for (int r = 0; r < R; ++r) { md[(warp * R + r) * 32 + lane] = top.d[r]; mi[(warp * R + r) * 32 + lane] = top.id[r]; }
    __syncthreads();
    if (warp == 0) {
      for (int w2 = 1; w2 < kWarps; ++w2)
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int32_t ci = mi[(w2 * R + r) * 32 + lane];
          top.offer(ci != INT32_MAX, md[(w2 * R + r) * 32 + lane], ci, a.nprobe, thd, thi);
        }
      // the selected lists re-ordered by their FP32-rule coarse distance (ties by l)
      WarpTopK<R, int32_t, float> fin;
      fin.init();
      float fd = INFINITY;
      int32_t fi = INT32_MAX;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int e = r * 32 + lane;
        const int32_t l = top.id[r];
        const bool ok = e < a.nprobe && l != INT32_MAX;
        float acc = 0.f;
        if (ok) {
          const float* c = a.C + (int64_t)l * a.dim;
          for (int d = 0; d < a.dim; ++d) {
            const float e2 = sub_rn(qf[d], c[d]);
            acc = add_rn(acc, mul_rn(e2, e2));
          }
        }
        fin.offer(ok, acc, l, a.nprobe, fd, fi);
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int e = r * 32 + lane;
        if (e < a.nprobe) {
          const bool ok = fin.id[r] != INT32_MAX;
          a.probes[q * a.nprobe + e] = ok ? fin.id[r] : -1;
          a.probe_d2[q * a.nprobe + e] = ok ? fin.d[r] : INFINITY;
        }
      }
      if (lane == 0 && a.low) atomicAdd(a.low, low_blk);
    }
    __syncthreads();
  }
}

struct LcArgs {
  const float* Q; const float* C; int64_t nq; int dim, nprobe, k, M, Mp, dsub, nchunk, Klc;
  float lo, inv, scale, th[3];
  const float* cent; const float* rad; const uint8_t* assign; const uint8_t* y8;
  const int32_t* probes; const uint8_t* codes; const int64_t* ids;
  const int32_t* list_len; const int64_t* vec_off; const int64_t* tile_off;
  int64_t* ids_out; float* dists_out; unsigned long long* low;
};

template <int R>
__global__ void __launch_bounds__(kThreads) subspace_lc_kernel(const LcArgs a) {
  unsigned char* sm = anns_dyn_smem;
  int32_t* T = (int32_t*)sm;                                             // [Mp * 256]
  float* rf = (float*)(sm + (size_t)a.Mp * 1024);                        // [dim]
  int* r8 = (int*)(rf + a.dim);                                          // [dim]
  uint8_t* gb = (uint8_t*)(r8 + a.dim);                                  // [kWarps * 256] group bits
  uint32_t* md = (uint32_t*)(gb + kWarps * 256);                         // [kWarps * R * 32]
  int64_t* mi = (int64_t*)(md + kWarps * R * 32);                        // [kWarps * R * 32]
  __shared__ unsigned long long low_blk;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t q = blockIdx.x; q < a.nq; q += gridDim.x) {
    WarpTopK<R, int64_t, uint32_t> top;
    top.init();
    uint32_t thd = 0xFFFFFFFFu;
    int64_t thi = INT64_MAX;
    unsigned long long low = 0;
    if (threadIdx.x == 0) low_blk = 0ull;
    for (int j = 0; j < a.nprobe; ++j) {
      const int l = a.probes[q * a.nprobe + j];
      if (l < 0) continue;
      const int n_l = a.list_len[l];
      if (n_l == 0) continue;
      __syncthreads();  // the previous pair is done with the table and the residual
      for (int d = threadIdx.x; d < a.dim; d += kThreads) {
        rf[d] = sub_rn(a.Q[q * a.dim + d], a.C[(int64_t)l * a.dim + d]);
        r8[d] = to_u8(rf[d], a.lo, a.inv);
      }
      __syncthreads();
      // per sub-space m (a warp each): bits of its entry groups, then its table row
      for (int m = warp; m < a.Mp; m += kWarps) {
        if (m >= a.M) {
          for (int c = lane; c < 256; c += 32) T[m * 256 + c] = 0;
          continue;
        }
        unsigned long long mine = ~0ull;
        for (int g = lane; g < a.Klc; g += 32) {
          const float* c = a.cent + ((int64_t)m * a.Klc + g) * a.dsub;
          float acc = 0.f;
          for (int jj = 0; jj < a.dsub; ++jj) {
            const float e = sub_rn(rf[m * a.dsub + jj], c[jj]);
            acc = add_rn(acc, mul_rn(e, e));
          }
          const unsigned long long key = key_of(acc, g);
          mine = key < mine ? key : mine;
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
          const unsigned long long y = __shfl_xor_sync(kFull, mine, o);
          mine = y < mine ? y : mine;
        }
        const int g1 = (int)(mine & 0xFFFFFFFFull);
        const float d1 = __fsqrt_rn(__uint_as_float((uint32_t)(mine >> 32)));
        const float r1 = a.rad[(int64_t)m * a.Klc + g1];
        for (int g = lane; g < a.Klc; g += 32) {
          const float* c = a.cent + ((int64_t)m * a.Klc + g) * a.dsub;
          float acc = 0.f;
          for (int jj = 0; jj < a.dsub; ++jj) {
            const float e = sub_rn(rf[m * a.dsub + jj], c[jj]);
            acc = add_rn(acc, mul_rn(e, e));
          }
          gb[warp * 256 + g] = (uint8_t)bits_of(__fsqrt_rn(acc), d1, r1, a.rad[(int64_t)m * a.Klc + g], a.th);
        }
        __syncwarp();
        for (int c = lane; c < 256; c += 32) {
          const int b = gb[warp * 256 + a.assign[m * 256 + c]];
          low += b < 8;
          const int t = 8 - b;
          const uint8_t* y = a.y8 + ((int64_t)m * 256 + c) * a.dsub;
          int acc = 0;
          for (int jj = 0; jj < a.dsub; ++jj) acc += sq_trunc(r8[m * a.dsub + jj], y[jj], t);
          T[m * 256 + c] = acc;
        }
        __syncwarp();
      }
      __syncthreads();
      // scan: warps over the list's tiles, one vector per lane
      const int ntile = (n_l + kTileVecs - 1) / kTileVecs;
      const int64_t t0 = a.tile_off[l], v0 = a.vec_off[l];
      for (int t = warp; t < ntile; t += kWarps) {
        const uint8_t* tp = a.codes + (t0 + t) * (int64_t)a.nchunk * kTileChunkBytes + lane * kChunkBytes;
        uint32_t S = 0;
        for (int ch = 0; ch < a.nchunk; ++ch) {
          const uint4 w4 = __ldg((const uint4*)(tp + ch * kTileChunkBytes));
          const uint32_t wd[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
          for (int bb = 0; bb < 16; ++bb) {
            const int m = ch * 16 + bb;
            const uint32_t code = (wd[bb >> 2] >> ((bb & 3) * 8)) & 0xFFu;
            S += (uint32_t)T[m * 256 + code];
          }
        }
        const int v = t * kTileVecs + lane;
        const bool ok = v < n_l;
        const int64_t id = ok ? a.ids[v0 + v] : INT64_MAX;
        top.offer(ok, S, id, a.k, thd, thi);
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) low += __shfl_xor_sync(kFull, low, o);
    if (lane == 0) atomicAdd(&low_blk, low);
#pragma unroll
    for (int r = 0; r < R; ++r) { md[(warp * R + r) * 32 + lane] = top.d[r]; mi[(warp * R + r) * 32 + lane] = top.id[r]; }
    __syncthreads();
    if (warp == 0) {
      for (int w2 = 1; w2 < kWarps; ++w2)
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int64_t ci = mi[(w2 * R + r) * 32 + lane];
          top.offer(ci != INT64_MAX, md[(w2 * R + r) * 32 + lane], ci, a.k, thd, thi);
        }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int e = r * 32 + lane;
        if (e < a.k) {
          const bool ok = top.id[r] != INT64_MAX;
          a.ids_out[q * a.k + e] = ok ? top.id[r] : -1;
          a.dists_out[q * a.k + e] = ok ? mul_rn(__uint2float_rn(top.d[r]), a.scale) : INFINITY;
        }
      }
      if (lane == 0 && a.low) atomicAdd(a.low + 1, low_blk);
    }
    __syncthreads();
  }
}

// Covering radius of each sub-space (FP64: squares summed over dimensions in
// ascending order, square root, rounded to FP32) and its size.
void host_stats(const std::vector<float>& X, int64_t n, int dim, const std::vector<float>& C, int K,
                const std::vector<int32_t>& a, float* rad, int64_t* size) {
  std::vector<double> r(K, 0.0);
  for (int k = 0; k < K; ++k) size[k] = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int k = a[i];
    double acc = 0.0;
    for (int j = 0; j < dim; ++j) {
      const double e = (double)X[i * dim + j] - (double)C[(int64_t)k * dim + j];
      acc = acc + e * e;
    }
    r[k] = std::max(r[k], std::sqrt(acc));
    size[k]++;
  }
  for (int k = 0; k < K; ++k) rad[k] = (float)r[k];
}

void host_map(const std::vector<float>& v, float* lo, float* inv) {
  float mn = v[0], mx = v[0];
  for (float x : v) { mn = std::min(mn, x); mx = std::max(mx, x); }
  const float span = mx - mn;
  *lo = mn;
  *inv = span > 0.f ? 255.0f / span : 1.0f;
}

int host_u8(float x, float lo, float inv) {
  const float y = std::nearbyint((x - lo) * inv);
  return y <= 0.f ? 0 : (y >= 255.f ? 255 : (int)y);
}

}  // namespace

void free_subspaces(Index& ix) {
  if (!ix.ss) return;
  if (ix.ss->dev) cudaFree(ix.ss->dev);
  if (ix.ss->ws) cudaFree(ix.ss->ws);
  delete ix.ss;
  ix.ss = nullptr;
}

}  // namespace anns

using namespace anns;

extern "C" int anns_build_subspaces(anns_index* ix, const anns_subspace_desc* d) {
  if (!ix || !d) return fail(ANNS_ERR_INVALID_ARG, "null index or desc");
  const int S = d->slices, K = d->K, Klc = d->K_lc;
  const int64_t D = ix->dim, nlist = ix->nlist, M = ix->M, dsub = ix->dsub;
  if (S < 1 || D % S || D > 4096) return fail(ANNS_ERR_INVALID_ARG, "slices must divide dim (dim <= 4096)");
  if (K < 1 || K > nlist || K > 1024 || (int64_t)S * K > 16384)
    return fail(ANNS_ERR_INVALID_ARG, "1 <= K <= min(nlist, 1024) and slices * K <= 16384 required");
  if (Klc < 1 || Klc > 256 || d->iters < 0) return fail(ANNS_ERR_INVALID_ARG, "1 <= K_lc <= 256, iters >= 0 required");
  if (ix->Mp * 1024 > 128 * 1024) return fail(ANNS_ERR_UNSUPPORTED, "M > 128");
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(ix->device) != cudaSuccess) return fail(ANNS_ERR_CUDA, "cudaSetDevice");
  const int w = (int)(D / S);
  auto* ss = new Subspaces();
  ss->S = S; ss->w = w; ss->K = K; ss->Klc = Klc;
  ss->cl_size.assign((size_t)S * K, 0);
  ss->lc_size.assign((size_t)M * Klc, 0);
  std::vector<float> cent((size_t)nlist * D), books((size_t)M * 256 * dsub);
  std::vector<float> cl_cent((size_t)S * K * w), cl_rad((size_t)S * K), lc_cent((size_t)M * Klc * dsub),
      lc_rad((size_t)M * Klc);
  std::vector<int32_t> cl_assign((size_t)S * nlist);
  std::vector<uint8_t> lc_assign((size_t)M * 256), c8((size_t)nlist * D), y8((size_t)M * 256 * dsub);
  int rc = ANNS_OK;
  float *dX = nullptr, *dC = nullptr, *dist = nullptr;
  int32_t* da = nullptr;
  cudaError_t e = cudaMemcpy(cent.data(), ix->centroids, cent.size() * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(books.data(), ix->codebooks, books.size() * 4, cudaMemcpyDeviceToHost);
  const int64_t rows = std::max<int64_t>(nlist, 256), width = std::max<int64_t>(D / S, dsub);
  if (e == cudaSuccess) e = cudaMalloc((void**)&dX, (size_t)rows * width * 4);
  if (e == cudaSuccess) e = cudaMalloc((void**)&dC, (size_t)std::max(K, Klc) * width * 4);
  if (e == cudaSuccess) e = cudaMalloc((void**)&da, (size_t)rows * 4);
  if (e == cudaSuccess) e = cudaMalloc((void**)&dist, (size_t)rows * 4);
  if (e != cudaSuccess) rc = cuda_fail(e, "sub-space build buffers");
  // one partition: k-means of the rows of X [n x dd] into k sub-spaces
  auto part = [&](const std::vector<float>& X, int64_t n, int dd, int k, float* centres, float* rad, int64_t* size,
                  std::vector<int32_t>& assign) -> int {
    cudaError_t ce = cudaMemcpy(dX, X.data(), (size_t)n * dd * 4, cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) return cuda_fail(ce, "sub-space rows");
    int r = kmeans(dX, n, dd, k, d->iters, dC, nullptr);
    if (r) return r;
    r = nearest(dX, n, dd, dC, k, da, dist, nullptr);
    if (r) return r;
    assign.resize(n);
    std::vector<float> C((size_t)k * dd);
    ce = cudaMemcpy(C.data(), dC, C.size() * 4, cudaMemcpyDeviceToHost);
    if (ce == cudaSuccess) ce = cudaMemcpy(assign.data(), da, (size_t)n * 4, cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) return cuda_fail(ce, "sub-space partition");
    std::copy(C.begin(), C.end(), centres);
    host_stats(X, n, dd, C, k, assign, rad, size);
    return ANNS_OK;
  };
  std::vector<float> Xs;
  std::vector<int32_t> as;
  for (int s = 0; s < S && rc == ANNS_OK; ++s) {
    Xs.assign((size_t)nlist * w, 0.f);
    for (int64_t l = 0; l < nlist; ++l)
      for (int j = 0; j < w; ++j) Xs[l * w + j] = cent[l * D + (int64_t)s * w + j];
    rc = part(Xs, nlist, w, K, cl_cent.data() + (size_t)s * K * w, cl_rad.data() + (size_t)s * K,
              ss->cl_size.data() + (size_t)s * K, as);
    if (rc == ANNS_OK) std::copy(as.begin(), as.end(), cl_assign.begin() + (size_t)s * nlist);
  }
  for (int64_t m = 0; m < M && rc == ANNS_OK; ++m) {
    Xs.assign(books.begin() + m * 256 * dsub, books.begin() + (m + 1) * 256 * dsub);
    rc = part(Xs, 256, (int)dsub, Klc, lc_cent.data() + (size_t)m * Klc * dsub, lc_rad.data() + (size_t)m * Klc,
              ss->lc_size.data() + (size_t)m * Klc, as);
    if (rc == ANNS_OK)
      for (int c = 0; c < 256; ++c) lc_assign[m * 256 + c] = (uint8_t)as[c];
  }
  if (dX) cudaFree(dX);
  if (dC) cudaFree(dC);
  if (da) cudaFree(da);
  if (dist) cudaFree(dist);
  if (rc == ANNS_OK) {
    host_map(cent, &ss->cl_lo, &ss->cl_inv);
    host_map(books, &ss->lc_lo, &ss->lc_inv);
    for (size_t i = 0; i < cent.size(); ++i) c8[i] = (uint8_t)host_u8(cent[i], ss->cl_lo, ss->cl_inv);
    for (size_t i = 0; i < books.size(); ++i) y8[i] = (uint8_t)host_u8(books[i], ss->lc_lo, ss->lc_inv);
    // one device allocation: floats first, then the int32 and byte arrays
    const size_t nf = cl_cent.size() + cl_rad.size() + lc_cent.size() + lc_rad.size();
    const size_t bytes = nf * 4 + cl_assign.size() * 4 + lc_assign.size() + c8.size() + y8.size() + 64;
    e = cudaMalloc(&ss->dev, bytes);
    if (e != cudaSuccess) {
      ss->dev = nullptr;
      rc = cuda_fail(e, "sub-space tables");
    } else {
      char* p = (char*)ss->dev;
      auto put = [&](const void* src, size_t n) {
        char* at = p;
        if (e == cudaSuccess) e = cudaMemcpy(at, src, n, cudaMemcpyHostToDevice);
        p += n;
        return at;
      };
      ss->cl_cent = (float*)put(cl_cent.data(), cl_cent.size() * 4);
      ss->cl_rad = (float*)put(cl_rad.data(), cl_rad.size() * 4);
      ss->lc_cent = (float*)put(lc_cent.data(), lc_cent.size() * 4);
      ss->lc_rad = (float*)put(lc_rad.data(), lc_rad.size() * 4);
      ss->cl_assign = (int32_t*)put(cl_assign.data(), cl_assign.size() * 4);
      ss->lc_assign = (uint8_t*)put(lc_assign.data(), lc_assign.size());
      ss->c8 = (uint8_t*)put(c8.data(), c8.size());
      ss->y8 = (uint8_t*)put(y8.data(), y8.size());
      if (e != cudaSuccess) rc = cuda_fail(e, "sub-space table copy");
    }
  }
  cudaSetDevice(prev);
  if (rc != ANNS_OK) {
    if (ss->dev) cudaFree(ss->dev);
    delete ss;
    return rc;
  }
  free_subspaces(*ix);
  ix->ss = ss;
  return ANNS_OK;
}

extern "C" int anns_subspace_sizes(anns_index* ix, int64_t* cl_size, int64_t* lc_size) {
  if (!ix || !ix->ss) return fail(ANNS_ERR_INVALID_ARG, "no sub-spaces built");
  if (cl_size) std::copy(ix->ss->cl_size.begin(), ix->ss->cl_size.end(), cl_size);
  if (lc_size) std::copy(ix->ss->lc_size.begin(), ix->ss->lc_size.end(), lc_size);
  return ANNS_OK;
}

extern "C" int anns_search_subspace(anns_index* ix, const float* Q, int64_t nq, int32_t nprobe, int32_t k,
                                    const anns_subspace_policy* pol, int64_t* ids_out, float* dists_out,
                                    unsigned long long* low_counts, void* stream) {
  if (!ix || !pol) return fail(ANNS_ERR_INVALID_ARG, "null index or policy");
  if (!ix->ss) return fail(ANNS_ERR_INVALID_ARG, "no sub-spaces built (anns_build_subspaces)");
  int rc = check_search_args(ix, Q, nq, nprobe, k, nullptr, ids_out, dists_out);
  if (rc) return rc;
  for (int i = 0; i < 3; ++i)
    if (std::isnan(pol->th_cl[i]) || std::isnan(pol->th_lc[i])) return fail(ANNS_ERR_INVALID_ARG, "NaN threshold");
  if (nq == 0) return ANNS_OK;
  Subspaces& ss = *ix->ss;
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(ix->device) != cudaSuccess) return fail(ANNS_ERR_CUDA, "cudaSetDevice");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t P = (size_t)nq * nprobe;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t d2b = pol->cl ? 0 : al((size_t)nq * ix->nlist * 4);
  const size_t qtb = pol->lc ? 0 : al((size_t)nq * ix->Mp * kKsub * 4);
  const size_t need = al(P * 4) * 2 + al(P) + d2b + qtb;
  if ((rc = grow(&ss.ws, &ss.ws_cap, need))) { cudaSetDevice(prev); return rc; }
  char* b = (char*)ss.ws;
  int32_t* probes = (int32_t*)b; b += al(P * 4);
  float* pd = (float*)b; b += al(P * 4);
  uint8_t* bits = (uint8_t*)b; b += al(P);
  float* d2 = (float*)b; b += d2b;
  float* qt = (float*)b;
  const unsigned grid = (unsigned)std::min<int64_t>(nq, 65535);
  cudaError_t e = cudaSuccess;
  if (pol->cl) {
    ClArgs a{};
    a.Q = Q; a.C = ix->centroids; a.nq = nq; a.nlist = ix->nlist; a.dim = (int)ix->dim; a.nprobe = nprobe;
    a.S = ss.S; a.w = ss.w; a.K = ss.K; a.lo = ss.cl_lo; a.inv = ss.cl_inv;
    for (int i = 0; i < 3; ++i) a.th[i] = pol->th_cl[i];
    a.cent = ss.cl_cent; a.rad = ss.cl_rad; a.assign = ss.cl_assign; a.c8 = ss.c8;
    a.probes = probes; a.probe_d2 = pd; a.low = low_counts;
    const int Rp = (nprobe + 31) / 32;
    const size_t smem = ((8 * (size_t)a.dim + 4 * (size_t)a.K + (size_t)a.S * a.K + 15) & ~size_t(15)) +
                        (size_t)kWarps * Rp * 32 * 8;
    auto go = [&](auto kern) {
      cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e2 == cudaSuccess) { kern<<<grid, kThreads, smem, s>>>(a); note_launch(); e2 = cudaGetLastError(); }
      return e2;
    };
    switch (Rp) {
      case 1: e = go(subspace_cl_kernel<1>); break;
      case 2: e = go(subspace_cl_kernel<2>); break;
      case 3: e = go(subspace_cl_kernel<3>); break;
      default: e = go(subspace_cl_kernel<4>); break;
    }
  } else {
    e = launch_coarse(*ix, Q, nq, nprobe, nullptr, d2, probes, pd, s);
  }
  if (e == cudaSuccess) {
    if (pol->lc) {
      LcArgs a{};
      a.Q = Q; a.C = ix->centroids; a.nq = nq; a.dim = (int)ix->dim; a.nprobe = nprobe; a.k = k;
      a.M = (int)ix->M; a.Mp = (int)ix->Mp; a.dsub = (int)ix->dsub; a.nchunk = (int)ix->nchunk; a.Klc = ss.Klc;
      a.lo = ss.lc_lo; a.inv = ss.lc_inv;
      a.scale = 1.0f / (ss.lc_inv * ss.lc_inv);
      for (int i = 0; i < 3; ++i) a.th[i] = pol->th_lc[i];
      a.cent = ss.lc_cent; a.rad = ss.lc_rad; a.assign = ss.lc_assign; a.y8 = ss.y8;
      a.probes = probes; a.codes = ix->codes; a.ids = ix->ids; a.list_len = ix->list_len;
      a.vec_off = ix->vec_off; a.tile_off = ix->tile_off; a.ids_out = ids_out; a.dists_out = dists_out;
      a.low = low_counts;
      const int Rk = (k + 31) / 32;
      const size_t smem = (size_t)a.Mp * 1024 + (size_t)a.dim * 8 + kWarps * 256 + (size_t)kWarps * Rk * 32 * 12;
      auto go = [&](auto kern) {
        cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e2 == cudaSuccess) { kern<<<grid, kThreads, smem, s>>>(a); note_launch(); e2 = cudaGetLastError(); }
        return e2;
      };
      switch (Rk) {
        case 1: e = go(subspace_lc_kernel<1>); break;
        case 2: e = go(subspace_lc_kernel<2>); break;
        case 3: e = go(subspace_lc_kernel<3>); break;
        default: e = go(subspace_lc_kernel<4>); break;
      }
    } else {
      e = cudaMemsetAsync(bits, 0, P, s);
      if (e == cudaSuccess) e = launch_query_tables(*ix, Q, nq, qt, s);
      if (e == cudaSuccess)
        e = launch_search(*ix, qt, nq, nprobe, nullptr, k, nullptr, probes, pd, bits, nullptr, ids_out, dists_out,
                          s);
    }
  }
  cudaSetDevice(prev);
  return e == cudaSuccess ? ANNS_OK : cuda_fail(e, "sub-space search");
}
