// IVF-PQ index training on the GPU (the offline index of Section 2.1): the
// coarse centroids and the PQ codebooks by Lloyd k-means, then the encoding
// of every vector into its list and M code bytes. The paper fixes neither the
// sample, the initialisation nor the rounding of the means; the rules below
// make training a deterministic function of the data and the seed, with
// results independent of thread scheduling:
//   * sample: row i is drawn when the SplitMix64 output (Steele, Lea and
//     Flood, 2014) of the state seed + (i + 1) * 0x9E3779B97F4A7C15 is below
//     floor(target * 2^64 / n); drawn rows keep their row order;
//   * initial centroid j = sample row floor(j * S / k);
//   * assignment: nearest centroid by the FP32 rule of CL (the CL kernels,
//     ties to the lower index);
//   * update: each coordinate the exact sum of the members' values (ExactSum
//     of common.cuh, any order) rounded once to FP32, then one FP32 division
//     by the member count; the e-th empty centroid takes the e-th farthest
//     sample row from its centroid (ties to the lower row);
//   * PQ: a second sample (seed + 1), residuals fl32(x - c) to their nearest
//     centroid, one k-means of 256 entries per sub-space;
//   * encoding: nearest centroid, then per sub-space the nearest codebook
//     entry of the residual (FP32 rule, ties to the lower index).
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace anns {
namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;
constexpr int kRowsPerBlock = 1024;

__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ bool drawn(int64_t i, uint64_t seed, uint64_t thr) {
  return splitmix64(seed + (uint64_t)(i + 1) * kGolden) < thr;
}

// Pass 1 of the sample: rows drawn per block of 1024 rows.
__global__ void __launch_bounds__(kRowsPerBlock) sample_count_kernel(int64_t n, uint64_t seed, uint64_t thr,
                                                                     int* __restrict__ cnt) {
  __shared__ int tot;
  if (threadIdx.x == 0) tot = 0;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * kRowsPerBlock + threadIdx.x;
  const bool f = i < n && drawn(i, seed, thr);
  const unsigned b = __ballot_sync(kFull, f);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(&tot, __popc(b));
  __syncthreads();
  if (threadIdx.x == 0) cnt[blockIdx.x] = tot;
}

// Exclusive scan of v[0..n) in place (one block of 1024 threads), total in v[n].
__global__ void __launch_bounds__(1024) scan_kernel(int* __restrict__ v, int64_t n) {
  __shared__ int part[1024];
  const int64_t per = (n + 1023) / 1024;
  const int64_t b = (int64_t)threadIdx.x * per, e = b + per < n ? b + per : n;
  int s = 0;
  for (int64_t i = b; i < e; ++i) s += v[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int t = 0; t < 1024; ++t) { const int x = part[t]; part[t] = run; run += x; }
    v[n] = run;
  }
  __syncthreads();
  int run = part[threadIdx.x];
  for (int64_t i = b; i < e; ++i) { const int x = v[i]; v[i] = run; run += x; }
}

// Pass 2: the drawn rows' indices in row order.
__global__ void __launch_bounds__(kRowsPerBlock) sample_write_kernel(int64_t n, uint64_t seed, uint64_t thr,
                                                                     const int* __restrict__ off,
                                                                     int64_t* __restrict__ rows) {
  __shared__ int wsum[kRowsPerBlock / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * kRowsPerBlock + threadIdx.x;
  const bool f = i < n && drawn(i, seed, thr);
  const unsigned b = __ballot_sync(kFull, f);
  if (lane == 0) wsum[warp] = __popc(b);
  __syncthreads();
  int before = 0;
  for (int w = 0; w < warp; ++w) before += wsum[w];
  if (f) rows[off[blockIdx.x] + before + __popc(b & ((1u << lane) - 1u))] = i;
}

// out[j][c] = X[rows[j]][c0 + c] for c < w (rows NULL: row j itself).
__global__ void gather_rows_kernel(const float* __restrict__ X, int64_t ldx, const int64_t* __restrict__ rows,
                                   int64_t nrows, int64_t c0, int64_t w, float* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nrows * w) return;
  const int64_t j = t / w, c = t % w;
  const int64_t r = rows ? rows[j] : j;
  out[t] = X[r * ldx + c0 + c];
}

// Residuals of rows to their assigned centroids: out = fl32(x - c_a).
__global__ void residual_kernel(const float* __restrict__ X, const int32_t* __restrict__ a,
                                const float* __restrict__ C, int64_t nrows, int64_t dim, float* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nrows * dim) return;
  const int64_t j = t / dim, c = t % dim;
  out[t] = sub_rn(X[t], C[(int64_t)a[j] * dim + c]);
}

__global__ void count_kernel(const int32_t* __restrict__ a, int64_t n, int* __restrict__ cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(&cnt[a[i]], 1);
}

__global__ void scatter_kernel(const int32_t* __restrict__ a, int64_t n, int* __restrict__ fill,
                               int32_t* __restrict__ members) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) members[atomicAdd(&fill[a[i]], 1)] = (int32_t)i;
}

// One block per centroid with members: each coordinate is the exact sum of
// the members' values rounded once, divided by the count (a warp per
// coordinate, lanes striding over the members in any order).
__global__ void __launch_bounds__(256) update_kernel(const float* __restrict__ X, int64_t dim,
                                                     const int* __restrict__ off, const int32_t* __restrict__ members,
                                                     float* __restrict__ C) {
  const int j = blockIdx.x;
  const int b = off[j], e = off[j + 1];
  if (e == b) return;  // empty: re-seeded on the host side
  const float cntf = (float)(e - b);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t c = warp; c < dim; c += 8) {
    ExactSum acc;
    xsum_init(acc);
    for (int i = b + lane; i < e; i += 32) xsum_add(acc, X[(int64_t)members[i] * dim + c]);
    xsum_warp(acc);
    const float s = xsum_round(acc);
    if (lane == 0) C[(int64_t)j * dim + c] = __fdiv_rn(s, cntf);
  }
}

// Largest key = (distance bits, ~row) over rows not yet taken (dist >= 0):
// the farthest row, ties to the lower row.
__global__ void farthest_kernel(const float* __restrict__ dist, int64_t n, unsigned long long* __restrict__ best) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long key = 0ull;
  if (i < n && dist[i] >= 0.f)
    key = ((unsigned long long)__float_as_uint(dist[i]) << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)i);
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(kFull, key, o);
    key = y > key ? y : key;
  }
  if ((threadIdx.x & 31) == 0 && key) atomicMax(best, key);
}

// Nearest codebook entry of each (row, sub-space): block (256 rows, m), the
// sub-space's 256 entries in shared memory; the residual's sub-vector is
// fl32(x - c_list) and the distance follows the FP32 rule, ties to the lower entry.
__global__ void __launch_bounds__(256) encode_kernel(const float* __restrict__ X, const int32_t* __restrict__ lst,
                                                     const float* __restrict__ C, const float* __restrict__ books,
                                                     int64_t n, int64_t dim, int M, int dsub,
                                                     uint8_t* __restrict__ codes) {
  float* cb = (float*)anns_dyn_smem;  // [256 * dsub]
  const int m = blockIdx.y;
  for (int t = threadIdx.x; t < 256 * dsub; t += blockDim.x) cb[t] = books[(int64_t)m * 256 * dsub + t];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float r[16];
  const int64_t l = lst[i];
#pragma unroll
  for (int j = 0; j < 16; ++j)
    if (j < dsub) r[j] = sub_rn(X[i * dim + (int64_t)m * dsub + j], C[l * dim + (int64_t)m * dsub + j]);
  float bd = INFINITY;
  int bc = 0;
  for (int c = 0; c < 256; ++c) {
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (j < dsub) {
        const float e = sub_rn(r[j], cb[c * dsub + j]);
        acc = add_rn(acc, mul_rn(e, e));
      }
    if (acc < bd) { bd = acc; bc = c; }
  }
  codes[i * M + m] = (uint8_t)bc;
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
  cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, std::max<size_t>(bytes, 16)); }
  template <typename T> T* as() const { return (T*)p; }
};

#define TRY(x)                                   \
  do {                                           \
    const cudaError_t e_ = (x);                  \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x); \
  } while (0)

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// Nearest centroid of rows X[0..nrows) (FP32 rule, ties to the lower index),
// chunked so that the distance matrix stays under about 1 GB.
int nearest(const float* X, int64_t nrows, int64_t dim, const float* C, int64_t k, int32_t* a, float* dist,
            cudaStream_t s) {
  Index tmp;
  tmp.centroids = const_cast<float*>(C);
  tmp.nlist = k;
  tmp.dim = dim;
  const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(nrows, ((int64_t)1 << 28) / k));
  DevBuf d2;
  TRY(d2.alloc((size_t)chunk * k * 4));
  for (int64_t r0 = 0; r0 < nrows; r0 += chunk) {
    const int64_t m = std::min(chunk, nrows - r0);
    TRY(launch_coarse(tmp, X + r0 * dim, m, 1, nullptr, d2.as<float>(), a + r0, dist + r0, s));
  }
  return ANNS_OK;
}

namespace {

// Rows of an n-row matrix drawn for a sample of `target` (ascending); *S is
// the count. rows must hold n entries.
int sample(int64_t n, int64_t target, uint64_t seed, int64_t* rows, int64_t* S, cudaStream_t s) {
  if (target >= n) {
    std::vector<int64_t> h(n);
    for (int64_t i = 0; i < n; ++i) h[i] = i;
    TRY(cudaMemcpyAsync(rows, h.data(), n * 8, cudaMemcpyHostToDevice, s));
    TRY(cudaStreamSynchronize(s));
    *S = n;
    return ANNS_OK;
  }
  const uint64_t thr = (uint64_t)(((unsigned __int128)target << 64) / (unsigned __int128)n);
  const int64_t nb = (n + kRowsPerBlock - 1) / kRowsPerBlock;
  DevBuf cnt;
  TRY(cnt.alloc((nb + 1) * 4));
  sample_count_kernel<<<(unsigned)nb, kRowsPerBlock, 0, s>>>(n, seed, thr, cnt.as<int>()); note_launch();
  scan_kernel<<<1, 1024, 0, s>>>(cnt.as<int>(), nb); note_launch();
  sample_write_kernel<<<(unsigned)nb, kRowsPerBlock, 0, s>>>(n, seed, thr, cnt.as<int>(), rows); note_launch();
  int tot = 0;
  TRY(cudaMemcpyAsync(&tot, cnt.as<int>() + nb, 4, cudaMemcpyDeviceToHost, s));
  TRY(cudaStreamSynchronize(s));
  *S = tot;
  return ANNS_OK;
}

}  // namespace

// Lloyd k-means of the S rows of X (device, [S x dim]) into C [k x dim].
int kmeans(const float* X, int64_t S, int64_t dim, int64_t k, int iters, float* C, cudaStream_t s) {
  if (S < k) return fail(ANNS_ERR_INVALID_ARG, "the training sample has fewer rows than clusters");
  // initial centroid j = row floor(j * S / k)
  std::vector<int64_t> init(k);
  for (int64_t j = 0; j < k; ++j) init[j] = (int64_t)(((unsigned __int128)j * (unsigned __int128)S) / (uint64_t)k);
  DevBuf irows, a, dist, cnt, fill, members, Cn, best;
  TRY(irows.alloc(k * 8));
  TRY(cudaMemcpyAsync(irows.p, init.data(), k * 8, cudaMemcpyHostToDevice, s));
  gather_rows_kernel<<<blocks_for(k * dim, 256), 256, 0, s>>>(X, dim, irows.as<int64_t>(), k, 0, dim, C);
  note_launch();
  TRY(a.alloc(S * 4));
  TRY(dist.alloc(S * 4));
  TRY(cnt.alloc((k + 1) * 4));
  TRY(fill.alloc((k + 1) * 4));
  TRY(members.alloc(S * 4));
  TRY(Cn.alloc(k * dim * 4));
  TRY(best.alloc(8));
  std::vector<int> hcnt(k + 1);
  for (int it = 0; it < iters; ++it) {
    int rc = nearest(X, S, dim, C, k, a.as<int32_t>(), dist.as<float>(), s);
    if (rc) return rc;
    TRY(cudaMemsetAsync(cnt.p, 0, (k + 1) * 4, s));
    count_kernel<<<blocks_for(S, 256), 256, 0, s>>>(a.as<int32_t>(), S, cnt.as<int>()); note_launch();
    TRY(cudaMemcpyAsync(hcnt.data(), cnt.p, k * 4, cudaMemcpyDeviceToHost, s));
    scan_kernel<<<1, 1024, 0, s>>>(cnt.as<int>(), k); note_launch();
    TRY(cudaMemcpyAsync(fill.p, cnt.p, (k + 1) * 4, cudaMemcpyDeviceToDevice, s));
    scatter_kernel<<<blocks_for(S, 256), 256, 0, s>>>(a.as<int32_t>(), S, fill.as<int>(), members.as<int32_t>());
    note_launch();
    TRY(cudaMemcpyAsync(Cn.p, C, k * dim * 4, cudaMemcpyDeviceToDevice, s));
    update_kernel<<<(unsigned)k, 256, 0, s>>>(X, dim, cnt.as<int>(), members.as<int32_t>(), Cn.as<float>());
    note_launch();
    TRY(cudaStreamSynchronize(s));
    // empty centroids, ascending: the farthest rows from their centroids, ties to the lower row
    for (int64_t j = 0; j < k; ++j) {
      if (hcnt[j] != 0) continue;
      TRY(cudaMemsetAsync(best.p, 0, 8, s));
      farthest_kernel<<<blocks_for(S, 256), 256, 0, s>>>(dist.as<float>(), S, best.as<unsigned long long>());
      note_launch();
      unsigned long long key = 0;
      TRY(cudaMemcpyAsync(&key, best.p, 8, cudaMemcpyDeviceToHost, s));
      TRY(cudaStreamSynchronize(s));
      if (key == 0) return fail(ANNS_ERR_INVALID_ARG, "more empty clusters than sample rows");
      const int64_t row = (int64_t)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull));
      TRY(cudaMemcpyAsync(Cn.as<float>() + j * dim, X + row * dim, dim * 4, cudaMemcpyDeviceToDevice, s));
      const float taken = -1.f;
      TRY(cudaMemcpyAsync(dist.as<float>() + row, &taken, 4, cudaMemcpyHostToDevice, s));
      TRY(cudaStreamSynchronize(s));
    }
    TRY(cudaMemcpyAsync(C, Cn.p, k * dim * 4, cudaMemcpyDeviceToDevice, s));
  }
  TRY(cudaStreamSynchronize(s));
  return ANNS_OK;
}

}  // namespace anns

using namespace anns;

extern "C" int anns_train_index(const float* base, int64_t n, int64_t dim, const anns_train_desc* t,
                                int32_t on_device, int32_t device, anns_index** out) {
  set_error("");
  if (!base || !t || !out) return fail(ANNS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (n < 1 || dim < 1 || t->nlist < 1 || t->M < 1 || dim % t->M) return fail(ANNS_ERR_INVALID_ARG, "bad shape");
  if (t->M > ANNS_MAX_M || dim / t->M > 16) return fail(ANNS_ERR_INVALID_ARG, "M <= 128 and dim / M <= 16 required");
  if (t->nlist > n || n > INT32_MAX || t->nlist > (1 << 20))
    return fail(ANNS_ERR_INVALID_ARG, "need nlist <= n <= 2^31 - 1 and nlist <= 2^20");
  if (t->iters < 0 || t->pq_iters < 0 || t->per_centroid < 1 || t->pq_sample < 256)
    return fail(ANNS_ERR_INVALID_ARG, "iters >= 0, per_centroid >= 1, pq_sample >= 256 required");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return fail(ANNS_ERR_INVALID_ARG, "bad device ordinal");
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return fail(ANNS_ERR_CUDA, "cudaSetDevice");
  const int64_t nlist = t->nlist, M = t->M, dsub = dim / M;
  cudaStream_t s = nullptr;
  int rc = ANNS_OK;
  {
    DevBuf Xown, rows, Xs, cent, books, R, Ra, Rd, res, Xm, lst, ldist, codes;
    const float* X = base;
    do {
      if (!on_device) {
        if (Xown.alloc((size_t)n * dim * 4) != cudaSuccess) { rc = fail(ANNS_ERR_OOM, "base copy"); break; }
        if (cudaMemcpy(Xown.p, base, (size_t)n * dim * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
          rc = fail(ANNS_ERR_CUDA, "base copy");
          break;
        }
        X = Xown.as<float>();
      }
      if (rows.alloc((size_t)n * 8) != cudaSuccess || cent.alloc((size_t)nlist * dim * 4) != cudaSuccess ||
          books.alloc((size_t)M * 256 * dsub * 4) != cudaSuccess) {
        rc = fail(ANNS_ERR_OOM, "training buffers");
        break;
      }
      // coarse centroids
      int64_t S = 0;
      if ((rc = sample(n, nlist * t->per_centroid, t->seed, rows.as<int64_t>(), &S, s))) break;
      if (Xs.alloc((size_t)S * dim * 4) != cudaSuccess) { rc = fail(ANNS_ERR_OOM, "sample"); break; }
      gather_rows_kernel<<<blocks_for(S * dim, 256), 256, 0, s>>>(X, dim, rows.as<int64_t>(), S, 0, dim,
                                                                   Xs.as<float>());
      note_launch();
      if ((rc = kmeans(Xs.as<float>(), S, dim, nlist, t->iters, cent.as<float>(), s))) break;
      // PQ codebooks on the residuals of a second sample
      int64_t S2 = 0;
      if ((rc = sample(n, t->pq_sample, t->seed + 1, rows.as<int64_t>(), &S2, s))) break;
      if (R.alloc((size_t)S2 * dim * 4) != cudaSuccess || Ra.alloc((size_t)S2 * 4) != cudaSuccess ||
          Rd.alloc((size_t)S2 * 4) != cudaSuccess || res.alloc((size_t)S2 * dim * 4) != cudaSuccess ||
          Xm.alloc((size_t)S2 * dsub * 4) != cudaSuccess) {
        rc = fail(ANNS_ERR_OOM, "PQ sample");
        break;
      }
      gather_rows_kernel<<<blocks_for(S2 * dim, 256), 256, 0, s>>>(X, dim, rows.as<int64_t>(), S2, 0, dim,
                                                                    R.as<float>());
      note_launch();
      if ((rc = nearest(R.as<float>(), S2, dim, cent.as<float>(), nlist, Ra.as<int32_t>(), Rd.as<float>(), s)))
        break;
      residual_kernel<<<blocks_for(S2 * dim, 256), 256, 0, s>>>(R.as<float>(), Ra.as<int32_t>(), cent.as<float>(),
                                                                 S2, dim, res.as<float>());
      note_launch();
      for (int64_t m = 0; m < M && rc == ANNS_OK; ++m) {
        gather_rows_kernel<<<blocks_for(S2 * dsub, 256), 256, 0, s>>>(res.as<float>(), dim, nullptr, S2, m * dsub,
                                                                       dsub, Xm.as<float>());
        note_launch();
        rc = kmeans(Xm.as<float>(), S2, dsub, 256, t->pq_iters, books.as<float>() + m * 256 * dsub, s);
      }
      if (rc) break;
      // encoding
      if (lst.alloc((size_t)n * 4) != cudaSuccess || ldist.alloc((size_t)n * 4) != cudaSuccess ||
          codes.alloc((size_t)n * M) != cudaSuccess) {
        rc = fail(ANNS_ERR_OOM, "encoding buffers");
        break;
      }
      if ((rc = nearest(X, n, dim, cent.as<float>(), nlist, lst.as<int32_t>(), ldist.as<float>(), s))) break;
      const size_t smem = (size_t)256 * dsub * 4;
      encode_kernel<<<dim3(blocks_for(n, 256), (unsigned)M), 256, smem, s>>>(
          X, lst.as<int32_t>(), cent.as<float>(), books.as<float>(), n, dim, (int)M, (int)dsub, codes.as<uint8_t>());
      note_launch();
      cudaError_t e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) { rc = cuda_fail(e, "training kernels"); break; }
      anns_build_desc d{};
      d.n = n; d.dim = dim; d.nlist = nlist; d.M = M; d.ksub = ANNS_KSUB;
      d.centroids = cent.as<float>(); d.codebooks = books.as<float>(); d.codes = codes.as<uint8_t>();
      d.list_of = lst.as<int32_t>(); d.ids = nullptr; d.on_device = 1; d.device = device;
      rc = anns_build_index_from_arrays(&d, out);
    } while (false);
  }
  cudaSetDevice(prev);
  return rc;
}
