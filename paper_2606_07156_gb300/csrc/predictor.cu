// Learned precision predictor: training set, labels and GPU training of the
// 5-32-32-5 MLP that picks each (query, list) LUT's bit width (the regressor
// of Section 3.4, here a classifier over 4/6/8/12/16 bits; features of
// Section 3.3; labels after Fig. 6, read as "fewest bits that keep the
// FP32 top-k").
//
// Labels: for probe rank j of query q, tau = (d_k + d_{k+1}) / 2 of the FP32
// search, margin = min over the list of |d - tau|, E(b) = max over the list of
// |dhat_b - d|; the label is the fewest b with E(b) < margin, 0 when none
// ("needs FP32"). Every FP32 value follows the search's rules exactly, the
// comparisons are FP64, so labels are exact integers.
//
// Training: FP16-operand forward (the inference rule of predictor.cuh, plus
// the pre-activation signs), FP32 backward of the mean softmax cross-entropy,
// per-block reduction of the per-sample gradients in shared memory, one FP32
// atomic add per parameter and block, then an Adam step on the FP32 master
// weights.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "predictor.cuh"

namespace anns {
namespace {

constexpr int kBitsN = 5;
__constant__ int kBitsTab[kBitsN] = {4, 6, 8, 12, 16};

// Parameter vector layout (FP32 master copy): W1 [32x5] | b1 [32] | W2 [32x32]
// | b2 [32] | W3 [5x32] | b3 [5].
constexpr int oW1 = 0, ob1 = 160, oW2 = 192, ob2 = 1216, oW3 = 1248, ob3 = 1408, kNP = 1413;

// ------------------------------------------------------------------ labels

struct LabelArgs {
  const float* qt; const float* ltab; const int32_t* probes; const float* probe_d2;
  const double* tau; const uint8_t* codes; const int32_t* list_len; const int64_t* tile_off;
  int nchunk, M, Mp, nprobe; int64_t nq;
  uint8_t* labels;
};

__global__ void __launch_bounds__(256) label_kernel(const LabelArgs a) {
  float* T = (float*)anns_dyn_smem;                          // [Mp * 256]
  float* bias = T + a.Mp * kKsub;                            // [Mp]
  float* rowmax = bias + a.Mp;                               // [Mp]
  float* scal = rowmax + a.Mp;                               // s32[5] | d32[5] | B32
  double* red = (double*)(scal + 16);                        // [8 warps][6]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;
  for (int64_t p = blockIdx.x; p < a.nq * a.nprobe; p += gridDim.x) {
    const int64_t q = p / a.nprobe;
    const int l = a.probes[p];
    if (l < 0) {
      if (tid == 0) a.labels[p] = 255;
      continue;
    }
    const int n_l = a.list_len[l];
    if (n_l == 0) {
      if (tid == 0) a.labels[p] = 4;
      continue;
    }
    const float d2 = a.probe_d2[p];
    const double tau = a.tau[q];
    const float* P = a.ltab + (size_t)l * a.Mp * kKsub;
    const float* Qt = a.qt + (size_t)q * a.Mp * kKsub;
    for (int m = warp; m < a.M; m += nwarps) {
      float t[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int c = e * 32 + lane;
        t[e] = sub_rn(__ldg(P + m * kKsub + c), __ldg(Qt + m * kKsub + c));
        T[m * kKsub + c] = t[e];
      }
      float mn = t[0];
#pragma unroll
      for (int e = 1; e < 8; ++e) mn = fminf(mn, t[e]);
      mn = warp_min(mn);
      float mx = 0.f;
#pragma unroll
      for (int e = 0; e < 8; ++e) mx = fmaxf(mx, sub_rn(t[e], mn));
      mx = warp_max(mx);
      if (lane == 0) { bias[m] = mn; rowmax[m] = mx; }
    }
    __syncthreads();
    if (warp == 0) {
      float range = 0.f;
      for (int m = lane; m < a.M; m += 32) range = fmaxf(range, rowmax[m]);
      const float B32 = warp_exact_sum(bias, a.M, d2, true);
      range = warp_max(range);
      if (lane < kBitsN) {
        const int L = (1 << kBitsTab[lane]) - 1;
        scal[lane] = range > 0.f ? __fdiv_rn((float)L, range) : 0.f;
        scal[kBitsN + lane] = range > 0.f ? __fdiv_rn(range, (float)L) : 0.f;
      }
      if (lane == 0) scal[2 * kBitsN] = B32;
    }
    __syncthreads();
    double err[kBitsN] = {0, 0, 0, 0, 0};
    double margin = INFINITY;
    const float B32 = scal[2 * kBitsN];
    const uint8_t* base = a.codes + (size_t)a.tile_off[l] * a.nchunk * kTileChunkBytes;
    for (int v = tid; v < n_l; v += blockDim.x) {
      const uint8_t* vc = base + (size_t)(v / kTileVecs) * a.nchunk * kTileChunkBytes + (v % kTileVecs) * kChunkBytes;
      float acc = 0.f;
      int S[kBitsN] = {0, 0, 0, 0, 0};
      for (int m = 0; m < a.M; ++m) {
        const int c = vc[(m >> 4) * kTileChunkBytes + (m & 15)];
        const float Tm = T[m * kKsub + c];
        acc = add_rn(acc, Tm);
        const float tp = sub_rn(Tm, bias[m]);
#pragma unroll
        for (int bi = 0; bi < kBitsN; ++bi)
          S[bi] += min(__float2int_rn(mul_rn(tp, scal[bi])), (1 << kBitsTab[bi]) - 1);
      }
      const float d = add_rn(d2, acc);
      margin = fmin(margin, fabs(__dsub_rn((double)d, tau)));
#pragma unroll
      for (int bi = 0; bi < kBitsN; ++bi) {
        const float dh = add_rn(mul_rn(scal[kBitsN + bi], __int2float_rn(S[bi])), B32);
        err[bi] = fmax(err[bi], fabs(__dsub_rn((double)dh, (double)d)));
      }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      margin = fmin(margin, __shfl_xor_sync(kFull, margin, o));
#pragma unroll
      for (int bi = 0; bi < kBitsN; ++bi) err[bi] = fmax(err[bi], __shfl_xor_sync(kFull, err[bi], o));
    }
    if (lane == 0) {
      red[warp * 6] = margin;
#pragma unroll
      for (int bi = 0; bi < kBitsN; ++bi) red[warp * 6 + 1 + bi] = err[bi];
    }
    __syncthreads();
    if (tid == 0) {
      double mg = INFINITY, e[kBitsN] = {0, 0, 0, 0, 0};
      for (int w = 0; w < nwarps; ++w) {
        mg = fmin(mg, red[w * 6]);
        for (int bi = 0; bi < kBitsN; ++bi) e[bi] = fmax(e[bi], red[w * 6 + 1 + bi]);
      }
      int lab = 0;
      for (int bi = 0; bi < kBitsN; ++bi)
        if (e[bi] < mg) { lab = kBitsTab[bi]; break; }
      a.labels[p] = (uint8_t)lab;
    }
    __syncthreads();
  }
}

// tau[q] = (d_k + d_{k+1}) / 2 from the FP32 top-(k+1) distances (FP64; +inf
// when fewer than k+1 candidates exist).
__global__ void tau_kernel(const float* dists, int64_t nq, int k, double* tau) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const double a = dists[q * (k + 1) + k - 1], b = dists[q * (k + 1) + k];
  tau[q] = __dmul_rn(__dadd_rn(a, b), 0.5);
}

// ------------------------------------------------------------------ training

struct GradArgs {
  const float* X; const uint8_t* cls; const int64_t* idx; int64_t n;
  const float* w;                 // FP32 master weights [kNP]
  float mean[5], inv_std[5];
  float inv_count;                // 1 / number of samples in the batch
  float high_w;                   // loss weight of classes 3 and 4
  float* grad; double* loss;
};

constexpr int kGT = 64;  // samples (threads) per block (static shared memory stays < 48 KB)

__global__ void __launch_bounds__(kGT) mlp_grad_kernel(const GradArgs a) {
  __shared__ float wh[kNP];                 // FP16-rounded weights, as floats
  __shared__ float xs[kGT][5];
  __shared__ float h1s[kGT][33], h2s[kGT][33], g1s[kGT][33], g2s[kGT][33];
  __shared__ float gzs[kGT][5];
  __shared__ double lsum[kGT / 32];
  const int t = threadIdx.x;
  for (int i = t; i < kNP; i += kGT) wh[i] = __half2float(__float2half_rn(a.w[i]));
  __syncthreads();
  const int64_t s = (int64_t)blockIdx.x * kGT + t;
  int y = 255;
  float x[5] = {0, 0, 0, 0, 0};
  if (s < a.n) {
    const int64_t r = a.idx ? a.idx[s] : s;
    y = a.cls[r];
#pragma unroll
    for (int i = 0; i < 5; ++i)
      x[i] = __half2float(__float2half_rn(mul_rn(sub_rn(a.X[r * 5 + i], a.mean[i]), a.inv_std[i])));
  }
  const bool live = y < 5;
  // forward (inference rule) keeping the ReLU masks
  float h1[32];
  unsigned m1 = 0, m2 = 0;
#pragma unroll
  for (int o = 0; o < 32; ++o) {
    float acc = wh[ob1 + o];
#pragma unroll
    for (int i = 0; i < 5; ++i) acc = fmaf(wh[oW1 + o * 5 + i], x[i], acc);
    if (acc > 0.f) m1 |= 1u << o;
    h1[o] = __half2float(__float2half_rn(fmaxf(acc, 0.f)));
  }
  float h2[32];
#pragma unroll 4
  for (int o = 0; o < 32; ++o) {
    float acc = wh[ob2 + o];
#pragma unroll
    for (int i = 0; i < 32; ++i) acc = fmaf(wh[oW2 + o * 32 + i], h1[i], acc);
    if (acc > 0.f) m2 |= 1u << o;
    h2[o] = __half2float(__float2half_rn(fmaxf(acc, 0.f)));
  }
  float z[5], zmax = -INFINITY;
#pragma unroll
  for (int o = 0; o < 5; ++o) {
    float acc = wh[ob3 + o];
#pragma unroll
    for (int i = 0; i < 32; ++i) acc = fmaf(wh[oW3 + o * 32 + i], h2[i], acc);
    z[o] = acc;
    zmax = fmaxf(zmax, acc);
  }
  float e[5], se = 0.f;
#pragma unroll
  for (int o = 0; o < 5; ++o) { e[o] = expf(z[o] - zmax); se += e[o]; }
  float gz[5];
  double l = 0.0;
  const float wy = y >= 3 ? a.high_w : 1.f;
#pragma unroll
  for (int o = 0; o < 5; ++o) gz[o] = live ? (e[o] / se - (o == y ? 1.f : 0.f)) * (a.inv_count * wy) : 0.f;
  if (live) l = -(double)wy * (double)(z[y] - zmax - logf(se));
  // backward to the hidden layers
  float g2[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    float acc = 0.f;
#pragma unroll
    for (int o = 0; o < 5; ++o) acc = fmaf(wh[oW3 + o * 32 + i], gz[o], acc);
    g2[i] = (m2 >> i & 1u) ? acc : 0.f;
  }
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    float acc = 0.f;
#pragma unroll 8
    for (int o = 0; o < 32; ++o) acc = fmaf(wh[oW2 + o * 32 + i], g2[o], acc);
    g1s[t][i] = (m1 >> i & 1u) ? acc : 0.f;
    h1s[t][i] = live ? h1[i] : 0.f;
    h2s[t][i] = live ? h2[i] : 0.f;
    g2s[t][i] = g2[i];
  }
#pragma unroll
  for (int i = 0; i < 5; ++i) { xs[t][i] = live ? x[i] : 0.f; gzs[t][i] = gz[i]; }
#pragma unroll
  for (int o = 16; o; o >>= 1) l += __shfl_xor_sync(kFull, l, o);
  if ((t & 31) == 0) lsum[t >> 5] = l;
  __syncthreads();
  // parameter gradients summed over the block's samples
  for (int p = t; p < kNP; p += kGT) {
    float acc = 0.f;
    if (p < ob1) { const int o = p / 5, i = p % 5; for (int s2 = 0; s2 < kGT; ++s2) acc = fmaf(g1s[s2][o], xs[s2][i], acc); }
    else if (p < oW2) { const int o = p - ob1; for (int s2 = 0; s2 < kGT; ++s2) acc += g1s[s2][o]; }
    else if (p < ob2) { const int o = (p - oW2) / 32, i = (p - oW2) % 32; for (int s2 = 0; s2 < kGT; ++s2) acc = fmaf(g2s[s2][o], h1s[s2][i], acc); }
    else if (p < oW3) { const int o = p - ob2; for (int s2 = 0; s2 < kGT; ++s2) acc += g2s[s2][o]; }
    else if (p < ob3) { const int o = (p - oW3) / 32, i = (p - oW3) % 32; for (int s2 = 0; s2 < kGT; ++s2) acc = fmaf(gzs[s2][o], h2s[s2][i], acc); }
    else { const int o = p - ob3; for (int s2 = 0; s2 < kGT; ++s2) acc += gzs[s2][o]; }
    atomicAdd(a.grad + p, acc);
  }
  if (t == 0) {
    double tot = 0.0;
    for (int w = 0; w < kGT / 32; ++w) tot += lsum[w];
    atomicAdd(a.loss, tot);
  }
}

__global__ void adam_kernel(float* w, const float* g, float* m, float* v, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNP) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Bits -> class (4, 6, 8, 12, 16 -> 0..4; "needs FP32" trains as 16 bits; 255 = no sample).
// map 1, the two tables of the GB300 width map: 4, 6, 8 -> 2; 12, 16, FP32 -> 4.
// map 2, its three tables: 4 -> 0 (nibble tables); 6, 8 -> 2; 12, 16, FP32 -> 4.
__global__ void class_kernel(const uint8_t* bits, int64_t n, int map, uint8_t* cls) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = bits[i];
  uint8_t c = b == 4 ? 0 : b == 6 ? 1 : b == 8 ? 2 : b == 12 ? 3 : (b == 16 || b == 0) ? 4 : 255;
  if (map == 1 && c < 5) c = c <= 2 ? 2 : 4;
  if (map == 2 && c < 5) c = c == 0 ? 0 : (c <= 2 ? 2 : 4);
  cls[i] = c;
}

void pack(const anns_predictor& p, std::vector<float>& w) {
  w.resize(kNP);
  std::memcpy(&w[oW1], p.W1, sizeof p.W1);
  std::memcpy(&w[ob1], p.b1, sizeof p.b1);
  std::memcpy(&w[oW2], p.W2, sizeof p.W2);
  std::memcpy(&w[ob2], p.b2, sizeof p.b2);
  std::memcpy(&w[oW3], p.W3, sizeof p.W3);
  std::memcpy(&w[ob3], p.b3, sizeof p.b3);
}
void unpack(const std::vector<float>& w, anns_predictor& p) {
  std::memcpy(p.W1, &w[oW1], sizeof p.W1);
  std::memcpy(p.b1, &w[ob1], sizeof p.b1);
  std::memcpy(p.W2, &w[oW2], sizeof p.W2);
  std::memcpy(p.b2, &w[ob2], sizeof p.b2);
  std::memcpy(p.W3, &w[oW3], sizeof p.W3);
  std::memcpy(p.b3, &w[ob3], sizeof p.b3);
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
  int alloc(size_t bytes) {
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(bytes, 16));
    return e == cudaSuccess ? ANNS_OK : cuda_fail(e, "cudaMalloc(training)");
  }
};

uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct DeviceGuardP {
  int prev = 0;
  explicit DeviceGuardP(int d) { cudaGetDevice(&prev); cudaSetDevice(d); }
  ~DeviceGuardP() { cudaSetDevice(prev); }
};

// Gradient of the mean loss over samples idx[0..n) (or 0..n) into grad (device, zeroed here).
cudaError_t launch_grad(const float* X, const uint8_t* cls, const int64_t* idx, int64_t n,
                        const float* w, const anns_predictor& norm, float* grad, double* loss,
                        float inv_count, float high_w, cudaStream_t s) {
  GradArgs a{};
  a.X = X; a.cls = cls; a.idx = idx; a.n = n; a.w = w; a.inv_count = inv_count;
  a.high_w = high_w > 0.f ? high_w : 1.f;
  for (int i = 0; i < 5; ++i) { a.mean[i] = norm.mean[i]; a.inv_std[i] = norm.inv_std[i]; }
  a.grad = grad; a.loss = loss;
  cudaError_t e = cudaMemsetAsync(grad, 0, kNP * sizeof(float), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  mlp_grad_kernel<<<(unsigned)((n + kGT - 1) / kGT), kGT, 0, s>>>(a); note_launch();
  return cudaGetLastError();
}

int train_on(Index& ix, const float* X, const uint8_t* cls, int64_t n, const anns_train_cfg& cfg,
             anns_predictor& io, cudaStream_t s) {
  std::vector<float> w;
  pack(io, w);
  DevBuf dw, dg, dm, dv, dl, didx;
  int rc;
  if ((rc = dw.alloc(kNP * 4)) || (rc = dg.alloc(kNP * 4)) || (rc = dm.alloc(kNP * 4)) ||
      (rc = dv.alloc(kNP * 4)) || (rc = dl.alloc(8)) || (rc = didx.alloc((size_t)n * 8)))
    return rc;
  cudaError_t e = cudaMemcpyAsync(dw.p, w.data(), kNP * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(dm.p, 0, kNP * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(dv.p, 0, kNP * 4, s);
  if (e != cudaSuccess) return cuda_fail(e, "training setup");
  std::vector<int64_t> perm(n);
  uint64_t st = cfg.seed ^ 0x5851F42D4C957F2Dull;
  const int64_t B = std::max<int32_t>(1, cfg.batch);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  int64_t step = 0;
  for (int ep = 0; ep < cfg.epochs; ++ep) {
    for (int64_t i = 0; i < n; ++i) perm[i] = i;
    for (int64_t i = n - 1; i > 0; --i) std::swap(perm[i], perm[splitmix(st) % (uint64_t)(i + 1)]);
    e = cudaMemcpyAsync(didx.p, perm.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "training permutation");
    for (int64_t b0 = 0; b0 < n; b0 += B) {
      const int64_t cnt = std::min<int64_t>(B, n - b0);
      e = launch_grad(X, cls, (const int64_t*)didx.p + b0, cnt, (const float*)dw.p, io, (float*)dg.p,
                      (double*)dl.p, 1.f / (float)cnt, cfg.high_weight, s);
      if (e != cudaSuccess) return cuda_fail(e, "gradient kernel");
      ++step;
      const float c1 = 1.f - std::pow(b1, (float)step), c2 = 1.f - std::pow(b2, (float)step);
      adam_kernel<<<(kNP + 255) / 256, 256, 0, s>>>((float*)dw.p, (const float*)dg.p, (float*)dm.p,
                                                     (float*)dv.p, cfg.lr, b1, b2, eps, c1, c2); note_launch();
      e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(e, "adam kernel");
    }
  }
  e = cudaMemcpyAsync(w.data(), dw.p, kNP * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "training result");
  unpack(w, io);
  return ANNS_OK;
}

int install(Index& ix, const anns_predictor& p) {
  MlpParams16 h;
  for (int i = 0; i < 160; ++i) h.W1[i] = __float2half_rn(p.W1[i]);
  for (int i = 0; i < 32; ++i) h.b1[i] = __float2half_rn(p.b1[i]);
  for (int i = 0; i < 1024; ++i) h.W2[i] = __float2half_rn(p.W2[i]);
  for (int i = 0; i < 32; ++i) h.b2[i] = __float2half_rn(p.b2[i]);
  for (int i = 0; i < 160; ++i) h.W3[i] = __float2half_rn(p.W3[i]);
  for (int i = 0; i < 5; ++i) h.b3[i] = __float2half_rn(p.b3[i]);
  for (int i = 0; i < 5; ++i) { h.mean[i] = p.mean[i]; h.inv_std[i] = p.inv_std[i]; }
  if (!ix.mlp_dev) {
    cudaError_t e = cudaMalloc(&ix.mlp_dev, sizeof(MlpParams16));
    if (e != cudaSuccess) { ix.mlp_dev = nullptr; return cuda_fail(e, "cudaMalloc(predictor)"); }
  }
  cudaError_t e = cudaMemcpy(ix.mlp_dev, &h, sizeof h, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "upload predictor");
  ix.mlp_host = p;
  ix.has_mlp = true;
  return ANNS_OK;
}

}  // namespace

int make_training_set(Index& ix, const float* Q, int64_t nq, int nprobe, int k, float* feat,
                      uint8_t* labels, cudaStream_t s);

}  // namespace anns

using namespace anns;

extern "C" int anns_set_predictor(anns_index* ix, const anns_predictor* p) {
  if (!ix || !p) return fail(ANNS_ERR_INVALID_ARG, "null index or predictor");
  DeviceGuardP g(ix->device);
  return install(*ix, *p);
}

extern "C" int anns_get_predictor(const anns_index* ix, anns_predictor* out) {
  if (!ix || !out) return fail(ANNS_ERR_INVALID_ARG, "null index or out");
  if (!ix->has_mlp) return fail(ANNS_ERR_INVALID_ARG, "no predictor trained or loaded");
  *out = ix->mlp_host;
  return ANNS_OK;
}

extern "C" int anns_mlp_grad(anns_index* ix, const anns_predictor* w, const float* X, const uint8_t* cls,
                             int64_t n, float high_weight, float* grad_out, double* loss_out, void* stream) {
  if (!ix || !w || !grad_out) return fail(ANNS_ERR_INVALID_ARG, "null argument");
  if (n <= 0 || !X || !cls) return fail(ANNS_ERR_INVALID_ARG, "need n > 0 samples");
  DeviceGuardP g(ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<float> hw;
  pack(*w, hw);
  DevBuf dw, dg, dl;
  int rc;
  if ((rc = dw.alloc(kNP * 4)) || (rc = dg.alloc(kNP * 4)) || (rc = dl.alloc(8))) return rc;
  cudaError_t e = cudaMemcpyAsync(dw.p, hw.data(), kNP * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = launch_grad(X, cls, nullptr, n, (const float*)dw.p, *w, (float*)dg.p, (double*)dl.p, 1.f / (float)n,
                    high_weight, s);
  double loss = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(grad_out, dg.p, kNP * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&loss, dl.p, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "gradient");
  if (loss_out) *loss_out = loss / (double)n;
  return ANNS_OK;
}

extern "C" int anns_mlp_train(anns_index* ix, const float* X, const uint8_t* cls, int64_t n,
                              const anns_train_cfg* cfg, anns_predictor* io, void* stream) {
  if (!ix || !cfg || !io || !X || !cls) return fail(ANNS_ERR_INVALID_ARG, "null argument");
  if (n <= 0 || cfg->epochs < 0 || cfg->batch <= 0) return fail(ANNS_ERR_INVALID_ARG, "bad sizes");
  DeviceGuardP g(ix->device);
  return train_on(*ix, X, cls, n, *cfg, *io, (cudaStream_t)stream);
}

extern "C" int anns_make_training_set(anns_index* ix, const float* Q, int64_t nq, int32_t nprobe,
                                      int32_t k, float* feat_out, uint8_t* label_out, void* stream) {
  if (!ix || !Q || !feat_out || !label_out) return fail(ANNS_ERR_INVALID_ARG, "null argument");
  if (nq <= 0 || nprobe < 1 || nprobe > ix->nlist || nprobe > ANNS_MAX_NPROBE || k < 1 || k + 1 > ANNS_MAX_K)
    return fail(ANNS_ERR_INVALID_ARG, "bad sizes");
  DeviceGuardP g(ix->device);
  return make_training_set(*ix, Q, nq, nprobe, k, feat_out, label_out, (cudaStream_t)stream);
}

extern "C" int anns_train_predictor(anns_index* ix, const float* Q, int64_t nq, int32_t nprobe, int32_t k,
                                    const anns_train_cfg* cfg, anns_predictor* out, void* stream) {
  if (!ix || !Q || !cfg) return fail(ANNS_ERR_INVALID_ARG, "null argument");
  if (nq <= 0 || nprobe < 1 || nprobe > ix->nlist || nprobe > ANNS_MAX_NPROBE || k < 1 || k + 1 > ANNS_MAX_K)
    return fail(ANNS_ERR_INVALID_ARG, "bad sizes");
  DeviceGuardP g(ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = nq * nprobe;
  DevBuf feat, lab, cls;
  int rc;
  if ((rc = feat.alloc((size_t)n * 5 * 4)) || (rc = lab.alloc((size_t)n)) || (rc = cls.alloc((size_t)n))) return rc;
  if ((rc = make_training_set(*ix, Q, nq, nprobe, k, (float*)feat.p, (uint8_t*)lab.p, s))) return rc;
  class_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const uint8_t*)lab.p, n, cfg->label_map,
                                                           (uint8_t*)cls.p); note_launch();
  // normalisation over the samples (host, FP64): a one-off set-up statistic
  std::vector<float> hf((size_t)n * 5);
  std::vector<uint8_t> hc((size_t)n);
  cudaError_t e = cudaMemcpyAsync(hf.data(), feat.p, hf.size() * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hc.data(), cls.p, hc.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "training set copy");
  anns_predictor p{};
  double s1[5] = {0}, s2[5] = {0};
  int64_t cnt = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (hc[i] >= 5) continue;
    ++cnt;
    for (int f = 0; f < 5; ++f) { const double x = hf[i * 5 + f]; s1[f] += x; s2[f] += x * x; }
  }
  if (cnt == 0) return fail(ANNS_ERR_INVALID_ARG, "no training samples");
  for (int f = 0; f < 5; ++f) {
    const double mu = s1[f] / cnt, var = std::max(0.0, s2[f] / cnt - mu * mu);
    p.mean[f] = (float)mu;
    p.inv_std[f] = var > 0 ? (float)(1.0 / std::sqrt(var)) : 1.f;
  }
  // He-uniform initial weights from the configured seed
  uint64_t st = cfg->seed;
  auto uni = [&](float lim) { return (float)((splitmix(st) >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0) * lim; };
  for (float& v : p.W1) v = uni(std::sqrt(6.f / 5.f));
  for (float& v : p.W2) v = uni(std::sqrt(6.f / 32.f));
  for (float& v : p.W3) v = uni(std::sqrt(6.f / 32.f));
  if ((rc = train_on(*ix, (const float*)feat.p, (const uint8_t*)cls.p, n, *cfg, p, s))) return rc;
  if ((rc = install(*ix, p))) return rc;
  if (out) *out = p;
  return ANNS_OK;
}

namespace anns {

// Features (policy kernel, Eq. 2 mode) and labels (label kernel) of the
// (query, probe rank) pairs of a batch of training queries.
int make_training_set(Index& ix, const float* Q, int64_t nq, int nprobe, int k, float* feat,
                      uint8_t* labels, cudaStream_t s) {
  // FP32 top-(k+1) distances of the plain search -> tau per query
  DevBuf ids, dists, tau;
  int rc;
  if ((rc = ids.alloc((size_t)nq * (k + 1) * 8)) || (rc = dists.alloc((size_t)nq * (k + 1) * 4)) ||
      (rc = tau.alloc((size_t)nq * 8)))
    return rc;
  anns_precision_policy plain{};
  plain.lut_mode = ANNS_LUT_PLAIN_FP32;
  if ((rc = anns_search(static_cast<anns_index*>(&ix), Q, nq, nprobe, nullptr, k + 1, nullptr, &plain,
                        (int64_t*)ids.p, (float*)dists.p, s)))
    return rc;
  tau_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, s>>>((const float*)dists.p, nq, k, (double*)tau.p);
  note_launch();
  // the workspace now holds this batch's probes, probe D2 and query tables
  anns_precision_policy eq2{};
  eq2.lut_mode = ANNS_LUT_HEURISTIC_EQ2;
  if ((rc = launch_policy(ix, eq2, nq, nprobe, nullptr, ix.ws_probes, ix.ws_probe_d2, ix.ws_bits, feat, s)))
    return rc;
  LabelArgs a{};
  a.qt = ix.ws_qt; a.ltab = ix.ltab; a.probes = ix.ws_probes; a.probe_d2 = ix.ws_probe_d2;
  a.tau = (const double*)tau.p; a.codes = ix.codes; a.list_len = ix.list_len; a.tile_off = ix.tile_off;
  a.nchunk = (int)ix.nchunk; a.M = (int)ix.M; a.Mp = (int)ix.Mp; a.nprobe = nprobe; a.nq = nq;
  a.labels = labels;
  const size_t smem = (size_t)ix.Mp * kKsub * 4 + 2 * ix.Mp * 4 + 16 * 4 + 8 * 6 * 8 + 64;
  cudaError_t e = cudaFuncSetAttribute(label_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "label kernel smem");
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t np = nq * nprobe;
  label_kernel<<<(unsigned)std::min<int64_t>(np, (int64_t)sms * 8), 256, smem, s>>>(a); note_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "label kernel");
  // make sure the temporaries outlive the kernels that read them
  e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? ANNS_OK : cuda_fail(e, "training set");
}

}  // namespace anns
