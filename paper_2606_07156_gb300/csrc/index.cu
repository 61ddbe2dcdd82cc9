// Index construction and facts (Section 2.1: IVF lists, PQ codes on residuals
// with one codebook shared by every cluster; covering radius r of Eq. 1).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

namespace anns {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }
int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? ANNS_ERR_OOM : ANNS_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

int grow(void** p, size_t* cap, size_t bytes) {
  if (*cap >= bytes && *p) return ANNS_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (bytes == 0) return ANNS_OK;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e, "cudaMalloc(workspace)");
  }
  *cap = bytes;
  return ANNS_OK;
}

static void free_index(anns_index* ix) {
  if (!ix) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(ix->device);
  void* ptrs[] = {ix->centroids, ix->codebooks, ix->codes, ix->ids, ix->list_len,
                  ix->vec_off, ix->tile_off, ix->radius, ix->ltab, ix->order, ix->mlp_dev,
                  ix->tc_mu, ix->tc_c[0], ix->tc_c[1], ix->tc_c[2], ix->tc_crows[0], ix->tc_crows[1],
                  ix->tc_crows[2], ix->dev_status, ix->svr_dev};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  free_workspace(*ix);
  free_subspaces(*ix);
  for (auto& set : ix->prof_ev)
    for (cudaEvent_t e : set)
      if (e) cudaEventDestroy(e);
  cudaSetDevice(prev);
  delete[] ix->h_list_len64;
  delete[] ix->h_radius;
  delete ix;
}

}  // namespace anns

using namespace anns;

namespace {

template <typename T>
int fetch(const T* src, size_t count, bool on_device, std::vector<T>& dst, const char* what) {
  dst.resize(count);
  if (count == 0) return ANNS_OK;
  if (on_device) {
    cudaError_t e = cudaMemcpy(dst.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, what);
  } else {
    std::memcpy(dst.data(), src, count * sizeof(T));
  }
  return ANNS_OK;
}

template <typename T>
int upload(T** dst, const T* src, size_t count, const char* what) {
  size_t bytes = std::max<size_t>(count * sizeof(T), 16);
  cudaError_t e = cudaMalloc((void**)dst, bytes);
  if (e != cudaSuccess) return cuda_fail(e, what);
  if (count) {
    e = cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, what);
  }
  return ANNS_OK;
}

// P_l[m][c] = fl32(yn[m][c] + fl32(2 * <c_lm, y_mc>)) with both inner products
// accumulated in FP32, j ascending, one rounding per operation; rows M..Mp-1 zero.
void list_tables(const std::vector<float>& cent, const std::vector<float>& books, int64_t nlist,
                 int64_t dim, int64_t M, int64_t Mp, std::vector<float>& out) {
  const int64_t dsub = dim / M;
  std::vector<float> yn((size_t)M * ANNS_KSUB);
  for (int64_t e = 0; e < M * ANNS_KSUB; ++e) {
    float acc = 0.f;
    for (int64_t j = 0; j < dsub; ++j) {
      const float y = books[(size_t)e * dsub + j];
      const float sq = y * y;
      acc = acc + sq;
    }
    yn[e] = acc;
  }
  out.assign((size_t)nlist * Mp * ANNS_KSUB, 0.f);
  auto work = [&](int64_t l0, int64_t l1) {
    for (int64_t l = l0; l < l1; ++l)
      for (int64_t m = 0; m < M; ++m)
        for (int c = 0; c < ANNS_KSUB; ++c) {
          float acc = 0.f;
          for (int64_t j = 0; j < dsub; ++j) {
            const float pr = cent[(size_t)l * dim + m * dsub + j] * books[((size_t)m * ANNS_KSUB + c) * dsub + j];
            acc = acc + pr;
          }
          const float two = 2.f * acc;
          out[((size_t)l * Mp + m) * ANNS_KSUB + c] = yn[(size_t)m * ANNS_KSUB + c] + two;
        }
  };
  const int64_t nt = std::max<int64_t>(1, std::min<int64_t>(std::thread::hardware_concurrency(), nlist));
  std::vector<std::thread> th;
  for (int64_t t = 0; t < nt; ++t) th.emplace_back(work, nlist * t / nt, nlist * (t + 1) / nt);
  for (auto& x : th) x.join();
}

}  // namespace

extern "C" int anns_build_index_from_arrays(const anns_build_desc* d, anns_index** out) {
  set_error("");
  if (!d || !out) return fail(ANNS_ERR_INVALID_ARG, "null desc or out");
  *out = nullptr;
  if (d->n < 0 || d->dim <= 0 || d->nlist <= 0 || d->M <= 0)
    return fail(ANNS_ERR_INVALID_ARG, "n must be >= 0 and dim, nlist, M > 0");
  if (d->ksub != ANNS_KSUB) return fail(ANNS_ERR_INVALID_ARG, "ksub must be 256");
  if (d->dim % d->M) return fail(ANNS_ERR_INVALID_ARG, "dim must be a multiple of M");
  if (d->M > ANNS_MAX_M) return fail(ANNS_ERR_INVALID_ARG, "M must be <= 128");
  if (d->nlist > INT32_MAX || d->n > INT32_MAX)
    return fail(ANNS_ERR_INVALID_ARG, "n and nlist must fit in int32");
  if (!d->centroids || !d->codebooks || (d->n > 0 && (!d->codes || !d->list_of)))
    return fail(ANNS_ERR_INVALID_ARG, "null array");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
    return fail(ANNS_ERR_CUDA, "no CUDA device");
  if (d->device < 0 || d->device >= ndev) return fail(ANNS_ERR_INVALID_ARG, "bad device ordinal");
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(d->device);

  const int64_t n = d->n, dim = d->dim, nlist = d->nlist, M = d->M, dsub = dim / M;
  const int64_t Mp = (M + 15) / 16 * 16, nchunk = Mp / 16;
  const bool dev = d->on_device != 0;
  std::vector<float> cent, books;
  std::vector<uint8_t> codes;
  std::vector<int32_t> list_of;
  std::vector<int64_t> uids;
  int rc;
  if ((rc = fetch(d->centroids, (size_t)(nlist * dim), dev, cent, "copy centroids")) ||
      (rc = fetch(d->codebooks, (size_t)(M * ANNS_KSUB * dsub), dev, books, "copy codebooks")) ||
      (rc = fetch(d->codes, (size_t)(n * M), dev, codes, "copy codes")) ||
      (rc = fetch(d->list_of, (size_t)n, dev, list_of, "copy list_of"))) {
    cudaSetDevice(prev);
    return rc;
  }
  if (d->ids && (rc = fetch(d->ids, (size_t)n, dev, uids, "copy ids"))) {
    cudaSetDevice(prev);
    return rc;
  }
  std::vector<int64_t> cnt(nlist, 0);
  for (int64_t i = 0; i < n; ++i) {
    const int32_t l = list_of[i];
    if (l < 0 || l >= nlist) {
      cudaSetDevice(prev);
      return fail(ANNS_ERR_INVALID_ARG, "list_of value outside [0, nlist)");
    }
    cnt[l]++;
  }
  std::vector<int64_t> voff(nlist + 1, 0), toff(nlist + 1, 0);
  int64_t max_list = 0;
  for (int64_t l = 0; l < nlist; ++l) {
    voff[l + 1] = voff[l] + cnt[l];
    toff[l + 1] = toff[l] + (cnt[l] + kTileVecs - 1) / kTileVecs;
    max_list = std::max(max_list, cnt[l]);
  }
  const int64_t ntiles = toff[nlist];
  std::vector<uint8_t> packed((size_t)ntiles * nchunk * kTileChunkBytes, 0);
  std::vector<int64_t> pids(n);
  std::vector<int64_t> fill(nlist, 0);
  // ||y_{m,c}||^2 in FP64 with j ascending; per member the sum over m ascending.
  std::vector<double> yn2((size_t)M * ANNS_KSUB, 0.0);
  for (int64_t m = 0; m < M; ++m)
    for (int c = 0; c < ANNS_KSUB; ++c) {
      double acc = 0.0;
      for (int64_t j = 0; j < dsub; ++j) {
        const double y = (double)books[((size_t)m * ANNS_KSUB + c) * dsub + j];
        const double sq = y * y;
        acc = acc + sq;
      }
      yn2[(size_t)m * ANNS_KSUB + c] = acc;
    }
  std::vector<double> rmax2(nlist, 0.0);
  for (int64_t i = 0; i < n; ++i) {
    const int32_t l = list_of[i];
    const int64_t rank = fill[l]++;
    const int64_t tile = toff[l] + rank / kTileVecs;
    const int lane = (int)(rank % kTileVecs);
    const uint8_t* src = &codes[(size_t)i * M];
    double rn2 = 0.0;
    for (int64_t m = 0; m < M; ++m) {
      packed[((size_t)tile * nchunk + m / 16) * kTileChunkBytes + lane * kChunkBytes + m % 16] = src[m];
      rn2 = rn2 + yn2[(size_t)m * ANNS_KSUB + src[m]];
    }
    rmax2[l] = std::max(rmax2[l], rn2);
    pids[voff[l] + rank] = d->ids ? uids[i] : i;
  }
  anns_index* ix = new anns_index();
  ix->device = d->device;
  ix->n = n; ix->dim = dim; ix->nlist = nlist; ix->M = M; ix->dsub = dsub; ix->Mp = Mp;
  ix->nchunk = nchunk; ix->ntiles = ntiles; ix->max_list = max_list;
  ix->ids32 = std::all_of(pids.begin(), pids.end(),
                          [](int64_t v) { return v >= (int64_t)INT32_MIN && v < (int64_t)INT32_MAX; });
  ix->h_list_len64 = new int64_t[nlist];
  ix->h_radius = new float[nlist];
  std::vector<int32_t> len32(nlist);
  for (int64_t l = 0; l < nlist; ++l) {
    ix->h_list_len64[l] = cnt[l];
    len32[l] = (int32_t)cnt[l];
    ix->h_radius[l] = (float)std::sqrt(rmax2[l]);
  }
  std::vector<float> ltab;
  list_tables(cent, books, nlist, dim, M, Mp, ltab);
  std::vector<int32_t> order(nlist);
  for (int64_t l = 0; l < nlist; ++l) order[l] = (int32_t)l;
  std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return cnt[x] > cnt[y]; });
  if ((rc = upload(&ix->ltab, ltab.data(), ltab.size(), "upload list tables")) ||
      (rc = upload(&ix->order, order.data(), order.size(), "upload list order")) ||
      (rc = upload(&ix->centroids, cent.data(), cent.size(), "upload centroids")) ||
      (rc = upload(&ix->codebooks, books.data(), books.size(), "upload codebooks")) ||
      (rc = upload(&ix->codes, packed.data(), packed.size(), "upload codes")) ||
      (rc = upload(&ix->ids, pids.data(), pids.size(), "upload ids")) ||
      (rc = upload(&ix->list_len, len32.data(), len32.size(), "upload list_len")) ||
      (rc = upload(&ix->vec_off, voff.data(), voff.size(), "upload vec_off")) ||
      (rc = upload(&ix->tile_off, toff.data(), toff.size(), "upload tile_off")) ||
      (rc = upload(&ix->radius, ix->h_radius, (size_t)nlist, "upload radius")) ||
      (rc = prepare_coarse_tc(*ix, cent))) {
    free_index(ix);
    cudaSetDevice(prev);
    return rc;
  }
  cudaSetDevice(prev);
  *out = ix;
  return ANNS_OK;
}

extern "C" void anns_free(anns_index* index) { free_index(index); }

extern "C" int anns_get_info(const anns_index* ix, anns_index_info* out) {
  if (!ix || !out) return fail(ANNS_ERR_INVALID_ARG, "null index or out");
  out->n = ix->n; out->dim = ix->dim; out->nlist = ix->nlist; out->M = ix->M;
  out->dsub = ix->dsub; out->Mp = ix->Mp;
  out->code_bytes = ix->ntiles * ix->nchunk * kTileChunkBytes;
  out->max_list = ix->max_list; out->device = ix->device;
  return ANNS_OK;
}

extern "C" int anns_debug_tap(anns_index* ix, int32_t what, void* out, size_t bytes) {
  if (!ix || !out) return fail(ANNS_ERR_INVALID_ARG, "null index or out");
  const void* src = nullptr;
  size_t need = 0;
  bool host = false;
  const size_t pairs = (size_t)(ix->ws_nq * ix->ws_nprobe);
  switch (what) {
    case ANNS_TAP_PROBES: src = ix->ws_probes; need = pairs * 4; break;
    case ANNS_TAP_PROBE_D2: src = ix->ws_probe_d2; need = pairs * 4; break;
    case ANNS_TAP_BITS: src = ix->ws_bits; need = pairs; break;
    case ANNS_TAP_FEATURES: src = ix->ws_feat; need = pairs * kNFeat * 4; break;
    case ANNS_TAP_LIST_SIZES: src = ix->h_list_len64; need = (size_t)ix->nlist * 8; host = true; break;
    case ANNS_TAP_LIST_RADIUS: src = ix->h_radius; need = (size_t)ix->nlist * 4; host = true; break;
    case ANNS_TAP_PACKED_IDS: src = ix->ids; need = (size_t)ix->n * 8; break;
    case ANNS_TAP_COARSE_APPROX:
      if (!ix->ws_tc_valid) return fail(ANNS_ERR_INVALID_ARG, "last search did not use the tensor-core CL");
      src = ix->ws_d2; need = (size_t)ix->ws_tc_nq * ix->nlist * 4; break;
    case ANNS_TAP_COARSE_CANDIDATES: {
      if (!ix->ws_tc_valid) return fail(ANNS_ERR_INVALID_ARG, "last search did not use the tensor-core CL");
      src = coarse_tc_candidates(*ix, ix->ws_tc, ix->ws_tc_nq);
      need = (size_t)ix->ws_tc_nq * 4;
      break;
    }
    case ANNS_TAP_STATUS: {
      if (bytes < 4) return fail(ANNS_ERR_INVALID_ARG, "tap buffer too small");
      int v = 0;
      cudaError_t e = cudaMemcpy(&v, ix->dev_status, 4, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) e = cudaMemset(ix->dev_status, 0, 4);
      if (e != cudaSuccess) return cuda_fail(e, "status tap");
      *(int32_t*)out = v;
      return ANNS_OK;
    }
    default: return fail(ANNS_ERR_INVALID_ARG, "unknown tap");
  }
  if (bytes < need) return fail(ANNS_ERR_INVALID_ARG, "tap buffer too small");
  if (need == 0) return ANNS_OK;
  if (!src) return fail(ANNS_ERR_INVALID_ARG, "tap not available (no search yet?)");
  if (host) {
    std::memcpy(out, src, need);
    return ANNS_OK;
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(ix->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(out, src, need, cudaMemcpyDeviceToHost);
  cudaSetDevice(prev);
  if (e != cudaSuccess) return cuda_fail(e, "tap copy");
  return ANNS_OK;
}

extern "C" int anns_sync_status(anns_index* ix, void* stream) {
  if (!ix) return fail(ANNS_ERR_INVALID_ARG, "null index");
  int prev = 0;
  cudaError_t e = cudaGetDevice(&prev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  e = cudaSetDevice(ix->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice(index device)");
  int v = 0;
  e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e == cudaSuccess && ix->dev_status) {
    e = cudaMemcpy(&v, ix->dev_status, 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && v != 0) e = cudaMemset(ix->dev_status, 0, 4);
  }
  cudaSetDevice(prev);
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  if (v == ANNS_DEV_TIMEOUT) return fail(ANNS_ERR_TIMEOUT, "a bounded wait in a kernel of this index ran out; its output is invalid");
  return ANNS_OK;
}

extern "C" const char* anns_last_error(void) { return anns::g_err.c_str(); }

namespace anns {
namespace {
std::atomic<int64_t> g_launches{0};
}
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace anns

extern "C" int64_t anns_kernel_launches(void) { return anns::launch_count(); }
