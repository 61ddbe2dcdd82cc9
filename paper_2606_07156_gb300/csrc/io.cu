// Index export, save and load (no counterpart in the paper, whose index is
// fixed in the accelerator's memory). The file is the index's arrays in list
// order plus the installed predictors, little-endian, closed by a 64-bit
// FNV-1a checksum of every preceding byte:
//   "ANNSAMP1" | u32 version 1 | u32 flags (1: MLP predictor, 2: SVR model)
//   | i64 n, dim, nlist, M | f32 centroids [nlist*dim] | f32 codebooks
//   [M*256*dsub] | i64 list_len [nlist] | u8 codes [n*M] | i64 ids [n]
//   | (flag 1) anns_predictor | (flag 2) i32 nsv, i32 table_n, f64 ratio,
//   f32 gamma, f32 inv_step, f32 mean[5], f32 inv_std[5], f32 sv [nsv*5],
//   f32 beta [nsv] | u64 checksum.
#include <cstdio>
#include <cstring>
#include <vector>

#include "internal.h"

namespace anns {
namespace {

constexpr char kMagic[8] = {'A', 'N', 'N', 'S', 'A', 'M', 'P', '1'};
constexpr uint32_t kVersion = 1;

struct Writer {
  std::vector<uint8_t> buf;
  void put(const void* p, size_t n) {
    const uint8_t* b = (const uint8_t*)p;
    buf.insert(buf.end(), b, b + n);
  }
  template <typename T> void val(T v) { put(&v, sizeof v); }
};

struct Reader {
  const std::vector<uint8_t>& buf;
  size_t pos = 0;
  bool ok = true;
  explicit Reader(const std::vector<uint8_t>& b) : buf(b) {}
  void get(void* p, size_t n) {
    if (!ok || n > buf.size() - pos) { ok = false; return; }
    std::memcpy(p, buf.data() + pos, n);
    pos += n;
  }
  template <typename T> T val() { T v{}; get(&v, sizeof v); return v; }
};

uint64_t fnv1a(const uint8_t* p, size_t n) {
  uint64_t h = 0xcbf29ce484222325ull;
  for (size_t i = 0; i < n; ++i) { h ^= p[i]; h *= 0x100000001b3ull; }
  return h;
}

}  // namespace
}  // namespace anns

using namespace anns;

extern "C" int anns_export_index(anns_index* ix, float* centroids, float* codebooks, uint8_t* codes, int64_t* ids,
                                 int64_t* list_len) {
  if (!ix) return fail(ANNS_ERR_INVALID_ARG, "null index");
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(ix->device) != cudaSuccess) return fail(ANNS_ERR_CUDA, "cudaSetDevice");
  const int64_t dsub = ix->dim / ix->M;
  cudaError_t e = cudaSuccess;
  if (centroids) e = cudaMemcpy(centroids, ix->centroids, (size_t)ix->nlist * ix->dim * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && codebooks)
    e = cudaMemcpy(codebooks, ix->codebooks, (size_t)ix->M * ANNS_KSUB * dsub * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && ids) e = cudaMemcpy(ids, ix->ids, (size_t)ix->n * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && codes && ix->n > 0) {
    // unpack the warp-interleaved tiles: byte m of vector v of list l sits in
    // tile tile_off[l] + v / 32, chunk m / 16, lane v % 32, byte m % 16
    std::vector<uint8_t> packed((size_t)ix->ntiles * ix->nchunk * kTileChunkBytes);
    std::vector<int64_t> toff(ix->nlist + 1);
    e = cudaMemcpy(packed.data(), ix->codes, packed.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(toff.data(), ix->tile_off, toff.size() * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) {
      int64_t row = 0;
      for (int64_t l = 0; l < ix->nlist; ++l)
        for (int64_t v = 0; v < ix->h_list_len64[l]; ++v, ++row) {
          const int64_t t = toff[l] + v / kTileVecs, lane = v % kTileVecs;
          for (int64_t m = 0; m < ix->M; ++m)
            codes[row * ix->M + m] = packed[((size_t)t * ix->nchunk + m / 16) * kTileChunkBytes +
                                            lane * kChunkBytes + m % 16];
        }
    }
  }
  cudaSetDevice(prev);
  if (e != cudaSuccess) return cuda_fail(e, "index export");
  if (list_len) std::memcpy(list_len, ix->h_list_len64, (size_t)ix->nlist * 8);
  return ANNS_OK;
}

extern "C" int anns_save(anns_index* ix, const char* path) {
  if (!ix || !path) return fail(ANNS_ERR_INVALID_ARG, "null index or path");
  const int64_t n = ix->n, dim = ix->dim, nlist = ix->nlist, M = ix->M, dsub = dim / M;
  std::vector<float> cent((size_t)nlist * dim), books((size_t)M * ANNS_KSUB * dsub);
  std::vector<uint8_t> codes((size_t)n * M);
  std::vector<int64_t> ids(n), llen(nlist);
  int rc = anns_export_index(ix, cent.data(), books.data(), codes.data(), ids.data(), llen.data());
  if (rc) return rc;
  Writer w;
  w.put(kMagic, 8);
  w.val<uint32_t>(kVersion);
  w.val<uint32_t>((ix->has_mlp ? 1u : 0u) | (ix->has_svr ? 2u : 0u));
  w.val<int64_t>(n); w.val<int64_t>(dim); w.val<int64_t>(nlist); w.val<int64_t>(M);
  w.put(cent.data(), cent.size() * 4);
  w.put(books.data(), books.size() * 4);
  w.put(llen.data(), llen.size() * 8);
  w.put(codes.data(), codes.size());
  w.put(ids.data(), ids.size() * 8);
  if (ix->has_mlp) w.put(&ix->mlp_host, sizeof(anns_predictor));
  if (ix->has_svr) {
    w.val<int32_t>(ix->svr_nsv); w.val<int32_t>(ix->svr_tn); w.val<double>(ix->svr_ratio);
    w.val<float>(ix->svr_gamma); w.val<float>(ix->svr_inv_step);
    w.put(ix->svr_mean, 20); w.put(ix->svr_inv_std, 20);
    w.put(ix->svr_host.data(), ix->svr_host.size() * 4);
  }
  w.val<uint64_t>(fnv1a(w.buf.data(), w.buf.size()));
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(ANNS_ERR_INVALID_ARG, std::string("cannot open for writing: ") + path);
  const size_t put = std::fwrite(w.buf.data(), 1, w.buf.size(), f);
  const int closed = std::fclose(f);
  if (put != w.buf.size() || closed != 0) return fail(ANNS_ERR_INVALID_ARG, std::string("write failed: ") + path);
  return ANNS_OK;
}

extern "C" int anns_load(const char* path, int32_t device, anns_index** out) {
  if (!path || !out) return fail(ANNS_ERR_INVALID_ARG, "null path or out");
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(ANNS_ERR_INVALID_ARG, std::string("cannot open: ") + path);
  std::vector<uint8_t> buf;
  uint8_t tmp[1 << 16];
  size_t got;
  while ((got = std::fread(tmp, 1, sizeof tmp, f)) > 0) buf.insert(buf.end(), tmp, tmp + got);
  std::fclose(f);
  if (buf.size() < 8 + 8 + 32 + 8) return fail(ANNS_ERR_INVALID_ARG, "file too short");
  uint64_t sum = 0;
  std::memcpy(&sum, buf.data() + buf.size() - 8, 8);
  if (sum != fnv1a(buf.data(), buf.size() - 8)) return fail(ANNS_ERR_INVALID_ARG, "checksum mismatch: corrupt file");
  Reader r(buf);
  char magic[8];
  r.get(magic, 8);
  if (std::memcmp(magic, kMagic, 8) != 0) return fail(ANNS_ERR_INVALID_ARG, "not an index file (magic)");
  if (r.val<uint32_t>() != kVersion) return fail(ANNS_ERR_INVALID_ARG, "unsupported file version");
  const uint32_t flags = r.val<uint32_t>();
  const int64_t n = r.val<int64_t>(), dim = r.val<int64_t>(), nlist = r.val<int64_t>(), M = r.val<int64_t>();
  if (!r.ok || n < 0 || dim < 1 || nlist < 1 || M < 1 || M > ANNS_MAX_M || dim % M || n > INT32_MAX ||
      nlist > INT32_MAX || dim > (1 << 20))
    return fail(ANNS_ERR_INVALID_ARG, "bad shape in file");
  const int64_t dsub = dim / M;
  const size_t need = (size_t)nlist * dim * 4 + (size_t)M * ANNS_KSUB * dsub * 4 + (size_t)nlist * 8 +
                      (size_t)n * M + (size_t)n * 8;
  if (need > buf.size()) return fail(ANNS_ERR_INVALID_ARG, "file shorter than its shapes");
  std::vector<float> cent((size_t)nlist * dim), books((size_t)M * ANNS_KSUB * dsub);
  std::vector<int64_t> llen(nlist), ids(n);
  std::vector<uint8_t> codes((size_t)n * M);
  r.get(cent.data(), cent.size() * 4);
  r.get(books.data(), books.size() * 4);
  r.get(llen.data(), llen.size() * 8);
  r.get(codes.data(), codes.size());
  r.get(ids.data(), ids.size() * 8);
  anns_predictor pred{};
  if (flags & 1u) r.get(&pred, sizeof pred);
  int32_t nsv = 0, tn = 0;
  double ratio = 0.0;
  float gamma = 0.f, inv_step = 0.f, mean[5] = {}, inv_std[5] = {};
  std::vector<float> svr;
  if (flags & 2u) {
    nsv = r.val<int32_t>(); tn = r.val<int32_t>(); ratio = r.val<double>();
    gamma = r.val<float>(); inv_step = r.val<float>();
    r.get(mean, 20); r.get(inv_std, 20);
    if (!r.ok || nsv < 1 || nsv > ANNS_SVR_MAX_SAMPLES) return fail(ANNS_ERR_INVALID_ARG, "bad SVR model in file");
    svr.resize((size_t)nsv * 6);
    r.get(svr.data(), svr.size() * 4);
  }
  if (!r.ok || r.pos != buf.size() - 8) return fail(ANNS_ERR_INVALID_ARG, "file size does not match its contents");
  std::vector<int32_t> list_of(n);
  int64_t row = 0;
  for (int64_t l = 0; l < nlist; ++l) {
    if (llen[l] < 0 || llen[l] > n - row) return fail(ANNS_ERR_INVALID_ARG, "bad list sizes in file");
    for (int64_t v = 0; v < llen[l]; ++v) list_of[row++] = (int32_t)l;
  }
  if (row != n) return fail(ANNS_ERR_INVALID_ARG, "list sizes do not add up to n");
  anns_build_desc d{};
  d.n = n; d.dim = dim; d.nlist = nlist; d.M = M; d.ksub = ANNS_KSUB;
  d.centroids = cent.data(); d.codebooks = books.data(); d.codes = codes.data(); d.list_of = list_of.data();
  d.ids = ids.data(); d.on_device = 0; d.device = device;
  anns_index* ix = nullptr;
  int rc = anns_build_index_from_arrays(&d, &ix);
  if (rc) return rc;
  if (flags & 1u) rc = anns_set_predictor(ix, &pred);
  if (rc == ANNS_OK && (flags & 2u)) {
    anns_svr_model m{};
    m.nsv = nsv; m.sv = svr.data(); m.beta = svr.data() + (size_t)nsv * 5; m.gamma = gamma;
    for (int i = 0; i < 5; ++i) { m.mean[i] = mean[i]; m.inv_std[i] = inv_std[i]; }
    m.table_n = tn; m.table_ratio = ratio; m.inv_step = inv_step;
    rc = anns_set_svr(ix, &m);
  }
  if (rc) {
    anns_free(ix);
    return rc;
  }
  *out = ix;
  return ANNS_OK;
}
