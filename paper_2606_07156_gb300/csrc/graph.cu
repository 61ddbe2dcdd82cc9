// Whole-search CUDA graphs and the autotuner (the batching side of the
// scheduling of Section 4.3).
//
// A graph is captured from the same launch sequence as anns_search, run on a
// private copy of the index handle: the copy shares the index arrays, options
// and predictor, but gets its own workspace, allocated before capture, so the
// captured kernels keep valid scratch pointers whatever else runs on the
// index. Nothing inside the captured sequence allocates or synchronises.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"

struct anns_graph {
  anns::Index shadow;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace anns {
namespace {

struct DeviceGuardG {
  int prev = 0;
  explicit DeviceGuardG(int d) { cudaGetDevice(&prev); cudaSetDevice(d); }
  ~DeviceGuardG() { cudaSetDevice(prev); }
};

// Copy of the handle with no workspace, staging or profiling state.
void make_shadow(const Index& ix, Index& sh) {
  sh = ix;
  sh.ws_d2 = nullptr; sh.ws_probes = nullptr; sh.ws_probe_d2 = nullptr; sh.ws_bits = nullptr;
  sh.ws_feat = nullptr; sh.ws_qt = nullptr; sh.ws_counter = nullptr; sh.ws_lists = nullptr;
  sh.ws_sched = nullptr; sh.ws_tc = nullptr; sh.st_q = nullptr; sh.st_out = nullptr; sh.st_pq = nullptr;
  sh.ws_tc_cap = 0;
  sh.ws_tc_valid = false;
  sh.ws_grp = nullptr;
  sh.ws_grp_cap = 0;
  sh.ws_qt_cap = sh.ws_d2_cap = sh.ws_pair_cap = sh.ws_counter_cap = sh.ws_lists_cap = 0;
  sh.ws_sched_cap = sh.st_q_cap = sh.st_out_cap = sh.st_pq_cap = 0;
  sh.ws_nq = sh.ws_nprobe = 0;
  sh.prof_on = false;
  sh.prof_pending = 0;
  for (auto& set : sh.prof_ev)
    for (cudaEvent_t& e : set) e = nullptr;
}

}  // namespace
}  // namespace anns

using namespace anns;

extern "C" int anns_graph_capture(anns_index* ix, const float* Q, int64_t nq, int32_t nprobe,
                                  const int32_t* nprobe_per_q, int32_t k, const int32_t* k_per_q,
                                  const anns_precision_policy* pol, int64_t* ids_out, float* dists_out,
                                  anns_graph** out) {
  if (!out) return fail(ANNS_ERR_INVALID_ARG, "null out");
  *out = nullptr;
  int rc = check_search_args(ix, Q, nq, nprobe, k, pol, ids_out, dists_out);
  if (rc) return rc;
  if (nq == 0) return fail(ANNS_ERR_INVALID_ARG, "cannot capture an empty batch");
  DeviceGuardG g(ix->device);
  anns_precision_policy plain{};
  plain.lut_mode = ANNS_LUT_PLAIN_FP32;
  const anns_precision_policy& P = pol ? *pol : plain;
  anns_graph* gr = new anns_graph();
  make_shadow(*ix, gr->shadow);
  cudaStream_t st = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete gr;
    return cuda_fail(e, "capture stream");
  }
  // one ordinary run: allocates the workspace and sets kernel attributes
  rc = search_sequence(gr->shadow, Q, nq, nprobe, nprobe_per_q, k, k_per_q, P, ids_out, dists_out, st, false);
  if (rc == ANNS_OK) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "search before capture");
  }
  if (rc == ANNS_OK) {
    e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "begin capture");
    } else {
      const int rs = search_sequence(gr->shadow, Q, nq, nprobe, nprobe_per_q, k, k_per_q, P, ids_out, dists_out,
                                     st, false);
      e = cudaStreamEndCapture(st, &gr->graph);
      if (rs != ANNS_OK) rc = rs;
      else if (e != cudaSuccess) rc = cuda_fail(e, "end capture");
    }
  }
  if (rc == ANNS_OK) {
    e = cudaGraphInstantiate(&gr->exec, gr->graph, 0);
    if (e != cudaSuccess) rc = cuda_fail(e, "graph instantiate");
  }
  cudaStreamDestroy(st);
  if (rc != ANNS_OK) {
    anns_graph_free(gr);
    return rc;
  }
  *out = gr;
  return ANNS_OK;
}

extern "C" int anns_graph_launch(anns_graph* gr, void* stream) {
  if (!gr || !gr->exec) return fail(ANNS_ERR_INVALID_ARG, "null graph");
  DeviceGuardG g(gr->shadow.device);
  cudaError_t e = cudaGraphLaunch(gr->exec, (cudaStream_t)stream);
  return e == cudaSuccess ? ANNS_OK : cuda_fail(e, "graph launch");
}

extern "C" void anns_graph_free(anns_graph* gr) {
  if (!gr) return;
  DeviceGuardG g(gr->shadow.device);
  if (gr->exec) cudaGraphExecDestroy(gr->exec);
  if (gr->graph) cudaGraphDestroy(gr->graph);
  free_workspace(gr->shadow);
  delete gr;
}

extern "C" int anns_autotune(anns_index* ix, const float* Q, int64_t nq, int32_t nprobe,
                             const int32_t* nprobe_per_q, int32_t k, const int32_t* k_per_q,
                             const anns_precision_policy* pol, int32_t reps, anns_tune_result* results,
                             int32_t cap, int32_t* n_results, void* stream) {
  // outputs go to temporary buffers: pass non-null placeholders to the checks
  int rc = check_search_args(ix, Q, nq, nprobe, k, pol, Q, Q);
  if (rc) return rc;
  if (nq == 0) return fail(ANNS_ERR_INVALID_ARG, "cannot tune on an empty batch");
  if (reps < 1 || reps > 1000) return fail(ANNS_ERR_INVALID_ARG, "reps must be in [1, 1000]");
  if (cap < 0 || (cap > 0 && !results)) return fail(ANNS_ERR_INVALID_ARG, "null results");
  DeviceGuardG g(ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  anns_precision_policy plain{};
  plain.lut_mode = ANNS_LUT_PLAIN_FP32;
  const anns_precision_policy& P = pol ? *pol : plain;
  void* ids = nullptr;
  void* dists = nullptr;
  cudaError_t e = cudaMalloc(&ids, (size_t)nq * k * 8);
  if (e == cudaSuccess) e = cudaMalloc(&dists, (size_t)nq * k * 4);
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  if (e != cudaSuccess) rc = cuda_fail(e, "autotune setup");
  const int kern0 = ix->opt_kernel, sched0 = ix->opt_schedule;
  const int64_t qchunk0 = ix->opt_qchunk;
  struct Cand { int kernel, schedule; int64_t qchunk; };
  std::vector<Cand> cands = {{ANNS_KERNEL_BASIC, ANNS_SCHED_NATURAL, 0}, {ANNS_KERNEL_BASIC, ANNS_SCHED_LPT, 0},
                             {ANNS_KERNEL_SPLIT, ANNS_SCHED_NATURAL, 0}, {ANNS_KERNEL_SPLIT, ANNS_SCHED_LPT, 0},
                             {ANNS_KERNEL_LIST_MAJOR, ANNS_SCHED_NATURAL, 0}};
  // the grouped kernel under both query orders, with its automatic work order
  // and with query chunks of a half and a quarter of the batch (at least 256)
  std::vector<int64_t> chunks = {0};
  for (int64_t c : {nq / 2, nq / 4})
    if (c >= 256 && std::find(chunks.begin(), chunks.end(), c) == chunks.end()) chunks.push_back(c);
  for (int sched : {ANNS_SCHED_NATURAL, ANNS_SCHED_LPT})
    for (int64_t c : chunks) cands.push_back({ANNS_KERNEL_GROUPED, sched, c});
  std::vector<anns_tune_result> got;
  for (const Cand& c : cands) {
    if (rc != ANNS_OK) break;
    ix->opt_kernel = c.kernel;
    ix->opt_schedule = c.schedule;
    ix->opt_qchunk = c.qchunk;
    // one untimed run (allocations, attributes); a configuration this index
    // cannot run (a list-major table too large) is skipped
    int r = search_sequence(*ix, Q, nq, nprobe, nprobe_per_q, k, k_per_q, P, (int64_t*)ids, (float*)dists, s,
                            false);
    if (r == ANNS_ERR_UNSUPPORTED) continue;
    if (r != ANNS_OK) { rc = r; break; }
    e = cudaEventRecord(t0, s);
    for (int i = 0; i < reps && e == cudaSuccess && r == ANNS_OK; ++i)
      r = search_sequence(*ix, Q, nq, nprobe, nprobe_per_q, k, k_per_q, P, (int64_t*)ids, (float*)dists, s,
                          false);
    if (r != ANNS_OK) { rc = r; break; }
    if (e == cudaSuccess) e = cudaEventRecord(t1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (e != cudaSuccess) { rc = cuda_fail(e, "autotune timing"); break; }
    anns_tune_result t;
    t.kernel = c.kernel;
    t.schedule = c.schedule;
    t.ms = ms / (float)reps;
    t.qchunk = c.qchunk;
    got.push_back(t);
  }
  ix->opt_kernel = kern0;
  ix->opt_schedule = sched0;
  ix->opt_qchunk = qchunk0;
  if (rc == ANNS_OK && !got.empty()) {
    size_t best = 0;
    for (size_t i = 1; i < got.size(); ++i)
      if (got[i].ms < got[best].ms) best = i;
    ix->opt_kernel = got[best].kernel;
    ix->opt_schedule = got[best].schedule;
    ix->opt_qchunk = got[best].qchunk;
    for (size_t i = 0; i < got.size() && (int)i < cap; ++i) results[i] = got[i];
    if (n_results) *n_results = (int32_t)got.size();
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (ids) cudaFree(ids);
  if (dists) cudaFree(dists);
  return rc;
}
