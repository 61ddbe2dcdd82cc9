// Library-internal declarations shared by the translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "anns_amp.h"

namespace anns {

struct Subspaces;  // sub-space partitions (subspace.cu)

constexpr int kKsub = 256;
constexpr int kTileVecs = 32;         // vectors per code tile (one per lane)
constexpr int kChunkBytes = 16;       // code bytes a lane loads at once
constexpr int kTileChunkBytes = 512;  // one 16-byte chunk for all 32 lanes
constexpr int kNFeat = 5, kH1 = 32, kH2 = 32, kNCls = 5;
// Device status word values (Index::dev_status, ANNS_TAP_STATUS).
constexpr int ANNS_DEV_TIMEOUT = 1;   // a bounded wait in a kernel ran out

// Device-resident index (Section 2.1: IVF lists + PQ codes, one shared codebook).
//
// Packed code layout: list l owns tiles [tile_off[l], tile_off[l+1]); a tile
// holds 32 vectors and nchunk = Mp/16 chunks of 512 bytes. Byte m of vector
// (tile t, lane i) sits at  codes + (t*nchunk + m/16)*512 + i*16 + m%16, so a
// warp reads one chunk of a tile with one coalesced 16-byte load per lane.
// Vectors past n_l in a list's last tile have all-zero codes and are masked.
struct Index {
  int device = 0;
  int64_t n = 0, dim = 0, nlist = 0, M = 0, dsub = 0, Mp = 0, nchunk = 0;
  int64_t ntiles = 0, max_list = 0;
  bool ids32 = false;           // every id in [INT32_MIN, INT32_MAX): 32-bit ids in the 128-entry top-k lists
  float* centroids = nullptr;   // [nlist*dim]
  float* codebooks = nullptr;   // [M*256*dsub]
  uint8_t* codes = nullptr;     // [ntiles*nchunk*512]
  int64_t* ids = nullptr;       // [n] user ids in list order
  int32_t* list_len = nullptr;  // [nlist]
  int64_t* vec_off = nullptr;   // [nlist+1]
  int64_t* tile_off = nullptr;  // [nlist+1]
  float* radius = nullptr;      // [nlist] covering radius, FP64-derived
  // Per-list table P_l[m][c] = fl32(||y_mc||^2 + fl32(2 <c_lm, y_mc>)), rows
  // M..Mp-1 zero: [nlist * Mp * 256]. With the per-query table Q it gives the
  // pair's LUT T' = P_l - 2 Q_q (the LUT shifted by ||r_m||^2, Section 2.1).
  float* ltab = nullptr;
  int32_t* order = nullptr;     // [nlist] list ids by size, largest first (ties by id)
  // CL fast path (coarse_tc.cu): centroid mean; per operand format (BF16,
  // FP16, FP8 E4M3) the centred, scaled, rounded centroids [nlist * Dp] and
  // their rows (cn, cd, cs: [3 * nlist]); device status word
  float* tc_mu = nullptr;
  void* tc_c[3] = {};
  float* tc_crows[3] = {};
  int* dev_status = nullptr;
  // host copies of the small per-list tables
  std::string err;
  int64_t* h_list_len64 = nullptr;
  float* h_radius = nullptr;
  // workspace of the last search
  int64_t ws_nq = 0, ws_nprobe = 0;
  float* ws_d2 = nullptr;        // [nq*nlist]
  int32_t* ws_probes = nullptr;  // [nq*nprobe]
  float* ws_probe_d2 = nullptr;  // [nq*nprobe]
  uint8_t* ws_bits = nullptr;    // [nq*nprobe]
  float* ws_feat = nullptr;      // [nq*nprobe*5]
  float* ws_qt = nullptr;        // [nq*Mp*256] per-query tables 2 Q_q
  size_t ws_qt_cap = 0;
  size_t ws_d2_cap = 0, ws_pair_cap = 0;
  int* ws_counter = nullptr;     // work counter of the list-major kernel
  size_t ws_counter_cap = 0;
  void* ws_lists = nullptr;      // list-major work: per-list counts/offsets, pairs, partial top-k
  size_t ws_lists_cap = 0;
  void* ws_sched = nullptr;      // query order of the LPT schedule (schedule.cu)
  size_t ws_sched_cap = 0;
  void* ws_grp = nullptr;        // query-major partial top-k of the grouped search
  size_t ws_grp_cap = 0;
  void* ws_tc = nullptr;         // BF16 centred queries, norms, candidate counts (coarse_tc.cu)
  size_t ws_tc_cap = 0;
  bool ws_tc_valid = false;      // the last search (or anns_locate) used the CL fast path
  int ws_tc_prec = 0;            // ... with this operand format
  int64_t ws_tc_nq = 0;          // ... for this many queries
  int opt_kernel = 0;            // ANNS_KERNEL_* (anns_set_option)
  int opt_schedule = 0;          // ANNS_SCHED_*
  int64_t opt_qchunk = 0;        // grouped kernel: queries per chunk (0 = automatic)
  int opt_nibble = 1;            // grouped search: pairs on <= 4-bit tables eight to a word
  long long opt_wait_cycles = 0; // limit of the CL GEMM's main-loop waits in clock cycles (0 = about 1 s)
  // staging for anns_search_host
  void* st_q = nullptr; size_t st_q_cap = 0;
  void* st_out = nullptr; size_t st_out_cap = 0;
  void* st_pq = nullptr; size_t st_pq_cap = 0;
  // stage timing (anns_profile): pending event sets, accumulated ms
  static constexpr int kProfSlots = 64, kStages = ANNS_PROFILE_STAGES;
  bool prof_on = false;
  cudaEvent_t prof_ev[kProfSlots][kStages + 1] = {};
  int prof_pending = 0;
  double prof_ms[kStages] = {};
  int64_t prof_count = 0;
  // learned predictor (FP16 inference copy + normalisation), see predictor.cu
  bool has_mlp = false;
  void* mlp_dev = nullptr;       // device MlpParams16
  anns_predictor mlp_host{};     // FP32 master copy of the installed predictor
  // SVR-RBF model (policy ANNS_LUT_SVR): device [sv nsv*5 | beta nsv | table tn] floats
  bool has_svr = false;
  float* svr_dev = nullptr;
  int svr_nsv = 0, svr_tn = 0;
  float svr_gamma = 0.f, svr_inv_step = 0.f, svr_mean[5] = {}, svr_inv_std[5] = {};
  double svr_ratio = 0.0;
  std::vector<float> svr_host;   // [sv nsv*5 | beta nsv]: the installed model, for anns_save
  Subspaces* ss = nullptr;       // the paper's sub-space partitions (anns_build_subspaces)
};

void free_subspaces(Index& ix);

void set_error(const std::string& msg);
// Counts one kernel launch enqueued by the library (host side; a launch into a
// stream being captured counts once, its replays not at all).
void note_launch();
int64_t launch_count();
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

// Grows *p to at least `bytes` (cudaFree + cudaMalloc). Returns 0 or an error.
int grow(void** p, size_t* cap, size_t bytes);

// ---- launchers (all asynchronous on `s`) ----
// CL: D2[q][l] by the FP32 rule, then per-query top-nprobe by (d, l).
cudaError_t launch_coarse(const Index& ix, const float* Q, int64_t nq, int nprobe,
                          const int32_t* nprobe_per_q, float* d2, int32_t* probes,
                          float* probe_d2, cudaStream_t s, cudaEvent_t between = nullptr);
// CL fast path: tensor-core distances with BF16, FP16 or FP8 E4M3 operands
// (ANNS_PREC_*), then the exact re-rank (coarse_tc.cu).
bool coarse_tc_format(int prec);
int coarse_tc_dp(const Index& ix, int prec);
int prepare_coarse_tc(Index& ix, const std::vector<float>& cent);
size_t coarse_tc_workspace_bytes(const Index& ix, int64_t nq);
const int* coarse_tc_candidates(const Index& ix, const void* ws, int64_t nq);
cudaError_t launch_coarse_tc(const Index& ix, int prec, const float* Q, int64_t nq, int nprobe,
                             const int32_t* nprobe_per_q, void* ws, float* dt, int32_t* probes,
                             float* probe_d2, cudaStream_t s);
// Per-query tables 2*Q_q[m][c] = 2 <q_m, y_mc> (FP32 dot rule), rows M..Mp-1 zero.
cudaError_t launch_query_tables(const Index& ix, const float* Q, int64_t nq, float* qt, cudaStream_t s);
// Precision choice per (query, probe rank).
int launch_policy(const Index& ix, const anns_precision_policy& pol, int64_t nq, int nprobe,
                  const int32_t* nprobe_per_q, const int32_t* probes, const float* probe_d2,
                  uint8_t* bits, float* feat, cudaStream_t s);
// Table widths a query-major launch serves: all (an FP32 table and a level
// table of up to 16 bits), FP32 pairs only, or 1..8-bit pairs only (no FP32
// table: fewer bytes of shared memory per block, more blocks per SM).
enum { QM_TABLES_ALL = 0, QM_TABLES_FP32 = 1, QM_TABLES_NARROW = 2 };
// RC + LC + quantise + DC + TS for every query; `order` (NULL = 0..nq-1) is
// the order in which blocks take the queries. skip_narrow 1 leaves out the
// 1..8-bit pairs of probe rank >= 1, 2 those of every rank. With
// QM_TABLES_NARROW only the 1..8-bit pairs are scanned, and part_d / part_i
// (or NULL), the query's top-k over its other pairs ([nq * k]), bound the
// scan and join the final merge.
cudaError_t launch_search(const Index& ix, const float* qt, int64_t nq, int nprobe,
                          const int32_t* nprobe_per_q, int k, const int32_t* k_per_q,
                          const int32_t* probes, const float* probe_d2, const uint8_t* bits,
                          const int32_t* order, int64_t* ids_out, float* dists_out, cudaStream_t s,
                          int skip_narrow = 0, int tables = QM_TABLES_ALL, const float* part_d = nullptr,
                          const int64_t* part_i = nullptr);
// Longest-first query order (schedule.cu) into a workspace of
// lpt_workspace_bytes(nq); the order is at lpt_order_ptr(ws, nq).
size_t lpt_workspace_bytes(int64_t nq);
int32_t* lpt_order_ptr(void* ws, int64_t nq);
// `bits` (NULL = every pair FP32) weights each pair's lookups by its table
// width; `skip_narrow` leaves out the pairs the grouped kernel takes.
cudaError_t launch_lpt_order(const Index& ix, const int32_t* probes, const int32_t* npq, int64_t nq,
                             int nprobe, void* ws, cudaStream_t s, const uint8_t* bits = nullptr,
                             bool skip_narrow = false);
// The whole search sequence of anns_search on stream s (abi.cu), for an index
// whose workspace is already large enough when `no_alloc` is set.
int search_sequence(Index& ix, const float* Q, int64_t nq, int nprobe, const int32_t* nprobe_per_q, int k,
                    const int32_t* k_per_q, const anns_precision_policy& P, int64_t* ids_out,
                    float* dists_out, cudaStream_t s, bool profile);
// Grows every workspace buffer a search of this shape needs.
int reserve_search(Index& ix, int64_t nq, int nprobe, int k, const anns_precision_policy& P,
                   const int32_t* nprobe_per_q);
// Frees the workspace buffers (not the index arrays).
void free_workspace(Index& ix);

// List-major search (search_lists.cu): work regrouped by list (invert.cu),
// one warp per (query, list) pair, then a per-query merge.
// Buckets are (query chunk, list) pairs, key c * nlist + l with c = q / qchunk
// (one chunk unless the grouped kernel asks for more).
struct ListWork {
  int* cnt; int* off; int* ioff; int* fill;  // [nbuckets + 1] each
  int32_t* pairs;                           // [nq * nprobe]
  float* part_d; int64_t* part_i;           // [nq * nprobe * k]
  int* counter;
  int64_t qchunk;                           // queries per chunk
  int nbuckets;                             // chunks * nlist
  int* gtab;                                // grouped kernel: bucket of each group [<= pairs + nbuckets]
  // a second set of buckets for the grouped search's pairs on tables of at
  // most 4 bits (groups of eight; the sets above then hold the 5..8-bit pairs)
  int *cnt4, *off4, *ioff4, *fill4, *gtab4, *counter4;
  int32_t* pairs4;
};
// With narrow_bits, only the pairs of probe rank >= 1 on tables of blo..bhi bits.
cudaError_t launch_invert(const Index& ix, const int32_t* probes, const int32_t* npq, int64_t nq,
                          int nprobe, int batch, const ListWork& w, cudaStream_t s,
                          const uint8_t* narrow_bits = nullptr, int blo = 1, int bhi = 8);
// Warps per block the list-major kernel gets for tables of `table_bytes_per_entry`.
int list_major_warps(const Index& ix, int table_bytes_per_entry);
cudaError_t launch_search_lists(const Index& ix, const float* qt, int64_t nq, int nprobe,
                                const int32_t* nprobe_per_q, int k, const int32_t* k_per_q,
                                const int32_t* probes, const float* probe_d2, const uint8_t* bits,
                                int table_bytes_per_entry, const ListWork& w, int64_t* ids_out,
                                float* dists_out, cudaStream_t s);
// Grouped search (search_grouped.cu): the pairs on 1..8-bit tables packed four
// queries to a shared-memory word per list, the wide pairs query-major, then a
// per-query merge. k <= 128.
bool grouped_supported(const Index& ix, int k);
// Queries per chunk of the grouped kernel's work order: chunks whose query
// tables fit in L2 beside the list tables and codes, when those fit; else nq.
int64_t grouped_qchunk(const Index& ix, int64_t nq);
size_t grouped_workspace_bytes(int64_t nq, int k);
cudaError_t launch_search_grouped(const Index& ix, const float* qt, int64_t nq, int nprobe,
                                  const int32_t* nprobe_per_q, int k, const int32_t* k_per_q,
                                  const int32_t* probes, const float* probe_d2, const uint8_t* bits,
                                  const ListWork& w, void* qm_ws, int64_t* ids_out, float* dists_out,
                                  cudaStream_t s, cudaEvent_t after_qm = nullptr,
                                  cudaEvent_t after_packed = nullptr, cudaEvent_t after_nibble = nullptr,
                                  const int32_t* qm_order = nullptr);
// Pair-level debug paths; qt are the queries' tables from launch_query_tables.
cudaError_t launch_compute_luts(const Index& ix, const float* Q, const float* qt, int64_t nq,
                                const int32_t* pq, const int32_t* pl, const uint8_t* pb,
                                int64_t npairs, float* T_out, uint16_t* t_out, double* scale_out,
                                cudaStream_t s);
cudaError_t launch_scan_pairs(const Index& ix, const float* Q, const float* qt, int64_t nq,
                              const int32_t* pq, const int32_t* pl, const uint8_t* pb,
                              int64_t npairs, const int64_t* off, float* dist_out, int32_t* S_out,
                              cudaStream_t s);

// Index training (train.cu): Lloyd k-means of the S rows of X [S x dim]
// (device) into C [k x dim] (device), and the nearest centroid of each row
// (FP32 rule, ties to the lower index) with its distance.
int kmeans(const float* X, int64_t S, int64_t dim, int64_t k, int iters, float* C, cudaStream_t s);
int nearest(const float* X, int64_t nrows, int64_t dim, const float* C, int64_t k, int32_t* a, float* dist,
            cudaStream_t s);

}  // namespace anns

// The opaque handle of the C ABI is the internal index.
struct anns_index : public anns::Index {};

namespace anns {
int check_search_args(anns_index* ix, const float* Q, int64_t nq, int32_t nprobe, int32_t k,
                      const anns_precision_policy* pol, const void* ids_out, const void* dists_out);
}
