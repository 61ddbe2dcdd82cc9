/*
 * anns_amp.h — C ABI of the GB300 (sm_103a) adaptive mixed-precision IVF-PQ search.
 *
 * The search is the five-stage cluster-based ANNS pipeline of Section 2.1
 * (Fig. 1): cluster locating (CL), residual calculation (RC), LUT construction
 * (LC), distance calculation (DC) and top-k selection (TS), with a per-(query,
 * probed list) precision choice in the spirit of Section 3 (cluster-level
 * precision predicted from scale, radius and query distance, Section 3.3).
 *
 * Conventions for every entry point:
 *  - Return ANNS_OK (0) on success or a negative ANNS_ERR_* code. The message
 *    of the last failure on the calling thread is returned by anns_last_error().
 *    No C++ exception crosses this boundary.
 *  - Pointers documented "device" must be CUDA device (or managed) memory on
 *    the index's device; "host" pointers are ordinary host memory. The caller
 *    owns every buffer it passes; the library copies what it keeps.
 *  - Distances are squared L2. Results are sorted by ascending (distance, id);
 *    missing results are padded with id -1 and distance +inf.
 *  - Work is enqueued on the given cudaStream_t (passed as void*, NULL = the
 *    legacy default stream) and is asynchronous unless stated otherwise.
 *  - Only one search may run on an index at a time: the index owns its
 *    workspace. Searches on distinct indexes may run concurrently.
 */
#ifndef ANNS_AMP_H
#define ANNS_AMP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ANNS_OK 0
#define ANNS_ERR_INVALID_ARG (-1)
#define ANNS_ERR_OOM (-2)
#define ANNS_ERR_CUDA (-3)
#define ANNS_ERR_TIMEOUT (-4)
#define ANNS_ERR_UNSUPPORTED (-5)

#define ANNS_KSUB 256      /* codebook entries per sub-space: codes are uint8 */
#define ANNS_MAX_M 128     /* sub-spaces per vector */
#define ANNS_MAX_NPROBE 128
#define ANNS_MAX_K 128

typedef struct anns_index anns_index; /* opaque, library-owned */

/* Index arrays (Section 2.1: IVF lists + PQ with one codebook shared by all
 * clusters, trained on residuals).
 *  centroids [nlist * dim] float32, row-major.
 *  codebooks [M * 256 * dsub] float32, dsub = dim / M; entry (m, c) holds the
 *            sub-vector for dimensions [m*dsub, (m+1)*dsub).
 *  codes     [n * M] uint8, row-major; codes[i*M + m] indexes codebook m.
 *  list_of   [n] int32 in [0, nlist): the list (cluster) of each vector.
 *  ids       [n] int64 user ids, or NULL for the row index. Ties in distance
 *            are broken by ascending id.
 *  on_device 1 if the five arrays are device pointers, 0 if host pointers. */
typedef struct {
  int64_t n, dim, nlist, M, ksub;
  const float* centroids;
  const float* codebooks;
  const uint8_t* codes;
  const int32_t* list_of;
  const int64_t* ids;
  int32_t on_device;
  int32_t device; /* CUDA device ordinal the index lives on */
} anns_build_desc;

/* Builds an index on desc->device: copies the arrays, packs each list's codes
 * into the warp-interleaved 16-byte layout and derives per-list sizes and
 * covering radii (FP64, the r of Eq. 1). Synchronous. Errors: INVALID_ARG
 * (shape or value out of range, dim % M != 0, ksub != 256, M > 128, a list id
 * outside [0, nlist)), OOM, CUDA. *out is set only on success. */
int anns_build_index_from_arrays(const anns_build_desc* desc, anns_index** out);

/* Index training on the GPU (the offline IVF-PQ index of Section 2.1: Lloyd
 * k-means for the nlist centroids, k-means of 256 entries per sub-space on
 * the residuals for the PQ codebooks, then every vector's list and codes).
 * The paper fixes none of the following; they make training a deterministic
 * function of (base, desc), identical however the GPU schedules its threads:
 *   sample: row i is drawn when the SplitMix64 output of the state
 *     seed + (i + 1) * 0x9E3779B97F4A7C15 (mod 2^64) is below
 *     floor(target * 2^64 / n), target = nlist * per_centroid (every row
 *     when target >= n); drawn rows keep their order;
 *   k-means over S rows and k clusters: initial centroid j = sample row
 *     floor(j * S / k); each of `iters` iterations assigns every row to its
 *     nearest centroid by the FP32 distance rule of CL (ties to the lower
 *     index), sets each coordinate of a centroid with members to the exact
 *     sum of the members' FP32 values rounded once to FP32, divided (one IEEE
 *     FP32 division) by the member count, and gives the e-th empty centroid
 *     (ascending) the e-th farthest row from its centroid (ties to the lower
 *     row);
 *   PQ: a second sample of pq_sample rows (seed + 1), the residuals
 *     fl32(x - c) to their nearest centroid, one k-means of 256 clusters and
 *     pq_iters iterations per sub-space on that sub-space's coordinates;
 *   encoding: each row's nearest centroid, then per sub-space the nearest
 *     entry to the residual's sub-vector (FP32 rule, ties to the lower entry).
 * The index is then built as by anns_build_index_from_arrays (ids = row
 * index).
 *  base  float32 [n * dim], host (on_device = 0) or device memory.
 * Synchronous. Errors: INVALID_ARG (dim % M != 0, M > 128, dim / M > 16,
 * nlist > n, n >= 2^31, nlist > 2^20, iters < 0, per_centroid < 1,
 * pq_sample < 256, a sample smaller than its cluster count), OOM, CUDA. */
typedef struct {
  int64_t nlist, M;
  int32_t iters, pq_iters;
  uint64_t seed;
  int64_t per_centroid;   /* coarse sample = nlist * per_centroid rows */
  int64_t pq_sample;      /* rows whose residuals train the codebooks */
} anns_train_desc;
int anns_train_index(const float* base, int64_t n, int64_t dim, const anns_train_desc* desc,
                     int32_t on_device, int32_t device, anns_index** out);

/* The index's arrays, in list order, into host buffers (each may be NULL):
 *  centroids float [nlist * dim], codebooks float [M * 256 * dsub],
 *  codes uint8 [n * M] (row-major per vector), ids int64 [n] (the ids the
 *  search returns), list_len int64 [nlist] (vectors per list; list l's
 *  vectors follow list l-1's). Synchronous. Errors: INVALID_ARG, CUDA. */
int anns_export_index(anns_index* index, float* centroids, float* codebooks, uint8_t* codes, int64_t* ids,
                      int64_t* list_len);

/* Saves the index to a file and loads it back (no counterpart in the paper).
 * The file holds the shapes, the arrays of anns_export_index, the installed
 * MLP predictor and SVR model if any, and a 64-bit FNV-1a checksum of all
 * preceding bytes; it is little-endian. anns_load builds the index on
 * `device` as anns_build_index_from_arrays would from those arrays, then
 * installs the predictor and the SVR model: every search returns what the
 * saved index returned. Errors: INVALID_ARG (null argument, unreadable or
 * corrupt file: bad magic, version, shape or checksum), OOM, CUDA. */
int anns_save(anns_index* index, const char* path);
int anns_load(const char* path, int32_t device, anns_index** out);

/* The paper's sub-space precision granularity (Section 3.2: the dimensions
 * cut into slices and, inside each slice, the vectors clustered into
 * sub-spaces; Section 3.3: features per sub-space; Section 4.2: precision as
 * the operands' most significant bits; Section 5.3, Fig. 13: slices x
 * sub-spaces per slice in CL, and LC alike). anns_build_subspaces partitions
 * the index's centroids and codebooks:
 *   CL: slice s (`slices` slices of dim / slices consecutive dimensions) of
 *     the nlist centroids into K sub-spaces; LC: the 256 entries of each
 *     codebook m into K_lc groups; both by the k-means rules of
 *     anns_train_index (`iters` iterations) on the GPU. Per sub-space: its
 *     centre, size, and covering radius (FP64, squares summed over dimensions
 *     in ascending order, square root, rounded to FP32).
 *   uint8 maps: x8 = clamp(rint(fl32(fl32(x - lo) * inv)), 0, 255) (half to
 *     even), inv = fl32(255 / fl32(hi - lo)); CL: lo / hi = the smallest /
 *     largest centroid coordinate (queries use the same map); LC: the
 *     codebook's, applied to residuals fl32(q - c).
 * Errors: INVALID_ARG (slices not dividing dim, dim > 4096, K outside
 * [1, min(nlist, 1024)], slices * K > 16384, K_lc outside [1, 256]), OOM,
 * CUDA. Synchronous; replaces earlier partitions. */
typedef struct {
  int32_t slices, K, K_lc, iters;
} anns_subspace_desc;
int anns_build_subspaces(anns_index* index, const anns_subspace_desc* desc);

/* Sizes of the sub-spaces (host int64 [slices * K] and [M * K_lc], either NULL). */
int anns_subspace_sizes(anns_index* index, int64_t* cl_size, int64_t* lc_size);

/* A search whose CL and/or LC + DC run at sub-space precision.
 * Bits per (query, slice, sub-space) (CL; in LC per (pair, codebook m,
 * group)): with D_k the FP32-rule squared distance from the query's slice
 * (the pair's residual sub-vector) to centre k, d_k = fl32(sqrt(D_k)), k1 the
 * nearest centre (ties to the lower index), g = fl32(fl32(fl32(fl32(d_k -
 * d_k1) - fl32(3 r_k1)) - r_k) / r_k) (Eq. 2 with the distance measured
 * beyond the nearest sub-space; -inf when r_k = 0): 2 bits if g >= th[0],
 * else 4 if g >= th[1], else 6 if g >= th[2], else 8. Keeping b bits:
 * x_b = (x8 >> (8 - b)) << (8 - b).
 *  cl != 0: D2_int[l] = sum over slices and their dimensions of
 *    (q_b - c_b)^2, b the bits of (query, slice, sub-space of c_l's slice);
 *    the nprobe smallest (D2_int, l) are probed, ordered by their FP32-rule
 *    coarse distance. cl == 0: the FP32 CL of anns_search.
 *  lc != 0: T_int[m][c] = sum over the sub-vector's dimensions of
 *    (r_b - y_b)^2, b the bits of (pair, m, group of entry c); a vector's
 *    distance is S = sum_m T_int[m][code_m] (exact), the top-k by (S, id),
 *    reported as fl32(fl32(S) * fl32(1 / inv^2)). lc == 0: the plain FP32
 *    LUT of anns_search on the probed lists.
 *  low_counts: device uint64 [2] or NULL; atomically increased by the number
 *    of (query, list, slice) partial distances (CL) and of table entries
 *    (LC) computed below 8 bits.
 * Queries, ids_out and dists_out as for anns_search (device). Asynchronous
 * on cuda_stream. Errors: INVALID_ARG (no partitions, NaN threshold, as
 * anns_search), CUDA. */
typedef struct {
  float th_cl[3], th_lc[3];
  int32_t cl, lc;
} anns_subspace_policy;
int anns_search_subspace(anns_index* index, const float* queries, int64_t nq, int32_t nprobe, int32_t k,
                         const anns_subspace_policy* policy, int64_t* ids_out, float* dists_out,
                         unsigned long long* low_counts, void* cuda_stream);

/* Frees the index and all device memory it owns. NULL is a no-op. */
void anns_free(anns_index* index);

/* Precision of each (query, probed list) LUT (Section 3: cluster-level
 * precision). */
enum {
  ANNS_LUT_PLAIN_FP32 = 0,    /* FP32 LUT, FP32 accumulation, every pair */
  ANNS_LUT_FIXED_BITS = 1,    /* every pair at fixed_bits */
  ANNS_LUT_HEURISTIC_EQ2 = 2, /* Eq. 2 feature f = d' - 3 r1 - r2 against thresholds */
  ANNS_LUT_MLP = 3,           /* learned predictor with full-precision fallback */
  ANNS_LUT_EXPLICIT = 4,      /* caller-provided bits per (query, probe rank) */
  ANNS_LUT_SVR = 5            /* the SVR-RBF regressor of Section 3.4 (anns_set_svr) */
};
enum { ANNS_PREC_FP32 = 0, ANNS_PREC_BF16 = 1, ANNS_PREC_FP8E4M3 = 2, ANNS_PREC_FP16 = 3 };

typedef struct {
  int32_t lut_mode;        /* ANNS_LUT_* */
  int32_t fixed_bits;      /* 4, 6, 8, 12 or 16 (FIXED_BITS) */
  int32_t cl_prec;         /* coarse distances: ANNS_PREC_FP32, or a tensor-core GEMM
                              on centred operands scaled per row by a power of two,
                              in ANNS_PREC_BF16, ANNS_PREC_FP16 or ANNS_PREC_FP8E4M3
                              with FP32 accumulation, then every list within the
                              GEMM's error bound of the nprobe-th re-ranked by the
                              FP32 rule: same probes and distances as FP32 */
  int32_t lc_prec;         /* ANNS_PREC_* for the LUT build; FP32 only */
  float eq2_thresholds[4]; /* HEURISTIC_EQ2: g thresholds for 4, 6, 8, 12 bits */
  float fallback_margin;   /* MLP round-up margin tau (not NaN): the fewest bits b such
                              that fl32(max logit over widths <= b - max logit over
                              wider widths) >= tau (16 bits if none); tau = 0 is the
                              argmax, ties to the narrower width. A larger tau rounds
                              uncertain pairs up, towards full precision; a negative
                              tau takes a narrower width while its best logit is
                              within -tau of the wider ones'. */
  const uint8_t* pair_bits;/* EXPLICIT: device [nq * nprobe], 0 = FP32 */
  int32_t width_map;       /* HEURISTIC_EQ2 / MLP: 0 = widths as chosen; 1 = widths
                              mapped to this GPU's tables: 6 -> 8 bits (same table
                              cost, finer levels), 12 and 16 -> FP32 (a 16-bit table
                              gathers as slowly as FP32 and FP32 is exact) */
} anns_precision_policy;

/* Batched search (Section 2.1, stages CL -> RC -> LC -> DC -> TS).
 *  queries      device float32 [nq * dim].
 *  nprobe       lists probed per query, 1 <= nprobe <= min(nlist, 128).
 *  nprobe_per_q NULL, or device int32 [nq]: per-query nprobe, clamped to [0, nprobe].
 *  k            results per query, 1 <= k <= 128.
 *  k_per_q      NULL, or device int32 [nq]: per-query k, clamped to [0, k];
 *               slots beyond a query's k are padding.
 *  policy       precision choice (NULL = plain FP32).
 *  ids_out      device int64 [nq * k], dists_out device float32 [nq * k].
 * Within one precision policy the output is deterministic and equals the
 * CPU oracle's bit for bit. Errors: INVALID_ARG, OOM, CUDA. */
int anns_search(anns_index* index, const float* queries, int64_t nq, int32_t nprobe,
                const int32_t* nprobe_per_q, int32_t k, const int32_t* k_per_q,
                const anns_precision_policy* policy, int64_t* ids_out, float* dists_out,
                void* cuda_stream);

/* anns_search with HOST buffers: queries (host float32 [nq*dim]),
 * nprobe_per_q / k_per_q (host int32 [nq] or NULL) and ids_out / dists_out
 * (host). Copies in, searches and copies out on cuda_stream, then waits for
 * the stream. Host buffers should be pinned for full copy speed.
 * policy->pair_bits, if used, is still a device pointer. */
int anns_search_host(anns_index* index, const float* queries, int64_t nq, int32_t nprobe,
                     const int32_t* nprobe_per_q, int32_t k, const int32_t* k_per_q,
                     const anns_precision_policy* policy, int64_t* ids_out, float* dists_out,
                     void* cuda_stream);

/* Index facts. */
typedef struct {
  int64_t n, dim, nlist, M, dsub, Mp; /* Mp = M rounded up to 16 (packed code row) */
  int64_t code_bytes;                 /* bytes of packed codes in device memory */
  int64_t max_list;                   /* largest list */
  int32_t device;
} anns_index_info;
int anns_get_info(const anns_index* index, anns_index_info* out);

/* Debug taps: copy library state to a HOST buffer of `bytes` bytes
 * (synchronous). Taps of the last search (valid until the next search):
 *   PROBES   int32 [nq * nprobe]  probed lists by rank (-1 past a query's nprobe)
 *   PROBE_D2 float [nq * nprobe]  their FP32 coarse distances
 *   BITS     uint8 [nq * nprobe]  chosen bits per pair (0 = FP32 LUT)
 *   FEATURES float [nq * nprobe * 5] predictor features (MLP / EQ2 modes)
 *   COARSE_APPROX     float [nq * nlist] tensor-core distances D~ (last
 *                     search with cl_prec = BF16, FP16 or FP8E4M3)
 *   COARSE_CANDIDATES int32 [nq] lists re-ranked in FP32 per query (same)
 * Index taps:
 *   LIST_SIZES int64 [nlist], LIST_RADIUS float [nlist],
 *   PACKED_IDS int64 [n] (ids in list order, lists ascending),
 *   STATUS int32: the device status word (0 = ok, 1 = a bounded wait in a
 *   kernel timed out), reset to 0 by the read. */
enum {
  ANNS_TAP_PROBES = 0, ANNS_TAP_PROBE_D2 = 1, ANNS_TAP_BITS = 2, ANNS_TAP_FEATURES = 3,
  ANNS_TAP_COARSE_APPROX = 4, ANNS_TAP_COARSE_CANDIDATES = 5,
  ANNS_TAP_LIST_SIZES = 10, ANNS_TAP_LIST_RADIUS = 11, ANNS_TAP_PACKED_IDS = 12, ANNS_TAP_STATUS = 13
};
int anns_debug_tap(anns_index* index, int32_t what, void* out, size_t bytes);

/* LUT construction + quantisation for explicit pairs (RC + LC of Section 2.1
 * and the per-pair precision), with the same device code the search uses.
 * The FP32 LUT is the one the search evaluates: T'[m][c] = ||r_m - y_mc||^2
 * - ||r_m||^2 (the ADC distance is the coarse distance D2 plus sum_m T'),
 * formed as fl32(P_l - 2 Q_q) from a per-list and a per-query table (the
 * IVFADC look-up-table decomposition for residual PQ); the offset B of a
 * quantised pair is the exact sum of D2 and the M row minima, rounded once
 * to FP32.
 *  queries  device float32 [nq * dim]; pair_q, pair_l device int32 [npairs];
 *  pair_bits device uint8 [npairs] (0 = FP32 only).
 *  T_out     device float32 [npairs * M * 256] FP32 LUT, or NULL.
 *  t_out     device uint16  [npairs * M * 256] quantised levels, or NULL.
 *  scale_out device float64 [npairs * 4]: (Delta in FP64, B32, range, s), or
 *            NULL. */
int anns_compute_luts(anns_index* index, const float* queries, int64_t nq,
                      const int32_t* pair_q, const int32_t* pair_l, const uint8_t* pair_bits,
                      int64_t npairs, float* T_out, uint16_t* t_out, double* scale_out,
                      void* cuda_stream);

/* The quantiser's offset rule on arbitrary values (a test tap for the rule
 * that forms each quantised pair's offset B from D2 and the row minima; the
 * quantiser itself is a reading, the paper states none, Section 3.3): for
 * each of `nsets` sets of `n` FP32 values, the exact sum rounded once to the
 * nearest FP32 value (ties to even), independent of summation order.
 *  vals device float32 [nsets * n], set-major; 0 <= n < 1024, nsets <= 2^30.
 *  out  device float32 [nsets].
 * Asynchronous on `cuda_stream`. Errors: INVALID_ARG (null pointer with
 * nsets > 0, n out of range), CUDA. */
int anns_debug_exact_sum(const float* vals, int64_t nsets, int32_t n, float* out, void* cuda_stream);

/* ADC scan of whole lists for explicit pairs (DC of Section 2.1): for pair p,
 * the n_l distances of list pair_l[p] in list order are written at
 * dist_out + out_off[p] (device int64 [npairs]), and, for quantised pairs,
 * the integer sums S at S_out + out_off[p] (device int32, or NULL). */
int anns_scan_pairs(anns_index* index, const float* queries, int64_t nq,
                    const int32_t* pair_q, const int32_t* pair_l, const uint8_t* pair_bits,
                    int64_t npairs, const int64_t* out_off, float* dist_out, int32_t* S_out,
                    void* cuda_stream);

/* Stage timing with CUDA events recorded on the search stream around each
 * stage of anns_search:
 *   0 CL distances, 1 CL selection (the tensor-core CL: the whole stage in 1),
 *   2 precision choice plus the per-query tables, 3 the search kernels up to
 *   the grouped kernels (the whole LUT + scan + top-k for the query-major and
 *   list-major kernels; pair regrouping plus the query-major pass for the
 *   grouped search; the wide pass of the split search), 4 the grouped kernel
 *   of the 5..8-bit tables (of all narrow tables without nibble packing; the
 *   narrow pass of the split search), 5 the grouped kernel of the 4-bit
 *   tables packed eight to a word, 6 the grouped search's per-query merge
 *   (4 to 6 are 0 on the other kernels).
 *  enable  1 = start recording (and clear the totals), 0 = stop, -1 = leave as is.
 *  out_ms  host double [ANNS_PROFILE_STAGES] or NULL: accumulated
 *          milliseconds per stage since recording started (waits for the
 *          recorded searches to finish).
 *  count   host int64 or NULL: number of searches accumulated. */
#define ANNS_PROFILE_STAGES 7
int anns_profile(anns_index* index, int32_t enable, double* out_ms, int64_t* count);

/* Number of CUDA kernels the library has enqueued since it was loaded, on
 * every index and stream (host-side count: a launch into a stream being
 * captured counts once, graph replays do not count). */
int64_t anns_kernel_launches(void);

/* Failure detection (no counterpart in the paper, whose accelerator has no
 * waits that can fail): waits for `cuda_stream` (NULL = the legacy default
 * stream), then reads and clears the index's device status word.
 * Returns ANNS_OK, or ANNS_ERR_TIMEOUT when a bounded wait inside a kernel of
 * this index ran out since the last read (that call's output is invalid; the
 * index and the context stay usable). Errors: INVALID_ARG, CUDA, TIMEOUT. */
int anns_sync_status(anns_index* index, void* cuda_stream);

/* Index options.
 *  ANNS_OPT_KERNEL: which search kernel anns_search launches.
 *    ANNS_KERNEL_AUTO (default): grouped when the policy can choose tables of
 *      at most 8 bits (k <= 128), else query-major.
 *    ANNS_KERNEL_BASIC: query-major, one block per query walking its probes.
 *    ANNS_KERNEL_GROUPED: the pairs on 1..8-bit tables taken four per list,
 *      their byte tables interleaved so that one shared-memory gather serves
 *      four queries; the other pairs query-major; then a per-query merge
 *      (k <= 128).
 *    ANNS_KERNEL_LIST_MAJOR: the probed pairs regrouped by list; one warp per
 *      (query, list) pair, blocks of pairs sharing a list, work items taken
 *      largest list first; then a per-query merge of the pairs' top-k.
 *      UNSUPPORTED at search time if one table does not fit.
 *    ANNS_KERNEL_SPLIT: query-major in two passes split by table width: the
 *      FP32 and 12/16-bit pairs into a per-query partial top-k, then the
 *      1..8-bit pairs with byte tables only (no FP32 table in shared memory,
 *      so more blocks per SM), bounded by and merged with the partial.
 *  ANNS_OPT_SCHEDULE: the order in which the query-major kernel takes queries
 *    (the greedy load scheduling of Section 4.3, applied to queries).
 *    ANNS_SCHED_AUTO (default): longest first when nprobe_per_q is given (an
 *      uneven batch), else in query order.
 *    ANNS_SCHED_NATURAL: query order.
 *    ANNS_SCHED_LPT: longest first by the estimated cost sum over the probed
 *      lists of (list size + 768), bucketed within 12.5 %.
 *  ANNS_OPT_QCHUNK: queries per chunk of the grouped kernel's work order (its
 *    groups run chunk by chunk, each chunk largest list first, so that one
 *    chunk's query tables are in use at a time). 0 (default) = automatic:
 *    chunks whose query tables take half of L2 (at least 256 queries) when
 *    the list tables and codes fit in the other half, else one chunk.
 *    Values >= 1 fix the chunk.
 *  ANNS_OPT_WAIT_CYCLES: the limit, in SM clock cycles, of each wait inside
 *    the tensor-core CL kernel's main loop (its mbarrier waits on TMA copies,
 *    stage releases and the accumulator). 0 (default) = 2e9 cycles (about
 *    one second). A wait that runs out makes the kernel record a timeout in
 *    the index's status word (anns_sync_status), wait with the long limit for
 *    the copies and MMAs it has issued, free its tensor memory and return;
 *    the coarse stage's output is then invalid. Small values serve tests of
 *    this failure path.
 *  ANNS_OPT_NIBBLE: 1 (default) = in the grouped search (k <= 32), the pairs
 *    on tables of at most 4 bits are taken eight per list, their levels
 *    interleaved as nibbles so that one gather serves eight queries (the
 *    5..8-bit pairs stay four per word); 0 = all 1..8-bit pairs four per word.
 * Every kernel, schedule, chunk size and packing returns identical results.
 * Errors: INVALID_ARG. */
enum { ANNS_OPT_KERNEL = 0, ANNS_OPT_SCHEDULE = 1, ANNS_OPT_QCHUNK = 2, ANNS_OPT_WAIT_CYCLES = 3,
       ANNS_OPT_NIBBLE = 4 };
enum { ANNS_KERNEL_AUTO = 0, ANNS_KERNEL_BASIC = 1, ANNS_KERNEL_LIST_MAJOR = 2, ANNS_KERNEL_GROUPED = 3,
       ANNS_KERNEL_SPLIT = 4 };
enum { ANNS_SCHED_AUTO = 0, ANNS_SCHED_NATURAL = 1, ANNS_SCHED_LPT = 2 };
int anns_set_option(anns_index* index, int32_t option, int64_t value);

/* A whole search (the calls of anns_search) captured once as a CUDA graph on
 * fixed device buffers and replayed with one launch. The graph owns its own
 * workspace (allocated at capture), so searches on the index and other
 * graphs do not disturb it; the index arrays, options and installed predictor
 * are shared (the graph uses the kernel and schedule options set at capture,
 * and the predictor's current weights at each replay). The caller keeps the
 * buffers alive and may rewrite queries / nprobe_per_q / k_per_q / pair_bits
 * between replays; the graph must be freed before the index. Capture runs the
 * search once (outputs are written) and synchronises. Errors as anns_search. */
typedef struct anns_graph anns_graph;
int anns_graph_capture(anns_index* index, const float* queries, int64_t nq, int32_t nprobe,
                       const int32_t* nprobe_per_q, int32_t k, const int32_t* k_per_q,
                       const anns_precision_policy* policy, int64_t* ids_out, float* dists_out,
                       anns_graph** out);
int anns_graph_launch(anns_graph* graph, void* cuda_stream);
void anns_graph_free(anns_graph* graph);

/* Autotuner: times every available configuration on the given batch (reps
 * timed searches each, after one untimed): the query-major kernel in query
 * order and longest first, the list-major kernel, and the grouped kernel in
 * both query orders with its automatic work order and with query chunks of
 * a half and a quarter of the batch (when >= 256 queries). Installs the
 * fastest as the index's options and reports all of them (at most cap, in
 * trial order) with their mean milliseconds. Uses temporary output buffers;
 * synchronous. Errors as anns_search, plus INVALID_ARG for reps outside
 * [1, 1000]. */
typedef struct {
  int32_t kernel, schedule; /* ANNS_KERNEL_*, ANNS_SCHED_* */
  float ms;                 /* mean time of one search */
  int64_t qchunk;           /* ANNS_OPT_QCHUNK of the trial (0 = automatic) */
} anns_tune_result;
int anns_autotune(anns_index* index, const float* queries, int64_t nq, int32_t nprobe,
                  const int32_t* nprobe_per_q, int32_t k, const int32_t* k_per_q,
                  const anns_precision_policy* policy, int32_t reps, anns_tune_result* results,
                  int32_t cap, int32_t* n_results, void* cuda_stream);

/* Learned precision predictor: the regressor of Section 3.4 as a 5-32-32-5 MLP
 * classifier over the bit widths {4, 6, 8, 12, 16}, on the features of
 * Section 3.3 for probe rank j: (sqrt(D2_j) - sqrt(D2_0), r_0, r_j, sqrt(n_j),
 * j / nprobe), normalised as fl32(fl32(x - mean) * inv_std). FP32 master
 * weights, row-major [out][in]. Inference (policy ANNS_LUT_MLP) uses FP16
 * operands with FP32 accumulation, then the round-up rule on the logits
 * (policy->fallback_margin) and, if requested, the width map. */
typedef struct {
  float W1[32 * 5], b1[32], W2[32 * 32], b2[32], W3[5 * 32], b3[5];
  float mean[5], inv_std[5];
} anns_predictor;
typedef struct {
  int32_t epochs, batch; /* passes over the samples, samples per Adam step */
  float lr;              /* Adam step size (beta1 0.9, beta2 0.999, eps 1e-8) */
  uint64_t seed;         /* initial weights and sample order */
  int32_t label_map;     /* anns_train_predictor: 0 = classes of the label widths 4, 6, 8,
                            12, 16 ("needs FP32" trains as 16); 1 = the two tables of
                            the GB300 width map: labels 4, 6, 8 -> the 8-bit class,
                            12, 16 and "needs FP32" -> the 16-bit class; 2 = its three
                            tables: 4 -> the 4-bit class (nibble tables), 6 and 8 ->
                            the 8-bit class, 12, 16 and "needs FP32" -> 16 bits */
  float high_weight;     /* loss weight of samples whose class is 12 or 16 bits (a
                            missed wide pair costs recall, a missed narrow one only
                            speed); 0 is read as 1 */
} anns_train_cfg;

/* Installs / returns the index's predictor (host structs). */
int anns_set_predictor(anns_index* index, const anns_predictor* p);
int anns_get_predictor(const anns_index* index, anns_predictor* out);

/* Training set from training queries (device float32 [nq * dim]), uniform
 * nprobe and k (k + 1 <= 128). For every (query, probe rank) pair:
 *  feat_out  device float32 [nq * nprobe * 5]: raw features,
 *  label_out device uint8  [nq * nprobe]: the label (Section 3.3 / Fig. 6,
 *            read as "the fewest bits that keep the FP32 top-k"):
 *            tau = (d_k + d_{k+1}) / 2 of the FP32 search, margin = min over the
 *            list of |d - tau|, E(b) = max over the list of |dhat_b - d|; the
 *            fewest b in {4,6,8,12,16} with E(b) < margin, 0 if none (needs the
 *            FP32 LUT), 255 for a rank the query does not probe.
 * Synchronous. Reuses the index's search workspace. */
int anns_make_training_set(anns_index* index, const float* train_q, int64_t nq, int32_t nprobe,
                           int32_t k, float* feat_out, uint8_t* label_out, void* cuda_stream);

/* Weighted softmax cross-entropy and its gradient over n samples with the
 * MLP in `w`: (1/n) sum_i w_i CE_i with w_i = high_weight for classes 3 and 4
 * (12 and 16 bits), else 1. X device float32 [n * 5] raw features, cls device
 * uint8 [n] classes 0..4 (255 = skipped). grad_out host float32 [1413] in the
 * order W1 b1 W2 b2 W3 b3; loss_out host (or NULL). FP16-operand forward,
 * FP32 backward. Synchronous. */
int anns_mlp_grad(anns_index* index, const anns_predictor* w, const float* X, const uint8_t* cls,
                  int64_t n, float high_weight, float* grad_out, double* loss_out, void* cuda_stream);

/* Adam training on given samples (as for anns_mlp_grad), starting from and
 * returning the weights in *io (its normalisation is used as is). Synchronous. */
int anns_mlp_train(anns_index* index, const float* X, const uint8_t* cls, int64_t n,
                   const anns_train_cfg* cfg, anns_predictor* io, void* cuda_stream);

/* Training set + normalisation statistics + seeded initial weights + Adam
 * training on the GPU, then installs the predictor in the index (and copies
 * it to *out if not NULL). Synchronous. */
int anns_train_predictor(anns_index* index, const float* train_q, int64_t nq, int32_t nprobe,
                         int32_t k, const anns_train_cfg* cfg, anns_predictor* out, void* cuda_stream);

/* The coarse stage (cluster locating, CL of Section 2.1) alone: the nprobe
 * nearest lists of each query by the FP32 rule, ties by list id, computed
 * with cl_prec = ANNS_PREC_FP32 (CUDA cores), or ANNS_PREC_BF16 / FP16 /
 * FP8E4M3 (tensor-core GEMM + exact re-rank; same output). probes_out device
 * int32 [nq * nprobe],
 * probe_d2_out device float32 [nq * nprobe] (padding -1 / +inf past a query's
 * nprobe_per_q). Uses the index workspace (asynchronous on cuda_stream). */
int anns_locate(anns_index* index, const float* queries, int64_t nq, int32_t nprobe,
                const int32_t* nprobe_per_q, int32_t cl_prec, int32_t* probes_out, float* probe_d2_out,
                void* cuda_stream);

/* The coarse stage (cluster locating) without any allocation, for callers
 * that cannot allocate device memory: real-time or embedded hosts that forbid
 * allocation after start-up (cudaMalloc and cudaFree take unbounded time and
 * may synchronise the device), and plugins whose host application owns every
 * memory pool. There is no counterpart in the paper;
 * it is the probe selection of anns_search (same kernels, same results as
 * the PROBES / PROBE_D2 taps) with its scratch — the nq * nlist coarse
 * distance matrix — in a fixed array of ANNS_STATIC_SCRATCH_FLOATS floats
 * (8 MiB) compiled into the library and held by every GPU that loads it
 * until the process exits. No cudaMalloc, cudaFree or allocating library
 * call is made.
 *  queries       device float32 [nq * dim].
 *  probes_out    device int32 [nq * nprobe]: the nprobe nearest lists by (D2, list id).
 *  probe_d2_out  device float32 [nq * nprobe]: their FP32 coarse distances.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture. All calls on a device share the array, so calls
 * that overlap on the GPU race; each call overwrites every element it reads.
 * Errors: INVALID_ARG (nq * nlist > ANNS_STATIC_SCRATCH_FLOATS, nprobe out of
 * range, null buffer), CUDA. */
#define ANNS_STATIC_SCRATCH_FLOATS (1 << 21)
int anns_locate_static(anns_index* index, const float* queries, int64_t nq, int32_t nprobe,
                       int32_t* probes_out, float* probe_d2_out, void* cuda_stream);

/* SVR-RBF precision model for inference on the GPU (policy ANNS_LUT_SVR; the
 * regressor of Section 3.4 with its exponential evaluated through a lookup
 * table). Per probed pair, with the same five features as the MLP policy:
 *   x = fl32(fl32(f - mean) * inv_std);  f = 0;  for i ascending:
 *     d2 = FP32 sum over the 5 features, ascending, of fl32(e * e),
 *          e = fl32(x_c - sv_ic);
 *     u = fl32(fl32(gamma * d2) * inv_step);
 *     ex = 0 if u >= table_n - 1, else with k = floor(u), w = fl32(u - k):
 *          fl32(fl32(tab_k * fl32(1 - w)) + fl32(tab_{k+1} * w));
 *     f = fl32(f + fl32(beta_i * fl32(ex + 1)));
 *   width index = clip(ceil(fl32(f - margin)), 0, 5) into (4, 6, 8, 12, 16,
 *   FP32), margin = the policy's fallback_margin; width_map applies after.
 * The table is built here from table_ratio rho: e_0 = 1, e_k = fl64(e_{k-1} *
 * rho) for k ascending, each rounded once to FP32, i.e. exp(-k step) with
 * step = -ln(rho) and no exponential function evaluated; inv_step = 1 / step
 * is given by the caller.
 *  sv    host float [nsv * 5]: the support vectors (normalised features)
 *  beta  host float [nsv]: their coefficients (anns_svr_fit's beta)
 * Copied to the device (synchronous). Errors: INVALID_ARG (nsv out of
 * [1, ANNS_SVR_MAX_SAMPLES], table_n out of [2, 4096], rho out of (0, 1),
 * non-finite parameter, null pointer), OOM, CUDA. */
typedef struct {
  int32_t nsv;
  const float* sv;
  const float* beta;
  float gamma;
  float mean[5], inv_std[5];
  int32_t table_n;
  double table_ratio;
  float inv_step;
} anns_svr_model;
int anns_set_svr(anns_index* index, const anns_svr_model* model);

/* SVR-RBF precision model (Section 3.4), training on the host (the paper's
 * predictor, a comparator to the MLP; at most ANNS_SVR_MAX_SAMPLES samples).
 * Model: f(x) = sum_i beta_i (exp(-gamma |x_i - x|^2) + 1), the constant 1
 * being the bias. Training solves the dual of epsilon-insensitive regression
 * over the box beta in [-C, C]^n,
 *   minimise 1/2 beta^T K1 beta - y^T beta + eps |beta|_1,  K1 = K + 1,
 * by exact coordinate descent: i ascending in sweeps, each step the
 * coordinate's minimiser (soft threshold, then the clip to the box), until
 * the largest change of a sweep is <= tol or max_sweeps sweeps ran. FP64.
 *  X          host double [n x dim], row-major features
 *  y          host double [n] targets
 *  beta_out   host double [n] (written)
 *  sweeps_out host int64 or NULL: sweeps run
 * No GPU is used. Errors: INVALID_ARG (n < 1, n > ANNS_SVR_MAX_SAMPLES,
 * dim < 1, C <= 0, gamma <= 0, eps < 0, tol < 0, max_sweeps < 1, null
 * pointer), OOM. */
#define ANNS_SVR_MAX_SAMPLES 4096
int anns_svr_fit(const double* X, const double* y, int64_t n, int32_t dim, double C, double gamma,
                 double eps, double tol, int64_t max_sweeps, double* beta_out, int64_t* sweeps_out);

/* Message of the last failure on the calling thread ("" if none). */
const char* anns_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* ANNS_AMP_H */
