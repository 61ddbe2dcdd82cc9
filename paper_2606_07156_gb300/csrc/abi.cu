// anns_search and friends: argument checks, workspace, and the launch sequence
// CL -> precision choice -> (RC + LC + quantise + DC + TS) of Section 2.1.
#include <cmath>
#include <cstring>
#include <utility>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "predictor.cuh"

namespace anns {
namespace {

struct PolicyArgs {
  int64_t nq; int nprobe; const int32_t* npq;
  const int32_t* probes; const float* probe_d2;
  const int32_t* list_len; const float* radius;
  int mode, fixed_bits; float th[4]; float margin; int width_map;
  const uint8_t* pair_bits; const void* mlp;
  uint8_t* bits; float* feat;
};

__device__ __forceinline__ uint8_t sanitize_bits(int b) { return (b >= 1 && b <= 16) ? (uint8_t)b : 0; }

// Features of probe rank j (Section 3.3: query distance d', radii r1 and r2,
// size n; plus the probe rank): (sqrt(D2_j) - sqrt(D2_0), r_0, r_j, sqrt(n_j), j/nprobe_q).
__device__ __forceinline__ void features_of(const PolicyArgs& p, int64_t q, int j, int np, float f[5]) {
  const int64_t row = q * p.nprobe;
  const int l0 = p.probes[row], lj = p.probes[row + j];
  if (l0 < 0 || lj < 0) return;
  f[0] = sub_rn(__fsqrt_rn(p.probe_d2[row + j]), __fsqrt_rn(p.probe_d2[row]));
  f[1] = p.radius[l0];
  f[2] = p.radius[lj];
  f[3] = __fsqrt_rn((float)p.list_len[lj]);
  f[4] = __fdiv_rn((float)j, (float)np);
}

// Eq. 2 heuristic: g = f / r_j with f = d' - 3 r_0 - r_j; the fewest bits whose
// threshold g reaches (thresholds non-increasing), else 16.
__device__ __forceinline__ uint8_t eq2_bits(const float f[5], const float th[4]) {
  const float fe = sub_rn(sub_rn(f[0], mul_rn(3.f, f[1])), f[2]);
  const float g = f[2] > 0.f ? __fdiv_rn(fe, f[2]) : -INFINITY;
  uint8_t b = 16;
  if (g >= th[3]) b = 12;
  if (g >= th[2]) b = 8;
  if (g >= th[1]) b = 6;
  if (g >= th[0]) b = 4;
  return b;
}

// Widths on this GPU's tables: 6 -> 8 bits (byte tables either way, finer
// levels), 12 and 16 -> FP32 (a 16-bit table gathers as slowly as FP32).
__device__ __forceinline__ uint8_t gpu_width(uint8_t b) { return b == 6 ? 8 : (b == 12 || b == 16) ? 0 : b; }

__global__ void policy_kernel(const PolicyArgs p) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= p.nq * p.nprobe) return;
  const int64_t q = idx / p.nprobe;
  const int j = (int)(idx % p.nprobe);
  const int np = p.npq ? min(max(p.npq[q], 0), p.nprobe) : p.nprobe;
  const int l = p.probes[idx];
  float f[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  uint8_t b = 0;
  if (j < np && l >= 0) {
    switch (p.mode) {
      case ANNS_LUT_PLAIN_FP32: b = 0; break;
      case ANNS_LUT_FIXED_BITS: b = (uint8_t)p.fixed_bits; break;
      case ANNS_LUT_EXPLICIT: b = sanitize_bits(p.pair_bits[idx]); break;
      case ANNS_LUT_HEURISTIC_EQ2:
        features_of(p, q, j, np, f);
        b = eq2_bits(f, p.th);
        if (p.width_map) b = gpu_width(b);
        break;
      case ANNS_LUT_MLP:
        features_of(p, q, j, np, f);
        b = mlp_decide(*(const MlpParams16*)p.mlp, f, p.margin);
        if (p.width_map) b = gpu_width(b);
        break;
    }
  }
  p.bits[idx] = b;
  if (p.feat) {
#pragma unroll
    for (int i = 0; i < 5; ++i) p.feat[idx * 5 + i] = f[i];
  }
}

// SVR-RBF policy (Section 3.4): one thread per pair, the support vectors,
// coefficients and exponential table staged in shared memory; the FP32 rule
// of anns_set_svr in anns_amp.h.
struct SvrArgs {
  const float* dev;  // [sv nsv*5 | beta nsv | table tn]
  int nsv, tn;
  float gamma, inv_step, mean[5], inv_std[5];
};

__global__ void __launch_bounds__(256) svr_policy_kernel(const PolicyArgs p, const SvrArgs m) {
  float* s_sv = (float*)anns_dyn_smem;
  float* s_beta = s_sv + m.nsv * 5;
  float* s_tab = s_beta + m.nsv;
  const int total = m.nsv * 6 + m.tn;
  for (int i = threadIdx.x; i < total; i += blockDim.x) s_sv[i] = m.dev[i];
  __syncthreads();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= p.nq * p.nprobe) return;
  const int64_t q = idx / p.nprobe;
  const int j = (int)(idx % p.nprobe);
  const int np = p.npq ? min(max(p.npq[q], 0), p.nprobe) : p.nprobe;
  const int l = p.probes[idx];
  float f[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  uint8_t b = 0;
  if (j < np && l >= 0) {
    features_of(p, q, j, np, f);
    float x[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) x[c] = mul_rn(sub_rn(f[c], m.mean[c]), m.inv_std[c]);
    const float ulim = (float)(m.tn - 1);
    float acc = 0.f;
    for (int i = 0; i < m.nsv; ++i) {
      float d2 = 0.f;
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const float e = sub_rn(x[c], s_sv[i * 5 + c]);
        d2 = add_rn(d2, mul_rn(e, e));
      }
      const float u = mul_rn(mul_rn(m.gamma, d2), m.inv_step);
      float ex = 0.f;
      if (u < ulim) {
        const int k = (int)floorf(u);
        const float w = sub_rn(u, (float)k);
        ex = add_rn(mul_rn(s_tab[k], sub_rn(1.f, w)), mul_rn(s_tab[k + 1], w));
      }
      acc = add_rn(acc, mul_rn(s_beta[i], add_rn(ex, 1.f)));
    }
    const float c = ceilf(sub_rn(acc, p.margin));
    const int wi = c >= 5.f ? 5 : (c > 0.f ? (int)c : 0);
    constexpr uint8_t kW[6] = {4, 6, 8, 12, 16, 0};
    b = kW[wi];
    if (p.width_map) b = gpu_width(b);
  }
  p.bits[idx] = b;
  if (p.feat) {
#pragma unroll
    for (int i = 0; i < 5; ++i) p.feat[idx * 5 + i] = f[i];
  }
}

bool valid_bits(int b) { return b == 4 || b == 6 || b == 8 || b == 12 || b == 16; }

struct DeviceGuard {
  int prev = 0;
  explicit DeviceGuard(int d) { cudaGetDevice(&prev); cudaSetDevice(d); }
  ~DeviceGuard() { cudaSetDevice(prev); }
};

int ensure_workspace(Index& ix, int64_t nq, int nprobe) {
  int rc = grow((void**)&ix.ws_d2, &ix.ws_d2_cap, (size_t)nq * ix.nlist * 4);
  if (rc) return rc;
  const size_t P = (size_t)nq * nprobe;
  // one block: probes (4P) | probe_d2 (4P) | features (20P) | bits (P)
  void* blk = ix.ws_probes;
  rc = grow(&blk, &ix.ws_pair_cap, P * 29 + 64);
  if (rc) return rc;
  ix.ws_probes = (int32_t*)blk;
  ix.ws_probe_d2 = (float*)((char*)blk + 4 * P);
  ix.ws_feat = (float*)((char*)blk + 8 * P);
  ix.ws_bits = (uint8_t*)((char*)blk + 28 * P);
  ix.ws_nq = nq;
  ix.ws_nprobe = nprobe;
  rc = grow((void**)&ix.ws_qt, &ix.ws_qt_cap, (size_t)nq * ix.Mp * kKsub * 4);
  if (rc) return rc;
  return grow((void**)&ix.ws_counter, &ix.ws_counter_cap, 64);
}

int table_bytes_for(const anns_precision_policy& P) {
  switch (P.lut_mode) {
    case ANNS_LUT_FIXED_BITS: return P.fixed_bits <= 8 ? 1 : 2;
    case ANNS_LUT_HEURISTIC_EQ2: return P.width_map ? 4 : 2;  // 4..16 bits, or FP32 when mapped
    default: return 4;                       // plain, explicit, MLP (with FP32 fallback)
  }
}

int list_workspace(Index& ix, int64_t nq, int nprobe, int k, ListWork& w, int64_t qchunk) {
  w.qchunk = std::max<int64_t>(qchunk, 1);
  const int64_t nchunks = std::max<int64_t>((nq + w.qchunk - 1) / w.qchunk, 1);
  if (nchunks * ix.nlist > INT32_MAX / 2) return fail(ANNS_ERR_INVALID_ARG, "too many (query chunk, list) buckets");
  w.nbuckets = (int)(nchunks * ix.nlist);
  const size_t L = (size_t)(w.nbuckets + 1) * 4, P = (size_t)nq * nprobe;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t G = (P + (size_t)w.nbuckets + 1) * 4;  // groups: at most one per pair plus one per bucket
  const size_t bytes = 2 * (4 * al(L) + al(P * 4) + al(G)) + al(P * k * 4) + al(P * k * 8);
  int rc = grow(&ix.ws_lists, &ix.ws_lists_cap, bytes);
  if (rc) return rc;
  char* b = (char*)ix.ws_lists;
  w.cnt = (int*)b; b += al(L);
  w.off = (int*)b; b += al(L);
  w.ioff = (int*)b; b += al(L);
  w.fill = (int*)b; b += al(L);
  w.pairs = (int32_t*)b; b += al(P * 4);
  w.part_d = (float*)b; b += al(P * k * 4);
  w.part_i = (int64_t*)b; b += al(P * k * 8);
  w.gtab = (int*)b; b += al(G);
  w.counter = ix.ws_counter;
  w.cnt4 = (int*)b; b += al(L);
  w.off4 = (int*)b; b += al(L);
  w.ioff4 = (int*)b; b += al(L);
  w.fill4 = (int*)b; b += al(L);
  w.pairs4 = (int32_t*)b; b += al(P * 4);
  w.gtab4 = (int*)b;
  w.counter4 = ix.ws_counter + 8;
  return ANNS_OK;
}

// Folds finished event sets into the totals; with `all`, waits for every set.
int drain_profile(Index& ix, bool all) {
  int keep = 0;
  for (int i = 0; i < ix.prof_pending; ++i) {
    cudaEvent_t* ev = ix.prof_ev[i];
    cudaError_t q = all ? cudaEventSynchronize(ev[Index::kStages]) : cudaEventQuery(ev[Index::kStages]);
    if (q == cudaSuccess) {
      for (int st = 0; st < Index::kStages; ++st) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[st], ev[st + 1]);
        ix.prof_ms[st] += ms;
      }
      ix.prof_count++;
    } else if (q == cudaErrorNotReady) {
      if (keep != i)
        for (int st = 0; st <= Index::kStages; ++st) std::swap(ix.prof_ev[keep][st], ix.prof_ev[i][st]);
      keep++;
    } else {
      return cuda_fail(q, "profile event");
    }
  }
  ix.prof_pending = keep;
  return ANNS_OK;
}

// Event set for the next search, or nullptr when profiling is off.
cudaEvent_t* next_profile_slot(Index& ix) {
  if (!ix.prof_on) return nullptr;
  if (ix.prof_pending == Index::kProfSlots && drain_profile(ix, true)) return nullptr;
  cudaEvent_t* ev = ix.prof_ev[ix.prof_pending];
  for (int st = 0; st <= Index::kStages; ++st)
    if (!ev[st] && cudaEventCreate(&ev[st]) != cudaSuccess) return nullptr;
  ix.prof_pending++;
  return ev;
}

}  // namespace

int launch_policy(const Index& ix, const anns_precision_policy& pol, int64_t nq, int nprobe,
                  const int32_t* nprobe_per_q, const int32_t* probes, const float* probe_d2,
                  uint8_t* bits, float* feat, cudaStream_t s) {
  PolicyArgs p{};
  p.nq = nq; p.nprobe = nprobe; p.npq = nprobe_per_q; p.probes = probes; p.probe_d2 = probe_d2;
  p.list_len = ix.list_len; p.radius = ix.radius; p.mode = pol.lut_mode;
  p.fixed_bits = pol.fixed_bits;
  for (int i = 0; i < 4; ++i) p.th[i] = pol.eq2_thresholds[i];
  p.margin = pol.fallback_margin; p.pair_bits = pol.pair_bits; p.mlp = ix.mlp_dev;
  p.width_map = pol.width_map;
  p.bits = bits; p.feat = feat;
  const int64_t n = nq * nprobe;
  if (pol.lut_mode == ANNS_LUT_SVR) {
    SvrArgs m{};
    m.dev = ix.svr_dev; m.nsv = ix.svr_nsv; m.tn = ix.svr_tn; m.gamma = ix.svr_gamma; m.inv_step = ix.svr_inv_step;
    for (int i = 0; i < 5; ++i) { m.mean[i] = ix.svr_mean[i]; m.inv_std[i] = ix.svr_inv_std[i]; }
    const size_t smem = (size_t)(m.nsv * 6 + m.tn) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(svr_policy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "svr policy kernel attribute");
    svr_policy_kernel<<<(unsigned)((n + 255) / 256), 256, smem, s>>>(p, m); note_launch();
  } else {
    policy_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p); note_launch();
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ANNS_OK : cuda_fail(e, "policy kernel");
}

}  // namespace anns

using namespace anns;

int anns::check_search_args(anns_index* ix, const float* Q, int64_t nq, int32_t nprobe, int32_t k,
                             const anns_precision_policy* pol, const void* ids_out,
                             const void* dists_out) {
  if (!ix) return fail(ANNS_ERR_INVALID_ARG, "null index");
  if (nq < 0) return fail(ANNS_ERR_INVALID_ARG, "nq must be >= 0");
  if (nq > 0 && (!Q || !ids_out || !dists_out)) return fail(ANNS_ERR_INVALID_ARG, "null buffer");
  if (nprobe < 1 || nprobe > ix->nlist || nprobe > ANNS_MAX_NPROBE)
    return fail(ANNS_ERR_INVALID_ARG, "nprobe must be in [1, min(nlist, 128)]");
  if (k < 1 || k > ANNS_MAX_K) return fail(ANNS_ERR_INVALID_ARG, "k must be in [1, 128]");
  if (nq > (int64_t)INT32_MAX) return fail(ANNS_ERR_INVALID_ARG, "nq too large");
  if (pol) {
    switch (pol->lut_mode) {
      case ANNS_LUT_PLAIN_FP32: case ANNS_LUT_HEURISTIC_EQ2: break;
      case ANNS_LUT_FIXED_BITS:
        if (!valid_bits(pol->fixed_bits)) return fail(ANNS_ERR_INVALID_ARG, "fixed_bits must be 4/6/8/12/16");
        break;
      case ANNS_LUT_EXPLICIT:
        if (!pol->pair_bits && nq > 0) return fail(ANNS_ERR_INVALID_ARG, "EXPLICIT needs pair_bits");
        break;
      case ANNS_LUT_MLP:
        if (!ix->has_mlp) return fail(ANNS_ERR_INVALID_ARG, "MLP policy needs a trained or loaded predictor");
        if (std::isnan(pol->fallback_margin)) return fail(ANNS_ERR_INVALID_ARG, "MLP round-up margin is NaN");
        break;
      case ANNS_LUT_SVR:
        if (!ix->has_svr) return fail(ANNS_ERR_INVALID_ARG, "SVR policy needs a model (anns_set_svr)");
        if (std::isnan(pol->fallback_margin)) return fail(ANNS_ERR_INVALID_ARG, "SVR margin is NaN");
        break;
      default: return fail(ANNS_ERR_INVALID_ARG, "unknown lut_mode");
    }
    if (pol->cl_prec != ANNS_PREC_FP32 && !coarse_tc_format(pol->cl_prec))
      return fail(ANNS_ERR_UNSUPPORTED, "CL operands: FP32, or BF16 / FP16 / FP8 E4M3 (with exact re-rank)");
    if (pol->lc_prec != ANNS_PREC_FP32) return fail(ANNS_ERR_UNSUPPORTED, "LC operands: FP32 only");
  }
  return ANNS_OK;
}

namespace anns {

// The grouped kernel (narrow pairs packed four to a word): on request, or by
// default for a policy that can choose 1..8-bit tables, when k <= 128.
static bool use_grouped(const Index& ix, const anns_precision_policy& P, int k) {
  if (ix.opt_kernel == ANNS_KERNEL_GROUPED) return grouped_supported(ix, k);
  if (ix.opt_kernel != ANNS_KERNEL_AUTO) return false;
  const bool narrow_possible = P.lut_mode == ANNS_LUT_MLP || P.lut_mode == ANNS_LUT_HEURISTIC_EQ2 ||
                               P.lut_mode == ANNS_LUT_EXPLICIT || P.lut_mode == ANNS_LUT_SVR ||
                               (P.lut_mode == ANNS_LUT_FIXED_BITS && P.fixed_bits <= 8);
  return narrow_possible && grouped_supported(ix, k);
}

// Whether every pair the policy can put outside 1..8 bits is an FP32 pair
// (no 12- or 16-bit tables): the split search's wide pass then needs no
// level table.
static bool wide_tables_fp32(const anns_precision_policy& P) {
  switch (P.lut_mode) {
    case ANNS_LUT_PLAIN_FP32: return true;
    case ANNS_LUT_FIXED_BITS: return P.fixed_bits <= 8;
    case ANNS_LUT_HEURISTIC_EQ2:
    case ANNS_LUT_MLP:
    case ANNS_LUT_SVR: return P.width_map != 0;
    default: return false;
  }
}

static bool use_lpt(const Index& ix, const int32_t* nprobe_per_q) {
  return ix.opt_schedule == ANNS_SCHED_LPT || (ix.opt_schedule == ANNS_SCHED_AUTO && nprobe_per_q);
}

int reserve_search(Index& ix, int64_t nq, int nprobe, int k, const anns_precision_policy& P,
                   const int32_t* nprobe_per_q) {
  int rc = ensure_workspace(ix, nq, nprobe);
  if (rc) return rc;
  if (ix.opt_kernel == ANNS_KERNEL_LIST_MAJOR || use_grouped(ix, P, k)) {
    ListWork w{};
    const int64_t qchunk = ix.opt_kernel == ANNS_KERNEL_LIST_MAJOR ? nq : grouped_qchunk(ix, nq);
    if ((rc = list_workspace(ix, nq, nprobe, k, w, qchunk))) return rc;
  }
  if (use_grouped(ix, P, k) || ix.opt_kernel == ANNS_KERNEL_SPLIT) {
    if ((rc = grow(&ix.ws_grp, &ix.ws_grp_cap, grouped_workspace_bytes(nq, k)))) return rc;
  }
  if (ix.opt_kernel != ANNS_KERNEL_LIST_MAJOR && use_lpt(ix, nprobe_per_q)) {
    if ((rc = grow(&ix.ws_sched, &ix.ws_sched_cap, lpt_workspace_bytes(nq)))) return rc;
  }
  if (coarse_tc_format(P.cl_prec)) {
    if ((rc = grow(&ix.ws_tc, &ix.ws_tc_cap, coarse_tc_workspace_bytes(ix, nq)))) return rc;
  }
  return ANNS_OK;
}

int search_sequence(Index& ix, const float* Q, int64_t nq, int nprobe, const int32_t* nprobe_per_q, int k,
                    const int32_t* k_per_q, const anns_precision_policy& P, int64_t* ids_out,
                    float* dists_out, cudaStream_t s, bool profile) {
  int rc = reserve_search(ix, nq, nprobe, k, P, nprobe_per_q);
  if (rc) return rc;
  cudaEvent_t* ev = profile ? next_profile_slot(ix) : nullptr;
  if (ev) cudaEventRecord(ev[0], s);
  cudaError_t e;
  ix.ws_tc_valid = coarse_tc_format(P.cl_prec);
  ix.ws_tc_prec = P.cl_prec;
  ix.ws_tc_nq = nq;
  if (ix.ws_tc_valid) {
    if (ev) cudaEventRecord(ev[1], s);
    e = launch_coarse_tc(ix, P.cl_prec, Q, nq, nprobe, nprobe_per_q, ix.ws_tc, ix.ws_d2, ix.ws_probes,
                         ix.ws_probe_d2, s);
  } else {
    e = launch_coarse(ix, Q, nq, nprobe, nprobe_per_q, ix.ws_d2, ix.ws_probes, ix.ws_probe_d2, s,
                      ev ? ev[1] : nullptr);
  }
  if (e != cudaSuccess) return cuda_fail(e, "coarse kernels");
  if (ev) cudaEventRecord(ev[2], s);
  const bool want_feat = P.lut_mode == ANNS_LUT_MLP || P.lut_mode == ANNS_LUT_HEURISTIC_EQ2 ||
                         P.lut_mode == ANNS_LUT_SVR;
  if ((rc = launch_policy(ix, P, nq, nprobe, nprobe_per_q, ix.ws_probes, ix.ws_probe_d2, ix.ws_bits,
                          want_feat ? ix.ws_feat : nullptr, s)))
    return rc;
  e = launch_query_tables(ix, Q, nq, ix.ws_qt, s);
  if (e != cudaSuccess) return cuda_fail(e, "query tables");
  // table width the policy may need: FP32 (4 bytes), 16-bit or 8-bit levels
  const int tbytes = table_bytes_for(P);
  // AUTO: query-major (measured faster on the SIFT-shaped workload for every
  // table width); list-major on request
  if (ix.opt_kernel == ANNS_KERNEL_LIST_MAJOR) {
    if (list_major_warps(ix, tbytes) < 1)
      return fail(ANNS_ERR_UNSUPPORTED, "list-major kernel: one table does not fit in shared memory");
    ListWork w{};
    if ((rc = list_workspace(ix, nq, nprobe, k, w, nq))) return rc;
    if (ev) cudaEventRecord(ev[3], s);
    e = launch_search_lists(ix, ix.ws_qt, nq, nprobe, nprobe_per_q, k, k_per_q, ix.ws_probes, ix.ws_probe_d2,
                            ix.ws_bits, tbytes, w, ids_out, dists_out, s);
  } else if (use_grouped(ix, P, k)) {
    ListWork w{};
    if ((rc = list_workspace(ix, nq, nprobe, k, w, grouped_qchunk(ix, nq)))) return rc;
    // longest-first order of the query-major pass, over the pairs it scans
    const int32_t* order = nullptr;
    if (use_lpt(ix, nprobe_per_q)) {
      e = launch_lpt_order(ix, ix.ws_probes, nprobe_per_q, nq, nprobe, ix.ws_sched, s, ix.ws_bits, true);
      if (e != cudaSuccess) return cuda_fail(e, "schedule kernels");
      order = lpt_order_ptr(ix.ws_sched, nq);
    }
    if (ev) cudaEventRecord(ev[3], s);
    e = launch_search_grouped(ix, ix.ws_qt, nq, nprobe, nprobe_per_q, k, k_per_q, ix.ws_probes, ix.ws_probe_d2,
                              ix.ws_bits, w, ix.ws_grp, ids_out, dists_out, s, ev ? ev[4] : nullptr,
                              ev ? ev[5] : nullptr, ev ? ev[6] : nullptr, order);
    if (e == cudaSuccess && ev) cudaEventRecord(ev[7], s);
    return e == cudaSuccess ? ANNS_OK : cuda_fail(e, "search kernel");
  } else {
    const int32_t* order = nullptr;
    if (use_lpt(ix, nprobe_per_q)) {
      e = launch_lpt_order(ix, ix.ws_probes, nprobe_per_q, nq, nprobe, ix.ws_sched, s, ix.ws_bits, false);
      if (e != cudaSuccess) return cuda_fail(e, "schedule kernels");
      order = lpt_order_ptr(ix.ws_sched, nq);
    }
    if (ev) cudaEventRecord(ev[3], s);
    if (ix.opt_kernel == ANNS_KERNEL_SPLIT) {
      // wide pairs (FP32, 12/16 bits) into a partial top-k per query, then
      // the 1..8-bit pairs with byte tables only, merged with it
      float* part_d = (float*)ix.ws_grp;
      int64_t* part_i = (int64_t*)((char*)ix.ws_grp + (((size_t)nq * k * 4 + 255) & ~size_t(255)));
      e = launch_search(ix, ix.ws_qt, nq, nprobe, nprobe_per_q, k, k_per_q, ix.ws_probes, ix.ws_probe_d2,
                        ix.ws_bits, order, part_i, part_d, s, 2, wide_tables_fp32(P) ? QM_TABLES_FP32 : QM_TABLES_ALL);
      if (e == cudaSuccess && ev) cudaEventRecord(ev[4], s);
      if (e == cudaSuccess)
        e = launch_search(ix, ix.ws_qt, nq, nprobe, nprobe_per_q, k, k_per_q, ix.ws_probes, ix.ws_probe_d2,
                          ix.ws_bits, order, ids_out, dists_out, s, 0, QM_TABLES_NARROW, part_d, part_i);
      if (e != cudaSuccess) return cuda_fail(e, "search kernel");
      if (ev)
        for (int st = 5; st <= Index::kStages; ++st) cudaEventRecord(ev[st], s);
      return ANNS_OK;
    }
    // a plain-FP32 policy needs no level table, a fixed <= 8-bit one no FP32 table
    const int tables = P.lut_mode == ANNS_LUT_PLAIN_FP32 ? QM_TABLES_FP32
                       : P.lut_mode == ANNS_LUT_FIXED_BITS && P.fixed_bits <= 8 ? QM_TABLES_NARROW
                                                                                 : QM_TABLES_ALL;
    e = launch_search(ix, ix.ws_qt, nq, nprobe, nprobe_per_q, k, k_per_q, ix.ws_probes, ix.ws_probe_d2,
                      ix.ws_bits, order, ids_out, dists_out, s, 0, tables);
  }
  if (e != cudaSuccess) return cuda_fail(e, "search kernel");
  if (ev)
    for (int st = 4; st <= Index::kStages; ++st) cudaEventRecord(ev[st], s);
  return ANNS_OK;
}

void free_workspace(Index& ix) {
  void* ptrs[] = {ix.ws_qt, ix.ws_lists, ix.ws_d2, ix.ws_probes /* base of the pair block */,
                  ix.ws_counter, ix.ws_sched, ix.ws_tc, ix.ws_grp, ix.st_q, ix.st_out, ix.st_pq};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  ix.ws_qt = nullptr; ix.ws_lists = nullptr; ix.ws_d2 = nullptr; ix.ws_probes = nullptr;
  ix.ws_probe_d2 = nullptr; ix.ws_bits = nullptr; ix.ws_feat = nullptr; ix.ws_counter = nullptr;
  ix.ws_sched = nullptr; ix.ws_tc = nullptr; ix.st_q = nullptr; ix.st_out = nullptr; ix.st_pq = nullptr;
  ix.ws_tc_cap = 0;
  ix.ws_tc_valid = false;
  ix.ws_grp = nullptr;
  ix.ws_grp_cap = 0;
  ix.ws_qt_cap = ix.ws_lists_cap = ix.ws_d2_cap = ix.ws_pair_cap = ix.ws_counter_cap = 0;
  ix.ws_sched_cap = ix.st_q_cap = ix.st_out_cap = ix.st_pq_cap = 0;
  ix.ws_nq = ix.ws_nprobe = 0;
}

}  // namespace anns

extern "C" int anns_search(anns_index* ix, const float* Q, int64_t nq, int32_t nprobe,
                           const int32_t* nprobe_per_q, int32_t k, const int32_t* k_per_q,
                           const anns_precision_policy* pol, int64_t* ids_out, float* dists_out,
                           void* stream) {
  int rc = check_search_args(ix, Q, nq, nprobe, k, pol, ids_out, dists_out);
  if (rc) return rc;
  if (nq == 0) return ANNS_OK;
  DeviceGuard g(ix->device);
  anns_precision_policy plain{};
  plain.lut_mode = ANNS_LUT_PLAIN_FP32;
  return search_sequence(*ix, Q, nq, nprobe, nprobe_per_q, k, k_per_q, pol ? *pol : plain, ids_out, dists_out,
                         (cudaStream_t)stream, true);
}

extern "C" int anns_locate(anns_index* ix, const float* Q, int64_t nq, int32_t nprobe,
                           const int32_t* nprobe_per_q, int32_t cl_prec, int32_t* probes_out,
                           float* probe_d2_out, void* stream) {
  if (!ix) return fail(ANNS_ERR_INVALID_ARG, "null index");
  if (nq < 0) return fail(ANNS_ERR_INVALID_ARG, "nq must be >= 0");
  if (nprobe < 1 || nprobe > ix->nlist || nprobe > ANNS_MAX_NPROBE)
    return fail(ANNS_ERR_INVALID_ARG, "nprobe must be in [1, min(nlist, 128)]");
  if (cl_prec != ANNS_PREC_FP32 && !coarse_tc_format(cl_prec))
    return fail(ANNS_ERR_UNSUPPORTED, "CL operands: FP32, or BF16 / FP16 / FP8 E4M3 (with exact re-rank)");
  if (nq == 0) return ANNS_OK;
  if (!Q || !probes_out || !probe_d2_out) return fail(ANNS_ERR_INVALID_ARG, "null buffer");
  DeviceGuard g(ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  int rc = grow((void**)&ix->ws_d2, &ix->ws_d2_cap, (size_t)nq * ix->nlist * 4);
  if (rc) return rc;
  cudaError_t e;
  ix->ws_tc_valid = coarse_tc_format(cl_prec);
  ix->ws_tc_prec = cl_prec;
  ix->ws_tc_nq = nq;
  if (ix->ws_tc_valid) {
    if ((rc = grow(&ix->ws_tc, &ix->ws_tc_cap, coarse_tc_workspace_bytes(*ix, nq)))) return rc;
    e = launch_coarse_tc(*ix, cl_prec, Q, nq, nprobe, nprobe_per_q, ix->ws_tc, ix->ws_d2, probes_out, probe_d2_out,
                         s);
  } else {
    e = launch_coarse(*ix, Q, nq, nprobe, nprobe_per_q, ix->ws_d2, probes_out, probe_d2_out, s);
  }
  return e == cudaSuccess ? ANNS_OK : cuda_fail(e, "coarse kernels");
}

extern "C" int anns_search_host(anns_index* ix, const float* Q, int64_t nq, int32_t nprobe,
                                const int32_t* nprobe_per_q, int32_t k, const int32_t* k_per_q,
                                const anns_precision_policy* pol, int64_t* ids_out,
                                float* dists_out, void* stream) {
  int rc = check_search_args(ix, Q, nq, nprobe, k, pol, ids_out, dists_out);
  if (rc) return rc;
  if (nq == 0) return ANNS_OK;
  DeviceGuard g(ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t qb = (size_t)nq * ix->dim * 4, ob = (size_t)nq * k * 12, pb = (size_t)nq * 8;
  if ((rc = grow(&ix->st_q, &ix->st_q_cap, qb)) || (rc = grow(&ix->st_out, &ix->st_out_cap, ob)) ||
      (rc = grow(&ix->st_pq, &ix->st_pq_cap, pb)))
    return rc;
  float* dq = (float*)ix->st_q;
  int64_t* di = (int64_t*)ix->st_out;
  float* dd = (float*)((char*)ix->st_out + (size_t)nq * k * 8);
  int32_t* dnp = nprobe_per_q ? (int32_t*)ix->st_pq : nullptr;
  int32_t* dk = k_per_q ? (int32_t*)ix->st_pq + nq : nullptr;
  cudaError_t e = cudaMemcpyAsync(dq, Q, qb, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && dnp) e = cudaMemcpyAsync(dnp, nprobe_per_q, nq * 4, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && dk) e = cudaMemcpyAsync(dk, k_per_q, nq * 4, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "copy queries in");
  if ((rc = anns_search(ix, dq, nq, nprobe, dnp, k, dk, pol, di, dd, stream))) return rc;
  e = cudaMemcpyAsync(ids_out, di, (size_t)nq * k * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dists_out, dd, (size_t)nq * k * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "copy results out");
  return ANNS_OK;
}

static int check_pairs(anns_index* ix, const float* Q, int64_t nq, const int32_t* pq,
                       const int32_t* pl, const uint8_t* pb, int64_t npairs) {
  if (!ix) return fail(ANNS_ERR_INVALID_ARG, "null index");
  if (npairs < 0 || nq < 0) return fail(ANNS_ERR_INVALID_ARG, "negative size");
  if (npairs > 0 && (!Q || !pq || !pl || !pb)) return fail(ANNS_ERR_INVALID_ARG, "null buffer");
  return ANNS_OK;
}

extern "C" int anns_compute_luts(anns_index* ix, const float* Q, int64_t nq, const int32_t* pq,
                                 const int32_t* pl, const uint8_t* pb, int64_t npairs,
                                 float* T_out, uint16_t* t_out, double* scale_out, void* stream) {
  int rc = check_pairs(ix, Q, nq, pq, pl, pb, npairs);
  if (rc) return rc;
  if (npairs == 0) return ANNS_OK;
  DeviceGuard g(ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = grow((void**)&ix->ws_qt, &ix->ws_qt_cap, (size_t)nq * ix->Mp * kKsub * 4))) return rc;
  cudaError_t e = launch_query_tables(*ix, Q, nq, ix->ws_qt, s);
  if (e == cudaSuccess)
    e = launch_compute_luts(*ix, Q, ix->ws_qt, nq, pq, pl, pb, npairs, T_out, t_out, scale_out, s);
  return e == cudaSuccess ? ANNS_OK : cuda_fail(e, "LUT kernel");
}

namespace anns {
// One warp per set: the exact sum of the set's values rounded once (common.cuh).
__global__ void debug_exact_sum_kernel(const float* __restrict__ vals, int64_t nsets, int n, float* __restrict__ out) {
  const int64_t set = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (set >= nsets) return;
  const float r = warp_exact_sum(vals + set * n, n, 0.f, false);
  if (lane == 0) out[set] = r;
}
}  // namespace anns

extern "C" int anns_debug_exact_sum(const float* vals, int64_t nsets, int32_t n, float* out, void* stream) {
  if (nsets < 0 || nsets > (int64_t(1) << 30) || n < 0 || n >= 1024)
    return fail(ANNS_ERR_INVALID_ARG, "0 <= nsets <= 2^30 and 0 <= n < 1024 required");
  if (nsets == 0) return ANNS_OK;
  if (!out || (!vals && n > 0)) return fail(ANNS_ERR_INVALID_ARG, "null buffer");
  debug_exact_sum_kernel<<<(unsigned)((nsets + 7) / 8), 256, 0, (cudaStream_t)stream>>>(vals, nsets, n, out);
  note_launch();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? ANNS_OK : cuda_fail(e, "exact sum kernel");
}

extern "C" int anns_scan_pairs(anns_index* ix, const float* Q, int64_t nq, const int32_t* pq,
                               const int32_t* pl, const uint8_t* pb, int64_t npairs,
                               const int64_t* off, float* dist_out, int32_t* S_out, void* stream) {
  int rc = check_pairs(ix, Q, nq, pq, pl, pb, npairs);
  if (rc) return rc;
  if (npairs == 0) return ANNS_OK;
  if (!off || !dist_out) return fail(ANNS_ERR_INVALID_ARG, "null buffer");
  DeviceGuard g(ix->device);
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = grow((void**)&ix->ws_qt, &ix->ws_qt_cap, (size_t)nq * ix->Mp * kKsub * 4))) return rc;
  cudaError_t e = launch_query_tables(*ix, Q, nq, ix->ws_qt, s);
  if (e == cudaSuccess)
    e = launch_scan_pairs(*ix, Q, ix->ws_qt, nq, pq, pl, pb, npairs, off, dist_out, S_out, s);
  return e == cudaSuccess ? ANNS_OK : cuda_fail(e, "scan kernel");
}

extern "C" int anns_profile(anns_index* ix, int32_t enable, double* out_ms, int64_t* count) {
  if (!ix) return fail(ANNS_ERR_INVALID_ARG, "null index");
  DeviceGuard g(ix->device);
  int rc = drain_profile(*ix, true);
  if (rc) return rc;
  if (enable == 1) {
    ix->prof_on = true;
    for (double& v : ix->prof_ms) v = 0.0;
    ix->prof_count = 0;
  } else if (enable == 0) {
    ix->prof_on = false;
  }
  if (out_ms)
    for (int st = 0; st < Index::kStages; ++st) out_ms[st] = ix->prof_ms[st];
  if (count) *count = ix->prof_count;
  return ANNS_OK;
}

extern "C" int anns_set_svr(anns_index* ix, const anns_svr_model* m) {
  if (!ix || !m) return fail(ANNS_ERR_INVALID_ARG, "null index or model");
  if (m->nsv < 1 || m->nsv > ANNS_SVR_MAX_SAMPLES) return fail(ANNS_ERR_INVALID_ARG, "nsv out of range");
  if (m->table_n < 2 || m->table_n > 4096) return fail(ANNS_ERR_INVALID_ARG, "table_n must be in [2, 4096]");
  if (!(m->table_ratio > 0.0 && m->table_ratio < 1.0)) return fail(ANNS_ERR_INVALID_ARG, "table_ratio must be in (0, 1)");
  if (!m->sv || !m->beta) return fail(ANNS_ERR_INVALID_ARG, "null support vectors or coefficients");
  bool finite = std::isfinite(m->gamma) && std::isfinite(m->inv_step);
  for (int i = 0; i < 5; ++i) finite = finite && std::isfinite(m->mean[i]) && std::isfinite(m->inv_std[i]);
  for (int64_t i = 0; i < (int64_t)m->nsv * 5 && finite; ++i) finite = std::isfinite(m->sv[i]);
  for (int i = 0; i < m->nsv && finite; ++i) finite = std::isfinite(m->beta[i]);
  if (!finite) return fail(ANNS_ERR_INVALID_ARG, "non-finite model parameter");
  std::vector<float> h((size_t)m->nsv * 6 + m->table_n);
  std::memcpy(h.data(), m->sv, (size_t)m->nsv * 5 * sizeof(float));
  std::memcpy(h.data() + (size_t)m->nsv * 5, m->beta, (size_t)m->nsv * sizeof(float));
  double e = 1.0;  // geometric table: e_k = fl64(e_{k-1} * rho), rounded once to FP32
  for (int k = 0; k < m->table_n; ++k) {
    h[(size_t)m->nsv * 6 + k] = (float)e;
    e = e * m->table_ratio;
  }
  DeviceGuard g(ix->device);
  if (ix->svr_dev) { cudaFree(ix->svr_dev); ix->svr_dev = nullptr; ix->has_svr = false; }
  cudaError_t ce = cudaMalloc((void**)&ix->svr_dev, h.size() * sizeof(float));
  if (ce != cudaSuccess) { ix->svr_dev = nullptr; return cuda_fail(ce, "cudaMalloc(svr model)"); }
  ce = cudaMemcpy(ix->svr_dev, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) return cuda_fail(ce, "svr model copy");
  ix->svr_nsv = m->nsv; ix->svr_tn = m->table_n; ix->svr_gamma = m->gamma; ix->svr_inv_step = m->inv_step;
  ix->svr_ratio = m->table_ratio;
  ix->svr_host.assign(h.begin(), h.begin() + (size_t)m->nsv * 6);
  for (int i = 0; i < 5; ++i) { ix->svr_mean[i] = m->mean[i]; ix->svr_inv_std[i] = m->inv_std[i]; }
  ix->has_svr = true;
  return ANNS_OK;
}

extern "C" int anns_set_option(anns_index* ix, int32_t option, int64_t value) {
  if (!ix) return fail(ANNS_ERR_INVALID_ARG, "null index");
  switch (option) {
    case ANNS_OPT_KERNEL:
      if (value < ANNS_KERNEL_AUTO || value > ANNS_KERNEL_SPLIT)
        return fail(ANNS_ERR_INVALID_ARG, "unknown kernel choice");
      ix->opt_kernel = (int)value;
      return ANNS_OK;
    case ANNS_OPT_SCHEDULE:
      if (value < ANNS_SCHED_AUTO || value > ANNS_SCHED_LPT) return fail(ANNS_ERR_INVALID_ARG, "unknown schedule");
      ix->opt_schedule = (int)value;
      return ANNS_OK;
    case ANNS_OPT_QCHUNK:
      if (value < 0) return fail(ANNS_ERR_INVALID_ARG, "query chunk must be >= 0");
      ix->opt_qchunk = value;
      return ANNS_OK;
    case ANNS_OPT_WAIT_CYCLES:
      if (value < 0) return fail(ANNS_ERR_INVALID_ARG, "wait limit must be >= 0");
      ix->opt_wait_cycles = value;
      return ANNS_OK;
    case ANNS_OPT_NIBBLE:
      if (value != 0 && value != 1) return fail(ANNS_ERR_INVALID_ARG, "nibble option must be 0 or 1");
      ix->opt_nibble = (int)value;
      return ANNS_OK;
    default: return fail(ANNS_ERR_INVALID_ARG, "unknown option");
  }
}
