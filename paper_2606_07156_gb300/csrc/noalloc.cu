// Cluster locating (the coarse stage) without any allocation.
//
// Some callers cannot allocate device memory: real-time or embedded hosts
// that forbid allocation after start-up (cudaMalloc and cudaFree take
// unbounded time and may synchronise the device), and plugins living inside
// a host application that owns every memory pool. For them, anns_locate_static
// runs the coarse-distance and top-nprobe kernels with their scratch (the
// nq x nlist distance matrix) in a fixed array compiled into this library,
// instead of the index workspace that anns_search grows with cudaMalloc.
//
// The array is a file-scope __device__ variable of ANNS_STATIC_SCRATCH_FLOATS
// floats (8 MiB); every GPU that loads the library holds it until the process
// exits. Host code cannot use the array's name as a device address, so the
// first call on each device, with that device current, looks the address up
// with cudaGetSymbolAddress and caches it; that first call should happen
// before any stream capture. Every call on a device shares the one array:
// calls whose work overlaps on the GPU (different streams, or different
// threads without ordering) race on it. Each call overwrites every element it
// later reads, so nothing needs clearing between calls.
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace anns {
namespace {

__device__ __align__(256) float g_static_scratch[ANNS_STATIC_SCRATCH_FLOATS];

constexpr int kMaxDevices = 64;
float* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of g_static_scratch on the current device (looked up once).
int static_scratch(int dev, float** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(ANNS_ERR_UNSUPPORTED, "device ordinal too large");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
    g_scratch_ptr[dev] = (float*)p;
  }
  *out = g_scratch_ptr[dev];
  return ANNS_OK;
}

}  // namespace
}  // namespace anns

using namespace anns;

extern "C" int anns_locate_static(anns_index* ix, const float* queries, int64_t nq, int32_t nprobe,
                                  int32_t* probes_out, float* probe_d2_out, void* stream) {
  if (!ix) return fail(ANNS_ERR_INVALID_ARG, "null index");
  if (nq < 0) return fail(ANNS_ERR_INVALID_ARG, "nq must be >= 0");
  if (nprobe < 1 || nprobe > ix->nlist || nprobe > ANNS_MAX_NPROBE)
    return fail(ANNS_ERR_INVALID_ARG, "nprobe must be in [1, min(nlist, 128)]");
  if (nq > 0 && (!queries || !probes_out || !probe_d2_out)) return fail(ANNS_ERR_INVALID_ARG, "null buffer");
  // nq <= scratch / nlist: the product nq * nlist is never formed, so no
  // overflow can let a huge nq through
  if (nq > (int64_t)ANNS_STATIC_SCRATCH_FLOATS / ix->nlist)
    return fail(ANNS_ERR_INVALID_ARG,
                "nq * nlist exceeds the static scratch (ANNS_STATIC_SCRATCH_FLOATS); use anns_search "
                "or smaller batches");
  if (nq == 0) return ANNS_OK;
  int prev = 0;
  cudaError_t se = cudaGetDevice(&prev);
  if (se != cudaSuccess) return cuda_fail(se, "cudaGetDevice");
  se = cudaSetDevice(ix->device);
  if (se != cudaSuccess) return cuda_fail(se, "cudaSetDevice(index device)");
  float* d2 = nullptr;
  int rc = static_scratch(ix->device, &d2);
  if (rc == ANNS_OK) {
    cudaError_t e = launch_coarse(*ix, queries, nq, nprobe, nullptr, d2, probes_out, probe_d2_out,
                                  (cudaStream_t)stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "coarse kernels");
  }
  cudaSetDevice(prev);
  return rc;
}
