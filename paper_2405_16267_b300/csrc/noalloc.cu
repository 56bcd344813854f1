// Allocation-free entry point: the consensus update (z, t, s, v) of one outer iteration,
// with its scratch memory in file-scope device arrays instead of buffers from cudaMalloc.
//
// Some callers cannot allocate device memory when they call in: code running while a
// stream is being captured into a CUDA graph (cudaMalloc is not allowed there), services
// whose device memory is owned by another allocator or pool (a raw cudaMalloc would step
// outside its accounting), and latency-bound loops that must not risk the implicit
// synchronisation of a cudaMalloc/cudaFree.  They pass their inputs and outputs and this
// file supplies the scratch.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>

#include "bicadmm.h"
#include "common.cuh"
#include "nspace.cuh"

using namespace bic;

namespace {

constexpr int kNoAllocThreads = 1024;
constexpr int64_t kNoAllocMaxN = 32768;  // largest n this entry point accepts
constexpr int kMaxDevices = 64;

// The scratch of the consensus update, shared by every call on a device:
//   breakpoints tau_r, their intercepts and slopes c_r, e_r (n doubles each), top-kappa
//   keys (n uint64), the scalar block, one residual record and the device status word.
//   About 1 MB per device, held by every GPU that loads the library until the process
//   exits.
struct NoAllocScratch {
  double tau_r[kNoAllocMaxN];
  double c_arr[kNoAllocMaxN];
  double e_arr[kNoAllocMaxN];
  uint64_t key[kNoAllocMaxN];
  GlobalState gs;
  Resid rec;
  int err;
};
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Device address of g_noalloc_scratch, looked up once per device (host code cannot use
// the symbol itself as a device pointer).  The first lookup on a device runs under a
// mutex, so first calls from several host threads are well defined.
std::atomic<NoAllocScratch*> g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

NoAllocScratch* scratch_for_device(int dev) {
  NoAllocScratch* sc = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (sc) return sc;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  sc = g_scratch_addr[dev].load(std::memory_order_relaxed);
  if (sc) return sc;
  void* ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
    cudaGetLastError();
    return nullptr;
  }
  sc = static_cast<NoAllocScratch*>(ptr);
  g_scratch_addr[dev].store(sc, std::memory_order_release);
  return sc;
}

__global__ void k_noalloc_prologue(NoAllocScratch* sc, const double* tvt) {
  // Clear everything the consensus kernel reads before writing; take v^k from the caller.
  sc->gs.t = 0.0;
  sc->gs.v = tvt[1];
  sc->gs.tau = 0.0;
  sc->gs.iter = 0;
  sc->gs.ticket = 0;
  sc->err = 0;
}

__global__ void k_noalloc_epilogue(const NoAllocScratch* sc, double* tvt) {
  tvt[0] = sc->gs.t;
  tvt[1] = sc->gs.v;
  tvt[2] = sc->gs.tau;
  tvt[3] = static_cast<double>(sc->err);
}

}  // namespace

extern "C" int bicadmm_consensus_step_noalloc(const double* w, double* z, double* s, double* tvt,
                                              int64_t n, int64_t kappa, int32_t N_shards,
                                              double rho_c, double rho_b, void* stream) {
  if (!w || !z || !s || !tvt) return BICADMM_ERR_ARG;
  if (n < 1 || n > kNoAllocMaxN) return BICADMM_ERR_ARG;
  if (kappa < 1 || kappa > n || N_shards < 1) return BICADMM_ERR_ARG;
  if (!(rho_c > 0.0) || !(rho_b > 0.0)) return BICADMM_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return BICADMM_ERR_CUDA;
  }
  NoAllocScratch* sc = scratch_for_device(dev);
  if (!sc) return BICADMM_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_noalloc_prologue<<<1, 1, 0, st>>>(sc, tvt);
  ConsensusArgs a{};
  a.x = nullptr;
  a.u = nullptr;
  a.w = const_cast<double*>(w);  // read only when x is null
  a.z = z;
  a.s = s;
  a.tau_r = sc->tau_r;
  a.c_arr = sc->c_arr;
  a.e_arr = sc->e_arr;
  a.key = sc->key;
  a.gs = &sc->gs;
  a.trace = &sc->rec;
  a.trace_cap = 1;
  a.N = N_shards;
  a.n = n;
  a.kappa = kappa;
  a.lda = n;
  a.rho_c = rho_c;
  a.rho_b = rho_b;
  a.err = &sc->err;
  a.enabled = 1;
  k_global<kNoAllocThreads, 1><<<1, kNoAllocThreads, 0, st>>>(a);
  k_noalloc_epilogue<<<1, 1, 0, st>>>(sc, tvt);
  return cudaGetLastError() == cudaSuccess ? BICADMM_OK : BICADMM_ERR_CUDA;
}
