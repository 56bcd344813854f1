// Host runtime of libbicadmm: handle state, device layout, kernel dispatch and the C ABI
// declared in include/bicadmm.h.
//
// Device layout (all row-major, all owned by the handle):
//   A       m x lda   (TA = double | float | bf16), lda = n rounded up to 32, zero padding
//   b       m (TM);  omega, nu  m x K (TM)
//   x, u, r  N x ldx  FP64, ldx = lda K (K = 1 except softmax: entry (c, k) at c K + k);
//            xlo N x ldx (TM copy of x read by the A pass)
//   z, s, w           ldx FP64;  tau_r, c_arr, e_arr ldx FP64 and key ldx uint64
//                     (scratch of the consensus CTA)
//   P       per block (i,j): n_j x ldp_j (TP = TM), ldp_j = n_j rounded up to 32
//   slots   (G + N) x ldx (TM): A'd partial sums, one row per (panel CTA, shard) pair
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <memory>
#include <mutex>
#include <functional>
#include <chrono>
#include <cmath>
#include <deque>
#include <thread>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "bicadmm.h"
#include "common.cuh"
#include "nspace.cuh"
#include "batch.cuh"
#include "multiclass.cuh"
#include "mc_tc.cuh"
#include "objective.cuh"
#include "mc_tc2.cuh"
#include "gram_tf32.cuh"
#include "pass.cuh"
#include "polish.cuh"
#include "setup.cuh"

using namespace bic;

namespace {

constexpr int kPassThreads = 256;
constexpr int kDualThreads = 256;
constexpr int kXupdThreads = 256;
constexpr int kCholSplitCols = 256;  // blocks this wide or wider: the GPU-wide Cholesky
constexpr int kCholChunk = 64;       // rows of a panel solved per CTA in the GPU-wide Cholesky
constexpr int kXupdRows = 32;
constexpr int kXupdRowsK = 512;  // K > 1: rows of P per CTA (one staging of R_ij per CTA)
constexpr int kXupdThreadsK = 512;  // K > 1: one CTA of 16 warps per block of a shard (500-column
                                    // blocks: 62 us against 69 us for 128-row tiles of 256 threads)
constexpr int kCholThreads = 256;
constexpr int kTraceCap = kTraceCapacity;
constexpr int64_t kMaxN = 32768;                 // single-CTA global step limit
constexpr size_t kPassSmemBudget = 200 * 1024;   // dynamic smem for A-pass stages
constexpr size_t kPassCtaTarget = 100 * 1024;    // auto sizing aims at two CTAs per SM
constexpr int kPolishRowBlocks = 592;
constexpr int kPolishChunks = 64;
constexpr int kMaxPolishKappa = 1024;

int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// Text of the last failed create (or batch / server create) on this host thread.
thread_local std::string g_create_error;

}  // namespace

struct bicadmm_ctx {
  bicadmm_params p{};
  cudaStream_t stream = nullptr;
  int device = 0, num_sms = 0;
  std::string err;
  bool ready = false;
  int64_t launches = 0;
  int64_t iters_done = 0;
  bool converged = false;
  // CUDA graph of graph_iters outer iterations, replayed by bicadmm_step (0 = eager)
  int graph_iters = 0;
  cudaGraphExec_t graph = nullptr;
  int64_t graph_launches = 0;  // kernels in one replay

  // geometry
  int N = 0, M = 0;
  int64_t lda = 0;
  int K = 1;          // classes (softmax), 1 otherwise
  int KC = 1;         // compile-time class bucket of the K > 1 kernels
  int64_t ldx = 0;    // n-space row stride, lda K
  bool use_tc = false;  // BF16 softmax: tensor-core A pass (k_fused_pass_tc)
  bool tc2 = false;     // ... on pairs of SMs (k_fused_pass_tc2, 128-row panels)
  bool tf32 = false;    // BICADMM_PREC_TF32: 32-bit storage of A rounded to TF32 (p.precision
                        // then reads FP32, whose kernels serve it unchanged)
  // a sparsity path (bicadmm_create_path): K = ninst instances of one problem that differ in
  // kappa, run as the K columns of the multi-column kernels; each has its own consensus CTA,
  // scalars and residual records; z_cm, s_cm hold their z and s instance-major
  bool path = false;
  int ninst = 1;
  std::vector<int64_t> kappas;
  int64_t* d_kappas = nullptr;
  double *z_cm = nullptr, *s_cm = nullptr;
  CUtensorMap tmap;     // 2D map of A (BF16, 64 x 128 boxes, 128-byte swizzle) for it
  double c0 = 0.0;
  size_t esz = 8;  // bytes per m-space / n-space low-precision element (TM)
  size_t asz = 8;  // bytes per stored A element (TA)
  std::vector<int64_t> shard_row0, panel_start, G_off, P_off;
  std::vector<int> blk_col0, blk_ldp, slot_lo, slot_hi;
  int R = 0, S = 0, VPT = 0, G = 0, nslots = 0, max_nj = 0, max_ldp = 0, dual_chunks = 0;
  int64_t P_panels = 0, G_total = 0, P_total = 0;
  size_t pass_smem = 0;
  // fault injection for tests (bicadmm_inject_pass_stall): the K = 1 pass never posts the
  // load of stall_panel and waits at most wait_limit cycles on a stage
  int64_t stall_panel = -1;
  long long wait_limit = kWaitLimitCycles;

  // device buffers
  void *A = nullptr, *b = nullptr, *omega = nullptr, *nu = nullptr, *slots = nullptr,
       *xlo = nullptr, *Pm = nullptr;
  unsigned char* wpk = nullptr;  // tensor-core pass: W_i as BF16 hi/lo MMA tiles per shard
  int nslab = 0;                 // 128-column slabs of a row (tensor-core pass)
  double *x = nullptr, *u = nullptr, *r = nullptr, *z = nullptr, *s = nullptr, *w = nullptr,
         *tau_r = nullptr, *c_arr = nullptr, *e_arr = nullptr, *cta_stats = nullptr,
         *dual_part = nullptr;
  uint64_t* key = nullptr;
  int64_t *d_shard_row0 = nullptr, *d_panel_start = nullptr, *d_P_off = nullptr,
          *d_G_off = nullptr;
  int *d_blk_col0 = nullptr, *d_blk_ldp = nullptr, *d_slot_lo = nullptr, *d_slot_hi = nullptr;
  GlobalState* gs = nullptr;
  Resid* trace = nullptr;
  int* d_err = nullptr;
  // objective F(z): compacted nonzero features, their count, per-CTA partial sums, and
  // out[0] = F(z), out[1] = ||z||^2
  int *obj_idx = nullptr, *obj_cnt = nullptr;
  double *obj_part = nullptr, *obj_out = nullptr;
  // entry lists of k_consensus_prep for the consensus CTA (K > 1): indices per instance
  // (n K entries, instance-major for a path) and u_nb counts per instance
  int *u_idx = nullptr, *u_cnt = nullptr;
  int u_nb = 0;
  int obj_blocks = 0;
  std::vector<void*> allocs;

  // polish buffers (allocated on first use)
  int64_t* supp = nullptr;
  double *AS = nullptr, *pq = nullptr, *pd1 = nullptr, *pd2 = nullptr, *pp = nullptr,
         *pxs = nullptr, *pstep = nullptr, *pfpart = nullptr, *pgpart = nullptr,
         *pHpart = nullptr, *pH = nullptr;
  int* pflag = nullptr;
  bool polish_ready = false;
  // softmax polish (allocated on first use): support in class order, its classes and class
  // offsets, A_S and U (kappa x m), per-row q, p, d1, P (m x K)
  int64_t* ssupp = nullptr;
  int *scls = nullptr, *skb = nullptr;
  double *sU = nullptr, *sq = nullptr, *sp = nullptr, *sd1 = nullptr, *sP = nullptr;
  bool spolish_ready = false;

  // profiling: CUDA events around kernel launches on the handle's stream
  int prof = 0;                 // 0 off, 1 the A pass only, 2 every kernel of the iteration
  std::vector<cudaEvent_t> ev;  // pairs (start, end)
  std::vector<int> ev_kind;     // kernel kind of each pair
  size_t ev_used = 0;           // events recorded
};

namespace {

int fail(bicadmm_ctx* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(h, BICADMM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
int dev_alloc(bicadmm_ctx* h, T** ptr, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, e == cudaErrorMemoryAllocation ? BICADMM_ERR_OOM : BICADMM_ERR_CUDA,
                "cudaMalloc(" + std::to_string(bytes) + " B): " + cudaGetErrorString(e));
  }
  h->allocs.push_back(p);
  *ptr = static_cast<T*>(p);
  return BICADMM_OK;
}

void free_all(bicadmm_ctx* h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  h->graph = nullptr;
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  h->ev.clear();
}

// ---------------------------------------------------------------- A-pass dispatch
// With K > 1 the pass that carries the consensus CTA is preceded by k_consensus_prep (w and
// the breakpoints given); with K = 1 the consensus CTA forms them itself from x and u.
ConsensusArgs consensus_args(bicadmm_ctx* h, bool enabled) {
  ConsensusArgs a{};
  a.x = h->K > 1 ? nullptr : h->x;
  a.prepared = h->K > 1 ? 1 : 0;
  a.u = h->u;
  a.w = h->w;
  a.z = h->z;
  a.s = h->s;
  a.tau_r = h->tau_r;
  a.c_arr = h->c_arr;
  a.e_arr = h->e_arr;
  a.key = h->key;
  a.gs = h->gs;
  a.trace = h->trace;
  a.trace_cap = kTraceCap;
  a.N = h->N;
  a.n = h->p.n * h->K;
  a.kappa = h->p.kappa;
  a.lda = h->ldx;
  a.rho_c = h->p.rho_c;
  a.rho_b = h->p.rho_b;
  a.err = h->d_err;
  a.enabled = enabled ? 1 : 0;
  // the pass kernels launch with pass_smem bytes of dynamic shared memory, which their
  // consensus CTA (it stages no panels) may fill with top-kappa candidates
  a.cand_bytes = static_cast<int64_t>(h->pass_smem);
  if (a.prepared) {
    a.u_idx = h->u_idx;
    a.u_cnt = h->u_cnt;
    a.u_nb = h->u_nb;
  }
  if (h->path) {  // instance q: n entries of the instance-major arrays from q n
    a.z = h->z_cm;
    a.s = h->s_cm;
    a.n = h->p.n;
    a.kappa = h->kappas[0];
    a.ninst = h->ninst;
    a.inst_n = h->p.n;
    a.kappas = h->d_kappas;
  }
  return a;
}

// Allow the largest dynamic shared memory the kernel can take next to its static part.
template <typename K>
cudaError_t allow_max_dynamic_smem(K kern) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              227 * 1024 - static_cast<int>(fa.sharedSizeBytes));
}

template <typename TA, typename TM, int R, int VPT>
int launch_pass_rv(bicadmm_ctx* h, bool with_consensus) {
  auto kern = k_fused_pass<TA, TM, R, VPT, kPassThreads>;
  static bool attr_set = false;  // per instantiation
  if (!attr_set) {
    CK(allow_max_dynamic_smem(kern));
    attr_set = true;
  }
  PassGeometry geo{h->d_shard_row0, h->d_panel_start, h->N, h->P_panels, h->stall_panel};
  kern<<<h->G + (with_consensus ? h->ninst : 0), kPassThreads, h->pass_smem, h->stream>>>(
      static_cast<const TA*>(h->A), h->lda, static_cast<const TM*>(h->xlo),
      static_cast<const TM*>(h->b), static_cast<TM*>(h->omega), static_cast<TM*>(h->nu),
      static_cast<TM*>(h->slots), h->cta_stats, geo, h->S, h->p.loss, static_cast<TM>(h->M),
      static_cast<TM>(h->p.rho_l), h->p.newton_iters, h->d_err, h->wait_limit,
      consensus_args(h, with_consensus));
  CK(cudaGetLastError());
  return BICADMM_OK;
}

template <typename TA, typename TM, int R>
int launch_pass_r(bicadmm_ctx* h, bool wc) {
  switch (h->VPT) {
    case 1: return launch_pass_rv<TA, TM, R, 1>(h, wc);
    case 2: return launch_pass_rv<TA, TM, R, 2>(h, wc);
    case 3: return launch_pass_rv<TA, TM, R, 3>(h, wc);
    case 4: return launch_pass_rv<TA, TM, R, 4>(h, wc);
    case 5: return launch_pass_rv<TA, TM, R, 5>(h, wc);
    case 6: return launch_pass_rv<TA, TM, R, 6>(h, wc);
    case 8: return launch_pass_rv<TA, TM, R, 8>(h, wc);
    case 12: return launch_pass_rv<TA, TM, R, 12>(h, wc);
    case 16: return launch_pass_rv<TA, TM, R, 16>(h, wc);
  }
  return fail(h, BICADMM_ERR_UNSUPPORTED, "no A-pass variant for this width");
}

template <typename TA, typename TM>
int launch_pass(bicadmm_ctx* h, bool with_consensus) {
  switch (h->R) {
    case 1: return launch_pass_r<TA, TM, 1>(h, with_consensus);
    case 2: return launch_pass_r<TA, TM, 2>(h, with_consensus);
    case 4: return launch_pass_r<TA, TM, 4>(h, with_consensus);
    case 8: return launch_pass_r<TA, TM, 8>(h, with_consensus);
  }
  return fail(h, BICADMM_ERR_UNSUPPORTED, "no A-pass variant for this panel height");
}

// K > 1 (softmax) pass: R is fixed at 8 rows per panel; (VPT, KC) chosen at geometry time.
constexpr int kPassRowsK = 8;

template <typename TA, typename TM, int VPT, int KC>
constexpr bool pass_k_fits() {
  // x and Q accumulators of VPT x VE columns x KC classes, twice, in registers
  return VPT * Vec16<TA>::n * KC * (sizeof(TM) == 8 ? 2 : 1) <= 80;
}

template <typename TA, typename TM, int VPT, int KC>
int launch_pass_k_v(bicadmm_ctx* h, bool with_consensus, int op, int* blocks) {
  if constexpr (!pass_k_fits<TA, TM, VPT, KC>()) {
    return fail(h, BICADMM_ERR_UNSUPPORTED, "softmax A-pass: n K too large for the register tiles");
  } else {
    auto kern = k_fused_pass_k<TA, TM, kPassRowsK, VPT, kPassThreads, KC>;
    CK(allow_max_dynamic_smem(kern));
    if (op == 1) {
      CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern, kPassThreads, h->pass_smem));
      return BICADMM_OK;
    }
    PassGeometry geo{h->d_shard_row0, h->d_panel_start, h->N, h->P_panels, -1};
    kern<<<h->G + (with_consensus ? h->ninst : 0), kPassThreads, h->pass_smem, h->stream>>>(
        static_cast<const TA*>(h->A), h->lda, static_cast<const TM*>(h->xlo), h->ldx, h->K,
        static_cast<const TM*>(h->b), static_cast<TM*>(h->omega), static_cast<TM*>(h->nu),
        static_cast<TM*>(h->slots), h->cta_stats, geo, h->S, static_cast<TM>(h->M),
        static_cast<TM>(h->p.rho_l), h->p.newton_iters, h->d_err, kWaitLimitCycles,
        consensus_args(h, with_consensus), h->path ? h->p.loss : -1);
    CK(cudaGetLastError());
    return BICADMM_OK;
  }
}

template <typename TA, typename TM, int KC>
int launch_pass_k_c(bicadmm_ctx* h, bool wc, int op, int* blocks) {
  switch (h->VPT) {
    case 1: return launch_pass_k_v<TA, TM, 1, KC>(h, wc, op, blocks);
    case 2: return launch_pass_k_v<TA, TM, 2, KC>(h, wc, op, blocks);
    case 4: return launch_pass_k_v<TA, TM, 4, KC>(h, wc, op, blocks);
  }
  return fail(h, BICADMM_ERR_UNSUPPORTED, "no softmax A-pass variant for this width");
}

// op 0 = launch, 1 = occupancy query
template <typename TA, typename TM>
int launch_pass_k(bicadmm_ctx* h, bool wc, int op = 0, int* blocks = nullptr) {
  switch (h->KC) {
    case 4: return launch_pass_k_c<TA, TM, 4>(h, wc, op, blocks);
    case 10: return launch_pass_k_c<TA, TM, 10>(h, wc, op, blocks);
    case 16: return launch_pass_k_c<TA, TM, 16>(h, wc, op, blocks);
  }
  return fail(h, BICADMM_ERR_UNSUPPORTED, "no softmax A-pass variant for this class count");
}

template <int KC>
int launch_pass_tc_c(bicadmm_ctx* h, bool with_consensus, int op, int* blocks) {
  auto kern = k_fused_pass_tc<KC>;
  CK(allow_max_dynamic_smem(kern));
  if (op == 1) {
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern, kTcThreads, h->pass_smem));
    return BICADMM_OK;
  }
  PassGeometry geo{h->d_shard_row0, h->d_panel_start, h->N, h->P_panels, -1};
  kern<<<h->G + (with_consensus ? h->ninst : 0), kTcThreads, h->pass_smem, h->stream>>>(
      h->tmap, h->lda, h->wpk, h->ldx, h->K,
      static_cast<const float*>(h->b), static_cast<float*>(h->omega), static_cast<float*>(h->nu),
      static_cast<float*>(h->slots), h->cta_stats, geo, static_cast<float>(h->M),
      static_cast<float>(h->p.rho_l), h->p.newton_iters, h->d_err, kWaitLimitCycles,
      consensus_args(h, with_consensus), h->path ? h->p.loss : -1);
  CK(cudaGetLastError());
  return BICADMM_OK;
}

// The pair kernel; op 1 returns the number of co-resident clusters of two CTAs.
template <int KC>
int launch_pass_tc2_c(bicadmm_ctx* h, bool with_consensus, int op, int* blocks) {
  auto kern = k_fused_pass_tc2<KC>;
  CK(allow_max_dynamic_smem(kern));
  if (op == 1) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(2 * static_cast<unsigned>(h->num_sms), 1, 1);
    cfg.blockDim = dim3(kTc2Threads, 1, 1);
    cfg.dynamicSmemBytes = h->pass_smem;
    cfg.stream = h->stream;
    CK(cudaOccupancyMaxActiveClusters(blocks, kern, &cfg));
    return BICADMM_OK;
  }
  PassGeometry geo{h->d_shard_row0, h->d_panel_start, h->N, h->P_panels, -1};
  const int ncons = with_consensus ? tc2_cons_ctas(h->ninst) : 0;
  kern<<<2 * h->G + ((ncons + 1) & ~1), kTc2Threads, h->pass_smem, h->stream>>>(
      h->tmap, h->lda, h->wpk, h->nslab, h->ldx, h->K,
      static_cast<const float*>(h->b), static_cast<float*>(h->omega), static_cast<float*>(h->nu),
      static_cast<float*>(h->slots), h->cta_stats, geo, static_cast<float>(h->M),
      static_cast<float>(h->p.rho_l), h->p.newton_iters, h->d_err, kWaitLimitCycles,
      consensus_args(h, with_consensus), h->path ? h->p.loss : -1);
  CK(cudaGetLastError());
  return BICADMM_OK;
}

int launch_pass_tc(bicadmm_ctx* h, bool wc, int op = 0, int* blocks = nullptr) {
  if (h->tc2) {
    switch (h->KC) {
      case 4: return launch_pass_tc2_c<4>(h, wc, op, blocks);
      case 10: return launch_pass_tc2_c<10>(h, wc, op, blocks);
      case 16: return launch_pass_tc2_c<16>(h, wc, op, blocks);
    }
  }
  switch (h->KC) {
    case 4: return launch_pass_tc_c<4>(h, wc, op, blocks);
    case 10: return launch_pass_tc_c<10>(h, wc, op, blocks);
    case 16: return launch_pass_tc_c<16>(h, wc, op, blocks);
  }
  return fail(h, BICADMM_ERR_UNSUPPORTED, "no tensor-core A-pass variant for this class count");
}

// Encode the TMA map of the BF16 A for the tensor-core pass (driver entry point fetched
// through the runtime, so the library does not link libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int make_tmap(bicadmm_ctx* h) {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q));
    if (!ptr || q != cudaDriverEntryPointSuccess) return fail(h, BICADMM_ERR_CUDA, "cuTensorMapEncodeTiled not available");
    fn = reinterpret_cast<EncodeTiledFn>(ptr);
  }
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(h->lda), static_cast<cuuint64_t>(h->p.m)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(h->lda) * 2};
  const cuuint32_t box[2] = {64, static_cast<cuuint32_t>(h->tc2 ? kTc2Rows : kTcRows)};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(&h->tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, h->A, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(h, BICADMM_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string(static_cast<int>(r)));
  return BICADMM_OK;
}

// Launch the A pass for the handle's precision and class count.
int launch_pass_any(bicadmm_ctx* h, bool last) {
  if (h->use_tc) return launch_pass_tc(h, last);
  const bool mc = h->K > 1;
  switch (h->p.precision) {
    case BICADMM_PREC_FP64: return mc ? launch_pass_k<double, double>(h, last) : launch_pass<double, double>(h, last);
    case BICADMM_PREC_FP32: return mc ? launch_pass_k<float, float>(h, last) : launch_pass<float, float>(h, last);
    default: return mc ? launch_pass_k<__nv_bfloat16, float>(h, last) : launch_pass<__nv_bfloat16, float>(h, last);
  }
}

template <typename TA, typename TM, int R, int VPT>
int occupancy_rv(bicadmm_ctx* h, int* blocks) {
  auto kern = k_fused_pass<TA, TM, R, VPT, kPassThreads>;
  CK(allow_max_dynamic_smem(kern));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern, kPassThreads, h->pass_smem));
  return BICADMM_OK;
}

template <typename TA, typename TM>
int pass_occupancy(bicadmm_ctx* h, int* blocks) {
  // Occupancy depends on registers (VPT) and shared memory; query the chosen variant.
#define OCC_CASE(RR, VV) \
  if (h->R == RR && h->VPT == VV) return occupancy_rv<TA, TM, RR, VV>(h, blocks);
#define OCC_R(RR) OCC_CASE(RR, 1) OCC_CASE(RR, 2) OCC_CASE(RR, 3) OCC_CASE(RR, 4) OCC_CASE(RR, 5) \
  OCC_CASE(RR, 6) OCC_CASE(RR, 8) OCC_CASE(RR, 12) OCC_CASE(RR, 16)
  OCC_R(1) OCC_R(2) OCC_R(4) OCC_R(8)
#undef OCC_R
#undef OCC_CASE
  return fail(h, BICADMM_ERR_UNSUPPORTED, "no A-pass variant");
}

int pick_vpt(int64_t nvec) {
  static const int opts[] = {1, 2, 3, 4, 5, 6, 8, 12, 16};
  for (int v : opts)
    if (static_cast<int64_t>(v) * kPassThreads >= nvec) return v;
  return -1;
}

// Softmax pass: the smallest of {1, 2, 4} vectors per thread covering the row, if its
// register tiles (VPT x VE columns x KC classes, x and Q, doubled for FP64) fit.
int pick_vpt_k(int64_t nvec, int ve, int kc, size_t tm_bytes) {
  static const int opts[] = {1, 2, 4};
  for (int v : opts)
    if (static_cast<int64_t>(v) * kPassThreads >= nvec)
      return v * ve * kc * (tm_bytes == 8 ? 2 : 1) <= 80 ? v : -1;
  return -1;
}

// ---------------------------------------------------------------- profiling events
enum KernelKind { KIND_PASS = 0, KIND_XUPD = 1, KIND_DUAL = 2, KIND_RHS = 3, KIND_COUNT = 4 };

bool prof_on(const bicadmm_ctx* h, int kind) {
  return h->prof == 2 || (h->prof == 1 && kind == KIND_PASS);
}

int prof_begin(bicadmm_ctx* h, int kind) {
  if (!prof_on(h, kind)) return BICADMM_OK;
  if (h->ev_used + 2 > h->ev.size()) {
    for (int q = 0; q < 64; ++q) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      h->ev.push_back(e);
    }
  }
  CK(cudaEventRecord(h->ev[h->ev_used], h->stream));
  return BICADMM_OK;
}

int prof_end(bicadmm_ctx* h, int kind) {
  if (!prof_on(h, kind)) return BICADMM_OK;
  CK(cudaEventRecord(h->ev[h->ev_used + 1], h->stream));
  h->ev_kind.push_back(kind);
  h->ev_used += 2;
  return BICADMM_OK;
}

// ---------------------------------------------------------------- one outer iteration
template <typename TM>
int run_iterations(bicadmm_ctx* h, int n_iters) {
  const int N = h->N, M = h->M;
  const int64_t lda = h->ldx, n = h->p.n * h->K;
  const dim3 rhs_grid(static_cast<unsigned>((lda + 255) / 256), N);
  const dim3 xupd_grid(static_cast<unsigned>((h->max_nj + kXupdRows - 1) / kXupdRows), M, N);
  const size_t xupd_smem = static_cast<size_t>(h->max_ldp) * sizeof(TM);
  const dim3 dual_grid(h->dual_chunks, N);
  for (int it = 0; it < n_iters; ++it) {
    for (int jj = 0; jj < h->p.inner_iters; ++jj) {
      // The first sweep's right-hand side was formed by the previous iteration's k_dual (or
      // is zero after setup); later sweeps form it from the previous pass's slots.
      int rc;
      if (jj > 0) {
        if ((rc = prof_begin(h, KIND_RHS)) != BICADMM_OK) return rc;
        k_rhs<TM><<<rhs_grid, 256, 0, h->stream>>>(static_cast<const TM*>(h->slots), h->d_slot_lo,
                                                     h->d_slot_hi, h->x, h->u, h->z, h->r, lda,
                                                     h->p.rho_l, h->p.rho_c, h->c0);
        if ((rc = prof_end(h, KIND_RHS)) != BICADMM_OK) return rc;
        h->launches += 1;
      }
      if ((rc = prof_begin(h, KIND_XUPD)) != BICADMM_OK) return rc;
      if (h->K == 1) {
        k_xupd<TM, TM, kXupdThreads, kXupdRows><<<xupd_grid, kXupdThreads, xupd_smem, h->stream>>>(
            static_cast<const TM*>(h->Pm), h->d_P_off, h->d_blk_col0, h->d_blk_ldp, h->r, h->x,
            static_cast<TM*>(h->xlo), M, lda);
      } else {
        const size_t sm = static_cast<size_t>(h->max_ldp + 4) * h->KC * sizeof(TM);
        const dim3 grid_k(static_cast<unsigned>((h->max_nj + kXupdRowsK - 1) / kXupdRowsK), M, N);
#define XUPD_K(KCV)                                                                                 \
  {                                                                                                 \
    CK(cudaFuncSetAttribute(k_xupd_k<TM, KCV, kXupdThreadsK, kXupdRowsK>,                            \
                            cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm)));    \
    k_xupd_k<TM, KCV, kXupdThreadsK, kXupdRowsK><<<grid_k, kXupdThreadsK, sm, h->stream>>>(          \
        static_cast<const TM*>(h->Pm), h->d_P_off, h->d_blk_col0, h->d_blk_ldp, h->r, h->x,       \
        static_cast<TM*>(h->xlo), M, lda, h->K, h->wpk, h->nslab);                                  \
  }
        if (h->KC == 4) XUPD_K(4) else if (h->KC == 10) XUPD_K(10) else XUPD_K(16)
#undef XUPD_K
      }
      CK(cudaGetLastError());
      if ((rc = prof_end(h, KIND_XUPD)) != BICADMM_OK) return rc;
      // The last sweep's pass also runs the global step in its spare CTA; its target w
      // is formed here by all SMs.
      const bool last = jj == h->p.inner_iters - 1;
      if (last && h->path) {
        k_consensus_prep_path<<<dim3(static_cast<unsigned>(h->u_nb), static_cast<unsigned>(h->K)),
                                kPrepBlock, 0, h->stream>>>(
            h->x, h->u, h->s_cm, h->z_cm, h->w, h->tau_r, h->c_arr, h->e_arr, h->gs, h->u_idx,
            h->u_cnt, N, h->p.n, h->K, lda);
        CK(cudaGetLastError());
        h->launches += 1;
      } else if (last && h->K > 1) {
        k_consensus_prep<<<static_cast<unsigned>(h->u_nb), kPrepBlock, 0, h->stream>>>(
            h->x, h->u, h->s, h->z, h->w, h->tau_r, h->c_arr, h->e_arr, h->gs, h->u_idx, h->u_cnt,
            N, n, lda);
        CK(cudaGetLastError());
        h->launches += 1;
      }
      if ((rc = prof_begin(h, KIND_PASS)) != BICADMM_OK) return rc;
      rc = launch_pass_any(h, last);
      if (rc != BICADMM_OK) return rc;
      if ((rc = prof_end(h, KIND_PASS)) != BICADMM_OK) return rc;
      h->launches += 2;
      if (last && h->path) {  // the instances' z and s back to the feature-major layout
        k_path_to_feature_major<<<static_cast<unsigned>((n + 255) / 256), 256, 0, h->stream>>>(
            h->z_cm, h->s_cm, h->z, h->s, h->p.n, h->K);
        CK(cudaGetLastError());
        h->launches += 1;
      }
    }
    int rc;
    if ((rc = prof_begin(h, KIND_DUAL)) != BICADMM_OK) return rc;
    k_dual<TM, kDualThreads><<<dual_grid, kDualThreads, 0, h->stream>>>(
        h->u, h->x, h->z, static_cast<const TM*>(h->slots), h->d_slot_lo, h->d_slot_hi, h->r,
        h->p.rho_l, h->c0, h->dual_part, h->cta_stats, h->G, h->gs, h->trace, kTraceCap, N, n,
        lda, h->p.rho_c, h->d_err, h->ninst);
    CK(cudaGetLastError());
    if ((rc = prof_end(h, KIND_DUAL)) != BICADMM_OK) return rc;
    h->launches += 1;
    h->iters_done += 1;
  }
  return BICADMM_OK;
}

int check_device_error(bicadmm_ctx* h) {
  int e = 0;
  CK(cudaMemcpyAsync(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  switch (e) {
    case DEV_OK: return BICADMM_OK;
    case DEV_TIMEOUT_PASS: return fail(h, BICADMM_ERR_TIMEOUT, "A-pass wait timed out on the device");
    case DEV_NONPOS_PIVOT: return fail(h, BICADMM_ERR_NUMERIC, "non-positive pivot in a block factorisation");
    case DEV_NONFINITE: return fail(h, BICADMM_ERR_NUMERIC, "non-finite residual (NaN/Inf in the iterates)");
    case DEV_ZT_NOCONV: return fail(h, BICADMM_ERR_NUMERIC, "(z,t) root iteration did not terminate");
    case DEV_BAD_LABEL: return fail(h, BICADMM_ERR_ARG, "softmax labels must be integers in [0, K)");
  }
  return fail(h, BICADMM_ERR_CUDA, "unknown device error " + std::to_string(e));
}

// F(z) of problem (p:SML) at the current consensus iterate, in FP64 (objective.cuh).  Its
// three launches are diagnostics: they are not counted in h->launches.
template <typename TA, typename TM>
int launch_obj_rows(bicadmm_ctx* h, const double* z, int K) {
  if (K == 1)
    k_obj_rows<TA, TM, 1><<<h->obj_blocks, kObjThreads, 0, h->stream>>>(
        static_cast<const TA*>(h->A), h->lda, static_cast<const TM*>(h->b), z, h->obj_idx,
        h->obj_cnt, h->p.m, 1, h->p.loss, h->obj_part);
  else
    k_obj_rows<TA, TM, 16><<<h->obj_blocks, kObjThreads, 0, h->stream>>>(
        static_cast<const TA*>(h->A), h->lda, static_cast<const TM*>(h->b), z, h->obj_idx,
        h->obj_cnt, h->p.m, K, h->p.loss, h->obj_part);
  CK(cudaGetLastError());
  return BICADMM_OK;
}

// inst: the instance of a path (its z, one column); the handle's z otherwise.
int compute_objective(bicadmm_ctx* h, double* out, int inst = 0) {
  const double* z = h->path ? h->z_cm + static_cast<int64_t>(inst) * h->p.n : h->z;
  const int K = h->path ? 1 : h->K;
  k_obj_compact<1024><<<1, 1024, 0, h->stream>>>(z, h->p.n, K, h->obj_idx, h->obj_cnt, h->obj_out);
  CK(cudaGetLastError());
  int rc;
  if (h->asz == 8) rc = launch_obj_rows<double, double>(h, z, K);
  else if (h->asz == 4) rc = launch_obj_rows<float, float>(h, z, K);
  else rc = launch_obj_rows<__nv_bfloat16, float>(h, z, K);
  if (rc != BICADMM_OK) return rc;
  k_obj_final<256><<<1, 256, 0, h->stream>>>(h->obj_part, h->obj_blocks, h->p.gamma, h->obj_out);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(out, h->obj_out, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  return BICADMM_OK;
}

int fill_info(bicadmm_ctx* h, bicadmm_info* info, bool objective = true, int inst = 0) {
  double obj = 0.0;
  if (objective) {
    const int rc = compute_objective(h, &obj, inst);
    if (rc != BICADMM_OK) return rc;
  }
  GlobalState g;
  const GlobalState* gsrc = h->gs + inst;
  const Resid* tbase = h->trace + static_cast<int64_t>(inst) * kTraceCap;
  CK(cudaMemcpyAsync(&g, gsrc, sizeof(g), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  std::memset(info, 0, sizeof(*info));
  info->iters = static_cast<int32_t>(g.iter);
  info->converged = h->converged ? 1 : 0;
  info->t = g.t;
  info->v = g.v;
  info->tau = g.tau;
  info->kernel_launches = h->launches;
  if (g.iter > 0) {
    Resid rec;
    CK(cudaMemcpyAsync(&rec, tbase + (g.iter - 1) % kTraceCap, sizeof(rec),
                       cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    info->p_r = rec.p_r; info->d_r = rec.d_r; info->b_r = rec.b_r; info->i_r = rec.i_r;
    info->p_rel = rec.p_rel; info->d_rel = rec.d_rel; info->b_rel = rec.b_rel;
    info->i_rel = rec.i_rel;
  }
  info->objective = obj;
  return check_device_error(h);
}

int validate(const bicadmm_params* p, std::string& why) {
  if (!p) { why = "params is NULL"; return BICADMM_ERR_ARG; }
  if (p->loss != BICADMM_LOSS_SQUARED && p->loss != BICADMM_LOSS_LOGISTIC && p->loss != BICADMM_LOSS_SQHINGE && p->loss != BICADMM_LOSS_SOFTMAX) { why = "unknown loss"; return BICADMM_ERR_ARG; }
  if (p->precision != BICADMM_PREC_FP64 && p->precision != BICADMM_PREC_FP32 && p->precision != BICADMM_PREC_BF16 && p->precision != BICADMM_PREC_TF32) { why = "unknown precision"; return BICADMM_ERR_ARG; }
  if (p->m < 1 || p->n < 1) { why = "m and n must be >= 1"; return BICADMM_ERR_ARG; }
  if (p->loss == BICADMM_LOSS_SOFTMAX ? (p->K < 2 || p->K > 16) : p->K != 1) { why = "K must be 2..16 for softmax and 1 otherwise"; return BICADMM_ERR_ARG; }
  if (p->N_shards < 1 || p->N_shards > p->m) { why = "need 1 <= N_shards <= m"; return BICADMM_ERR_ARG; }
  if (p->M_blocks < 1 || p->M_blocks > p->n) { why = "need 1 <= M_blocks <= n"; return BICADMM_ERR_ARG; }
  if (p->kappa < 1 || p->kappa > p->n * p->K) { why = "need 1 <= kappa <= n K"; return BICADMM_ERR_ARG; }
  if (!(p->gamma > 0) || !(p->rho_c > 0) || !(p->rho_b >= 0) || !(p->rho_l >= 0)) { why = "gamma, rho_c must be > 0 and rho_b, rho_l >= 0"; return BICADMM_ERR_ARG; }
  if (p->inner_iters < 1 || p->newton_iters < 1) { why = "inner_iters and newton_iters must be >= 1"; return BICADMM_ERR_ARG; }
  if (p->max_iters < 0 || p->check_every < 1) { why = "max_iters >= 0 and check_every >= 1 required"; return BICADMM_ERR_ARG; }
  if (p->n * p->K > kMaxN) { why = "n K > 32768 is not supported by this build"; return BICADMM_ERR_UNSUPPORTED; }
  if (p->pass_rows != 0 && p->pass_rows != 1 && p->pass_rows != 2 && p->pass_rows != 4 && p->pass_rows != 8 && p->pass_rows != 64 && p->pass_rows != 128) { why = "pass_rows must be 0, 1, 2, 4, 8, 64 or 128"; return BICADMM_ERR_ARG; }
  if (p->pass_stages < 0 || p->pass_stages > 8) { why = "pass_stages must be in [0, 8]"; return BICADMM_ERR_ARG; }
  return BICADMM_OK;
}

int build_geometry(bicadmm_ctx* h) {
  const bicadmm_params& p = h->p;
  h->N = p.N_shards;
  h->M = p.M_blocks;
  h->esz = p.precision == BICADMM_PREC_FP64 ? 8 : 4;
  h->asz = p.precision == BICADMM_PREC_FP64 ? 8 : (p.precision == BICADMM_PREC_BF16 ? 2 : 4);
  h->lda = round_up(p.n, 32);
  h->K = static_cast<int>(p.K);
  h->KC = h->K == 1 ? 1 : (h->K <= 4 ? 4 : (h->K <= 10 ? 10 : 16));
  h->ldx = h->lda * h->K;
  h->c0 = 1.0 / (h->N * p.gamma) + p.rho_c;
  // shards / blocks: contiguous, first (total mod parts) one longer
  h->shard_row0.assign(h->N + 1, 0);
  for (int i = 0; i < h->N; ++i) h->shard_row0[i + 1] = h->shard_row0[i] + p.m / h->N + (i < p.m % h->N ? 1 : 0);
  h->blk_col0.assign(h->M + 1, 0);
  h->blk_ldp.assign(h->M, 0);
  h->max_nj = 0;
  h->max_ldp = 0;
  for (int j = 0; j < h->M; ++j) {
    const int nj = static_cast<int>(p.n / h->M + (j < p.n % h->M ? 1 : 0));
    h->blk_col0[j + 1] = h->blk_col0[j] + nj;
    h->blk_ldp[j] = static_cast<int>(round_up(nj, 32));
    h->max_nj = std::max(h->max_nj, nj);
    h->max_ldp = std::max(h->max_ldp, h->blk_ldp[j]);
  }
  if (h->max_nj > 8192) return fail(h, BICADMM_ERR_UNSUPPORTED, "feature blocks wider than 8192 columns are not supported; raise M_blocks");
  if (h->K > 1 && static_cast<size_t>(h->max_ldp + 4) * h->KC * h->esz > 200 * 1024)
    return fail(h, BICADMM_ERR_UNSUPPORTED, "feature blocks too wide for K classes (x-update tile); raise M_blocks");
  h->G_off.assign(static_cast<size_t>(h->N) * h->M, 0);
  h->P_off.assign(static_cast<size_t>(h->N) * h->M, 0);
  int64_t go = 0, po = 0;
  for (int i = 0; i < h->N; ++i)
    for (int j = 0; j < h->M; ++j) {
      const int nj = h->blk_col0[j + 1] - h->blk_col0[j];
      h->G_off[i * h->M + j] = go;
      h->P_off[i * h->M + j] = po;
      go += static_cast<int64_t>(nj) * nj;
      po += static_cast<int64_t>(nj) * h->blk_ldp[j];
    }
  h->G_total = go;
  h->P_total = po;

  // A-pass panel geometry
  const size_t row_bytes = static_cast<size_t>(h->lda) * h->asz;
  int R = p.pass_rows;
  // BF16 multi-column rows of <= 2048 columns: tensor-core pass unless 8-row CUDA-core
  // panels are asked for; 128-row panels on pairs of SMs (k_fused_pass_tc2) when the row
  // has at least two 128-column slabs, 64-row panels on single SMs when asked for
  // (pass_rows 64) or the row is narrower.
  h->use_tc = h->K > 1 && p.precision == BICADMM_PREC_BF16 && h->lda <= 128 * kTcMaxSlabs &&
              (R == 0 || R == kTcRows || R == kTc2Rows);
  h->tc2 = h->use_tc && R != kTcRows && h->lda > 128;
  if ((R == kTcRows || R == kTc2Rows) && !h->use_tc)
    return fail(h, BICADMM_ERR_UNSUPPORTED, "64- and 128-row panels are the tensor-core pass (BF16, K > 1, n <= 2048)");
  if (R == kTc2Rows && !h->tc2)
    return fail(h, BICADMM_ERR_UNSUPPORTED, "128-row panels need rows of more than 128 columns");
  if (h->K > 1 && !h->use_tc) {
    // Softmax pass: one CTA per SM (register tiles), 8-row panels, up to 4 stages in the
    // single-CTA budget.
    if (R != 0 && R != kPassRowsK) return fail(h, BICADMM_ERR_UNSUPPORTED, "the softmax A pass uses 8-row panels (pass_rows 0 or 8)");
    R = kPassRowsK;
  }
  if (h->use_tc) R = h->tc2 ? kTc2Rows : kTcRows;
  // Auto (one class): the tallest panel (at most 8 rows) of at most 96 KB, so that two CTAs
  // fit an SM.  A panel of 32 KB or more gets one stage: the two CTAs of an SM alternate
  // between loading and computing, and a panel held in registers (FP32) has its stage reloaded
  // right after the forward; smaller panels get up to four stages within 64 KB.  Measured on
  // FP32 logistic passes over 3 GB of A: n = 2000, 8 rows x 1 stage 0.47 ms against 0.67
  // for 4 x 2; n = 5000, 4 x 1 0.49 ms against 0.58 for 2 x 2.
  if (R == 0) {
    R = 1;
    for (int cand : {8, 4, 2}) {
      if (cand * row_bytes <= 96 * 1024) { R = cand; break; }
    }
  }
  int S = h->use_tc ? kTcStages : p.pass_stages;
  if (S == 0 && h->K == 1) {
    const size_t panel = static_cast<size_t>(R) * row_bytes;
    S = panel >= 32 * 1024 ? 1 : static_cast<int>(std::min<size_t>(4, (64 * 1024) / panel));
    if (S < 1) S = 1;
  } else if (S == 0) {
    const size_t budget = 2 * R * row_bytes <= kPassCtaTarget ? kPassCtaTarget : kPassSmemBudget;
    S = static_cast<int>(std::min<size_t>(4, budget / (R * row_bytes)));
    if (S < 1) S = 1;
  }
  if (!h->use_tc && static_cast<size_t>(S) * R * row_bytes > kPassSmemBudget)
    return fail(h, BICADMM_ERR_UNSUPPORTED, "A-pass stages do not fit in shared memory (rows too wide)");
  h->R = R;
  h->S = S;
  const int ve = static_cast<int>(16 / h->asz);
  const int64_t nvec = h->lda / ve;
  h->VPT = h->use_tc ? 1 : (h->K == 1 ? pick_vpt(nvec) : pick_vpt_k(nvec, ve, h->KC, h->esz));
  if (h->VPT < 0) return fail(h, BICADMM_ERR_UNSUPPORTED, "rows too wide for the register-resident A-pass accumulators");
  if (h->use_tc) {
    h->pass_smem = h->tc2 ? fused_pass_tc2_smem(h->KC) : fused_pass_tc_smem();
    h->nslab = 2 * static_cast<int>((h->lda + kTcStageCols - 1) / kTcStageCols);  // even
  } else if (h->K > 1) {
    const int C = h->KC <= 4 ? 4 : 16;
    h->pass_smem = static_cast<size_t>(S) * R * row_bytes + S * sizeof(uint64_t) +
                   static_cast<size_t>(R) * (kPassThreads / 32 + 1) * C * h->esz + 16;
  } else {
    h->pass_smem = static_cast<size_t>(S) * R * row_bytes + S * sizeof(uint64_t) +
                   static_cast<size_t>(R) * (kPassThreads / 32 + 1) * h->esz + 16;
  }
  h->panel_start.assign(h->N + 1, 0);
  for (int i = 0; i < h->N; ++i) {
    const int64_t mi = h->shard_row0[i + 1] - h->shard_row0[i];
    h->panel_start[i + 1] = h->panel_start[i] + (mi + R - 1) / R;
  }
  h->P_panels = h->panel_start[h->N];
  int occ = 0;
  int rc;
  if (h->use_tc) {
    rc = launch_pass_tc(h, false, 1, &occ);
  } else if (h->K > 1) {
    switch (h->p.precision) {
      case BICADMM_PREC_FP64: rc = launch_pass_k<double, double>(h, false, 1, &occ); break;
      case BICADMM_PREC_FP32: rc = launch_pass_k<float, float>(h, false, 1, &occ); break;
      default: rc = launch_pass_k<__nv_bfloat16, float>(h, false, 1, &occ); break;
    }
  } else {
    switch (h->p.precision) {
      case BICADMM_PREC_FP64: rc = pass_occupancy<double, double>(h, &occ); break;
      case BICADMM_PREC_FP32: rc = pass_occupancy<float, float>(h, &occ); break;
      default: rc = pass_occupancy<__nv_bfloat16, float>(h, &occ); break;
    }
  }
  if (rc != BICADMM_OK) return rc;
  if (occ < 1) return fail(h, BICADMM_ERR_UNSUPPORTED, "A-pass variant cannot be resident on an SM");
  // One resident slot is kept for each consensus CTA that rides on the last pass (the pair
  // kernel: occ co-resident pairs, its at most two consensus CTAs taking one pair).
  const int64_t slots_total = h->tc2 ? static_cast<int64_t>(occ) - (tc2_cons_ctas(h->ninst) + 1) / 2
                                     : static_cast<int64_t>(occ) * h->num_sms - h->ninst;
  if (slots_total < 1) return fail(h, BICADMM_ERR_UNSUPPORTED, "A-pass needs at least two resident CTAs");
  // At least 4 panels per CTA: a shard's A'd partial sums are spread over one slot per CTA
  // that touches it, and every x-update right-hand side sums them (small problems had
  // ~60 slots per shard with one panel per CTA).
  h->G = static_cast<int>(std::min<int64_t>(slots_total, std::max<int64_t>(1, (h->P_panels + 3) / 4)));
  // slots: CTA c writes slot (c + shard) for every shard it touches
  h->slot_lo.assign(h->N, 0);
  h->slot_hi.assign(h->N, 0);
  auto owner = [&](int64_t panel) {
    // CTA c owns [c*P/G, (c+1)*P/G)
    int64_t c = panel * h->G / h->P_panels;
    while (c > 0 && c * h->P_panels / h->G > panel) --c;
    while ((c + 1) * h->P_panels / h->G <= panel) ++c;
    return static_cast<int>(c);
  };
  for (int i = 0; i < h->N; ++i) {
    h->slot_lo[i] = owner(h->panel_start[i]) + i;
    h->slot_hi[i] = owner(h->panel_start[i + 1] - 1) + i;
  }
  h->nslots = h->G + h->N;
  // CTAs per shard of k_dual (each loops over its columns): at most 32, so that a thread has
  // a few columns (their loads are latency-bound) and the last-CTA ticket stays short, and
  // no more than the GPU holds at once over all shards (a second wave of CTAs would start
  // only as the first one finishes)
  int dual_occ = 0;
  if (h->esz == 8)
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&dual_occ, k_dual<double, kDualThreads>, kDualThreads, 0));
  else
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&dual_occ, k_dual<float, kDualThreads>, kDualThreads, 0));
  const int64_t dual_wave = std::max<int64_t>(1, static_cast<int64_t>(dual_occ) * h->num_sms / h->N);
  h->dual_chunks = static_cast<int>(std::min<int64_t>(
      std::min<int64_t>(32, dual_wave), (h->ldx + kDualThreads - 1) / kDualThreads));
  return BICADMM_OK;
}

// Device bytes a handle allocates (including the polish buffers of one polished get_x),
// and the extra bytes its setup holds temporarily.
void handle_bytes(const bicadmm_ctx* h, int64_t* persistent, int64_t* setup_extra) {
  const int64_t m = h->p.m, lda = h->lda, ldx = h->ldx, N = h->N, kappa = h->p.kappa;
  const int64_t es = static_cast<int64_t>(h->esz), as = static_cast<int64_t>(h->asz);
  int64_t b = 0;
  b += m * lda * as + m * es + 2 * m * h->K * es;       // A, b, omega, nu
  b += static_cast<int64_t>(h->nslots) * ldx * es;      // slots
  b += N * ldx * es + h->P_total * es;                  // xlo, P
  b += static_cast<int64_t>(N) * h->nslab * kTcWBytes;  // packed W (tensor-core pass)
  b += 3 * N * ldx * 8 + 7 * ldx * 8;                   // x, u, r; z, s, w, tau_r, c, e, key
  if (h->K > 1) b += ldx * 4 + static_cast<int64_t>(h->ninst) * ((ldx + kPrepBlock - 1) / kPrepBlock + 1) * 4;  // entry lists
  b += static_cast<int64_t>(h->G) * 32 + N * h->dual_chunks * 16 + 4096 * 112 + 4096;
  // polish: supp, A_S, q, d1, d2, p, x_S, step, partials, H
  b += kappa * 8 + kappa * m * 8 + 4 * m * 8 + 2 * kappa * 8 + kPolishRowBlocks * 8 +
       static_cast<int64_t>(kPolishChunks) * kappa * 8 + (kPolishChunks + 1) * kappa * kappa * 8;
  if (h->K > 1)  // softmax polish: U (kappa x m) and q, p, d1, P (m x K)
    b += kappa * m * 8 + 4 * m * h->K * 8 + kappa * 12;
  if (persistent) *persistent = b;
  // two staging slots of the input, the Gram matrices and the factor inverse Y = L^-1
  if (setup_extra) *setup_extra = 2 * std::min<int64_t>(256ll << 20, m * lda * 8) + 2 * h->G_total * 8;
}

int allocate(bicadmm_ctx* h) {
  const int64_t m = h->p.m, lda = h->ldx, N = h->N;  // n-space arrays use the stride lda K
  const size_t es = h->esz;
  int rc;
#define AL(ptr, bytes) if ((rc = dev_alloc(h, &(ptr), (bytes))) != BICADMM_OK) return rc
  AL(h->A, static_cast<size_t>(m) * h->lda * h->asz);
  AL(h->b, m * es);
  AL(h->omega, m * h->K * es);
  AL(h->nu, m * h->K * es);
  AL(h->slots, static_cast<size_t>(h->nslots) * lda * es);
  AL(h->xlo, static_cast<size_t>(N) * lda * es);
  AL(h->Pm, static_cast<size_t>(h->P_total) * es);
  AL(h->x, N * lda * sizeof(double));
  AL(h->u, N * lda * sizeof(double));
  AL(h->r, N * lda * sizeof(double));
  AL(h->z, lda * sizeof(double));
  AL(h->s, lda * sizeof(double));
  AL(h->w, lda * sizeof(double));
  AL(h->tau_r, lda * sizeof(double));
  AL(h->c_arr, lda * sizeof(double));
  AL(h->e_arr, lda * sizeof(double));
  AL(h->key, lda * sizeof(uint64_t));
  if (h->use_tc) AL(h->wpk, static_cast<size_t>(N) * h->nslab * kTcWBytes);
  AL(h->cta_stats, static_cast<size_t>(h->G) * 4 * sizeof(double));
  AL(h->dual_part, static_cast<size_t>(N) * h->dual_chunks * 2 * sizeof(double));
  AL(h->d_shard_row0, (N + 1) * sizeof(int64_t));
  AL(h->d_panel_start, (N + 1) * sizeof(int64_t));
  AL(h->d_P_off, h->P_off.size() * sizeof(int64_t));
  AL(h->d_G_off, h->G_off.size() * sizeof(int64_t));
  AL(h->d_blk_col0, h->blk_col0.size() * sizeof(int));
  AL(h->d_blk_ldp, h->blk_ldp.size() * sizeof(int));
  AL(h->d_slot_lo, N * sizeof(int));
  AL(h->d_slot_hi, N * sizeof(int));
  AL(h->gs, static_cast<size_t>(h->ninst) * sizeof(GlobalState));
  AL(h->trace, static_cast<size_t>(h->ninst) * kTraceCap * sizeof(Resid));
  if (h->path) {
    AL(h->z_cm, h->p.n * h->K * sizeof(double));
    AL(h->s_cm, h->p.n * h->K * sizeof(double));
    AL(h->d_kappas, h->ninst * sizeof(int64_t));
  }
  AL(h->d_err, sizeof(int));
  if (h->K > 1) {
    const int64_t n_inst = h->path ? h->p.n : h->p.n * h->K;
    h->u_nb = static_cast<int>((n_inst + kPrepBlock - 1) / kPrepBlock);
    AL(h->u_idx, static_cast<size_t>(h->p.n) * h->K * sizeof(int));
    AL(h->u_cnt, static_cast<size_t>(h->ninst) * h->u_nb * sizeof(int));
  }
  h->obj_blocks = std::max(1, h->num_sms) * 4;
  AL(h->obj_idx, h->p.n * sizeof(int));
  AL(h->obj_cnt, sizeof(int));
  AL(h->obj_part, static_cast<size_t>(h->obj_blocks) * sizeof(double));
  AL(h->obj_out, 2 * sizeof(double));
#undef AL
  auto up = [&](void* dst, const void* src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, h->stream);
  };
  CK(up(h->d_shard_row0, h->shard_row0.data(), (N + 1) * sizeof(int64_t)));
  CK(up(h->d_panel_start, h->panel_start.data(), (N + 1) * sizeof(int64_t)));
  CK(up(h->d_P_off, h->P_off.data(), h->P_off.size() * sizeof(int64_t)));
  CK(up(h->d_G_off, h->G_off.data(), h->G_off.size() * sizeof(int64_t)));
  CK(up(h->d_blk_col0, h->blk_col0.data(), h->blk_col0.size() * sizeof(int)));
  CK(up(h->d_blk_ldp, h->blk_ldp.data(), h->blk_ldp.size() * sizeof(int)));
  CK(up(h->d_slot_lo, h->slot_lo.data(), N * sizeof(int)));
  CK(up(h->d_slot_hi, h->slot_hi.data(), N * sizeof(int)));
  if (h->path) CK(up(h->d_kappas, h->kappas.data(), h->ninst * sizeof(int64_t)));
  CK(cudaStreamSynchronize(h->stream));
  return BICADMM_OK;
}

int reset_state(bicadmm_ctx* h) {
  const int64_t m = h->p.m, lda = h->ldx, N = h->N;
  const size_t es = h->esz;
  CK(cudaMemsetAsync(h->omega, 0, m * h->K * es, h->stream));
  CK(cudaMemsetAsync(h->nu, 0, m * h->K * es, h->stream));
  CK(cudaMemsetAsync(h->slots, 0, static_cast<size_t>(h->nslots) * lda * es, h->stream));
  CK(cudaMemsetAsync(h->xlo, 0, static_cast<size_t>(N) * lda * es, h->stream));
  CK(cudaMemsetAsync(h->x, 0, N * lda * sizeof(double), h->stream));
  if (h->wpk) CK(cudaMemsetAsync(h->wpk, 0, static_cast<size_t>(N) * h->nslab * kTcWBytes, h->stream));
  CK(cudaMemsetAsync(h->u, 0, N * lda * sizeof(double), h->stream));
  CK(cudaMemsetAsync(h->r, 0, N * lda * sizeof(double), h->stream));
  CK(cudaMemsetAsync(h->z, 0, lda * sizeof(double), h->stream));
  CK(cudaMemsetAsync(h->s, 0, lda * sizeof(double), h->stream));
  CK(cudaMemsetAsync(h->w, 0, lda * sizeof(double), h->stream));
  CK(cudaMemsetAsync(h->cta_stats, 0, static_cast<size_t>(h->G) * 4 * sizeof(double), h->stream));
  CK(cudaMemsetAsync(h->gs, 0, static_cast<size_t>(h->ninst) * sizeof(GlobalState), h->stream));
  CK(cudaMemsetAsync(h->trace, 0, static_cast<size_t>(h->ninst) * kTraceCap * sizeof(Resid), h->stream));
  if (h->path) {
    CK(cudaMemsetAsync(h->z_cm, 0, h->p.n * h->K * sizeof(double), h->stream));
    CK(cudaMemsetAsync(h->s_cm, 0, h->p.n * h->K * sizeof(double), h->stream));
  }
  CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream));
  h->iters_done = 0;
  h->converged = false;
  return BICADMM_OK;
}

// Copy rows [0, m) of a caller matrix (host or device, dtype) into the padded device layout.
template <typename TOUT>
int load_matrix(bicadmm_ctx* h, const void* src, int dtype, int64_t lda_src, int on_device,
                TOUT* dst, int64_t rows, int64_t cols, int64_t lda_dst) {
  const size_t in_es = dtype == BICADMM_DTYPE_F64 ? 8 : (dtype == BICADMM_DTYPE_BF16 ? 2 : 4);
  auto convert = [&](const void* s, TOUT* d, int64_t nr) -> int {
    const int64_t total = nr * lda_dst;
    const unsigned grid = static_cast<unsigned>(std::min<int64_t>((total + 255) / 256, 65535));
    if (dtype == BICADMM_DTYPE_F64)
      k_convert_rows<double, TOUT><<<grid, 256, 0, h->stream>>>(static_cast<const double*>(s), lda_src, d, lda_dst, nr, cols);
    else if (dtype == BICADMM_DTYPE_BF16)
      k_convert_rows<__nv_bfloat16, TOUT><<<grid, 256, 0, h->stream>>>(static_cast<const __nv_bfloat16*>(s), lda_src, d, lda_dst, nr, cols);
    else
      k_convert_rows<float, TOUT><<<grid, 256, 0, h->stream>>>(static_cast<const float*>(s), lda_src, d, lda_dst, nr, cols);
    CK(cudaGetLastError());
    h->launches += 1;
    return BICADMM_OK;
  };
  if (on_device) return convert(src, dst, rows);
  // Host source: stream chunks through a device staging buffer (at most 256 MB).
  const int64_t row_in = lda_src * static_cast<int64_t>(in_es);
  int64_t chunk = std::max<int64_t>(1, (256ll << 20) / std::max<int64_t>(row_in, 1));
  chunk = std::min(chunk, rows);
  void* stage = nullptr;
  cudaError_t e = cudaMalloc(&stage, static_cast<size_t>(chunk) * row_in);
  if (e != cudaSuccess) { cudaGetLastError(); return fail(h, BICADMM_ERR_OOM, "staging buffer allocation failed"); }
  int rc = BICADMM_OK;
  for (int64_t r0 = 0; r0 < rows && rc == BICADMM_OK; r0 += chunk) {
    const int64_t nr = std::min(chunk, rows - r0);
    // the last row may be shorter than lda_src: copy exactly (nr-1)*lda_src + cols elements
    const size_t bytes = (static_cast<size_t>(nr - 1) * lda_src + cols) * in_es;
    e = cudaMemcpyAsync(stage, static_cast<const char*>(src) + r0 * row_in, bytes,
                        cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) { rc = fail(h, BICADMM_ERR_CUDA, std::string("H2D copy: ") + cudaGetErrorString(e)); break; }
    rc = convert(stage, dst + r0 * lda_dst, nr);
    if (rc == BICADMM_OK) {
      e = cudaStreamSynchronize(h->stream);
      if (e != cudaSuccess) rc = fail(h, BICADMM_ERR_CUDA, std::string("sync: ") + cudaGetErrorString(e));
    }
  }
  cudaStreamSynchronize(h->stream);
  cudaFree(stage);
  return rc;
}

// Softmax: every b_r must be an integral class index in [0, K).
template <typename TM>
int check_labels(bicadmm_ctx* h) {
  if (h->K == 1 || h->path) return BICADMM_OK;
  const unsigned grid = static_cast<unsigned>(std::min<int64_t>((h->p.m + 255) / 256, 4096));
  k_check_labels<TM><<<grid, 256, 0, h->stream>>>(static_cast<const TM*>(h->b), h->p.m, h->K, h->d_err);
  CK(cudaGetLastError());
  h->launches += 1;
  return check_device_error(h);
}

// load_shard (optional): enqueues the arrival of shard i's rows of A on the handle's stream;
// the Gram matrices are then formed shard by shard right behind it, so they overlap the
// transfers of later shards.
template <typename TA, typename TM>
int build_factors(bicadmm_ctx* h, const std::function<int(int)>* load_shard = nullptr) {
  double* G = nullptr;
  cudaError_t e = cudaMalloc(&G, std::max<int64_t>(h->G_total, 1) * sizeof(double));
  if (e != cudaSuccess) { cudaGetLastError(); return fail(h, BICADMM_ERR_OOM, "Gram buffer allocation failed"); }

  int rc = BICADMM_OK;
  Gram32Item* d_items32 = nullptr;
  double* gscratch = nullptr;  // the split Gram tiles' partials and tickets
  int* gtick = nullptr;

  // Blocked factorisation when an NB-column panel of the widest block fits in shared memory:
  // Cholesky, Y = L^-1 by columns, P = Y'Y by tiles (n^3/2 FMAs per block); otherwise the
  // column-by-column kernels (Cholesky, then both triangular solves per column of P).
  int nb_panel = 0;
  for (int cand : {32, 16, 8})
    if (static_cast<size_t>(cand) * (h->max_nj + 1) * sizeof(double) <= (200u << 10)) { nb_panel = cand; break; }
  double* YT = nullptr;
  int* tick = nullptr;  // per block: tickets of the GPU-wide Cholesky's panel CTAs
  if (nb_panel > 0) {
    e = cudaMalloc(&YT, std::max<int64_t>(h->G_total, 1) * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&tick, static_cast<size_t>(h->N) * h->M * sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(tick, 0, static_cast<size_t>(h->N) * h->M * sizeof(int), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (YT) cudaFree(YT);
      if (tick) cudaFree(tick);
      YT = nullptr;
      tick = nullptr;
      nb_panel = 0;
      e = cudaSuccess;
    }
  }
  // P = Y'Y items (the same for every shard): long tile sums cut into parts of kspan columns,
  // kspan grown until every block's partial tiles fit its region of G (nj x nj doubles)
  std::vector<YtyItem> yitems;
  int yspan = 0, ytiles = 0;
  for (int U = std::max(4, (h->max_nj + 63) / 64 / 3);; ++U) {
    yitems.clear();
    yspan = 64 * U;
    ytiles = 0;
    bool fits = true;
    for (int j = 0; j < h->M; ++j) {
      const int nj = h->blk_col0[j + 1] - h->blk_col0[j], T = (nj + 63) / 64;
      int scr = 0;
      for (int ti = 0; ti < T; ++ti)
        for (int tj = ti; tj < T; ++tj) {
          const int len = nj - 64 * tj, np = (len + yspan - 1) / yspan;
          for (int pt = 0; pt < np; ++pt) yitems.push_back(YtyItem{j, ti, tj, pt, np, ytiles, scr, 0});
          if (np > 1) scr += np;
          ++ytiles;
        }
      if (static_cast<int64_t>(scr) * 64 * 64 > static_cast<int64_t>(nj) * nj) fits = false;
    }
    if (fits) break;
  }
  YtyItem* d_yitems = nullptr;
  int* ytick = nullptr;
  if (nb_panel > 0) {
    e = cudaMalloc(&d_yitems, yitems.size() * sizeof(YtyItem));
    if (e == cudaSuccess) e = cudaMalloc(&ytick, static_cast<size_t>(h->N) * ytiles * sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(ytick, 0, static_cast<size_t>(h->N) * ytiles * sizeof(int), h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_yitems, yitems.data(), yitems.size() * sizeof(YtyItem), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaFree(G);
      if (YT) cudaFree(YT);
      if (tick) cudaFree(tick);
      if (d_yitems) cudaFree(d_yitems);
      if (ytick) cudaFree(ytick);
      return fail(h, BICADMM_ERR_OOM, "factor tables allocation failed");
    }
  }
  const size_t chol_sm = static_cast<size_t>(nb_panel) * (h->max_nj + 1) * sizeof(double);
  const int inv_warps = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(8, (200 << 10) / (8 * h->max_nj))));
  const size_t inv_sm = static_cast<size_t>(inv_warps) * h->max_nj * sizeof(double);
  if (nb_panel > 0) {
    if (nb_panel == 32) e = cudaFuncSetAttribute(k_chol_blk<kCholThreads, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(chol_sm));
    else if (nb_panel == 16) e = cudaFuncSetAttribute(k_chol_blk<kCholThreads, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(chol_sm));
    else e = cudaFuncSetAttribute(k_chol_blk<kCholThreads, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(chol_sm));
    if (e == cudaSuccess && inv_sm > 48 * 1024)
      e = cudaFuncSetAttribute(k_inv_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(inv_sm));
  }
  // The blocked factorisation of shards [s0, s0 + ns) on stream st: every kernel finds its
  // block through G_off / P_off, so the shard range is an offset of those tables.
  auto factor_shards = [&](int s0, int ns, cudaStream_t st) -> cudaError_t {
    const int64_t* goff = h->d_G_off + static_cast<int64_t>(s0) * h->M;
    const int64_t* poff = h->d_P_off + static_cast<int64_t>(s0) * h->M;
    const unsigned nb = static_cast<unsigned>(ns * h->M);
    // Blocks of at least kCholSplitCols columns: the Cholesky over the whole GPU (scale, then
    // per NB-column panel one panel launch, a CTA per block, and one trailing-update launch, a
    // CTA per 64 x 64 tile per block); narrower blocks: one CTA per block for the whole
    // factorisation (fewer launches; the same arithmetic)
    if (h->max_nj < kCholSplitCols) {
      if (nb_panel == 32) k_chol_blk<kCholThreads, 32><<<nb, kCholThreads, chol_sm, st>>>(G, goff, h->d_blk_col0, h->M, h->p.rho_l, h->c0, h->d_err);
      else if (nb_panel == 16) k_chol_blk<kCholThreads, 16><<<nb, kCholThreads, chol_sm, st>>>(G, goff, h->d_blk_col0, h->M, h->p.rho_l, h->c0, h->d_err);
      else k_chol_blk<kCholThreads, 8><<<nb, kCholThreads, chol_sm, st>>>(G, goff, h->d_blk_col0, h->M, h->p.rho_l, h->c0, h->d_err);
      h->launches += 1;
    } else {
    const unsigned sc_chunks = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(64,
        (static_cast<int64_t>(h->max_nj) * h->max_nj + 256 * 64 - 1) / (256 * 64))));
    k_chol_scale<kCholThreads><<<dim3(nb, sc_chunks), kCholThreads, 0, st>>>(G, goff, h->d_blk_col0, h->M, h->p.rho_l, h->c0);
    h->launches += 1;
    for (int kb = 0; kb < h->max_nj; kb += nb_panel) {
      const int below = std::max(0, h->max_nj - kb - nb_panel);
      const dim3 pg(nb, static_cast<unsigned>(std::max(1, (below + kCholChunk - 1) / kCholChunk)));
      int* tk = tick + static_cast<int64_t>(s0) * h->M;
      if (nb_panel == 32) k_chol_panel<kCholThreads, 32, kCholChunk><<<pg, kCholThreads, 0, st>>>(G, goff, h->d_blk_col0, h->M, kb, h->d_err, tk);
      else if (nb_panel == 16) k_chol_panel<kCholThreads, 16, kCholChunk><<<pg, kCholThreads, 0, st>>>(G, goff, h->d_blk_col0, h->M, kb, h->d_err, tk);
      else k_chol_panel<kCholThreads, 8, kCholChunk><<<pg, kCholThreads, 0, st>>>(G, goff, h->d_blk_col0, h->M, kb, h->d_err, tk);
      h->launches += 1;
      const int nt = h->max_nj - kb - nb_panel;
      if (nt > 0) {
        const int Tt = (nt + 63) / 64;
        const dim3 ug(static_cast<unsigned>(Tt * (Tt + 1) / 2), nb);
        if (nb_panel == 32) k_chol_update<kCholThreads, 32><<<ug, kCholThreads, 0, st>>>(G, goff, h->d_blk_col0, h->M, kb);
        else if (nb_panel == 16) k_chol_update<kCholThreads, 16><<<ug, kCholThreads, 0, st>>>(G, goff, h->d_blk_col0, h->M, kb);
        else k_chol_update<kCholThreads, 8><<<ug, kCholThreads, 0, st>>>(G, goff, h->d_blk_col0, h->M, kb);
        h->launches += 1;
      }
    }
    }
    cudaError_t ee = cudaGetLastError();
    if (ee != cudaSuccess) return ee;
    k_inv_fwd<<<dim3(nb, (h->max_nj + inv_warps - 1) / inv_warps), 32 * inv_warps, inv_sm, st>>>(G, goff, h->d_blk_col0, h->M, YT);
    if ((ee = cudaGetLastError()) != cudaSuccess) return ee;
    k_yty<TM><<<dim3(static_cast<unsigned>(yitems.size()), 1, ns), 256, 0, st>>>(
        YT, goff, h->d_blk_col0, h->d_blk_ldp, h->M, static_cast<TM*>(h->Pm), poff, d_yitems, yspan, G,
        ytick + static_cast<int64_t>(s0) * ytiles, ytiles);
    h->launches += 2;
    return cudaGetLastError();
  };
  // With the host pipeline (shards arriving one by one), each shard is factorised as soon as
  // its Gram matrices are formed, on its own side stream (up to 16, then round robin), so the
  // FP64 factorisation (a block's Cholesky is one CTA at one SM's FP64 rate, about 17 ms for
  // 625 columns) overlaps the copies of later shards and only the last shard's follows them.
  constexpr int kFactorStreams = 16;
  const bool per_shard = load_shard != nullptr && nb_panel > 0 && h->N > 1;
  cudaStream_t fst[kFactorStreams] = {};
  std::vector<cudaEvent_t> fev;
  const int nfs = per_shard ? std::min(kFactorStreams, h->N) : 0;
  for (int q = 0; q < nfs && e == cudaSuccess; ++q) e = cudaStreamCreateWithFlags(&fst[q], cudaStreamNonBlocking);
  auto after_gram = [&](int i) -> cudaError_t {
    if (!per_shard) return cudaSuccess;
    cudaEvent_t ev;
    cudaError_t ee = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (ee != cudaSuccess) return ee;
    fev.push_back(ev);
    if ((ee = cudaEventRecord(ev, h->stream)) != cudaSuccess) return ee;
    cudaStream_t st = fst[i % nfs];
    if ((ee = cudaStreamWaitEvent(st, ev, 0)) != cudaSuccess) return ee;
    return factor_shards(i, 1, st);
  };

  if constexpr (!std::is_same<TA, double>::value) {
    // tensor cores, kind::tf32 (gram_tf32.cuh): (shard, block, 128-column strip, 128-column
    // chunk) items over each block's own columns, chunks at or right of the strip.  FP32
    // storage splits A into TF32 hi + lo (three products); TF32 storage (rounded first) and
    // BF16 storage (exact in TF32) take one product.
    // A launch with few tiles splits each tile's rows into parts (at most
    // 8, at least four 32-row stages each), a CTA per part: the softmax shape's four
    // 500-column blocks give 40 tiles per shard, and one CTA per tile walking all 15625 rows
    // made each shard's Gram matrices 1.9 ms on the setup stream, longer than its copy.
    int tiles_shard = 0;
    for (int j = 0; j < h->M; ++j) {
      const int t = (h->blk_col0[j + 1] - h->blk_col0[j] + 127) / 128;
      tiles_shard += t * (t + 1) / 2;
    }
    const int64_t tiles_launch = static_cast<int64_t>(tiles_shard) * (load_shard ? 1 : h->N);
    int64_t min_rows = h->p.m;
    for (int i = 0; i < h->N; ++i) min_rows = std::min<int64_t>(min_rows, h->shard_row0[i + 1] - h->shard_row0[i]);
    // (only below half an SM count: the partials cost scratch traffic, and 120 tiles of the
    // 200000 x 5000 shards already kept the Gram under the copy time)
    int nparts = tiles_launch * 2 >= h->num_sms ? 1 :
        static_cast<int>(std::min<int64_t>(8, (2 * h->num_sms + tiles_launch - 1) / std::max<int64_t>(tiles_launch, 1)));
    nparts = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(nparts, min_rows / (4 * kG32StageRows))));
    std::vector<Gram32Item> items;
    std::vector<size_t> first(h->N + 1, 0);  // items of shard i: [first[i], first[i + 1])
    for (int i = 0; i < h->N; ++i) {
      first[i] = items.size();
      int g = load_shard ? 0 : i * tiles_shard;  // tile index within its launch
      for (int j = 0; j < h->M; ++j) {
        const int nj = h->blk_col0[j + 1] - h->blk_col0[j];
        for (int a = 0; a < (nj + 127) / 128; ++a)
          for (int bq = a; bq < (nj + 127) / 128; ++bq, ++g)
            for (int pt = 0; pt < nparts; ++pt) items.push_back(Gram32Item{i, j, a, bq, pt, nparts, g});
      }
    }
    first[h->N] = items.size();
    if (nparts > 1) {
      e = cudaMalloc(&gscratch, static_cast<size_t>(tiles_launch) * nparts * 128 * 128 * sizeof(double));
      if (e == cudaSuccess) e = cudaMalloc(&gtick, static_cast<size_t>(tiles_launch) * sizeof(int));
      if (e == cudaSuccess) e = cudaMemsetAsync(gtick, 0, static_cast<size_t>(tiles_launch) * sizeof(int), h->stream);
    }
    constexpr bool kBf16 = std::is_same<TA, __nv_bfloat16>::value;
    const int terms = (kBf16 || h->tf32) ? 1 : 3;
    e = cudaMalloc(&d_items32, std::max<size_t>(items.size(), 1) * sizeof(Gram32Item));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_items32, items.data(), items.size() * sizeof(Gram32Item), cudaMemcpyHostToDevice, h->stream);
    const size_t sm = gram_tf32_smem(128, terms);
    if (e == cudaSuccess)
      e = terms == 3 ? cudaFuncSetAttribute(k_gram_tf32<3, TA>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm))
                     : cudaFuncSetAttribute(k_gram_tf32<1, TA>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
    // one launch for all shards, or one per shard after its rows have arrived (TF32 storage:
    // the rows are rounded first)
    for (int i = 0; e == cudaSuccess && rc == BICADMM_OK && i < (load_shard ? h->N : 1); ++i) {
      const size_t i0 = load_shard ? first[i] : 0, i1 = load_shard ? first[i + 1] : items.size();
      if (load_shard) rc = (*load_shard)(i);
      if constexpr (!kBf16) {
        if (rc == BICADMM_OK && h->tf32) {
          const int64_t r0 = load_shard ? h->shard_row0[i] : 0, r1 = load_shard ? h->shard_row0[i + 1] : h->p.m;
          const unsigned grid = static_cast<unsigned>(std::min<int64_t>(((r1 - r0) * h->lda + 255) / 256, 8192));
          k_round_tf32<<<grid, 256, 0, h->stream>>>(reinterpret_cast<float*>(h->A), h->lda, r0, r1);
          e = cudaGetLastError();
          h->launches += 1;
        }
      }
      if (e == cudaSuccess && rc == BICADMM_OK && i1 > i0) {
        const unsigned grid = static_cast<unsigned>(i1 - i0);
        const TA* Ap = static_cast<const TA*>(h->A);
        if (terms == 3)
          k_gram_tf32<3, TA><<<grid, kG32Threads, sm, h->stream>>>(Ap, h->lda, d_items32 + i0, h->d_shard_row0,
              h->d_blk_col0, G, h->d_G_off, h->M, gscratch, gtick, h->d_err, kWaitLimitCycles);
        else
          k_gram_tf32<1, TA><<<grid, kG32Threads, sm, h->stream>>>(Ap, h->lda, d_items32 + i0, h->d_shard_row0,
              h->d_blk_col0, G, h->d_G_off, h->M, gscratch, gtick, h->d_err, kWaitLimitCycles);
        e = cudaGetLastError();
        h->launches += 1;
      }
      if (e == cudaSuccess && rc == BICADMM_OK && load_shard) e = after_gram(i);
    }
  } else {
    const int T = (h->max_nj + 63) / 64;
    for (int i = 0; e == cudaSuccess && rc == BICADMM_OK && i < (load_shard ? h->N : 1); ++i) {
      if (load_shard && (rc = (*load_shard)(i)) != BICADMM_OK) break;
      const dim3 ggrid(T * (T + 1) / 2, h->M, load_shard ? 1 : h->N);
      k_gram<TA, TM><<<ggrid, 256, 0, h->stream>>>(static_cast<const TA*>(h->A), h->lda, h->d_shard_row0,
                                                   h->d_blk_col0, G, h->d_G_off, h->M, load_shard ? i : 0);
      e = cudaGetLastError();
      h->launches += 1;
      if (e == cudaSuccess && load_shard) e = after_gram(i);
    }
  }
  if (rc != BICADMM_OK) {
    cudaStreamSynchronize(h->stream);
    for (cudaStream_t st : fst)
      if (st) { cudaStreamSynchronize(st); cudaStreamDestroy(st); }
    for (cudaEvent_t ev : fev) cudaEventDestroy(ev);
    cudaFree(G);
    if (YT) cudaFree(YT);
    if (tick) cudaFree(tick);
    if (d_yitems) cudaFree(d_yitems);
    if (ytick) cudaFree(ytick);
    if (d_items32) cudaFree(d_items32);
    if (gscratch) cudaFree(gscratch);
    if (gtick) cudaFree(gtick);
    return rc;
  }
  if (per_shard) {
    // the handle's stream waits for every shard's factorisation
    for (int q = 0; q < nfs && e == cudaSuccess; ++q) {
      cudaEvent_t ev;
      e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e != cudaSuccess) break;
      fev.push_back(ev);
      if ((e = cudaEventRecord(ev, fst[q])) == cudaSuccess) e = cudaStreamWaitEvent(h->stream, ev, 0);
    }
  } else if (e == cudaSuccess && nb_panel > 0) {
    e = factor_shards(0, h->N, h->stream);
  } else {
    if (e == cudaSuccess) {
      auto kc = k_chol<kCholThreads>;
      const size_t sm = static_cast<size_t>(h->max_nj) * sizeof(double);
      if (sm > 48 * 1024) e = cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
      if (e == cudaSuccess) {
        kc<<<h->N * h->M, kCholThreads, sm, h->stream>>>(G, h->d_G_off, h->d_blk_col0, h->M,
                                                      h->p.rho_l, h->c0, h->d_err);
        h->launches += 1;
        e = cudaGetLastError();
      }
    }
    if (e == cudaSuccess) {
      // one warp per column; as many warps as fit 200 KB of column vectors (at most 8)
      const int warps = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(8, (200 << 10) / (8 * h->max_nj))));
      const size_t sm = static_cast<size_t>(warps) * h->max_nj * sizeof(double);
      auto ki = k_inv_cols<TM>;
      if (sm > 48 * 1024) e = cudaFuncSetAttribute(ki, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(sm));
      if (e == cudaSuccess) {
        const dim3 grid(h->N * h->M, (h->max_nj + warps - 1) / warps);
        ki<<<grid, 32 * warps, sm, h->stream>>>(G, h->d_G_off, h->d_blk_col0, h->d_blk_ldp, h->M,
                                                static_cast<TM*>(h->Pm), h->d_P_off);
        h->launches += 1;
        e = cudaGetLastError();
      }
    }
  }
  if (e != cudaSuccess) rc = fail(h, BICADMM_ERR_CUDA, std::string("factor kernels: ") + cudaGetErrorString(e));
  cudaError_t e2 = cudaStreamSynchronize(h->stream);
  if (rc == BICADMM_OK && e2 != cudaSuccess) rc = fail(h, BICADMM_ERR_CUDA, std::string("factor sync: ") + cudaGetErrorString(e2));
  for (cudaStream_t st : fst)
    if (st) { cudaStreamSynchronize(st); cudaStreamDestroy(st); }
  for (cudaEvent_t ev : fev) cudaEventDestroy(ev);
  cudaFree(G);
  if (YT) cudaFree(YT);
  if (tick) cudaFree(tick);
  if (d_yitems) cudaFree(d_yitems);
  if (ytick) cudaFree(ytick);
  if (d_items32) cudaFree(d_items32);
  if (gscratch) cudaFree(gscratch);
  if (gtick) cudaFree(gtick);
  if (rc != BICADMM_OK) return rc;
  return check_device_error(h);
}

// ---------------------------------------------------------------- support and polish

int compute_support(bicadmm_ctx* h) {
  if (!h->supp) {
    int rc = dev_alloc(h, &h->supp, h->p.kappa * sizeof(int64_t));
    if (rc != BICADMM_OK) return rc;
  }
  k_support<1024, 1><<<1, 1024, 0, h->stream>>>(h->z, h->key, h->p.n * h->K, h->p.kappa, h->supp);
  CK(cudaGetLastError());
  h->launches += 1;
  return BICADMM_OK;
}

template <typename TA, typename TM>
int run_polish(bicadmm_ctx* h, std::vector<double>& xs_out) {
  const int64_t m = h->p.m;
  const int kappa = static_cast<int>(h->p.kappa);
  const double gamma = h->p.gamma;
  const int nblk = static_cast<int>(std::min<int64_t>(kPolishRowBlocks, (m + 255) / 256));
  const int nch = static_cast<int>(std::min<int64_t>(kPolishChunks, (m + 255) / 256));
  const int64_t chunk = (m + nch - 1) / nch;
  if (!h->polish_ready) {
    int rc;
#define AL(ptr, bytes) if ((rc = dev_alloc(h, &(ptr), (bytes))) != BICADMM_OK) return rc
    AL(h->AS, static_cast<size_t>(kappa) * m * sizeof(double));
    AL(h->pq, m * sizeof(double));
    AL(h->pd1, m * sizeof(double));
    AL(h->pd2, m * sizeof(double));
    AL(h->pp, m * sizeof(double));
    AL(h->pxs, kappa * sizeof(double));
    AL(h->pstep, kappa * sizeof(double));
    AL(h->pfpart, nblk * sizeof(double));
    AL(h->pgpart, static_cast<size_t>(nch) * kappa * sizeof(double));
    AL(h->pHpart, static_cast<size_t>(nch) * kappa * kappa * sizeof(double));
    AL(h->pH, static_cast<size_t>(kappa) * kappa * sizeof(double));
    AL(h->pflag, sizeof(int));
#undef AL
    h->polish_ready = true;
  }
  int rc = compute_support(h);
  if (rc != BICADMM_OK) return rc;
  const dim3 ggrid(static_cast<unsigned>(std::min<int64_t>((m + 255) / 256, 1024)), kappa);
  k_gather_support<TA><<<ggrid, 256, 0, h->stream>>>(static_cast<const TA*>(h->A), h->lda, h->supp, m, h->AS);
  CK(cudaGetLastError());
  h->launches += 1;
  std::vector<double> xs(kappa, 0.0), step(kappa), fpart(nblk);
  CK(cudaMemsetAsync(h->pxs, 0, kappa * sizeof(double), h->stream));
  const int T = (kappa + 31) / 32;
  const size_t ksm = kappa * sizeof(double);
  auto objective = [&](double alpha, double* out) -> int {
    k_polish_rows<TM, 256><<<nblk, 256, ksm, h->stream>>>(h->AS, h->pxs, kappa, m,
        static_cast<const TM*>(h->b), h->p.loss, h->pq, h->pd1, h->pd2, h->pp, alpha, h->pfpart);
    CK(cudaGetLastError());
    h->launches += 1;
    CK(cudaMemcpyAsync(fpart.data(), h->pfpart, nblk * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    double f = 0.0;
    for (double v : fpart) f += v;
    *out = f;
    return BICADMM_OK;
  };
  for (int it = 0; it < 100; ++it) {
    double f0;
    if ((rc = objective(0.0, &f0)) != BICADMM_OK) return rc;  // also fills q, l', l''
    double xx = 0.0;
    for (double v : xs) xx += v * v;
    f0 += xx / (2.0 * gamma);
    k_polish_grad<256><<<dim3(nch, kappa), 256, 0, h->stream>>>(h->AS, h->pd1, kappa, m, chunk, h->pgpart);
    k_polish_hess<<<dim3(T * (T + 1) / 2, nch), 256, 0, h->stream>>>(h->AS, h->pd2, kappa, m, chunk, h->pHpart);
    k_polish_solve<256><<<1, 256, 2 * ksm, h->stream>>>(h->pHpart, h->pgpart, nch, h->pxs, kappa, gamma,
                                                        h->pH, h->pstep, h->pflag);
    k_polish_dir<256><<<nblk, 256, ksm, h->stream>>>(h->AS, h->pstep, kappa, m, h->pp);
    CK(cudaGetLastError());
    h->launches += 4;
    int flag = 0;
    CK(cudaMemcpyAsync(step.data(), h->pstep, kappa * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&flag, h->pflag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (flag) return fail(h, BICADMM_ERR_NUMERIC, "polish: restricted Hessian is not positive definite");
    double alpha = 1.0;
    for (;;) {
      double ft;
      if ((rc = objective(alpha, &ft)) != BICADMM_OK) return rc;
      double x2 = 0.0;
      for (int k = 0; k < kappa; ++k) {
        const double v = xs[k] - alpha * step[k];
        x2 += v * v;
      }
      ft += x2 / (2.0 * gamma);
      if (!(ft > f0 + 1e-16 * std::fabs(f0)) || !(alpha > 1e-12)) break;
      alpha *= 0.5;
    }
    double sn = 0.0, xn = 0.0;
    for (int k = 0; k < kappa; ++k) {
      xs[k] -= alpha * step[k];
      sn += (alpha * step[k]) * (alpha * step[k]);
      xn += xs[k] * xs[k];
    }
    CK(cudaMemcpyAsync(h->pxs, xs.data(), kappa * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (std::sqrt(sn) <= 1e-13 * std::max(1.0, std::sqrt(xn))) break;
  }
  CK(cudaStreamSynchronize(h->stream));
  xs_out = xs;
  return BICADMM_OK;
}

// Softmax polish: the same damped Newton on the kappa support entries of W (polish.cuh,
// softmax section).  supp_out receives the support in class order (matching xs_out).
template <typename TA, typename TM, int KC>
int run_polish_softmax(bicadmm_ctx* h, std::vector<double>& xs_out, std::vector<int64_t>& supp_out) {
  const int64_t m = h->p.m;
  const int kappa = static_cast<int>(h->p.kappa), K = h->K;
  const double gamma = h->p.gamma;
  const int nblk = static_cast<int>(std::min<int64_t>(kPolishRowBlocks, (m + 255) / 256));
  const int nch = static_cast<int>(std::min<int64_t>(kPolishChunks, (m + 255) / 256));
  const int64_t chunk = (m + nch - 1) / nch;
  int rc;
  if (!h->polish_ready) {  // shared buffers of the K = 1 polish (sizes in kappa only) + A_S
#define AL(ptr, bytes) if ((rc = dev_alloc(h, &(ptr), (bytes))) != BICADMM_OK) return rc
    AL(h->AS, static_cast<size_t>(kappa) * m * sizeof(double));
    AL(h->pxs, kappa * sizeof(double));
    AL(h->pstep, kappa * sizeof(double));
    AL(h->pfpart, nblk * sizeof(double));
    AL(h->pgpart, static_cast<size_t>(nch) * kappa * sizeof(double));
    AL(h->pHpart, static_cast<size_t>(nch) * kappa * kappa * sizeof(double));
    AL(h->pH, static_cast<size_t>(kappa) * kappa * sizeof(double));
    AL(h->pflag, sizeof(int));
    AL(h->pq, m * sizeof(double));  // unused by the softmax polish; keeps the K = 1 set complete
    AL(h->pd1, m * sizeof(double));
    AL(h->pd2, m * sizeof(double));
    AL(h->pp, m * sizeof(double));
    h->polish_ready = true;
  }
  if (!h->spolish_ready) {
    AL(h->ssupp, kappa * sizeof(int64_t));
    AL(h->scls, kappa * sizeof(int));
    AL(h->skb, (K + 1) * sizeof(int));
    AL(h->sU, static_cast<size_t>(kappa) * m * sizeof(double));
    AL(h->sq, static_cast<size_t>(m) * K * sizeof(double));
    AL(h->sp, static_cast<size_t>(m) * K * sizeof(double));
    AL(h->sd1, static_cast<size_t>(m) * K * sizeof(double));
    AL(h->sP, static_cast<size_t>(m) * K * sizeof(double));
#undef AL
    h->spolish_ready = true;
  }
  if ((rc = compute_support(h)) != BICADMM_OK) return rc;
  std::vector<int64_t> sp(kappa);
  CK(cudaMemcpyAsync(sp.data(), h->supp, kappa * sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  // class order (stable within a class: ascending flat index)
  std::vector<int64_t> ord;
  std::vector<int> cls, kb(K + 1, 0);
  for (int k = 0; k < K; ++k) {
    kb[k] = static_cast<int>(ord.size());
    for (int e = 0; e < kappa; ++e)
      if (sp[e] % K == k) { ord.push_back(sp[e]); cls.push_back(k); }
  }
  kb[K] = kappa;
  CK(cudaMemcpyAsync(h->ssupp, ord.data(), kappa * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->scls, cls.data(), kappa * sizeof(int), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->skb, kb.data(), (K + 1) * sizeof(int), cudaMemcpyHostToDevice, h->stream));
  const dim3 ggrid(static_cast<unsigned>(std::min<int64_t>((m + 255) / 256, 1024)), kappa);
  k_gather_support<TA><<<ggrid, 256, 0, h->stream>>>(static_cast<const TA*>(h->A), h->lda, h->ssupp, m, h->AS, K);
  CK(cudaGetLastError());
  h->launches += 1;
  std::vector<double> xs(kappa, 0.0), step(kappa), fpart(nblk);
  CK(cudaMemsetAsync(h->pxs, 0, kappa * sizeof(double), h->stream));
  const int T = (kappa + 31) / 32;
  const size_t ksm = kappa * sizeof(double);
  auto objective = [&](double alpha, double* out) -> int {
    k_polish_rows_sm<TM, KC, 256><<<nblk, 256, ksm, h->stream>>>(
        h->AS, h->pxs, h->skb, K, m, static_cast<const TM*>(h->b), h->sq, h->sp, h->sd1, h->sP,
        alpha, h->pfpart, kappa);
    CK(cudaGetLastError());
    h->launches += 1;
    CK(cudaMemcpyAsync(fpart.data(), h->pfpart, nblk * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    double f = 0.0;
    for (double v : fpart) f += v;
    *out = f;
    return BICADMM_OK;
  };
  for (int it = 0; it < 100; ++it) {
    double f0;
    if ((rc = objective(0.0, &f0)) != BICADMM_OK) return rc;  // also fills q, p, d1
    double xx = 0.0;
    for (double v : xs) xx += v * v;
    f0 += xx / (2.0 * gamma);
    k_polish_grad_sm<256><<<dim3(nch, kappa), 256, 0, h->stream>>>(h->AS, h->sd1, h->scls, K, kappa, m, chunk, h->pgpart);
    k_polish_u_sm<<<dim3(static_cast<unsigned>(std::min<int64_t>((m + 255) / 256, 256)), kappa), 256, 0, h->stream>>>(
        h->AS, h->sp, h->scls, K, kappa, m, h->sU);
    k_polish_hess_sm<<<dim3(T * (T + 1) / 2, nch), 256, 0, h->stream>>>(h->AS, h->sU, h->scls, kappa, m, chunk, h->pHpart);
    k_polish_solve<256><<<1, 256, 2 * ksm, h->stream>>>(h->pHpart, h->pgpart, nch, h->pxs, kappa, gamma,
                                                        h->pH, h->pstep, h->pflag);
    k_polish_dir_sm<KC, 256><<<nblk, 256, ksm, h->stream>>>(h->AS, h->pstep, h->skb, K, kappa, m, h->sP);
    CK(cudaGetLastError());
    h->launches += 5;
    int flag = 0;
    CK(cudaMemcpyAsync(step.data(), h->pstep, kappa * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(&flag, h->pflag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (flag) return fail(h, BICADMM_ERR_NUMERIC, "polish: restricted Hessian is not positive definite");
    double alpha = 1.0;
    for (;;) {
      double ft;
      if ((rc = objective(alpha, &ft)) != BICADMM_OK) return rc;
      double x2 = 0.0;
      for (int k = 0; k < kappa; ++k) {
        const double v = xs[k] - alpha * step[k];
        x2 += v * v;
      }
      ft += x2 / (2.0 * gamma);
      if (!(ft > f0 + 1e-16 * std::fabs(f0)) || !(alpha > 1e-12)) break;
      alpha *= 0.5;
    }
    double sn = 0.0, xn = 0.0;
    for (int k = 0; k < kappa; ++k) {
      xs[k] -= alpha * step[k];
      sn += (alpha * step[k]) * (alpha * step[k]);
      xn += xs[k] * xs[k];
    }
    CK(cudaMemcpyAsync(h->pxs, xs.data(), kappa * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (std::sqrt(sn) <= 1e-13 * std::max(1.0, std::sqrt(xn))) break;
  }
  CK(cudaStreamSynchronize(h->stream));
  xs_out = xs;
  supp_out = ord;
  return BICADMM_OK;
}

template <typename TA, typename TM>
int run_polish_softmax_k(bicadmm_ctx* h, std::vector<double>& xs, std::vector<int64_t>& sp) {
  switch (h->KC) {
    case 4: return run_polish_softmax<TA, TM, 4>(h, xs, sp);
    case 10: return run_polish_softmax<TA, TM, 10>(h, xs, sp);
    default: return run_polish_softmax<TA, TM, 16>(h, xs, sp);
  }
}

}  // namespace

// ============================================================================ batches

struct bicadmm_batch_ctx {
  std::vector<bicadmm_t> hs;
  cudaStream_t stream = nullptr;
  int esz = 8;   // bytes of the arithmetic type (m-space, slots)
  int asz = 8;   // bytes of the stored A element
  int prec = 0;  // BICADMM_PREC_* of every handle
  int R = 0, S = 0, VPT = 0, G = 0, nseg = 0, n_xitems = 0, n_ditems = 0, max_ldp = 0;
  int stage_kb = 0;
  int64_t P = 0;
  size_t stage_bytes = 0, smem = 0;
  std::vector<int> lsh;            // per instance: log2 of the pass's threads per row group
  // the narrow-instance pass: its own panel list, grid and shared memory
  BatchSeg* d_seg_n = nullptr;
  int nseg_n = 0, G_n = 0;
  int64_t P_n = 0;
  size_t smem_n = 0;
  int launches_per_iter = 4;
  std::vector<void*> allocs;       // batch-owned device memory (tables, slots, stats)
  std::vector<void*> table_allocs; // tables rebuilt on retiling
  BatchInst* d_inst = nullptr;
  BatchSeg* d_seg = nullptr;
  XItem* d_xitems = nullptr;
  DItem* d_ditems = nullptr;
  ConsensusArgs* d_cons = nullptr;
  std::vector<std::pair<int, int>> candidates;  // (R, S) tilings still to try
  std::vector<std::pair<double, std::pair<int, int>>> timings;
  int tune_iters = 0;
  bool use_graph = false;
  bool profile = false;                 // events around each kernel kind (eager launches)
  std::vector<cudaEvent_t> ev;          // pairs
  std::vector<int> ev_kind;
  double kind_ms[4] = {0, 0, 0, 0};
  int64_t kind_n[4] = {0, 0, 0, 0};
  cudaGraphExec_t graph = nullptr;
  int64_t launches = 0, iters = 0;
  std::string err;
};

namespace {

int bfail(bicadmm_batch_ctx* b, int code, const std::string& msg) {
  if (b) b->err = msg;
  return code;
}

#define BCK(call)                                                                                 \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess)                                                                        \
      return bfail(b, BICADMM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));      \
  } while (0)

template <typename T>
int bdev_alloc(bicadmm_batch_ctx* b, T** ptr, size_t bytes, bool table) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, BICADMM_ERR_OOM, "batch allocation failed");
  }
  (table ? b->table_allocs : b->allocs).push_back(p);
  *ptr = static_cast<T*>(p);
  return BICADMM_OK;
}

template <typename TA, typename TM, int R, int VPT>
int launch_pass_batch_rv(bicadmm_batch_ctx* b) {
  if (b->P == 0) return BICADMM_OK;
  auto kern = k_fused_pass_batch<TA, TM, R, VPT, kPassThreads>;
  BCK(allow_max_dynamic_smem(kern));
  kern<<<b->G, kPassThreads, b->smem, b->stream>>>(b->d_inst, b->d_seg, b->nseg, b->P, b->S,
                                                   b->stage_bytes, kWaitLimitCycles);
  BCK(cudaGetLastError());
  return BICADMM_OK;
}

template <typename TA, typename TM, int R, int VPT>
int occupancy_batch_rv(bicadmm_batch_ctx* b, int* blocks) {
  auto kern = k_fused_pass_batch<TA, TM, R, VPT, kPassThreads>;
  BCK(allow_max_dynamic_smem(kern));
  BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern, kPassThreads, b->smem));
  return BICADMM_OK;
}

// dispatch on (R, VPT); op 0 = launch, 1 = occupancy
template <typename TA, typename TM>
int batch_pass_dispatch(bicadmm_batch_ctx* b, int op, int* blocks) {
#define BP_CASE(RR, VV)                                                                \
  if (b->R == RR && b->VPT == VV)                                                      \
    return op == 0 ? launch_pass_batch_rv<TA, TM, RR, VV>(b) : occupancy_batch_rv<TA, TM, RR, VV>(b, blocks);
#define BP_R(RR) BP_CASE(RR, 1) BP_CASE(RR, 2) BP_CASE(RR, 3) BP_CASE(RR, 4) BP_CASE(RR, 5) \
  BP_CASE(RR, 6) BP_CASE(RR, 8) BP_CASE(RR, 12) BP_CASE(RR, 16)
  BP_R(8)
#undef BP_R
#undef BP_CASE
  return bfail(b, BICADMM_ERR_UNSUPPORTED, "no batched A-pass variant for this tiling");
}

int batch_pass_any(bicadmm_batch_ctx* b, int op, int* blocks) {
  switch (b->prec) {
    case BICADMM_PREC_FP64: return batch_pass_dispatch<double, double>(b, op, blocks);
    case BICADMM_PREC_FP32: return batch_pass_dispatch<float, float>(b, op, blocks);
    default: return batch_pass_dispatch<__nv_bfloat16, float>(b, op, blocks);
  }
}

// The narrow-instance pass; op 0 = launch (nothing when the list is empty), 1 = occupancy.
template <typename TA, typename TM>
int batch_pass_narrow(bicadmm_batch_ctx* b, int op, int* blocks) {
  auto kern = k_fused_pass_batch_narrow<TA, TM, 8, kPassThreads>;
  BCK(allow_max_dynamic_smem(kern));
  if (op == 1) {
    BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern, kPassThreads, b->smem_n));
    return BICADMM_OK;
  }
  if (b->P_n == 0) return BICADMM_OK;
  kern<<<b->G_n, kPassThreads, b->smem_n, b->stream>>>(b->d_inst, b->d_seg_n, b->nseg_n, b->P_n, b->S,
                                                       b->stage_bytes, kWaitLimitCycles);
  BCK(cudaGetLastError());
  return BICADMM_OK;
}

int batch_pass_narrow_any(bicadmm_batch_ctx* b, int op, int* blocks) {
  switch (b->prec) {
    case BICADMM_PREC_FP64: return batch_pass_narrow<double, double>(b, op, blocks);
    case BICADMM_PREC_FP32: return batch_pass_narrow<float, float>(b, op, blocks);
    default: return batch_pass_narrow<__nv_bfloat16, float>(b, op, blocks);
  }
}

constexpr int kBatchMaxRows = 8;  // rows per panel at most (the batched kernel's R)

// Build the panel partition and every table for a tiling: stages of `stage_kb` KB, S of
// them; each instance's panels take as many rows (<= 8) as fit in a stage.
int batch_build(bicadmm_batch_ctx* b, int stage_kb, int S) {
  for (void* p : b->table_allocs) cudaFree(p);
  b->table_allocs.clear();
  const int B = static_cast<int>(b->hs.size());
  int64_t max_lda = 0;
  int max_ldp = 0;
  for (bicadmm_t h : b->hs) {
    max_lda = std::max(max_lda, h->lda);
    max_ldp = std::max(max_ldp, h->max_ldp);
  }
  const int R = kBatchMaxRows;
  b->R = R;
  b->stage_kb = stage_kb;
  b->S = S;
  b->max_ldp = max_ldp;
  b->stage_bytes = static_cast<size_t>(stage_kb) * 1024;
  if (b->stage_bytes < static_cast<size_t>(max_lda) * b->asz)
    return bfail(b, BICADMM_ERR_UNSUPPORTED, "stage smaller than the widest row");
  const int ve = static_cast<int>(16 / b->asz);
  constexpr int NW = kPassThreads / 32;
  // wide pass: ring of S stages | kBatchSlots mbarriers and ring offsets | the issuer's
  // cursor | red[R][NW] | d[R]
  b->smem = S * b->stage_bytes + kBatchSlots * (sizeof(uint64_t) + sizeof(uint32_t)) + sizeof(BatchCursor) +
            static_cast<size_t>(R) * (NW + 1) * b->esz + 16;
  // narrow pass: stages | mbarriers | red and d (R * 32 rows each) | the row groups' A'd
  // partial sums (one vector per thread) | per-warp statistics
  b->smem_n = S * b->stage_bytes + S * sizeof(uint64_t) +
              (2 * static_cast<size_t>(R) * 32 + static_cast<size_t>(kPassThreads) * ve + 3 * NW) * b->esz + 16;
  // Row groups: an instance whose rows hold at most kPassThreads / 2 vectors runs in the
  // narrow pass with groups of L = max(R, next power of two >= its vectors) threads.
  int lg_nt = 0;
  while ((1 << lg_nt) < kPassThreads) ++lg_nt;
  b->lsh.assign(B, lg_nt);
  int64_t max_lda_w = 0;
  for (int q = 0; q < B; ++q) {
    const int64_t nv = b->hs[q]->lda / ve;
    if (2 * nv <= kPassThreads) {
      int l = 0;
      while ((int64_t{1} << l) < std::max<int64_t>(nv, R)) ++l;
      b->lsh[q] = l;
    } else {
      max_lda_w = std::max(max_lda_w, b->hs[q]->lda);
    }
  }
  b->VPT = max_lda_w > 0 ? pick_vpt(max_lda_w / ve) : 1;
  if (b->VPT < 0) return bfail(b, BICADMM_ERR_UNSUPPORTED, "instance rows too wide for the batched pass");
  // segments, one list per pass
  std::vector<BatchSeg> seg, seg_n;
  int64_t P = 0, P_n = 0;
  for (int q = 0; q < B; ++q) {
    bicadmm_t h = b->hs[q];
    const bool nar = b->lsh[q] < lg_nt;
    const int64_t rows_max = nar ? static_cast<int64_t>(R) * (kPassThreads >> b->lsh[q]) : R;
    const int rpp = static_cast<int>(std::min<int64_t>(
        rows_max, static_cast<int64_t>(b->stage_bytes / (static_cast<size_t>(h->lda) * b->asz))));
    for (int i = 0; i < h->N; ++i) {
      const int64_t rows = h->shard_row0[i + 1] - h->shard_row0[i];
      int64_t& PP = nar ? P_n : P;
      (nar ? seg_n : seg).push_back(BatchSeg{q, i, PP, h->shard_row0[i], rows, rpp, 0});
      PP += (rows + rpp - 1) / rpp;
    }
  }
  b->P = P;
  b->nseg = static_cast<int>(seg.size());
  b->P_n = P_n;
  b->nseg_n = static_cast<int>(seg_n.size());
  b->G = b->G_n = 0;
  int rc = BICADMM_OK;
  if (P > 0) {
    int occ = 0;
    if ((rc = batch_pass_any(b, 1, &occ)) != BICADMM_OK) return rc;
    if (occ < 1) return bfail(b, BICADMM_ERR_UNSUPPORTED, "batched A-pass cannot be resident");
    b->G = static_cast<int>(std::min<int64_t>(static_cast<int64_t>(occ) * b->hs[0]->num_sms, P));
  }
  if (P_n > 0) {
    int occ = 0;
    if ((rc = batch_pass_narrow_any(b, 1, &occ)) != BICADMM_OK) return rc;
    if (occ < 1) return bfail(b, BICADMM_ERR_UNSUPPORTED, "batched narrow A-pass cannot be resident");
    b->G_n = static_cast<int>(std::min<int64_t>(static_cast<int64_t>(occ) * b->hs[0]->num_sms, P_n));
  }
  b->launches_per_iter = 3 + (P > 0) + (P_n > 0);
  // CTA of a pass that owns a panel of its list
  auto owner = [](int64_t panel, int64_t PP, int GG) {
    int64_t c = panel * GG / PP;
    while (c > 0 && c * PP / GG > panel) --c;
    while ((c + 1) * PP / GG <= panel) ++c;
    return static_cast<int>(c);
  };
  // per-instance tables
  std::vector<BatchInst> inst(B);
  std::vector<ConsensusArgs> cons(B);
  std::vector<XItem> xitems;
  std::vector<DItem> ditems;
  size_t si_w = 0, si_n = 0;
  for (int q = 0; q < B; ++q) {
    bicadmm_t h = b->hs[q];
    const bool nar = b->lsh[q] < lg_nt;
    const std::vector<BatchSeg>& list = nar ? seg_n : seg;
    size_t& si = nar ? si_n : si_w;
    const int64_t PP = nar ? P_n : P;
    const int GG = nar ? b->G_n : b->G;
    const BatchSeg& s0 = list[si];
    const BatchSeg& s1 = list[si + h->N - 1];
    const int c_lo = owner(s0.first_panel, PP, GG);
    const int c_hi = owner(s1.first_panel + (s1.rows + s1.rpp - 1) / s1.rpp - 1, PP, GG);
    std::vector<int> lo(h->N), hi(h->N);
    for (int i = 0; i < h->N; ++i) {
      const BatchSeg& g = list[si + i];
      lo[i] = owner(g.first_panel, PP, GG) - c_lo + i;
      hi[i] = owner(g.first_panel + (g.rows + g.rpp - 1) / g.rpp - 1, PP, GG) - c_lo + i;
    }
    si += h->N;
    const int G_inst = c_hi - c_lo + 1;
    void* slots = nullptr;
    double* stats = nullptr;
    int* d_lo = nullptr;
    int* d_hi = nullptr;
    if ((rc = bdev_alloc(b, &slots, static_cast<size_t>(G_inst + h->N) * h->lda * b->esz, true)) != BICADMM_OK) return rc;
    if ((rc = bdev_alloc(b, &stats, static_cast<size_t>(G_inst) * 4 * sizeof(double), true)) != BICADMM_OK) return rc;
    if ((rc = bdev_alloc(b, &d_lo, h->N * sizeof(int), true)) != BICADMM_OK) return rc;
    if ((rc = bdev_alloc(b, &d_hi, h->N * sizeof(int), true)) != BICADMM_OK) return rc;
    BCK(cudaMemcpyAsync(d_lo, lo.data(), h->N * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    BCK(cudaMemcpyAsync(d_hi, hi.data(), h->N * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    BatchInst& I = inst[q];
    I.A = h->A; I.lda = h->lda; I.xlo = h->xlo; I.b = h->b; I.omega = h->omega; I.nu = h->nu;
    I.slots = slots; I.cta_stats = stats; I.c_lo = c_lo; I.G_inst = G_inst;
    I.loss = h->p.loss; I.newton_iters = h->p.newton_iters; I.M = h->M; I.rho_l = h->p.rho_l;
    I.lsh = b->lsh[q];
    I.P = h->Pm; I.P_off = h->d_P_off; I.blk_col0 = h->d_blk_col0; I.blk_ldp = h->d_blk_ldp;
    I.M_blocks = h->M; I.N = h->N; I.x = h->x; I.u = h->u; I.r = h->r; I.z = h->z;
    I.rho_c = h->p.rho_c; I.c0 = h->c0; I.slot_lo = d_lo; I.slot_hi = d_hi;
    I.dual_part = h->dual_part; I.dual_chunks = h->dual_chunks; I.n = h->p.n; I.gs = h->gs;
    I.trace = h->trace; I.err = h->d_err;
    cons[q] = consensus_args(h, true);
    cons[q].x = h->x;  // batched consensus CTAs form w and the breakpoints themselves
    cons[q].prepared = 0;
    for (int i = 0; i < h->N; ++i)
      for (int j = 0; j < h->M; ++j) {
        const int nj = h->blk_col0[j + 1] - h->blk_col0[j];
        for (int r0 = 0; r0 < nj; r0 += kXupdRows) xitems.push_back(XItem{q, i, j, r0});
      }
    for (int i = 0; i < h->N; ++i)
      for (int cidx = 0; cidx < h->dual_chunks; ++cidx) ditems.push_back(DItem{q, i, cidx});
  }
  b->n_xitems = static_cast<int>(xitems.size());
  b->n_ditems = static_cast<int>(ditems.size());
  if ((rc = bdev_alloc(b, &b->d_inst, B * sizeof(BatchInst), true)) != BICADMM_OK) return rc;
  if (!seg.empty() && (rc = bdev_alloc(b, &b->d_seg, seg.size() * sizeof(BatchSeg), true)) != BICADMM_OK) return rc;
  if (!seg_n.empty() && (rc = bdev_alloc(b, &b->d_seg_n, seg_n.size() * sizeof(BatchSeg), true)) != BICADMM_OK) return rc;
  if ((rc = bdev_alloc(b, &b->d_xitems, xitems.size() * sizeof(XItem), true)) != BICADMM_OK) return rc;
  if ((rc = bdev_alloc(b, &b->d_ditems, ditems.size() * sizeof(DItem), true)) != BICADMM_OK) return rc;
  if ((rc = bdev_alloc(b, &b->d_cons, B * sizeof(ConsensusArgs), true)) != BICADMM_OK) return rc;
  BCK(cudaMemcpyAsync(b->d_inst, inst.data(), B * sizeof(BatchInst), cudaMemcpyHostToDevice, b->stream));
  if (!seg.empty())
    BCK(cudaMemcpyAsync(b->d_seg, seg.data(), seg.size() * sizeof(BatchSeg), cudaMemcpyHostToDevice, b->stream));
  if (!seg_n.empty())
    BCK(cudaMemcpyAsync(b->d_seg_n, seg_n.data(), seg_n.size() * sizeof(BatchSeg), cudaMemcpyHostToDevice, b->stream));
  BCK(cudaMemcpyAsync(b->d_xitems, xitems.data(), xitems.size() * sizeof(XItem), cudaMemcpyHostToDevice, b->stream));
  BCK(cudaMemcpyAsync(b->d_ditems, ditems.data(), ditems.size() * sizeof(DItem), cudaMemcpyHostToDevice, b->stream));
  BCK(cudaMemcpyAsync(b->d_cons, cons.data(), B * sizeof(ConsensusArgs), cudaMemcpyHostToDevice, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  return BICADMM_OK;
}

int bprof(bicadmm_batch_ctx* b, int kind, bool end) {
  if (!b->profile) return BICADMM_OK;
  if (!end) {
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    b->ev.push_back(e0);
    b->ev.push_back(e1);
    b->ev_kind.push_back(kind);
    BCK(cudaEventRecord(e0, b->stream));
  } else {
    BCK(cudaEventRecord(b->ev.back(), b->stream));
  }
  return BICADMM_OK;
}

// One outer iteration of every instance: 4 or 5 launches (kinds: 1 x-update, 0 pass over
// the wide and over the narrow instances, 3 consensus, 2 dual).
template <typename TM>
int batch_iteration(bicadmm_batch_ctx* b) {
  int rc;
  auto kx = k_xupd_batch<TM, kXupdThreads, kXupdRows>;
  const size_t xsm = static_cast<size_t>(b->max_ldp) * sizeof(TM);
  if (xsm > 48 * 1024) BCK(cudaFuncSetAttribute(kx, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(xsm)));
  if ((rc = bprof(b, 1, false)) != BICADMM_OK) return rc;
  kx<<<b->n_xitems, kXupdThreads, xsm, b->stream>>>(b->d_inst, b->d_xitems);
  BCK(cudaGetLastError());
  if ((rc = bprof(b, 1, true)) != BICADMM_OK) return rc;
  if ((rc = bprof(b, 0, false)) != BICADMM_OK) return rc;
  if ((rc = batch_pass_any(b, 0, nullptr)) != BICADMM_OK) return rc;
  if ((rc = batch_pass_narrow_any(b, 0, nullptr)) != BICADMM_OK) return rc;
  if ((rc = bprof(b, 0, true)) != BICADMM_OK) return rc;
  if ((rc = bprof(b, 3, false)) != BICADMM_OK) return rc;
  k_global_batch<512, 2><<<static_cast<unsigned>(b->hs.size()), 512, 0, b->stream>>>(b->d_cons);
  if ((rc = bprof(b, 3, true)) != BICADMM_OK) return rc;
  if ((rc = bprof(b, 2, false)) != BICADMM_OK) return rc;
  k_dual_batch<TM, kDualThreads><<<b->n_ditems, kDualThreads, 0, b->stream>>>(b->d_inst, b->d_ditems);
  BCK(cudaGetLastError());
  if ((rc = bprof(b, 2, true)) != BICADMM_OK) return rc;
  b->launches += b->launches_per_iter;
  return BICADMM_OK;
}

int batch_run(bicadmm_batch_ctx* b, int n) {
  for (int it = 0; it < n; ++it) {
    int rc = b->esz == 8 ? batch_iteration<double>(b) : batch_iteration<float>(b);
    if (rc != BICADMM_OK) return rc;
  }
  return BICADMM_OK;
}

int batch_capture(bicadmm_batch_ctx* b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  if (!b->use_graph) return BICADMM_OK;
  // attributes are set by an eager launch before capture
  cudaGraph_t g = nullptr;
  BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  const int64_t before = b->launches;
  int rc = b->esz == 8 ? batch_iteration<double>(b) : batch_iteration<float>(b);
  cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  b->launches = before;
  if (rc != BICADMM_OK) return rc;
  if (e != cudaSuccess) return bfail(b, BICADMM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return bfail(b, BICADMM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return BICADMM_OK;
}

}  // namespace

// =============================================================================== C ABI

// Host A: copied in chunks of rows (within one shard, at most 256 MB) on a side stream into
// two alternating device staging slots; each chunk is converted into the padded device
// layout on the handle's stream as soon as it lands, and a shard's Gram matrices follow its
// last chunk there, so that they overlap the copies of later shards.  b first (small).
template <typename TA, typename TM>
int setup_host_pipelined(bicadmm_ctx* h, const void* A, int32_t A_dtype, int64_t lda_src,
                         const void* b, int32_t b_dtype, int32_t b_on_device) {
  int rc = load_matrix<TM>(h, b, b_dtype, 1, b_on_device, static_cast<TM*>(h->b), h->p.m, 1, 1);
  if (rc == BICADMM_OK) rc = check_labels<TM>(h);
  if (rc != BICADMM_OK) return rc;
  const size_t in_es = A_dtype == BICADMM_DTYPE_F64 ? 8 : (A_dtype == BICADMM_DTYPE_BF16 ? 2 : 4);
  const int64_t row_in = lda_src * static_cast<int64_t>(in_es);
  const int64_t cap_rows = std::max<int64_t>(1, (256ll << 20) / std::max<int64_t>(row_in, 1));
  struct Chunk { int64_t r0, nr; };
  std::vector<std::vector<Chunk>> chunks(h->N);
  int64_t max_rows = 1;
  for (int i = 0; i < h->N; ++i)
    for (int64_t r = h->shard_row0[i]; r < h->shard_row0[i + 1]; r += cap_rows) {
      const int64_t nr = std::min(cap_rows, h->shard_row0[i + 1] - r);
      chunks[i].push_back(Chunk{r, nr});
      max_rows = std::max(max_rows, nr);
    }
  void* stage[2] = {nullptr, nullptr};
  cudaStream_t cs = nullptr;
  std::vector<cudaEvent_t> evs;
  auto new_event = [&](cudaEvent_t* ev) -> cudaError_t {
    cudaError_t e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e == cudaSuccess) evs.push_back(*ev);
    return e;
  };
  cudaError_t e = cudaMalloc(&stage[0], static_cast<size_t>(max_rows) * row_in);
  if (e == cudaSuccess) e = cudaMalloc(&stage[1], static_cast<size_t>(max_rows) * row_in);
  if (e != cudaSuccess) {
    cudaGetLastError();
    for (void* p : stage)
      if (p) cudaFree(p);
    return fail(h, BICADMM_ERR_OOM, "staging buffer allocation failed");
  }
  e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  // the copies start after earlier work on the handle's stream (which may still read A)
  cudaEvent_t start_ev = nullptr;
  if (e == cudaSuccess) e = new_event(&start_ev);
  if (e == cudaSuccess) e = cudaEventRecord(start_ev, h->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, start_ev, 0);
  cudaEvent_t converted[2] = {nullptr, nullptr};  // last conversion out of each slot
  long long q = 0;
  std::function<int(int)> load_shard = [&](int i) -> int {
    for (const Chunk& ch : chunks[i]) {
      const int slot = static_cast<int>(q & 1);
      cudaEvent_t copied = nullptr;
      if (e == cudaSuccess && converted[slot]) e = cudaStreamWaitEvent(cs, converted[slot], 0);
      // the last row may be shorter than lda_src: copy exactly (nr-1)*lda_src + n elements
      const size_t bytes = (static_cast<size_t>(ch.nr - 1) * lda_src + h->p.n) * in_es;
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(stage[slot], static_cast<const char*>(A) + ch.r0 * row_in, bytes,
                            cudaMemcpyHostToDevice, cs);
      if (e == cudaSuccess) e = new_event(&copied);
      if (e == cudaSuccess) e = cudaEventRecord(copied, cs);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, copied, 0);
      if (e != cudaSuccess) return fail(h, BICADMM_ERR_CUDA, std::string("H2D copy: ") + cudaGetErrorString(e));
      const int64_t total = ch.nr * h->lda;
      const unsigned grid = static_cast<unsigned>(std::min<int64_t>((total + 255) / 256, 65535));
      TA* dst = static_cast<TA*>(h->A) + ch.r0 * h->lda;
      if (A_dtype == BICADMM_DTYPE_F64)
        k_convert_rows<double, TA><<<grid, 256, 0, h->stream>>>(static_cast<const double*>(stage[slot]), lda_src, dst, h->lda, ch.nr, h->p.n);
      else if (A_dtype == BICADMM_DTYPE_BF16)
        k_convert_rows<__nv_bfloat16, TA><<<grid, 256, 0, h->stream>>>(static_cast<const __nv_bfloat16*>(stage[slot]), lda_src, dst, h->lda, ch.nr, h->p.n);
      else
        k_convert_rows<float, TA><<<grid, 256, 0, h->stream>>>(static_cast<const float*>(stage[slot]), lda_src, dst, h->lda, ch.nr, h->p.n);
      e = cudaGetLastError();
      h->launches += 1;
      if (e == cudaSuccess) e = new_event(&converted[slot]);
      if (e == cudaSuccess) e = cudaEventRecord(converted[slot], h->stream);
      if (e != cudaSuccess) return fail(h, BICADMM_ERR_CUDA, std::string("convert: ") + cudaGetErrorString(e));
      ++q;
    }
    return BICADMM_OK;
  };
  if (e != cudaSuccess) rc = fail(h, BICADMM_ERR_CUDA, std::string("copy stream: ") + cudaGetErrorString(e));
  if (rc == BICADMM_OK) rc = build_factors<TA, TM>(h, &load_shard);
  cudaStreamSynchronize(h->stream);
  if (cs) {
    cudaStreamSynchronize(cs);
    cudaStreamDestroy(cs);
  }
  for (cudaEvent_t x : evs) cudaEventDestroy(x);
  for (void* p : stage) cudaFree(p);
  return rc;
}

extern "C" {

int bicadmm_default_params(bicadmm_params* p) {
  if (!p) return BICADMM_ERR_ARG;
  std::memset(p, 0, sizeof(*p));
  p->loss = BICADMM_LOSS_SQUARED;
  p->precision = BICADMM_PREC_FP64;
  p->K = 1;
  p->N_shards = 1;
  p->M_blocks = 1;
  p->gamma = 10.0;
  p->rho_c = 1.0;
  p->rho_b = 0.0;
  p->rho_l = 0.0;
  p->inner_iters = 1;
  p->newton_iters = 50;
  p->max_iters = 10000;
  p->check_every = 10;
  p->tol_rel = 1e-6;
  return BICADMM_OK;
}

int bicadmm_estimate_bytes(const bicadmm_params* params, int64_t* device_bytes,
                           int64_t* setup_extra_bytes) {
  std::string why;
  int rc = validate(params, why);
  if (rc != BICADMM_OK) { g_create_error = why; return rc; }
  bicadmm_ctx tmp;
  tmp.p = *params;
  if (tmp.p.rho_b == 0.0) tmp.p.rho_b = 0.5 * tmp.p.rho_c;
  if (tmp.p.rho_l == 0.0) tmp.p.rho_l = tmp.p.rho_c;
  cudaError_t e = cudaGetDevice(&tmp.device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&tmp.num_sms, cudaDevAttrMultiProcessorCount, tmp.device);
  if (e != cudaSuccess) { cudaGetLastError(); g_create_error = "no usable CUDA device"; return BICADMM_ERR_CUDA; }
  rc = build_geometry(&tmp);
  if (rc != BICADMM_OK) { g_create_error = tmp.err; return rc; }
  handle_bytes(&tmp, device_bytes, setup_extra_bytes);
  return BICADMM_OK;
}

// The part of create shared by single handles and paths: h->p (and the path fields) set.
static int create_handle(bicadmm_ctx* h, void* stream, bicadmm_t* out) {
  if (h->p.precision == BICADMM_PREC_TF32) {
    h->tf32 = true;
    h->p.precision = BICADMM_PREC_FP32;
  }
  if (h->p.rho_b == 0.0) h->p.rho_b = 0.5 * h->p.rho_c;
  if (h->p.rho_l == 0.0) h->p.rho_l = h->p.rho_c;
  h->stream = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e != cudaSuccess) {
    g_create_error = std::string("no usable CUDA device: ") + cudaGetErrorString(e);
    delete h;
    return BICADMM_ERR_CUDA;
  }
  int rc = build_geometry(h);
  if (rc == BICADMM_OK) rc = allocate(h);
  // the 2D tensor map of A serves the tensor-core softmax pass
  if (rc == BICADMM_OK && h->use_tc) rc = make_tmap(h);
  if (rc == BICADMM_OK) rc = reset_state(h);
  if (rc != BICADMM_OK) {
    g_create_error = h->err;
    free_all(h);
    delete h;
    return rc;
  }
  *out = h;
  return BICADMM_OK;
}

int bicadmm_create(const bicadmm_params* params, void* stream, bicadmm_t* out) {
  g_create_error.clear();
  if (!out) { g_create_error = "out is NULL"; return BICADMM_ERR_ARG; }
  *out = nullptr;
  std::string why;
  int rc = validate(params, why);
  if (rc != BICADMM_OK) { g_create_error = why; return rc; }
  bicadmm_ctx* h = new bicadmm_ctx();
  h->p = *params;
  return create_handle(h, stream, out);
}

int bicadmm_create_path(const bicadmm_params* params, int32_t count, const int64_t* kappas,
                        void* stream, bicadmm_t* out) {
  g_create_error.clear();
  if (!out) { g_create_error = "out is NULL"; return BICADMM_ERR_ARG; }
  *out = nullptr;
  if (!params || !kappas) { g_create_error = "params and kappas are required"; return BICADMM_ERR_ARG; }
  if (count < 2 || count > 16) { g_create_error = "a path holds 2..16 instances"; return BICADMM_ERR_ARG; }
  if (params->loss == BICADMM_LOSS_SOFTMAX || params->K != 1) {
    g_create_error = "a path runs a one-column loss (K = 1: squared, logistic, squared hinge)";
    return BICADMM_ERR_ARG;
  }
  int64_t kmax = 0;
  for (int q = 0; q < count; ++q) {
    if (kappas[q] < 1 || kappas[q] > params->n) { g_create_error = "need 1 <= kappa <= n for every instance"; return BICADMM_ERR_ARG; }
    kmax = std::max(kmax, kappas[q]);
  }
  bicadmm_params v = *params;
  v.kappa = kmax;
  std::string why;
  int rc = validate(&v, why);
  if (rc != BICADMM_OK) { g_create_error = why; return rc; }
  if (params->n * count > kMaxN) { g_create_error = "n times the instance count must be <= 32768"; return BICADMM_ERR_UNSUPPORTED; }
  bicadmm_ctx* h = new bicadmm_ctx();
  h->p = v;
  h->p.K = count;  // the instances are the columns of the multi-column kernels
  h->path = true;
  h->ninst = count;
  h->kappas.assign(kappas, kappas + count);
  return create_handle(h, stream, out);
}

int bicadmm_path_info(bicadmm_t h, int32_t instance, bicadmm_info* info) {
  if (!h || !info) return BICADMM_ERR_ARG;
  if (!h->path || instance < 0 || instance >= h->ninst) return fail(h, BICADMM_ERR_ARG, "not an instance of a path");
  if (!h->ready) return fail(h, BICADMM_ERR_STATE, "bicadmm_path_info before setup");
  int rc = fill_info(h, info, true, instance);
  info->converged = h->converged ? 1 : 0;
  return rc;
}

int bicadmm_path_get_x(bicadmm_t h, int32_t instance, double* x_host, int64_t len, int64_t* support_out) {
  if (!h) return BICADMM_ERR_ARG;
  if (!h->path || instance < 0 || instance >= h->ninst) return fail(h, BICADMM_ERR_ARG, "not an instance of a path");
  if (!h->ready) return fail(h, BICADMM_ERR_STATE, "bicadmm_path_get_x before setup");
  if (!x_host || len != h->p.n) return fail(h, BICADMM_ERR_ARG, "x_host must hold n doubles");
  const double* zq = h->z_cm + static_cast<int64_t>(instance) * h->p.n;
  CK(cudaMemcpyAsync(x_host, zq, h->p.n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  if (support_out) {
    const int64_t kq = h->kappas[static_cast<size_t>(instance)];
    if (!h->supp) {
      int rc = dev_alloc(h, &h->supp, h->p.kappa * sizeof(int64_t));  // p.kappa: the largest
      if (rc != BICADMM_OK) return rc;
    }
    k_support<1024, 1><<<1, 1024, 0, h->stream>>>(zq, h->key, h->p.n, kq, h->supp);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(support_out, h->supp, kq * sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  return check_device_error(h);
}

int bicadmm_setup(bicadmm_t h, const void* A, int32_t A_dtype, int64_t lda, int32_t A_on_device,
                  const void* b, int32_t b_dtype, int32_t b_on_device) {
  if (!h) return BICADMM_ERR_ARG;
  if (!A || !b) return fail(h, BICADMM_ERR_ARG, "A and b must be non-NULL");
  if (A_dtype != BICADMM_DTYPE_F64 && A_dtype != BICADMM_DTYPE_F32 && A_dtype != BICADMM_DTYPE_BF16) return fail(h, BICADMM_ERR_ARG, "A_dtype must be F64, F32 or BF16");
  if (b_dtype != BICADMM_DTYPE_F64 && b_dtype != BICADMM_DTYPE_F32) return fail(h, BICADMM_ERR_ARG, "b_dtype must be F64 or F32");
  if (lda < h->p.n) return fail(h, BICADMM_ERR_ARG, "lda must be >= n");
  h->ready = false;
  h->err.clear();
  int rc = reset_state(h);
  if (rc != BICADMM_OK) return rc;
  if (!A_on_device) {
    switch (h->p.precision) {
      case BICADMM_PREC_FP64: rc = setup_host_pipelined<double, double>(h, A, A_dtype, lda, b, b_dtype, b_on_device); break;
      case BICADMM_PREC_FP32: rc = setup_host_pipelined<float, float>(h, A, A_dtype, lda, b, b_dtype, b_on_device); break;
      default: rc = setup_host_pipelined<__nv_bfloat16, float>(h, A, A_dtype, lda, b, b_dtype, b_on_device); break;
    }
  } else if (h->p.precision == BICADMM_PREC_FP64) {
    rc = load_matrix<double>(h, A, A_dtype, lda, A_on_device, static_cast<double*>(h->A), h->p.m, h->p.n, h->lda);
    if (rc == BICADMM_OK) rc = load_matrix<double>(h, b, b_dtype, 1, b_on_device, static_cast<double*>(h->b), h->p.m, 1, 1);
    if (rc == BICADMM_OK) rc = check_labels<double>(h);
    if (rc == BICADMM_OK) rc = build_factors<double, double>(h);
  } else if (h->p.precision == BICADMM_PREC_FP32) {
    rc = load_matrix<float>(h, A, A_dtype, lda, A_on_device, static_cast<float*>(h->A), h->p.m, h->p.n, h->lda);
    if (rc == BICADMM_OK) rc = load_matrix<float>(h, b, b_dtype, 1, b_on_device, static_cast<float*>(h->b), h->p.m, 1, 1);
    if (rc == BICADMM_OK) rc = check_labels<float>(h);
    if (rc == BICADMM_OK) rc = build_factors<float, float>(h);
  } else {
    rc = load_matrix<__nv_bfloat16>(h, A, A_dtype, lda, A_on_device, static_cast<__nv_bfloat16*>(h->A), h->p.m, h->p.n, h->lda);
    if (rc == BICADMM_OK) rc = load_matrix<float>(h, b, b_dtype, 1, b_on_device, static_cast<float*>(h->b), h->p.m, 1, 1);
    if (rc == BICADMM_OK) rc = check_labels<float>(h);
    if (rc == BICADMM_OK) rc = build_factors<__nv_bfloat16, float>(h);
  }
  if (rc != BICADMM_OK) return rc;
  h->ready = true;
  return BICADMM_OK;
}

// Capture graph_iters outer iterations of the handle into a CUDA graph (the launches are
// recorded, not run; the counters are restored).
static int capture_graph(bicadmm_ctx* h) {
  const int64_t l0 = h->launches, i0 = h->iters_done;
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  int rc = h->esz == 8 ? run_iterations<double>(h, h->graph_iters) : run_iterations<float>(h, h->graph_iters);
  const cudaError_t ce = cudaStreamEndCapture(h->stream, &g);
  h->graph_launches = h->launches - l0;
  h->launches = l0;
  h->iters_done = i0;
  if (rc != BICADMM_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (ce != cudaSuccess) return fail(h, BICADMM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
  const cudaError_t ie = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    h->graph = nullptr;
    return fail(h, BICADMM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
  }
  return BICADMM_OK;
}

static int step_impl(bicadmm_t h, int32_t n_iters, bicadmm_info* info, bool objective);

int bicadmm_step(bicadmm_t h, int32_t n_iters, bicadmm_info* info) {
  return step_impl(h, n_iters, info, true);
}

static int step_impl(bicadmm_t h, int32_t n_iters, bicadmm_info* info, bool objective) {
  if (!h) return BICADMM_ERR_ARG;
  if (!h->ready) return fail(h, BICADMM_ERR_STATE, "bicadmm_step before a successful bicadmm_setup");
  if (n_iters < 0) return fail(h, BICADMM_ERR_ARG, "n_iters must be >= 0");
  int rc = BICADMM_OK;
  int done = 0;
  if (h->graph_iters > 0 && h->prof == 0) {
    // the first iteration runs eagerly (kernel attributes are set outside any capture)
    if (!h->graph && n_iters >= 1) {
      rc = h->esz == 8 ? run_iterations<double>(h, 1) : run_iterations<float>(h, 1);
      if (rc != BICADMM_OK) return rc;
      ++done;
      if ((rc = capture_graph(h)) != BICADMM_OK) return rc;
    }
    if (h->graph) {
      for (; done + h->graph_iters <= n_iters; done += h->graph_iters) {
        CK(cudaGraphLaunch(h->graph, h->stream));
        h->launches += h->graph_launches;
        h->iters_done += h->graph_iters;
      }
    }
  }
  if (done < n_iters)
    rc = h->esz == 8 ? run_iterations<double>(h, n_iters - done) : run_iterations<float>(h, n_iters - done);
  if (rc != BICADMM_OK) return rc;
  if (info) return fill_info(h, info, objective);
  return BICADMM_OK;
}

int bicadmm_set_graph(bicadmm_t h, int32_t iters_per_graph) {
  if (!h) return BICADMM_ERR_ARG;
  if (iters_per_graph < 0) return fail(h, BICADMM_ERR_ARG, "iters_per_graph must be >= 0");
  if (iters_per_graph > 0 && h->stream == nullptr)
    return fail(h, BICADMM_ERR_ARG, "graph replay needs a non-default stream");
  if (h->graph) {
    CK(cudaStreamSynchronize(h->stream));
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  h->graph_iters = iters_per_graph;
  return BICADMM_OK;
}

int bicadmm_solve(bicadmm_t h, bicadmm_info* info) {
  if (!h) return BICADMM_ERR_ARG;
  if (!h->ready) return fail(h, BICADMM_ERR_STATE, "bicadmm_solve before a successful bicadmm_setup");
  bicadmm_info loc;
  int done = 0;
  h->converged = false;
  while (done < h->p.max_iters) {
    const int k = std::min(h->p.check_every, h->p.max_iters - done);
    int rc = step_impl(h, k, &loc, false);
    if (rc != BICADMM_OK) return rc;
    done += k;
    double mx = std::max(std::max(loc.p_rel, loc.d_rel), std::max(loc.b_rel, loc.i_rel));
    for (int q = 1; q < h->ninst; ++q) {  // a path stops when every instance has
      bicadmm_info lq;
      if ((rc = fill_info(h, &lq, false, q)) != BICADMM_OK) return rc;
      mx = std::max(mx, std::max(std::max(lq.p_rel, lq.d_rel), std::max(lq.b_rel, lq.i_rel)));
    }
    if (mx <= h->p.tol_rel) { h->converged = true; break; }
  }
  loc.converged = h->converged ? 1 : 0;
  if (info) {
    int rc = fill_info(h, info);
    if (rc != BICADMM_OK) return rc;
  }
  return BICADMM_OK;
}

int bicadmm_get_x(bicadmm_t h, double* x_host, int64_t len, int32_t polished, int64_t* support_out) {
  if (!h) return BICADMM_ERR_ARG;
  if (!h->ready) return fail(h, BICADMM_ERR_STATE, "bicadmm_get_x before setup");
  const int64_t nK = h->p.n * h->K;
  if (!x_host || len != nK) return fail(h, BICADMM_ERR_ARG, "x_host must hold n K doubles");
  if (polished && h->p.kappa > kMaxPolishKappa)
    return fail(h, BICADMM_ERR_UNSUPPORTED, "polish supports kappa <= 1024");
  if (h->path && (polished || support_out))
    return fail(h, BICADMM_ERR_UNSUPPORTED, "a path's instances are read with bicadmm_path_get_x (no polish)");
  if (!polished) {
    CK(cudaMemcpyAsync(x_host, h->z, nK * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (support_out) {
      int rc = compute_support(h);
      if (rc != BICADMM_OK) return rc;
    }
  } else if (h->K > 1) {
    std::vector<double> xs;
    std::vector<int64_t> sp;
    int rc = h->p.precision == BICADMM_PREC_FP64 ? run_polish_softmax_k<double, double>(h, xs, sp)
             : h->p.precision == BICADMM_PREC_FP32 ? run_polish_softmax_k<float, float>(h, xs, sp)
                                                   : run_polish_softmax_k<__nv_bfloat16, float>(h, xs, sp);
    if (rc != BICADMM_OK) return rc;
    std::fill(x_host, x_host + nK, 0.0);
    for (int64_t k = 0; k < h->p.kappa; ++k) x_host[sp[k]] = xs[k];
  } else {
    std::vector<double> xs;
    int rc = h->p.precision == BICADMM_PREC_FP64 ? run_polish<double, double>(h, xs)
             : h->p.precision == BICADMM_PREC_FP32 ? run_polish<float, float>(h, xs)
                                                   : run_polish<__nv_bfloat16, float>(h, xs);
    if (rc != BICADMM_OK) return rc;
    std::vector<int64_t> sp(h->p.kappa);
    CK(cudaMemcpyAsync(sp.data(), h->supp, h->p.kappa * sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    std::fill(x_host, x_host + h->p.n, 0.0);
    for (int64_t k = 0; k < h->p.kappa; ++k) x_host[sp[k]] = xs[k];
  }
  if (support_out)
    CK(cudaMemcpyAsync(support_out, h->supp, h->p.kappa * sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return check_device_error(h);
}

int bicadmm_get_state(bicadmm_t h, int32_t field, double* out_host, int64_t len) {
  if (!h) return BICADMM_ERR_ARG;
  if (!out_host) return fail(h, BICADMM_ERR_ARG, "out_host is NULL");
  const int64_t n = h->p.n * h->K, m = h->p.m * h->K, N = h->N;  // n K and m K entries
  auto need = [&](int64_t L) { return len == L; };
  switch (field) {
    case BICADMM_FIELD_X:
    case BICADMM_FIELD_U: {
      if (!need(N * n)) return fail(h, BICADMM_ERR_ARG, "length must be N*n*K");
      const double* src = field == BICADMM_FIELD_X ? h->x : h->u;
      CK(cudaMemcpy2DAsync(out_host, n * sizeof(double), src, h->ldx * sizeof(double), n * sizeof(double), N,
                           cudaMemcpyDeviceToHost, h->stream));
      break;
    }
    case BICADMM_FIELD_Z:
    case BICADMM_FIELD_S:
      if (!need(n)) return fail(h, BICADMM_ERR_ARG, "length must be n*K");
      CK(cudaMemcpyAsync(out_host, field == BICADMM_FIELD_Z ? h->z : h->s, n * sizeof(double),
                         cudaMemcpyDeviceToHost, h->stream));
      break;
    case BICADMM_FIELD_OMEGA:
    case BICADMM_FIELD_NU: {
      if (!need(m)) return fail(h, BICADMM_ERR_ARG, "length must be m*K");
      const void* src = field == BICADMM_FIELD_OMEGA ? h->omega : h->nu;
      if (h->esz == 8) {
        CK(cudaMemcpyAsync(out_host, src, m * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      } else {
        std::vector<float> tmp(m);
        CK(cudaMemcpyAsync(tmp.data(), src, m * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        for (int64_t q = 0; q < m; ++q) out_host[q] = tmp[q];
      }
      break;
    }
    case BICADMM_FIELD_SCALARS: {
      if (!need(3)) return fail(h, BICADMM_ERR_ARG, "length must be 3");
      GlobalState g;
      CK(cudaMemcpyAsync(&g, h->gs, sizeof(g), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      out_host[0] = g.t;
      out_host[1] = g.v;
      out_host[2] = g.tau;
      break;
    }
    case BICADMM_FIELD_P: {
      int64_t total = 0;
      for (int j = 0; j < h->M; ++j) {
        const int64_t nj = h->blk_col0[j + 1] - h->blk_col0[j];
        total += N * nj * nj;
      }
      if (!need(total)) return fail(h, BICADMM_ERR_ARG, "length must be the sum of n_j^2 over shards and blocks");
      std::vector<unsigned char> tmp(static_cast<size_t>(h->P_total) * h->esz);
      CK(cudaMemcpyAsync(tmp.data(), h->Pm, tmp.size(), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      int64_t o = 0;
      for (int i = 0; i < N; ++i)
        for (int j = 0; j < h->M; ++j) {
          const int nj = h->blk_col0[j + 1] - h->blk_col0[j], ldp = h->blk_ldp[j];
          const int64_t base = h->P_off[static_cast<size_t>(i) * h->M + j];
          for (int a = 0; a < nj; ++a)
            for (int c = 0; c < nj; ++c) {
              const int64_t q = base + static_cast<int64_t>(a) * ldp + c;
              out_host[o++] = h->esz == 8 ? reinterpret_cast<const double*>(tmp.data())[q]
                                          : static_cast<double>(reinterpret_cast<const float*>(tmp.data())[q]);
            }
        }
      return BICADMM_OK;
    }
    default:
      return fail(h, BICADMM_ERR_ARG, "unknown field");
  }
  CK(cudaStreamSynchronize(h->stream));
  return check_device_error(h);
}

int bicadmm_get_trace(bicadmm_t h, double* out_host, int64_t max_records, int64_t* n_out) {
  if (!h) return BICADMM_ERR_ARG;
  if (!out_host || max_records < 0) return fail(h, BICADMM_ERR_ARG, "out_host is NULL or max_records < 0");
  GlobalState g;
  CK(cudaMemcpyAsync(&g, h->gs, sizeof(g), cudaMemcpyDeviceToHost, h->stream));
  std::vector<Resid> recs(kTraceCap);
  CK(cudaMemcpyAsync(recs.data(), h->trace, kTraceCap * sizeof(Resid), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  const int64_t avail = std::min<int64_t>(g.iter, kTraceCap);
  const int64_t cnt = std::min<int64_t>(avail, max_records);
  for (int64_t q = 0; q < cnt; ++q) {
    const Resid& r = recs[(g.iter - cnt + q) % kTraceCap];
    double* o = out_host + q * 15;
    o[0] = static_cast<double>(r.iter);
    o[1] = r.p_r; o[2] = r.d_r; o[3] = r.b_r; o[4] = r.i_r;
    o[5] = r.p_rel; o[6] = r.d_rel; o[7] = r.b_rel; o[8] = r.i_rel;
    o[9] = r.t; o[10] = r.v; o[11] = r.tau; o[12] = r.znorm;
    o[13] = static_cast<double>(r.zt_steps);
    o[14] = static_cast<double>(r.zt_lists);
  }
  if (n_out) *n_out = cnt;
  return check_device_error(h);
}

int bicadmm_set_profiling(bicadmm_t h, int32_t on) {
  if (!h) return BICADMM_ERR_ARG;
  if (on < 0 || on > 2) return fail(h, BICADMM_ERR_ARG, "profiling mode must be 0, 1 or 2");
  h->prof = on;
  h->ev_used = 0;
  h->ev_kind.clear();
  return BICADMM_OK;
}

int bicadmm_get_kernel_times(bicadmm_t h, double* ms_out, int64_t* launches_out, int32_t reset) {
  if (!h) return BICADMM_ERR_ARG;
  CK(cudaStreamSynchronize(h->stream));
  double tot[KIND_COUNT] = {0.0, 0.0, 0.0, 0.0};
  int64_t cnt[KIND_COUNT] = {0, 0, 0, 0};
  for (size_t q = 0; q + 1 < h->ev_used; q += 2) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev[q], h->ev[q + 1]));
    const int kind = h->ev_kind[q / 2];
    tot[kind] += ms;
    cnt[kind] += 1;
  }
  for (int k = 0; k < KIND_COUNT; ++k) {
    if (ms_out) ms_out[k] = tot[k];
    if (launches_out) launches_out[k] = cnt[k];
  }
  if (reset) {
    h->ev_used = 0;
    h->ev_kind.clear();
  }
  return BICADMM_OK;
}

int bicadmm_inject_pass_stall(bicadmm_t h, int64_t panel, int64_t wait_limit_cycles) {
  if (!h) return BICADMM_ERR_ARG;
  if (panel >= 0 && (!h->ready || h->K != 1 || panel >= h->P_panels))
    return fail(h, BICADMM_ERR_ARG, "stall panel must be a panel of a set-up K = 1 handle");
  if (panel >= 0 && wait_limit_cycles < 1000)
    return fail(h, BICADMM_ERR_ARG, "wait limit must be at least 1000 cycles");
  if (panel >= 0 && h->graph) return fail(h, BICADMM_ERR_STATE, "not with graph replay");
  h->stall_panel = panel >= 0 ? panel : -1;
  h->wait_limit = panel >= 0 ? static_cast<long long>(wait_limit_cycles) : kWaitLimitCycles;
  return BICADMM_OK;
}

int bicadmm_get_pass_time(bicadmm_t h, double* ms_out, int64_t* launches_out) {
  double ms[KIND_COUNT];
  int64_t cnt[KIND_COUNT];
  int rc = bicadmm_get_kernel_times(h, ms, cnt, 1);
  if (rc != BICADMM_OK) return rc;
  if (ms_out) *ms_out = ms[KIND_PASS];
  if (launches_out) *launches_out = cnt[KIND_PASS];
  return BICADMM_OK;
}

int bicadmm_batch_create(bicadmm_t* handles, int32_t count, void* stream, int32_t flags,
                         bicadmm_batch_t* out) {
  g_create_error.clear();
  if (!out || !handles || count < 1) { g_create_error = "handles, count >= 1 and out are required"; return BICADMM_ERR_ARG; }
  *out = nullptr;
  for (int q = 0; q < count; ++q) {
    bicadmm_t h = handles[q];
    if (!h || !h->ready) { g_create_error = "every handle must be set up"; return BICADMM_ERR_STATE; }
    if (h->p.precision != handles[0]->p.precision || h->device != handles[0]->device) { g_create_error = "handles must share precision and device"; return BICADMM_ERR_ARG; }
    if (h->K != 1) { g_create_error = "batches take handles with K = 1"; return BICADMM_ERR_UNSUPPORTED; }
    if (h->p.inner_iters != 1) { g_create_error = "batched handles must use inner_iters = 1"; return BICADMM_ERR_UNSUPPORTED; }
    for (int q2 = 0; q2 < q; ++q2)
      if (handles[q2] == h) { g_create_error = "a handle appears twice"; return BICADMM_ERR_ARG; }
  }
  bicadmm_batch_ctx* b = new bicadmm_batch_ctx();
  b->hs.assign(handles, handles + count);
  b->stream = static_cast<cudaStream_t>(stream);
  b->esz = static_cast<int>(handles[0]->esz);
  b->asz = static_cast<int>(handles[0]->asz);
  b->prec = handles[0]->p.precision;
  b->use_graph = (flags & BICADMM_BATCH_GRAPH) != 0;
  b->profile = (flags & BICADMM_BATCH_PROFILE) != 0;
  if (b->use_graph && b->profile) { g_create_error = "profiling needs eager launches (no graph)"; delete b; return BICADMM_ERR_ARG; }
  if (b->use_graph && !stream) { g_create_error = "graph capture needs a non-default stream"; delete b; return BICADMM_ERR_ARG; }
  int64_t max_lda = 0;
  for (bicadmm_t h : b->hs) max_lda = std::max(max_lda, h->lda);
  const size_t row_bytes = static_cast<size_t>(max_lda) * b->asz;
  // tilings (stage KB, S stages) that hold the widest row and fit the shared memory; one
  // stage of 32 KB or more lets the two CTAs of an SM alternate between loading and computing
  for (int kb : {16, 24, 32, 40, 48, 64, 96})
    for (int S : {1, 2, 3, 4}) {
      if (S == 1 && kb < 32) continue;
      const size_t st = static_cast<size_t>(kb) * 1024;
      if (st >= row_bytes && S * st <= kPassSmemBudget) b->candidates.push_back({kb, S});
    }
  if (b->candidates.empty()) { g_create_error = "rows too wide for the batched pass"; delete b; return BICADMM_ERR_UNSUPPORTED; }
  // default (the autotuner's choice on a 256-instance mix): one 96 KB stage for 4- and
  // 8-byte storage, two 48 KB stages for BF16 (or one widest row per stage); two CTAs per SM
  const bool bf16 = b->asz == 2;
  const int kb0 = static_cast<int>(std::max<size_t>(bf16 ? 48 : 96, (row_bytes + 1023) / 1024));
  const int S0 = bf16 && 2 * kb0 <= 200 ? 2 : 1;
  if (!(flags & BICADMM_BATCH_AUTOTUNE)) b->candidates.clear();
  int rc = batch_build(b, kb0, S0);
  if (rc != BICADMM_OK) {
    g_create_error = b->err;
    for (void* p : b->allocs) cudaFree(p);
    for (void* p : b->table_allocs) cudaFree(p);
    delete b;
    return rc;
  }
  b->tune_iters = 2;
  *out = b;
  return BICADMM_OK;
}

int bicadmm_batch_step(bicadmm_batch_t b, int32_t n_iters, int64_t* launches_out) {
  if (!b) return BICADMM_ERR_ARG;
  if (n_iters < 0) return bfail(b, BICADMM_ERR_ARG, "n_iters must be >= 0");
  int done = 0;
  int rc = BICADMM_OK;
  // Autotuning: the first iterations run each candidate tiling for tune_iters iterations
  // (each is an ordinary iteration of every instance), timed with CUDA events; the fastest
  // tiling is kept.
  while (!b->candidates.empty() && done < n_iters) {
    const auto cand = b->candidates.back();
    b->candidates.pop_back();
    if ((rc = batch_build(b, cand.first, cand.second)) != BICADMM_OK) {
      if (rc == BICADMM_ERR_UNSUPPORTED) continue;
      return rc;
    }
    const int k = std::min(b->tune_iters, n_iters - done);
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    BCK(cudaEventRecord(e0, b->stream));
    rc = batch_run(b, k);
    BCK(cudaEventRecord(e1, b->stream));
    BCK(cudaEventSynchronize(e1));
    float ms = 0.f;
    BCK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != BICADMM_OK) return rc;
    b->timings.push_back({ms / k, cand});
    done += k;
    b->iters += k;
    if (b->candidates.empty()) {
      auto best = *std::min_element(b->timings.begin(), b->timings.end());
      if ((rc = batch_build(b, best.second.first, best.second.second)) != BICADMM_OK) return rc;
    }
  }
  if (done < n_iters && b->use_graph && !b->graph) {
    // one eager iteration sets kernel attributes, then one iteration is captured
    if ((rc = batch_run(b, 1)) != BICADMM_OK) return rc;
    ++done;
    ++b->iters;
    if ((rc = batch_capture(b)) != BICADMM_OK) return rc;
  }
  for (; done < n_iters; ++done) {
    if (b->graph) {
      BCK(cudaGraphLaunch(b->graph, b->stream));
      b->launches += b->launches_per_iter;
    } else if ((rc = batch_run(b, 1)) != BICADMM_OK) {
      return rc;
    }
    ++b->iters;
  }
  for (bicadmm_t h : b->hs) h->iters_done += n_iters;
  if (launches_out) *launches_out = b->launches;
  return BICADMM_OK;
}

int bicadmm_batch_tiling(bicadmm_batch_t b, int32_t* rows_out, int32_t* stages_out) {
  if (!b) return BICADMM_ERR_ARG;
  if (rows_out) *rows_out = b->stage_kb;
  if (stages_out) *stages_out = b->S;
  return BICADMM_OK;
}

int bicadmm_batch_kernel_times(bicadmm_batch_t b, double* ms_out, int64_t* launches_out) {
  if (!b) return BICADMM_ERR_ARG;
  BCK(cudaStreamSynchronize(b->stream));
  double ms[4] = {0, 0, 0, 0};
  int64_t cnt[4] = {0, 0, 0, 0};
  for (size_t q = 0; q + 1 < b->ev.size(); q += 2) {
    float t = 0.f;
    BCK(cudaEventElapsedTime(&t, b->ev[q], b->ev[q + 1]));
    ms[b->ev_kind[q / 2]] += t;
    cnt[b->ev_kind[q / 2]] += 1;
  }
  for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
  b->ev.clear();
  b->ev_kind.clear();
  for (int k = 0; k < 4; ++k) {
    if (ms_out) ms_out[k] = ms[k];
    if (launches_out) launches_out[k] = cnt[k];
  }
  return BICADMM_OK;
}

int bicadmm_batch_destroy(bicadmm_batch_t b) {
  if (!b) return BICADMM_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  else cudaDeviceSynchronize();
  for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (void* p : b->allocs) cudaFree(p);
  for (void* p : b->table_allocs) cudaFree(p);
  delete b;
  return BICADMM_OK;
}

const char* bicadmm_batch_last_error(bicadmm_batch_t b) {
  if (!b) return g_create_error.c_str();
  return b->err.c_str();
}

// ============================================================================ serving

struct ServerReq {
  bicadmm_params p{};
  const void* A = nullptr;
  const void* b = nullptr;
  int32_t A_dtype = 0, b_dtype = 0, A_dev = 0, b_dev = 0;
  int64_t lda = 0;
  // arrival; admission (= setup start); setup end; retirement start (polish, copy-out);
  // completion: seconds on the server's clock, -1 until reached
  double arrival = 0.0, admitted = -1.0, setup_done = -1.0, retiring = -1.0, done = -1.0;
  bicadmm_t h = nullptr;
  int64_t bytes = 0;
  int iters = 0, rounds = 0;
  int status = BICADMM_OK;
  std::vector<double> x;
  std::vector<int64_t> support;
  bicadmm_info info{};
};

// Request records live behind stable pointers: another host thread may submit (append a
// record, under mu) while run() works on the records it holds.  Fields of a request are
// written by the thread in run() only; its completion time is published under mu after
// its results, and bicadmm_server_result reads them under mu once it sees it.
struct bicadmm_server_ctx {
  bicadmm_server_params sp{};
  cudaStream_t round_stream = nullptr, setup_stream = nullptr;
  std::mutex mu;                                 // guards reqs (the vector), waiting, completed
  std::vector<std::unique_ptr<ServerReq>> reqs;
  std::deque<int64_t> waiting;   // submitted, not yet admitted, ordered by arrival
  std::vector<int64_t> active;   // run() thread only
  bicadmm_batch_t batch = nullptr;
  bool dirty = true;
  std::atomic<int> open{0};      // run() waits for submissions while set
  int64_t bytes_in_use = 0, peak_bytes = 0;
  int64_t rounds = 0, completed = 0, launches = 0;
  // where the host loop's time goes (seconds): batch rebuilds and their count, waiting for
  // rounds on the device, admissions (create + setup), retirements (polish + copy-out)
  double rebuild_s = 0.0, round_wait_s = 0.0, admit_s = 0.0, retire_s = 0.0;
  int64_t rebuilds = 0;
  std::chrono::steady_clock::time_point t0;
  std::string err;
  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  ServerReq* req(int64_t id) {
    std::lock_guard<std::mutex> g(mu);
    return reqs[static_cast<size_t>(id)].get();
  }
};

namespace {

int sfail(bicadmm_server_ctx* s, int code, const std::string& msg) {
  if (s) s->err = msg;
  return code;
}

void server_drop_batch(bicadmm_server_ctx* s) {
  if (s->batch) {
    bicadmm_batch_destroy(s->batch);
    s->batch = nullptr;
  }
  s->dirty = true;
}

// Publish a request's completion (after its results are written).
void server_finish(bicadmm_server_ctx* s, ServerReq& r) {
  std::lock_guard<std::mutex> g(s->mu);
  r.done = s->now();
  ++s->completed;
}

// Admit arrived requests in arrival order while the device-memory budget and slot count allow.
int server_admit(bicadmm_server_ctx* s) {
  const double t = s->now();
  while (static_cast<int>(s->active.size()) < s->sp.max_active) {
    int64_t id;
    {
      std::lock_guard<std::mutex> g(s->mu);
      if (s->waiting.empty()) break;
      id = s->waiting.front();
      if (s->reqs[static_cast<size_t>(id)]->arrival > t) break;
    }
    ServerReq& r = *s->req(id);
    int64_t need = 0, extra = 0;
    int rc = bicadmm_estimate_bytes(&r.p, &need, &extra);
    if (rc == BICADMM_OK && need + extra > s->sp.hbm_budget_bytes) rc = BICADMM_ERR_OOM;
    if (rc != BICADMM_OK) {  // an invalid or never-fitting request fails alone
      r.status = rc;
      {
        std::lock_guard<std::mutex> g(s->mu);
        s->waiting.pop_front();
      }
      server_finish(s, r);
      continue;
    }
    if (s->bytes_in_use + need + extra > s->sp.hbm_budget_bytes) break;  // wait for memory
    const double t_adm = s->now();
    bicadmm_t h = nullptr;
    rc = bicadmm_create(&r.p, s->setup_stream, &h);
    if (rc == BICADMM_OK) {
      rc = bicadmm_setup(h, r.A, r.A_dtype, r.lda, r.A_dev, r.b, r.b_dtype, r.b_dev);
      if (rc != BICADMM_OK) {
        s->err = h->err;
        bicadmm_destroy(h);
        h = nullptr;
      }
    } else {
      s->err = g_create_error;
    }
    {
      std::lock_guard<std::mutex> g(s->mu);
      s->waiting.pop_front();
    }
    r.admitted = t_adm;
    r.setup_done = s->now();
    s->admit_s += r.setup_done - t_adm;
    if (rc != BICADMM_OK) {
      r.status = rc;
      server_finish(s, r);
      continue;
    }
    r.h = h;
    r.bytes = need;
    s->bytes_in_use += need;
    s->peak_bytes = std::max(s->peak_bytes, s->bytes_in_use + extra);
    s->active.push_back(id);
    s->dirty = true;
  }
  return BICADMM_OK;
}

// Residual check of every active request after a round; retire the finished ones.
int server_retire(bicadmm_server_ctx* s) {
  std::vector<int64_t> still, finished;
  for (int64_t id : s->active) {
    ServerReq& r = *s->req(id);
    bicadmm_info inf;
    int rc = fill_info(r.h, &inf, false);
    const double mx = std::max(std::max(inf.p_rel, inf.d_rel), std::max(inf.b_rel, inf.i_rel));
    const bool conv = r.iters > 1 && mx <= r.p.tol_rel;
    if (rc != BICADMM_OK || conv || r.iters >= r.p.max_iters) {
      r.status = rc;
      r.info = inf;
      r.info.converged = conv ? 1 : 0;
      finished.push_back(id);
    } else {
      still.push_back(id);
    }
  }
  if (finished.empty()) return BICADMM_OK;
  const double t_ret = s->now();
  server_drop_batch(s);  // the batch references the handles
  for (int64_t id : finished) {
    ServerReq& r = *s->req(id);
    r.retiring = s->now();
    if (r.status == BICADMM_OK) {
      // the objective at the final iterate (FP64, on the device), then the model
      bicadmm_info inf;
      r.status = fill_info(r.h, &inf, true);
      r.info.objective = inf.objective;
    }
    if (r.status == BICADMM_OK) {
      r.x.assign(r.p.n, 0.0);
      r.support.assign(r.p.kappa, 0);
      const int pol = s->sp.polish && r.p.kappa <= kMaxPolishKappa ? 1 : 0;
      r.status = bicadmm_get_x(r.h, r.x.data(), r.p.n, pol, r.support.data());
    }
    bicadmm_destroy(r.h);
    r.h = nullptr;
    s->bytes_in_use -= r.bytes;
    server_finish(s, r);
  }
  s->retire_s += s->now() - t_ret;
  s->active = still;
  return BICADMM_OK;
}

}  // namespace

int bicadmm_server_create(const bicadmm_server_params* sp, bicadmm_server_t* out) {
  g_create_error.clear();
  if (!sp || !out) { g_create_error = "params and out are required"; return BICADMM_ERR_ARG; }
  *out = nullptr;
  if (sp->hbm_budget_bytes <= 0 || sp->max_active < 1 || sp->iters_per_round < 1) {
    g_create_error = "need hbm_budget_bytes > 0, max_active >= 1, iters_per_round >= 1";
    return BICADMM_ERR_ARG;
  }
  bicadmm_server_ctx* s = new bicadmm_server_ctx();
  s->sp = *sp;
  if (cudaStreamCreateWithFlags(&s->round_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->setup_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    g_create_error = "stream creation failed";
    delete s;
    return BICADMM_ERR_CUDA;
  }
  s->t0 = std::chrono::steady_clock::now();
  *out = s;
  return BICADMM_OK;
}

double bicadmm_server_clock(bicadmm_server_t s) { return s ? s->now() : 0.0; }

int bicadmm_server_submit(bicadmm_server_t s, const bicadmm_params* p, const void* A,
                          int32_t A_dtype, int64_t lda, int32_t A_on_device, const void* b,
                          int32_t b_dtype, int32_t b_on_device, double arrival, int64_t* id_out) {
  if (!s) return BICADMM_ERR_ARG;
  if (!p || !A || !b || !id_out) return BICADMM_ERR_ARG;
  if (p->precision != s->sp.precision) return BICADMM_ERR_ARG;
  if (p->inner_iters != 1 || p->K != 1) return BICADMM_ERR_UNSUPPORTED;
  std::unique_ptr<ServerReq> r(new ServerReq());
  r->p = *p;
  r->A = A;
  r->b = b;
  r->A_dtype = A_dtype;
  r->b_dtype = b_dtype;
  r->A_dev = A_on_device;
  r->b_dev = b_on_device;
  r->lda = lda;
  r->arrival = arrival;
  std::lock_guard<std::mutex> g(s->mu);
  s->reqs.push_back(std::move(r));
  const int64_t id = static_cast<int64_t>(s->reqs.size()) - 1;
  // keep the waiting list ordered by arrival (stable for equal times)
  auto it = s->waiting.end();
  while (it != s->waiting.begin() && s->reqs[static_cast<size_t>(*(it - 1))]->arrival > arrival) --it;
  s->waiting.insert(it, id);
  *id_out = id;
  return BICADMM_OK;
}

int bicadmm_server_set_open(bicadmm_server_t s, int32_t open) {
  if (!s) return BICADMM_ERR_ARG;
  s->open.store(open ? 1 : 0);
  return BICADMM_OK;
}

int bicadmm_server_run(bicadmm_server_t s, double until, int64_t* completed_out) {
  if (!s) return BICADMM_ERR_ARG;
  int rc;
  for (;;) {
    if ((rc = server_admit(s)) != BICADMM_OK) return rc;
    if (s->active.empty()) {
      double next = -1.0;
      {
        std::lock_guard<std::mutex> g(s->mu);
        if (!s->waiting.empty()) next = s->reqs[static_cast<size_t>(s->waiting.front())]->arrival;
      }
      if (next < 0.0) {  // nothing submitted is waiting
        if (!s->open.load() || s->now() > until) break;
        std::this_thread::sleep_for(std::chrono::duration<double>(0.0005));
        continue;
      }
      if (next > until) break;
      const double wait = next - s->now();
      if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(std::min(wait, 0.001)));
      continue;
    }
    if (s->dirty || !s->batch) {
      const double t_rb = s->now();
      server_drop_batch(s);
      std::vector<bicadmm_t> hs;
      for (int64_t id : s->active) hs.push_back(s->req(id)->h);
      rc = bicadmm_batch_create(hs.data(), static_cast<int32_t>(hs.size()), s->round_stream,
                                s->sp.use_graph ? BICADMM_BATCH_GRAPH : 0, &s->batch);
      if (rc != BICADMM_OK) return sfail(s, rc, std::string("batch: ") + g_create_error);
      s->dirty = false;
      s->rebuild_s += s->now() - t_rb;
      ++s->rebuilds;
    }
    // a round: as many iterations as the closest request to its cap still needs (<= the
    // round length), so every request stops exactly at its iteration cap
    int k = s->sp.iters_per_round;
    for (int64_t id : s->active) {
      const ServerReq& r = *s->req(id);
      k = std::min(k, r.p.max_iters - r.iters);
    }
    k = std::max(k, 1);
    int64_t launches = 0;
    if ((rc = bicadmm_batch_step(s->batch, k, &launches)) != BICADMM_OK) return sfail(s, rc, s->batch->err);
    s->launches += static_cast<int64_t>(s->batch->launches_per_iter) * k;
    for (int64_t id : s->active) {
      ServerReq& r = *s->req(id);
      r.iters += k;
      ++r.rounds;
    }
    ++s->rounds;
    // new arrivals are set up (setup stream) while the round runs on the device
    if ((rc = server_admit(s)) != BICADMM_OK) return rc;
    const double t_w = s->now();
    if (cudaStreamSynchronize(s->round_stream) != cudaSuccess) return sfail(s, BICADMM_ERR_CUDA, "round failed");
    s->round_wait_s += s->now() - t_w;
    if ((rc = server_retire(s)) != BICADMM_OK) return rc;
    bool idle;
    {
      std::lock_guard<std::mutex> g(s->mu);
      idle = s->active.empty() && s->waiting.empty();
    }
    if (idle && (!s->open.load() || s->now() > until)) break;
    if (s->now() > until && s->active.empty()) break;
  }
  if (completed_out) {
    std::lock_guard<std::mutex> g(s->mu);
    *completed_out = s->completed;
  }
  return BICADMM_OK;
}

int bicadmm_server_result(bicadmm_server_t s, int64_t id, double* x_host, int64_t len,
                          int64_t* support_out, bicadmm_info* info, double* times_out) {
  if (!s) return BICADMM_ERR_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  if (id < 0 || id >= static_cast<int64_t>(s->reqs.size())) return BICADMM_ERR_ARG;
  const ServerReq& r = *s->reqs[static_cast<size_t>(id)];
  if (r.done < 0) return BICADMM_ERR_STATE;
  if (times_out) {
    times_out[0] = r.arrival;
    times_out[1] = r.admitted;
    times_out[2] = r.done;
  }
  if (info) *info = r.info;
  if (r.status != BICADMM_OK) return r.status;
  if (x_host) {
    if (len != r.p.n) return BICADMM_ERR_ARG;
    std::copy(r.x.begin(), r.x.end(), x_host);
  }
  if (support_out) std::copy(r.support.begin(), r.support.end(), support_out);
  return BICADMM_OK;
}

int bicadmm_server_timing(bicadmm_server_t s, int64_t id, double* out) {
  if (!s || !out) return BICADMM_ERR_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  if (id < 0) {
    out[0] = static_cast<double>(s->rebuilds);
    out[1] = s->rebuild_s;
    out[2] = s->round_wait_s;
    out[3] = s->admit_s;
    out[4] = s->retire_s;
    out[5] = static_cast<double>(s->rounds);
    out[6] = s->now();
    return BICADMM_OK;
  }
  if (id >= static_cast<int64_t>(s->reqs.size())) return BICADMM_ERR_ARG;
  const ServerReq& r = *s->reqs[static_cast<size_t>(id)];
  if (r.done < 0) return BICADMM_ERR_STATE;
  out[0] = r.arrival;
  out[1] = r.admitted;
  out[2] = r.setup_done;
  out[3] = r.retiring;
  out[4] = r.done;
  out[5] = static_cast<double>(r.iters);
  out[6] = static_cast<double>(r.rounds);
  return BICADMM_OK;
}

int bicadmm_server_stats(bicadmm_server_t s, int64_t* counters_out) {
  if (!s) return BICADMM_ERR_ARG;
  if (counters_out) {
    std::lock_guard<std::mutex> g(s->mu);
    counters_out[0] = static_cast<int64_t>(s->reqs.size());
    counters_out[1] = s->completed;
    counters_out[2] = s->rounds;
    counters_out[3] = s->peak_bytes;
    counters_out[4] = s->launches;
  }
  return BICADMM_OK;
}

int bicadmm_server_destroy(bicadmm_server_t s) {
  if (!s) return BICADMM_OK;
  server_drop_batch(s);
  for (auto& r : s->reqs)
    if (r->h) bicadmm_destroy(r->h);
  cudaStreamDestroy(s->round_stream);
  cudaStreamDestroy(s->setup_stream);
  delete s;
  return BICADMM_OK;
}

const char* bicadmm_server_last_error(bicadmm_server_t s) {
  if (!s) return g_create_error.c_str();
  return s->err.c_str();
}

int bicadmm_destroy(bicadmm_t h) {
  if (!h) return BICADMM_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  free_all(h);
  delete h;
  return BICADMM_OK;
}

const char* bicadmm_last_error(bicadmm_t h) {
  if (!h) return g_create_error.c_str();
  return h->err.c_str();
}

}  // extern "C"
