// Tensor-core (tcgen05) variant of the softmax A pass for BF16 storage, K <= 16 classes,
// rows of at most 2048 columns.  Same arithmetic as k_fused_pass_k (Sec. 3.1 with K
// right-hand sides: eqs. p:GPU;x, p:GPU;omega, p:GPU;nu), with the two products on the
// 5th-generation tensor cores:
//
//   forward   D1[64 x 16] = A_panel[64 x n] W_i[n x 16]              (row dots, FP32 in TMEM)
//   backward  D2[n x 16] += A_panel'[n x 64] d_panel[64 x 16]          (A'd, FP32 in TMEM)
//
// A stays BF16.  W_i and d are split into BF16 pairs hi + lo (hi = bf16(v), lo =
// bf16(v - hi)) and both halves are accumulated into the same TMEM columns, so the
// products carry about 16 bits of the FP32 operand instead of 8.
//
// Data movement: the row is cut into 128-column slabs, each moved by two 2D TMA loads
// (64-column boxes, 128-byte swizzle) into one stage of an S-stage mbarrier ring.  The same
// swizzled slab serves as the K-major A operand of the forward (rows = M) and as the
// MN-major A operand of the backward (columns = M, the two boxes LBO apart).  The backward
// needs d, which needs the whole forward, so each slab is loaded twice per panel: the
// second load normally hits L2 (two panels, 512 KB, per SM are in flight).
//
// Warp roles, panel size and the MMA order are described at k_fused_pass_tc.
#pragma once

#include <cuda.h>

#include "common.cuh"
#include "nspace.cuh"
#include "pass.cuh"

namespace bic {

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_addr(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

// The same with an L2 cache policy (from createpolicy).
__device__ __forceinline__ void tma_load_2d_hint(void* dst, const CUtensorMap* map, int x, int y,
                                                 uint64_t* bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(
          smem_addr(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_addr(bar)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Generic-proxy shared-memory writes -> visible to the async proxy (tensor core operands).
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D[tmem] = (accumulate ? D : 0) + A[smem] B[smem], BF16 inputs, FP32 accumulator.
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// The same, issued by one elected lane of a converged warp (the warp runs the issuing loop
// uniformly, which keeps the operands in uniform registers; a loop in one thread of a
// divergent branch issued MMAs at a fraction of the rate).
__device__ __forceinline__ void umma_bf16_warp(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                               uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p, e;\n\tsetp.ne.b32 p, %4, 0;\n\telect.sync _|e, 0xffffffff;\n\t"
      "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit_warp(uint64_t* bar) {
  asm volatile(
      "{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
      "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(
          smem_addr(bar))
      : "memory");
}

// Arrive once on *bar when every tcgen05.mma issued so far by this thread has completed.
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}
// This warp's 32 TMEM lanes x 16 consecutive 32-bit columns from taddr.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor (sm_100 format) for a 128-byte-swizzled operand:
// start address, leading and stride byte offsets (>> 4), version 1, layout SWIZZLE_128B.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((saddr >> 4) & 0x3FFFu) |
         (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | (2ull << 61);
}
// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, operand majorness,
// N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool a_mn_major, bool b_mn_major) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn_major ? 1u : 0u) << 15) |
         ((b_mn_major ? 1u : 0u) << 16) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

// ------------------------------------------------------------------ per-row softmax prox
// omega-bar prox of eq. (p:GPU;omega) for one row held by one thread (K classes in
// registers): argmin_w CE(M w; y) + (M rho_l / 2) ||w - a||^2.  Newton with the
// Sherman-Morrison step of the Hessian diag(M^2 p + M rho_l) - M^2 p p', damped by halving
// until ||g|| decreases, stopped once every step is within a few ulps of w.
template <int KC>
__device__ __forceinline__ void softmax_prox_row(float (&w)[KC], const float (&a)[KC], int y, int K,
                                                 float M, float rho_l, int newton_iters) {
  const float Mr = M * rho_l, M2 = M * M;
  float p[KC], g[KC];
  // gradient at wv (and p = softmax(M wv)); returns ||g||^2.  exp and the reciprocal use
  // the fast hardware approximations (a few ulp); the minimiser is then that of phi up to
  // that relative accuracy.
  auto grad = [&](const float (&wv)[KC], float (&pk)[KC], float (&gk)[KC]) -> float {
    float mx = -FpLim<float>::big;
#pragma unroll
    for (int k = 0; k < KC; ++k)
      if (k < K) mx = fmaxf(mx, M * wv[k]);
    float S = 0.f;
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      pk[k] = k < K ? __expf(M * wv[k] - mx) : 0.f;
      S += pk[k];
    }
    const float inv = __fdividef(1.f, S);
    float gn = 0.f;
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      pk[k] *= inv;
      gk[k] = k < K ? M * (pk[k] - (k == y ? 1.f : 0.f)) + Mr * (wv[k] - a[k]) : 0.f;
      gn = fmaf(gk[k], gk[k], gn);
    }
    return gn;
  };
  float gn2 = grad(w, p, g);
  for (int it = 0; it < newton_iters; ++it) {
    float iD[KC], t = 0.f, sp = 0.f;
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      iD[k] = __fdividef(1.f, M2 * p[k] + Mr);
      if (k < K) {
        t = fmaf(p[k] * g[k], iD[k], t);
        sp = fmaf(p[k], iD[k], sp);
      }
    }
    const float coef = __fdividef(M2 * t, Mr * sp);
    float delta[KC];
    bool small = true;
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      delta[k] = k < K ? (g[k] + coef * p[k]) * iD[k] : 0.f;
      small = small && fabsf(delta[k]) <= 4.f * FpLim<float>::eps * fmaxf(fabsf(w[k]), 1.f);
    }
    if (small) break;
    // damped step: halve until ||g|| decreases; no decrease within 8 halvings means g is
    // at its rounding level, and w is kept
    float alpha = 1.f, wt[KC], pt[KC], gt[KC], gt2 = gn2;
    bool accepted = false;
    for (int bt = 0; bt < 8; ++bt) {
#pragma unroll
      for (int k = 0; k < KC; ++k) wt[k] = w[k] - alpha * delta[k];
      gt2 = grad(wt, pt, gt);
      const float shrink = 1.f - 1e-4f * alpha;
      if (gt2 <= shrink * shrink * gn2) { accepted = true; break; }
      alpha *= 0.5f;
    }
    if (!accepted) break;
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      w[k] = wt[k];
      p[k] = pt[k];
      g[k] = gt[k];
    }
    gn2 = gt2;
  }
}

// ------------------------------------------------------------------ k_fused_pass_tc
// Warp roles (256 threads): warps 0-3 own the 128 TMEM lanes (epilogue and slot flush),
// warp 4 lane 0 issues the loads, warp 5 lane 0 issues tcgen05.mma, warps 6-7 idle.
//
// Panels are 64 rows.  The forward MMA has M = 64; its accumulator puts row r in TMEM lane
// 32 (r / 16) + r % 16 (measured), so each of the four epilogue warps owns 16 panel rows
// (lanes 0-15 of its sub-partition) and all four run the per-row prox of every panel.
//
// W_i is read from global memory in its MMA layout (per 64-column box a 32 x 64 BF16 tile:
// rows 0-15 the hi parts of the 16 classes, rows 16-31 the lo parts; written by
// k_xupd_k): each forward stage brings the 8 KB W slab with the 16 KB A slab, so nothing
// per shard stays resident and the ring can hold S stages of 24 KB.  The forward MMA has
// N = 32 and produces A W_hi and A W_lo side by side; the epilogue adds the two halves.
//
// MMA order per CTA: F(0); then for each later panel k: F(k), B(k-1) inside a shard, or
// B(k-1), F(k) when k starts a new shard; B(last) at the end.  The producer loads slabs in
// exactly that order.  D1 and d are double-buffered by panel parity; the prox of panel k
// overlaps the loads and forward MMAs of panel k+1.  At a shard end all four epilogue
// warps wait for the shard's last backward and copy D2 to the shard's slot.
constexpr int kTcRows = 64;                        // panel rows
constexpr int kTcThreads = 256;
constexpr int kTcStages = 4;
constexpr int kTcBoxBytes = kTcRows * 128;         // one 64 x 64 BF16 box = 8 KB
constexpr int kTcWBytes = 2 * 4096;                // W of a 128-column slab: [box] 32 x 64 BF16 (hi | lo)
constexpr int kTcStageCols = 256;                  // columns per stage: two slabs, four boxes
constexpr int kTcStageABytes = 4 * kTcBoxBytes;
constexpr int kTcStageBytes = kTcStageABytes + 2 * kTcWBytes;  // A (256 columns) + its W
constexpr int kTcMaxSlabs = 16;                    // lda <= 2048
constexpr int kTcDBytes = 2 * 2 * 2048;            // [buffer][split] 16 x 64 BF16 tiles
constexpr int kTcTmemCols = 512;                   // D1 x2 at 0 / 32, D2 slab s at 64 + 16 s
constexpr int kTcD2Col = 64;

inline size_t fused_pass_tc_smem() {
  // alignment, ring, d tiles, barriers
  return 1024 + static_cast<size_t>(kTcStages) * kTcStageBytes + kTcDBytes + 256;
}

// Bounded wait that also gives up once another role has raised *abort.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity, long long limit,
                                                   volatile int* abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort || clock64() - t0 > limit) return false;
  }
  return true;
}

template <int KC>
__global__ void __launch_bounds__(kTcThreads, 1)
k_fused_pass_tc(const __grid_constant__ CUtensorMap tmap, int64_t lda,
                const unsigned char* __restrict__ wpk, int64_t ldx, int K,
                const float* __restrict__ b, float* __restrict__ omega, float* __restrict__ nu,
                float* __restrict__ slots, double* __restrict__ cta_stats, PassGeometry geo,
                float Mf, float rho_l, int newton_iters, int* __restrict__ err,
                long long wait_limit, ConsensusArgs cons, int path_loss) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // the last consensus_ctas(cons) CTAs run the global step (one per instance of a path)
  if (cons.enabled && blockIdx.x >= gridDim.x - consensus_ctas(cons)) {
    const int q = blockIdx.x - (gridDim.x - consensus_ctas(cons));
    consensus_block<kTcThreads, kConsMW, true>(consensus_instance(cons, q), smem_raw);  // its dynamic smem holds the top-kappa candidates
    return;
  }
  constexpr int S = kTcStages;
  constexpr uint32_t IDESC_FWD = idesc_bf16(64, 32, false, false);
  constexpr uint32_t IDESC_BWD = idesc_bf16(128, 16, true, false);
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  unsigned char* ring = base;
  unsigned char* ds = ring + S * kTcStageBytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(ds + kTcDBytes);
  uint64_t* empty = full + S;
  uint64_t* d1full = empty + S;   // [2]
  uint64_t* dready = d1full + 2;  // [2]
  uint64_t* bwddone = dready + 2;
  uint64_t* flushed = bwddone + 1;  // all 128 epilogue threads have copied D2 out
  uint64_t* drainbar = flushed + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drainbar + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  long long* counts = reinterpret_cast<long long*>(tmem_slot + 2);  // [0] issued, [1] consumed
  float* red = reinterpret_cast<float*>(counts + 2);               // [4 warps][3]

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c = blockIdx.x, G = gridDim.x - consensus_ctas(cons);
  const int64_t p_begin = static_cast<int64_t>(c) * geo.P / G;
  const int64_t p_end = static_cast<int64_t>(c + 1) * geo.P / G;
  const int np = static_cast<int>(p_end - p_begin);
  const int nstage = static_cast<int>((lda + kTcStageCols - 1) / kTcStageCols);  // stages per phase
  const int nslab = 2 * nstage;  // 128-column slabs (D2 tiles; W is stored for all of them)
  volatile int* abort_v = abort_flag;

  if (tid == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], 1);
    }
    mbar_init(&d1full[0], 1);
    mbar_init(&d1full[1], 1);
    mbar_init(&dready[0], 128);
    mbar_init(&dready[1], 128);
    mbar_init(bwddone, 1);
    mbar_init(flushed, 128);
    mbar_init(drainbar, 1);
    *abort_flag = 0;
    counts[0] = counts[1] = 0;
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, kTcTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // Shard of this CTA's first panel (binary search over the shards' first panels): every
  // walker starts there, so a lookup walks at most the shards the CTA spans, not all shards
  // before it (a walk from shard 0 per lookup made the last CTAs a quarter slower).
  int shard0 = 0;
  {
    int lo = 0, hi = geo.N - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (geo.panel_start[mid] <= p_begin) lo = mid; else hi = mid - 1;
    }
    shard0 = lo;
  }
  // Panel k -> (first row, rows, shard) with a forward-moving shard hint.
  struct PanelWalk {
    int hint;
    __device__ void at(const PassGeometry& g, int64_t p, int64_t& row0, int& nrows, int& shard) {
      locate_panel<kTcRows>(g, p, hint, row0, nrows);
      shard = hint;
    }
  };
  // shard of panel k (k < np) or -1
  auto shard_of = [&](int k) -> int {
    if (k < 0 || k >= np) return -1;
    PanelWalk t{shard0};
    int64_t r0;
    int nr, sh;
    t.at(geo, p_begin + k, r0, nr, sh);
    return sh;
  };
  // Step order shared by the producer and the MMA issuer: calls fn(is_forward, k).
  auto schedule = [&](auto&& fn) {
    PanelWalk pw{shard0};
    int prev_shard = -1;
    for (int k = 0; k < np; ++k) {
      int64_t r0;
      int nr, sh;
      pw.at(geo, p_begin + k, r0, nr, sh);
      const bool boundary = sh != prev_shard;
      if (k > 0 && boundary && !fn(false, k - 1)) return;
      if (!fn(true, k)) return;
      if (k > 0 && !boundary && !fn(false, k - 1)) return;
      prev_shard = sh;
    }
    if (np > 0) fn(false, np - 1);
  };

  float st_res = 0.f, st_om = 0.f, st_ax = 0.f;

  if (warp == 4) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      long long j = 0;
      PanelWalk pw{shard0};
      // forward loads are read again by the backward of the same panel: keep them in L2;
      // the backward load is their last use
      const uint64_t keep = l2_policy_evict_last(), drop = l2_policy_evict_first();
      schedule([&](bool fwd, int k) -> bool {
        int64_t row0;
        int nr, sh;
        pw.at(geo, p_begin + k, row0, nr, sh);  // non-decreasing shard along the schedule
        const unsigned char* wsrc = wpk + static_cast<int64_t>(sh) * nslab * kTcWBytes;
        for (int sg = 0; sg < nstage; ++sg, ++j) {
          const int st = static_cast<int>(j % S);
          if (j >= S && !mbar_wait_or_abort(&empty[st], static_cast<uint32_t>(((j / S) - 1) & 1), wait_limit, abort_v)) {
            *abort_v = 1;
            counts[0] = j;
            return false;
          }
          unsigned char* dst = ring + st * kTcStageBytes;
          mbar_arrive_expect_tx(&full[st], kTcStageABytes + (fwd ? 2 * kTcWBytes : 0));
#pragma unroll
          for (int bx = 0; bx < 4; ++bx)
            tma_load_2d_hint(dst + bx * kTcBoxBytes, &tmap, sg * kTcStageCols + bx * 64,
                             static_cast<int>(row0), &full[st], fwd ? keep : drop);
          if (fwd) bulk_copy_g2s(dst + kTcStageABytes, wsrc + 2 * sg * kTcWBytes, 2 * kTcWBytes, &full[st]);
        }
        counts[0] = j;
        return true;
      });
    }
  } else if (warp == 5) {
    // ---------------------------------------------------------------- MMA issuer (whole warp)
    {
      // descriptor templates: only the 14-bit start address field changes per MMA
      const uint64_t tk = sdesc_sw128(0, 16, 1024);          // K-major operands
      const uint64_t tm_ = sdesc_sw128(0, kTcBoxBytes, 1024);  // MN-major slab (backward A)
      const uint32_t ring_a = smem_addr(ring), ds_a = smem_addr(ds);
      auto dsc = [](uint64_t t, uint32_t addr) -> uint64_t { return t | ((addr >> 4) & 0x3FFFu); };
      long long j = 0;
      int bwd_shard = -1, fseg = 0;
      auto consume = [&](bool fwd, int k) -> bool {
        bool first_bwd = false;
        if (!fwd) {
          if (!mbar_wait_or_abort(&dready[k & 1], static_cast<uint32_t>((k >> 1) & 1), wait_limit, abort_v)) return false;
          const int sh = shard_of(k);
          first_bwd = sh != bwd_shard;
          if (first_bwd && bwd_shard >= 0) {  // D2 of the previous shard has been copied out
            if (!mbar_wait_or_abort(flushed, static_cast<uint32_t>(fseg & 1), wait_limit, abort_v)) return false;
            ++fseg;
          }
          bwd_shard = sh;
        }
        tc_fence_after();
        for (int sg = 0; sg < nstage; ++sg, ++j) {
          const int st = static_cast<int>(j % S);
          // TMA completion on the stage barrier makes the data visible to the MMAs (both
          // async proxy); no tcgen05 fence is needed here
          if (!mbar_wait_or_abort(&full[st], static_cast<uint32_t>((j / S) & 1), wait_limit, abort_v)) return false;
          const uint32_t sa = ring_a + st * kTcStageBytes;
          if (fwd) {
            const uint32_t d1 = tmem + 32 * (k & 1);
#pragma unroll
            for (int bx = 0; bx < 4; ++bx)
#pragma unroll
              for (int ks = 0; ks < 4; ++ks)
                umma_bf16_warp(d1, dsc(tk, sa + bx * kTcBoxBytes + ks * 32),
                               dsc(tk, sa + kTcStageABytes + bx * 4096 + ks * 32), IDESC_FWD,
                               (sg | bx | ks) != 0 ? 1u : 0u);
          } else {
            const uint32_t db = ds_a + (k & 1) * 4096;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int sl = 2 * sg + h;
              {
                const uint32_t d2 = tmem + kTcD2Col + 16 * sl;
#pragma unroll
                for (int sp = 0; sp < 2; ++sp)
#pragma unroll
                  for (int ks = 0; ks < 4; ++ks)
                    umma_bf16_warp(d2, dsc(tm_, sa + h * 2 * kTcBoxBytes + ks * 2048),
                                   dsc(tk, db + sp * 2048 + ks * 32), IDESC_BWD,
                                   (first_bwd && sp == 0 && ks == 0) ? 0u : 1u);
              }
            }
          }
          umma_commit_warp(&empty[st]);
        }
        if (fwd) {
          umma_commit_warp(&d1full[k & 1]);
        } else if (k + 1 >= np || shard_of(k + 1) != bwd_shard) {
          umma_commit_warp(bwddone);  // last backward of a shard
        }
        return true;
      };
      schedule([&](bool fwd, int k) -> bool {
        const bool okk = consume(fwd, k);
        counts[1] = j;
        if (!okk) *abort_v = 1;
        return okk;
      });
    }
  } else if (warp < 4) {
    // ---------------------------------------------------------------- epilogue warps
    const uint32_t lane_base = static_cast<uint32_t>(warp * 32) << 16;
    const bool has_row = lane < 16;        // M = 64 accumulator: lanes 0-15 of each warp
    const int r = warp * 16 + (lane & 15);  // panel row of this thread
    int seg = 0;
    bool eok = true;
    PanelWalk pw{shard0};
    // prefetched row data of the next panel
    float nur[KC], wv[KC];
    int y = 0;
    float yb = 0.f;
    auto prefetch = [&](int k) {
      int64_t row0 = 0;
      int nrows = 0, sh;
      if (k < np) {
        PanelWalk t{shard0};
        t.at(geo, p_begin + k, row0, nrows, sh);
      }
      const bool valid = has_row && k < np && r < nrows;
#pragma unroll
      for (int q = 0; q < KC; ++q) {
        nur[q] = (valid && q < K) ? nu[(row0 + r) * K + q] : 0.f;
        wv[q] = (valid && q < K) ? omega[(row0 + r) * K + q] : 0.f;
      }
      y = valid ? static_cast<int>(b[row0 + r]) : 0;
      yb = valid ? b[row0 + r] : 0.f;
    };
    prefetch(0);
    for (int k = 0; k < np && eok; ++k) {
      int64_t row0;
      int nrows, shard;
      pw.at(geo, p_begin + k, row0, nrows, shard);
      {
        if (!mbar_wait_or_abort(&d1full[k & 1], static_cast<uint32_t>((k >> 1) & 1), wait_limit, abort_v)) { eok = false; break; }
        tc_fence_after();
        uint32_t v[16], vl[16];
        tmem_ld16(tmem + lane_base + 32 * (k & 1), v);
        tmem_ld16(tmem + lane_base + 32 * (k & 1) + 16, vl);
        const bool valid = has_row && r < nrows;
        float Axb[KC], aa[KC], w[KC], nk[KC];
        const int yk = y;
        const float ybk = yb;
#pragma unroll
        for (int q = 0; q < KC; ++q) {
          Axb[q] = (__uint_as_float(v[q]) + __uint_as_float(vl[q])) / Mf;
          nk[q] = nur[q];
          w[q] = wv[q];
          aa[q] = Axb[q] + nk[q];
        }
        prefetch(k + 1);  // the next panel's rows: the loads overlap the prox
        if (valid) {
          if (path_loss < 0) {
            softmax_prox_row<KC>(w, aa, yk, K, Mf, rho_l, newton_iters);
          } else {  // a path: K instances, each column its own scalar prox on target b_r
#pragma unroll
            for (int q = 0; q < KC; ++q)
              if (q < K) w[q] = omega_prox<float>(path_loss, aa[q], ybk, Mf, rho_l, newton_iters, w[q]);
          }
        }
        unsigned char* dbuf = ds + (k & 1) * 4096;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          float dv = 0.f;
          if (q < KC && q < K && valid) {
            const float nun = nk[q] + Axb[q] - w[q];
            omega[(row0 + r) * K + q] = w[q];
            nu[(row0 + r) * K + q] = nun;
            dv = w[q] - Axb[q] - nun;
            const float rr = Axb[q] - w[q];
            st_res = fmaf(rr, rr, st_res);
            st_om = fmaf(w[q], w[q], st_om);
            st_ax = fmaf(Axb[q], Axb[q], st_ax);
          }
          const __nv_bfloat16 hi = __float2bfloat16_rn(dv);
          const __nv_bfloat16 lo = __float2bfloat16_rn(dv - __bfloat162float(hi));
          if (has_row) {
            const uint32_t off = sw128_off(q, r);
            *reinterpret_cast<__nv_bfloat16*>(dbuf + off) = hi;
            *reinterpret_cast<__nv_bfloat16*>(dbuf + 2048 + off) = lo;
          }
        }
        fence_async_smem();
        tc_fence_before();
        mbar_arrive(&dready[k & 1]);
      }
      // end of a shard: every epilogue warp copies its 32 columns of each slab of D2
      if (k + 1 >= np || shard_of(k + 1) != shard) {
        if (!mbar_wait_or_abort(bwddone, static_cast<uint32_t>(seg & 1), wait_limit, abort_v)) { eok = false; break; }
        ++seg;
        tc_fence_after();
        float* dst = slots + static_cast<int64_t>(c + shard) * ldx;
        for (int sl = 0; sl < nslab; ++sl) {
          uint32_t u[16];
          tmem_ld16(tmem + lane_base + kTcD2Col + 16 * sl, u);
          const int64_t col = static_cast<int64_t>(sl) * 128 + tid;
          if (col < lda) {
#pragma unroll
            for (int q = 0; q < KC; ++q)
              if (q < K) dst[col * K + q] = __uint_as_float(u[q]);
          }
        }
        tc_fence_before();
        if (k + 1 < np) mbar_arrive(flushed);
      }
    }
    if (!eok) *abort_v = 1;
    st_res = warp_sum(st_res);
    st_om = warp_sum(st_om);
    st_ax = warp_sum(st_ax);
    if (lane == 0) {
      red[warp * 3 + 0] = st_res;
      red[warp * 3 + 1] = st_om;
      red[warp * 3 + 2] = st_ax;
    }
  }
  __syncthreads();

  if (*abort_v) {
    // Report, then let the copies and MMAs this CTA issued finish before freeing TMEM.
    if (tid == 0) {
      set_err(err, DEV_TIMEOUT_PASS);
      for (long long q = counts[1]; q < counts[0]; ++q)
        mbar_wait_bounded(&full[q % S], static_cast<uint32_t>((q / S) & 1), wait_limit);
    }
    if (warp == 5) {
      umma_commit_warp(drainbar);  // arrives once every MMA this warp issued has completed
      mbar_wait_bounded(drainbar, 0, wait_limit);
    }
    __syncthreads();
  }
  if (tid == 0) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int w = 0; w < 4; ++w) {
      s0 += static_cast<double>(red[w * 3 + 0]);
      s1 += static_cast<double>(red[w * 3 + 1]);
      s2 += static_cast<double>(red[w * 3 + 2]);
    }
    cta_stats[c * 4 + 0] = s0;
    cta_stats[c * 4 + 1] = s1;
    cta_stats[c * 4 + 2] = s2;
    cta_stats[c * 4 + 3] = 0.0;
  }
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kTcTmemCols);
  }
}

}  // namespace bic
