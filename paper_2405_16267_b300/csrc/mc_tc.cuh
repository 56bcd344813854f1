// Tensor-core (tcgen05) variant of the softmax A pass for BF16 storage, K <= 16 classes,
// rows of at most 2048 columns.  Same arithmetic as k_fused_pass_k (Sec. 3.1 with K
// right-hand sides: eqs. p:GPU;x, p:GPU;omega, p:GPU;nu), with the two products on the
// 5th-generation tensor cores:
//
//   forward   D1[128 x 16] = A_panel[128 x n] W_i[n x 16]            (row dots, FP32 in TMEM)
//   backward  D2[n x 16]  += A_panel'[n x 128] d_panel[128 x 16]      (A'd, FP32 in TMEM)
//
// A stays BF16.  W_i and d are split into BF16 pairs hi + lo (hi = bf16(v), lo =
// bf16(v - hi)) and both halves are accumulated into the same TMEM columns, so the
// products carry about 16 bits of the FP32 operand instead of 8.
//
// Data movement: a panel is 128 rows; the row is cut into 128-column slabs, each moved by
// two 2D TMA loads (64 x 128 boxes, 128-byte swizzle) into one 32 KB stage of an S-stage
// mbarrier ring.  The same swizzled slab serves as the K-major A operand of the forward
// (rows = M) and as the MN-major A operand of the backward (columns = M, two boxes LBO
// apart).  The backward needs d, which needs the whole forward, so each slab is loaded twice
// per panel: the second load normally hits L2 (one panel is 512 KB per SM).
//
// Roles: thread 0 issues TMA loads and tcgen05.mma; all four warps read TMEM (warp w owns
// TMEM lanes 32w..32w+31 = panel rows / slab columns) and run the per-row softmax prox.
// TMEM (512 columns): D1 at column 0, D2 slab c at column 32 + 16c.
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

// Byte offset of element (row q, column c) inside a tile of rows of 64 BF16 (128 bytes)
// with the 128-byte swizzle: the 16-byte chunk index is XORed with the row index mod 8.
__device__ __forceinline__ uint32_t sw128_off(int q, int c) {
  return static_cast<uint32_t>((q >> 3) * 1024 + (q & 7) * 128 + ((((c >> 3) ^ q) & 7) << 4) + (c & 7) * 2);
}

// ------------------------------------------------------------------ per-row softmax prox
// omega-bar prox of eq. (p:GPU;omega) for one row held by one thread (K classes in
// registers): argmin_w CE(M w; y) + (M rho_l / 2) ||w - a||^2.  Newton with the
// Sherman-Morrison step of the Hessian diag(M^2 p + M rho_l) - M^2 p p', damped by halving
// until ||g|| decreases, stopped once every step is within a few ulps of w.
template <int KC, typename T>
__device__ __forceinline__ void softmax_prox_row(T (&w)[KC], const T (&a)[KC], int y, int K, T M,
                                                 T rho_l, int newton_iters) {
  const T Mr = M * rho_l, M2 = M * M;
  T p[KC], g[KC];
  auto grad = [&](const T (&wv)[KC], T (&pk)[KC], T (&gk)[KC]) -> T {
    T mx = -FpLim<T>::big;
#pragma unroll
    for (int k = 0; k < KC; ++k)
      if (k < K) mx = fmax(mx, M * wv[k]);
    T S = T(0);
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      pk[k] = k < K ? dev_exp<T>(M * wv[k] - mx) : T(0);
      S += pk[k];
    }
    const T inv = T(1) / S;
    T gn = T(0);
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      pk[k] *= inv;
      gk[k] = k < K ? M * (pk[k] - (k == y ? T(1) : T(0))) + Mr * (wv[k] - a[k]) : T(0);
      gn = fma(gk[k], gk[k], gn);
    }
    return gn;
  };
  T gn2 = grad(w, p, g);
  for (int it = 0; it < newton_iters; ++it) {
    T D[KC], t = T(0), sp = T(0);
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      D[k] = M2 * p[k] + Mr;
      if (k < K) {
        t += p[k] * g[k] / D[k];
        sp += p[k] / D[k];
      }
    }
    const T coef = M2 * t / (Mr * sp);
    T delta[KC];
    bool small = true;
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      delta[k] = k < K ? (g[k] + coef * p[k]) / D[k] : T(0);
      const T aw = fabs(w[k]);
      small = small && fabs(delta[k]) <= T(4) * FpLim<T>::eps * (aw > T(1) ? aw : T(1));
    }
    if (small) break;
    T alpha = T(1), wt[KC], pt[KC], gt[KC], gt2 = gn2;
    for (int bt = 0; bt < 40; ++bt) {
#pragma unroll
      for (int k = 0; k < KC; ++k) wt[k] = w[k] - alpha * delta[k];
      gt2 = grad(wt, pt, gt);
      const T shrink = T(1) - T(1e-4) * alpha;
      if (gt2 <= shrink * shrink * gn2) break;
      alpha *= T(0.5);
    }
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
constexpr int kTcRows = 128;                       // panel rows = MMA M
constexpr int kTcThreads = 128;                    // 4 warps = the 128 TMEM lanes
constexpr int kTcStages = 2;
constexpr int kTcStageBytes = 2 * kTcRows * 128;   // two 64-column BF16 boxes
constexpr int kTcMaxSlabs = 16;                    // 128-column slabs: lda <= 2048
constexpr int kTcXBytes = kTcMaxSlabs * 2 * 2 * 2048;  // [box][split] 16 x 64 BF16 tiles
constexpr int kTcDBytes = 2 * 2 * 2048;            // [split][row half] 16 x 64 BF16 tiles
constexpr int kTcTmemCols = 512;
constexpr int kTcConsMW = 8;                       // consensus masks: n K <= 32 * 8 * 128

inline size_t fused_pass_tc_smem() {
  return 1024 + static_cast<size_t>(kTcStages) * kTcStageBytes + kTcXBytes + kTcDBytes + 256;
}

template <int KC>
__global__ void __launch_bounds__(kTcThreads, 1)
k_fused_pass_tc(const __grid_constant__ CUtensorMap tmap, int64_t lda, const float* __restrict__ xlo,
                int64_t ldx, int K, const float* __restrict__ b, float* __restrict__ omega,
                float* __restrict__ nu, float* __restrict__ slots, double* __restrict__ cta_stats,
                PassGeometry geo, float Mf, float rho_l, int newton_iters, int* __restrict__ err,
                long long wait_limit, ConsensusArgs cons) {
  if (cons.enabled && blockIdx.x == gridDim.x - 1) {
    consensus_block<kTcThreads, kTcConsMW>(cons);
    return;
  }
  constexpr int S = kTcStages;
  constexpr uint32_t IDESC_FWD = idesc_bf16(128, 16, false, false);
  constexpr uint32_t IDESC_BWD = idesc_bf16(128, 16, true, false);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment for the swizzled tiles
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  unsigned char* ring = base;
  unsigned char* xs = ring + S * kTcStageBytes;
  unsigned char* ds = xs + kTcXBytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(ds + kTcDBytes);
  uint64_t* empty = full + S;
  uint64_t* d1bar = empty + S;
  uint64_t* bwdbar = d1bar + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bwdbar + 1);
  float* red = reinterpret_cast<float*>(tmem_slot + 4);  // [4 warps][3]

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c = blockIdx.x, G = gridDim.x - (cons.enabled ? 1 : 0);
  const int64_t p_begin = static_cast<int64_t>(c) * geo.P / G;
  const int64_t p_end = static_cast<int64_t>(c + 1) * geo.P / G;
  const int64_t np = p_end - p_begin;
  const int nslab = static_cast<int>((lda + 127) / 128);
  const int64_t nload = np * 2 * nslab;

  if (tid == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], 1);
    }
    mbar_init(d1bar, 1);
    mbar_init(bwdbar, 1);
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
  const uint32_t lane_base = static_cast<uint32_t>(warp * 32) << 16;

  // producer state (thread 0)
  int64_t j_issue = 0, j_cons = 0;
  int issue_shard = 0;
  auto issue = [&](int64_t j) -> bool {
    const int st = static_cast<int>(j % S);
    if (j >= S && !mbar_wait_bounded(&empty[st], static_cast<uint32_t>(((j / S) - 1) & 1), wait_limit))
      return false;
    const int64_t k = j / (2 * nslab);
    const int sl = static_cast<int>(j % nslab);
    int64_t row0;
    int nr;
    locate_panel<kTcRows>(geo, p_begin + k, issue_shard, row0, nr);
    unsigned char* dst = ring + st * kTcStageBytes;
    mbar_arrive_expect_tx(&full[st], kTcStageBytes);
    tma_load_2d(dst, &tmap, sl * 128, static_cast<int>(row0), &full[st]);
    tma_load_2d(dst + kTcStageBytes / 2, &tmap, sl * 128 + 64, static_cast<int>(row0), &full[st]);
    return true;
  };

  bool ok = true;
  if (tid == 0) {
    for (; j_issue < nload && j_issue < S; ++j_issue) ok = ok && issue(j_issue);
  }

  uint32_t d1_phase = 0, bwd_phase = 0;
  int cur = -1, shard = 0;
  bool first_bwd = true;
  float st_res = 0.f, st_om = 0.f, st_ax = 0.f;

  // Wait until every issued MMA has completed, then copy the D2 accumulators of shard i to
  // its slot (column col = 128 slab + TMEM lane, classes along TMEM columns).
  auto flush = [&](int i) -> bool {
    if (tid == 0) umma_commit(bwdbar);
    const bool w_ok = mbar_wait_bounded(bwdbar, bwd_phase, wait_limit);
    bwd_phase ^= 1u;
    tc_fence_after();
    float* dst = slots + static_cast<int64_t>(c + i) * ldx;
    for (int sl = 0; sl < nslab; ++sl) {
      uint32_t v[16];
      tmem_ld16(tmem + lane_base + 32 + 16 * sl, v);
      const int64_t col = static_cast<int64_t>(sl) * 128 + warp * 32 + lane;
      if (col < lda) {
#pragma unroll
        for (int k = 0; k < KC; ++k)
          if (k < K) dst[col * K + k] = __uint_as_float(v[k]);
      }
    }
    tc_fence_before();
    return w_ok;
  };

  for (int64_t k = 0; k < np && ok; ++k) {
    int64_t row0;
    int nrows;
    locate_panel<kTcRows>(geo, p_begin + k, shard, row0, nrows);
    if (shard != cur) {
      if (cur >= 0) ok = flush(cur) && ok;
      // W_i of the new shard as BF16 hi/lo tiles [box][split][16 classes x 64 columns]
      const float* xsrc = xlo + static_cast<int64_t>(shard) * ldx;
      for (int e = tid; e < nslab * 128 * 16; e += kTcThreads) {
        const int col = e >> 4, q = e & 15;
        const float v = (col < lda && q < K) ? xsrc[static_cast<int64_t>(col) * K + q] : 0.f;
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
        const int bx = col >> 6;
        const uint32_t off = sw128_off(q, col & 63);
        *reinterpret_cast<__nv_bfloat16*>(xs + (bx * 2 + 0) * 2048 + off) = hi;
        *reinterpret_cast<__nv_bfloat16*>(xs + (bx * 2 + 1) * 2048 + off) = lo;
      }
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      cur = shard;
      first_bwd = true;
    }

    // ---- forward: D1 = A_panel W_i (hi + lo)
    if (tid == 0 && ok) {
      for (int sl = 0; sl < nslab && ok; ++sl) {
        const int st = static_cast<int>(j_cons % S);
        if (!mbar_wait_bounded(&full[st], static_cast<uint32_t>((j_cons / S) & 1), wait_limit)) { ok = false; break; }
        tc_fence_after();
        const uint32_t sa = smem_addr(ring + st * kTcStageBytes);
#pragma unroll
        for (int bx = 0; bx < 2; ++bx)
#pragma unroll
          for (int sp = 0; sp < 2; ++sp)
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
              const uint64_t ad = sdesc_sw128(sa + bx * (kTcStageBytes / 2) + ks * 32, 16, 1024);
              const uint64_t bd = sdesc_sw128(smem_addr(xs + ((sl * 2 + bx) * 2 + sp) * 2048) + ks * 32, 16, 1024);
              umma_bf16(tmem, ad, bd, IDESC_FWD, (sl | bx | sp | ks) != 0 ? 1u : 0u);
            }
        umma_commit(&empty[st]);
        ++j_cons;
        if (j_issue < nload) { ok = issue(j_issue) && ok; ++j_issue; }
      }
      umma_commit(d1bar);
    }
    ok = __syncthreads_and(ok);
    if (!ok) break;
    ok = mbar_wait_bounded(d1bar, d1_phase, wait_limit);
    d1_phase ^= 1u;
    tc_fence_after();

    // ---- epilogue: thread = panel row
    {
      uint32_t v[16];
      tmem_ld16(tmem + lane_base, v);
      const int r = tid;
      const bool valid = r < nrows;
      float Axb[KC], aa[KC], w[KC], nur[KC];
#pragma unroll
      for (int q = 0; q < KC; ++q) {
        Axb[q] = __uint_as_float(v[q]) / Mf;
        nur[q] = (valid && q < K) ? nu[(row0 + r) * K + q] : 0.f;
        w[q] = (valid && q < K) ? omega[(row0 + r) * K + q] : 0.f;
        aa[q] = Axb[q] + nur[q];
      }
      const int y = valid ? static_cast<int>(b[row0 + r]) : 0;
      if (valid) softmax_prox_row<KC, float>(w, aa, y, K, Mf, rho_l, newton_iters);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        float dv = 0.f;
        if (q < KC && q < K && valid) {
          const float nun = nur[q] + Axb[q] - w[q];
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
        // d tile: [split][row half][16 classes x 64 rows], K-major (rows contiguous)
        const uint32_t off = sw128_off(q, r & 63) + (r >> 6) * 2048;
        *reinterpret_cast<__nv_bfloat16*>(ds + off) = hi;
        *reinterpret_cast<__nv_bfloat16*>(ds + 4096 + off) = lo;
      }
    }
    fence_async_smem();
    tc_fence_before();
    ok = __syncthreads_and(ok);
    if (!ok) break;

    // ---- backward: D2[slab] += A_slab' d (hi + lo)
    if (tid == 0) {
      tc_fence_after();
      for (int sl = 0; sl < nslab && ok; ++sl) {
        const int st = static_cast<int>(j_cons % S);
        if (!mbar_wait_bounded(&full[st], static_cast<uint32_t>((j_cons / S) & 1), wait_limit)) { ok = false; break; }
        tc_fence_after();
        const uint32_t sa = smem_addr(ring + st * kTcStageBytes);
#pragma unroll
        for (int sp = 0; sp < 2; ++sp)
#pragma unroll
          for (int ks = 0; ks < 8; ++ks) {
            const uint64_t ad = sdesc_sw128(sa + ks * 2048, kTcStageBytes / 2, 1024);
            const uint64_t bd = sdesc_sw128(smem_addr(ds + sp * 4096 + (ks >> 2) * 2048) + (ks & 3) * 32, 16, 1024);
            umma_bf16(tmem + 32 + 16 * sl, ad, bd, IDESC_BWD, (first_bwd && sp == 0 && ks == 0) ? 0u : 1u);
          }
        umma_commit(&empty[st]);
        ++j_cons;
        if (j_issue < nload) { ok = issue(j_issue) && ok; ++j_issue; }
      }
    }
    first_bwd = false;
    ok = __syncthreads_and(ok);
  }
  if (ok && cur >= 0) ok = flush(cur) && ok;
  ok = __syncthreads_and(ok);

  if (!ok) {
    // Report, then let this CTA's copies and MMAs in flight finish before freeing TMEM.
    if (tid == 0) {
      set_err(err, DEV_TIMEOUT_PASS);
      for (int64_t q = j_cons; q < j_issue; ++q)
        mbar_wait_bounded(&full[q % S], static_cast<uint32_t>((q / S) & 1), wait_limit);
      umma_commit(bwdbar);
      mbar_wait_bounded(bwdbar, bwd_phase, wait_limit);
    }
    __syncthreads();
  }

  st_res = warp_sum(st_res);
  st_om = warp_sum(st_om);
  st_ax = warp_sum(st_ax);
  if (lane == 0) {
    red[warp * 3 + 0] = st_res;
    red[warp * 3 + 1] = st_om;
    red[warp * 3 + 2] = st_ax;
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int w = 0; w < kTcThreads / 32; ++w) {
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
