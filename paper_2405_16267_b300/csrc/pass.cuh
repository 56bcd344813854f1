// Fused A pass: one streaming read of A per inner sweep of the sharing ADMM (Sec. 3.1).
//
// For every row r of shard i (rows grouped in panels of R consecutive rows):
//   Axbar_r = (1/M) a_r . x_i                     block products summed over j (Alg. 2 "Allreduce")
//   omega_r = prox of l(M w; b_r) at Axbar_r+nu_r eq. (p:GPU;omega), separable per row
//   nu_r   += Axbar_r - omega_r                    eq. (p:GPU;nu)
//   d_r     = omega_r - Axbar_r - nu_r             the target shift of eq. (p:GPU;x)
// and the residual product q_i = A_i' d_i is accumulated from the same panel while it is
// still in shared memory.  q_i feeds the next x_ij solve:
//   x_ij += P_ij (rho_l q_ij + rho_c (z_j - u_ij) - c0 x_ij),  P_ij = (rho_l A_ij'A_ij + c0 I)^-1,
// which equals eq. (p:GPU;x) because A_ij'(A_ij x_ij + d_i) = G_ij x_ij + q_ij and
// P_ij rho_l G_ij = I - c0 P_ij.
//
// Data movement: panels are contiguous (row stride lda, a multiple of 32 elements), so one
// bulk TMA copy moves a whole panel into a shared-memory stage; S stages per CTA are kept
// in flight behind mbarriers.  Each CTA is persistent over a contiguous range of panels;
// its A'd partial sums live in registers (VPT 16-byte vectors per thread) and are flushed
// to slot (cta + shard) whenever the CTA leaves a shard.  Slots are summed in a fixed order
// by the next kernel, so results are deterministic.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "nspace.cuh"

namespace bic {

enum : int { LOSS_SQUARED = 0, LOSS_LOGISTIC = 1, LOSS_SOFTMAX = 2, LOSS_SQHINGE = 3 };

template <typename T> struct FpLim;
template <> struct FpLim<float> {
  static constexpr float eps = 1.1920929e-7f;
  static constexpr float tiny = 1.17549435e-38f;
  static constexpr float big = 3.4028234e38f;
};
template <> struct FpLim<double> {
  static constexpr double eps = 2.220446049250313e-16;
  static constexpr double tiny = 2.2250738585072014e-308;
  static constexpr double big = 1.7976931348623157e308;
};

template <typename T> __device__ __forceinline__ T dev_exp(T x);
template <> __device__ __forceinline__ float dev_exp<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double dev_exp<double>(double x) { return exp(x); }

// Quotient for a Newton step (its rounding does not enter the root: the bracket and the
// stopping test use phi' itself): the fast approximate division in FP32.
template <typename T> __device__ __forceinline__ T step_div(T g, T h);
template <> __device__ __forceinline__ float step_div<float>(float g, float h) { return __fdividef(g, h); }
template <> __device__ __forceinline__ double step_div<double>(double g, double h) { return g / h; }

// omega-bar prox of eq. (p:GPU;omega) for one row:
//   argmin_w  l(M w; b) + (M rho_l / 2) (w - a)^2,
// w0: a starting point (the previous outer iteration's omega for this row).
template <typename T>
__device__ __forceinline__ T omega_prox(int loss, T a, T b, T M, T rho_l, int newton_iters, T w0) {
  if (loss == LOSS_SQUARED) return (T(2) * b + rho_l * a) / (T(2) * M + rho_l);
  if (loss == LOSS_SQHINGE) {
    if (T(1) - b * M * a > T(0)) return (T(2) * b + rho_l * a) / (T(2) * M + rho_l);
    return a;
  }
  // Logistic: phi'(w) = -b M sig(-b M w) + M rho_l (w - a) is increasing with its root in
  // [min(a, a + b/rho_l), max(...)].  Safeguarded Newton: a bisection step replaces the
  // Newton step when the latter leaves the bracket or does not shrink at least half as fast
  // as bisection would (plain Newton can cycle on this function); the bracket follows the
  // sign of phi'.  Stops once the step is below a few ulps of the bracket's scale.
  const T step0 = b / rho_l;
  T lo = a < a + step0 ? a : a + step0;
  T hi = a < a + step0 ? a + step0 : a;
  const T scale = (a < T(0) ? -a : a) + (step0 < T(0) ? -step0 : step0);
  const T stop = T(4) * FpLim<T>::eps * scale;
  T w = w0 > lo ? (w0 < hi ? w0 : hi) : lo;
  T dx_old = hi - lo, dx = dx_old;
  for (int it = 0; it < newton_iters; ++it) {
    const T sg = T(1) / (T(1) + dev_exp<T>(b * M * w));   // sigma(-b M w)
    const T g = -b * M * sg + M * rho_l * (w - a);
    if (g == T(0)) break;  // landed on the root
    const T h = M * M * sg * (T(1) - sg) + M * rho_l;
    if (g > T(0)) hi = w; else lo = w;
    T wn = w - step_div<T>(g, h);
    const T ag2 = g < T(0) ? T(-2) * g : T(2) * g;
    const T adh = (dx_old < T(0) ? -dx_old : dx_old) * h;
    if (!(wn >= lo && wn <= hi) || ag2 > adh) {
      dx_old = dx;
      dx = T(0.5) * (hi - lo);
      wn = lo + dx;
    } else {
      dx_old = dx;
      dx = w - wn;
    }
    w = wn;
    if ((dx < T(0) ? -dx : dx) <= stop || hi - lo <= stop) break;
  }
  return w;
}

struct PassGeometry {
  const int64_t* shard_row0;   // N + 1 row offsets of the shards
  const int64_t* panel_start;  // N + 1 first panel index of each shard
  int N;
  int64_t P;                   // total panels
  int64_t stall_panel;         // test hook: this panel's load is never posted (-1: none)
};

// Locate panel p: its shard i (searching forward from `hint`), first row and row count.
template <int R>
__device__ __forceinline__ void locate_panel(const PassGeometry& g, int64_t p, int& i,
                                             int64_t& row0, int& nrows) {
  while (i + 1 < g.N && g.panel_start[i + 1] <= p) ++i;
  row0 = g.shard_row0[i] + (p - g.panel_start[i]) * R;
  const int64_t rem = g.shard_row0[i + 1] - row0;
  nrows = rem < R ? static_cast<int>(rem) : R;
}

// Consensus-step mask words for NT threads: n <= 32 * kConsMW * NT.
constexpr int kConsMW = 4;

// FP32 storage with few vectors per thread: the forward keeps the thread's vectors of the
// panel in registers for the backward, so the stage is released (and the panel S ahead is
// loaded into it) right after the forward, while the row epilogue and the backward run.
// Taken when x, the A'd sums and the held vectors fit the 128 registers of two CTAs per SM
// (estimate: 4-byte words of x and A'd, 4 per held vector, 40 for the rest).
template <typename TA, int R, int VPT>
__host__ __device__ constexpr bool pass_holds_panel() {
  return sizeof(TA) == 4 && 2 * VPT * 4 + 4 * R * VPT + 40 <= 128;
}

template <typename TA, typename TM, int R, int VPT, int NT>
__global__ void __launch_bounds__(NT, pass_holds_panel<TA, R, VPT>() ? 2 : 1)
k_fused_pass(const TA* __restrict__ A, int64_t lda, const TM* __restrict__ xlo_in,
             const TM* __restrict__ b, TM* __restrict__ omega, TM* __restrict__ nu,
             TM* __restrict__ slots, double* __restrict__ cta_stats, PassGeometry geo,
             int S, int loss, TM Mf, TM rho_l, int newton_iters, int* __restrict__ err,
             long long wait_limit, ConsensusArgs cons) {
  // x_i is held in the storage type when it is the arithmetic type (FP32, FP64) and in the
  // arithmetic type otherwise (BF16 storage).
  using XT = typename std::conditional<std::is_same<TA, __nv_bfloat16>::value, TM, TA>::type;
  const XT* xlo = reinterpret_cast<const XT*>(xlo_in);
  // With cons.enabled the last CTA runs the global (z, t, s, v) step of this outer
  // iteration, which needs only x and u, concurrently with the A stream of the others.
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // the last consensus_ctas(cons) CTAs run the global step (one per instance of a path)
  if (cons.enabled && blockIdx.x >= gridDim.x - consensus_ctas(cons)) {
    const int q = blockIdx.x - (gridDim.x - consensus_ctas(cons));
    consensus_block<NT, kConsMW>(consensus_instance(cons, q), smem_raw);  // its dynamic smem holds the top-kappa candidates
    return;
  }
  using V = typename Vec16<TA>::type;
  constexpr int VE = Vec16<TA>::n;
  constexpr int NW = NT / 32;

  const int64_t nvec = lda / VE;
  const size_t stage_elems = static_cast<size_t>(R) * lda;
  TA* stages = reinterpret_cast<TA*>(smem_raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + S * stage_elems * sizeof(TA));
  TM* red = reinterpret_cast<TM*>(bars + S);  // [R][NW]
  TM* d_s = red + R * NW;                     // [R]

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c = blockIdx.x, G = gridDim.x - consensus_ctas(cons);
  const int64_t p_begin = static_cast<int64_t>(c) * geo.P / G;
  const int64_t p_end = static_cast<int64_t>(c + 1) * geo.P / G;
  const int64_t np = p_end - p_begin;

  if (tid == 0) {
    for (int st = 0; st < S; ++st) mbar_init(&bars[st], 1);
    fence_barrier_init();
  }
  __syncthreads();

  // Producer state (thread 0 only): next panel to issue and its shard hint.
  int64_t n_issued = 0;
  int issue_shard = 0;
  auto issue = [&](int64_t k) {
    int64_t row0;
    int nrows;
    locate_panel<R>(geo, p_begin + k, issue_shard, row0, nrows);
    const int st = static_cast<int>(k % S);
    if (p_begin + k == geo.stall_panel) return;  // test hook: no transaction, no copy
    const uint32_t bytes = static_cast<uint32_t>(nrows * lda * sizeof(TA));
    mbar_arrive_expect_tx(&bars[st], bytes);
    bulk_copy_g2s(stages + st * stage_elems, A + row0 * lda, bytes, &bars[st]);
  };
  if (tid == 0) {
    for (; n_issued < np && n_issued < S; ++n_issued) issue(n_issued);
  }

  XT xr[VPT][VE];
  TM acc[VPT][VE];
  int cur = -1, shard = 0;

  TM st_res = TM(0), st_om = TM(0), st_ax = TM(0);  // lane r of warp 0: inner-residual sums

  auto flush = [&](int i) {
    TM* dst = slots + static_cast<int64_t>(c + i) * lda;
#pragma unroll
    for (int kk = 0; kk < VPT; ++kk) {
      const int64_t v = tid + static_cast<int64_t>(kk) * NT;
      if (v < nvec) {
#pragma unroll
        for (int e = 0; e < VE; ++e) dst[v * VE + e] = acc[kk][e];
      }
    }
  };

  for (int64_t k = 0; k < np; ++k) {
    int64_t row0;
    int nrows;
    locate_panel<R>(geo, p_begin + k, shard, row0, nrows);
    if (shard != cur) {
      if (cur >= 0) flush(cur);
      cur = shard;
#pragma unroll
      for (int kk = 0; kk < VPT; ++kk) {
        const int64_t v = tid + static_cast<int64_t>(kk) * NT;
        if constexpr (std::is_same<XT, TA>::value) {  // one 16-byte load per vector
          const V* xv = reinterpret_cast<const V*>(xlo + static_cast<int64_t>(shard) * lda);
          V t;
          if (v < nvec) t = xv[v]; else t = V{};
          const TA* te = reinterpret_cast<const TA*>(&t);
#pragma unroll
          for (int e = 0; e < VE; ++e) { xr[kk][e] = te[e]; acc[kk][e] = TM(0); }
        } else {
          const XT* xs = xlo + static_cast<int64_t>(shard) * lda;
#pragma unroll
          for (int e = 0; e < VE; ++e) {
            xr[kk][e] = v < nvec ? xs[v * VE + e] : XT(0);
            acc[kk][e] = TM(0);
          }
        }
      }
    }
    // Per-row scalars for the epilogue (the previous omega warm-starts the prox).
    TM b_r = TM(0), nu_r = TM(0), om_r = TM(0);
    if (warp == 0 && lane < nrows) {
      b_r = b[row0 + lane];
      nu_r = nu[row0 + lane];
      om_r = omega[row0 + lane];
    }
    const int st = static_cast<int>(k % S);
    const uint32_t parity = static_cast<uint32_t>((k / S) & 1);
    const bool ok = mbar_wait_bounded(&bars[st], parity, wait_limit);
    if (__syncthreads_or(!ok)) {
      // Give up: report, then let every copy in flight land before exiting (each with the
      // full wait limit, whatever limit the pass ran with; a panel whose load was never
      // posted has nothing to wait for).
      if (tid == 0) {
        set_err(err, DEV_TIMEOUT_PASS);
        for (int64_t q = k; q < n_issued; ++q) {
          if (p_begin + q == geo.stall_panel) continue;
          mbar_wait_bounded(&bars[q % S], static_cast<uint32_t>((q / S) & 1), kWaitLimitCycles);
        }
      }
      return;
    }
    const V* sv = reinterpret_cast<const V*>(stages + st * stage_elems);

    // Forward: partial dots of the panel rows with x_i.
    constexpr bool kHoldA = pass_holds_panel<TA, R, VPT>();
    V areg[kHoldA ? VPT : 1][kHoldA ? R : 1];
    TM dot[R];
#pragma unroll
    for (int r = 0; r < R; ++r) dot[r] = TM(0);
#pragma unroll
    for (int kk = 0; kk < VPT; ++kk) {
      const int64_t v = tid + static_cast<int64_t>(kk) * NT;
      if (v < nvec) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (r < nrows) {
            const V a = sv[r * nvec + v];
            if constexpr (kHoldA) areg[kk][r] = a;
            const TA* ae = reinterpret_cast<const TA*>(&a);
#pragma unroll
            for (int e = 0; e < VE; ++e) dot[r] = fma(conv<TM>(ae[e]), conv<TM>(xr[kk][e]), dot[r]);
          }
        }
      }
    }
    if constexpr ((R & (R - 1)) == 0) {
      // the warp's R row sums in one reduce-scatter: lane r (32 / R) holds row r's
      const TM dsum = warp_reduce_scatter<R>(dot, lane);
      if ((lane & (32 / R - 1)) == 0) red[(lane / (32 / R)) * NW + warp] = dsum;
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) dot[r] = warp_sum(dot[r]);
      if (lane == 0) {
#pragma unroll
        for (int r = 0; r < R; ++r) red[r * NW + warp] = dot[r];
      }
    }
    __syncthreads();
    if constexpr (kHoldA) {  // every thread holds its part of the panel: reload the stage
      if (tid == 0 && n_issued < np) {
        issue(n_issued);
        ++n_issued;
      }
    }

    // Row epilogue: mean block product, omega prox, nu update, target shift d.
    if (warp == 0) {
      // row totals: lanes [r*NW, (r+1)*NW) hold row r's per-warp partials; reduce in groups
      TM tot = TM(0);
#pragma unroll
      for (int base = 0; base < R * NW; base += 32) {
        TM pv = base + lane < R * NW ? red[base + lane] : TM(0);
#pragma unroll
        for (int off = NW / 2; off > 0; off >>= 1) pv += __shfl_xor_sync(0xffffffffu, pv, off);
#pragma unroll
        for (int rr = 0; rr < 32 / NW; ++rr) {
          const TM t = __shfl_sync(0xffffffffu, pv, rr * NW);
          if (lane == base / NW + rr) tot = t;
        }
      }
      if (lane < nrows) {
      const TM Axb = tot / Mf;
      const TM om = omega_prox<TM>(loss, Axb + nu_r, b_r, Mf, rho_l, newton_iters, om_r);
      const TM nun = nu_r + Axb - om;
      omega[row0 + lane] = om;
      nu[row0 + lane] = nun;
      d_s[lane] = om - Axb - nun;
      const TM rr = Axb - om;
      st_res = fma(rr, rr, st_res);
      st_om = fma(om, om, st_om);
      st_ax = fma(Axb, Axb, st_ax);
      }
    }
    __syncthreads();

    // Backward: q_i += A_panel' d.
    TM dr[R];
#pragma unroll
    for (int r = 0; r < R; ++r) dr[r] = r < nrows ? d_s[r] : TM(0);
#pragma unroll
    for (int kk = 0; kk < VPT; ++kk) {
      const int64_t v = tid + static_cast<int64_t>(kk) * NT;
      if (v < nvec) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (r < nrows) {
            V a;
            if constexpr (kHoldA) a = areg[kk][r]; else a = sv[r * nvec + v];
            const TA* ae = reinterpret_cast<const TA*>(&a);
#pragma unroll
            for (int e = 0; e < VE; ++e) acc[kk][e] = fma(dr[r], conv<TM>(ae[e]), acc[kk][e]);
          }
        }
      }
    }
    if constexpr (!kHoldA) {
      __syncthreads();  // every thread is done with this stage
      if (tid == 0 && n_issued < np) {
        issue(n_issued);
        ++n_issued;
      }
    }
  }
  if (cur >= 0) flush(cur);

  if (warp == 0) {
    st_res = warp_sum(st_res);
    st_om = warp_sum(st_om);
    st_ax = warp_sum(st_ax);
    if (lane == 0) {
      cta_stats[c * 4 + 0] = static_cast<double>(st_res);
      cta_stats[c * 4 + 1] = static_cast<double>(st_om);
      cta_stats[c * 4 + 2] = static_cast<double>(st_ax);
      cta_stats[c * 4 + 3] = 0.0;
    }
  }
}

// Shared-memory bytes of one k_fused_pass launch.
template <typename TA, typename TM>
inline size_t fused_pass_smem(int R, int S, int64_t lda, int NT) {
  return static_cast<size_t>(S) * R * lda * sizeof(TA) + S * sizeof(uint64_t) +
         static_cast<size_t>(R) * (NT / 32 + 1) * sizeof(TM) + 16;
}

}  // namespace bic
