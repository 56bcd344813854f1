// Multi-class (softmax, K > 1 classes) kernels of one outer iteration.
//
// The decision variable is the n x K matrix W; every n-space vector holds it flattened
// feature-major (entry (c, k) at c*K + k, row stride ldx = lda*K per shard), so the
// consensus step, the duals and the residuals run unchanged on vectors of length n*K.
// What changes with K (Sec. 3.1 with K right-hand sides):
//   k_xupd_k        X_ij += P_ij R_ij, the same block inverse applied to K columns
//                   (eq. p:GPU;x)
//   k_fused_pass_k  per row r: Axbar_r = (1/M) a_r W_i (a K-vector), the softmax omega
//                   prox of eq. (p:GPU;omega) (a K-vector Newton solve), nu_r += Axbar_r -
//                   omega_r (eq. p:GPU;nu), d_r = omega_r - Axbar_r - nu_r, and the
//                   residual product Q_i += a_r' d_r (n x K) from the same smem panel.
// m-space arrays (b = class index per row; omega, nu m x K) are row-major in TM.
#pragma once

#include "common.cuh"
#include "nspace.cuh"
#include "pass.cuh"

namespace bic {

// Classes padded to the reduction width C (a power of two) used by the warp reductions.
template <int KC> struct ClassPad { static constexpr int C = KC <= 4 ? 4 : (KC <= 8 ? 8 : 16); };

// Setup check of the softmax labels: b_r integral and in [0, K).
template <typename TM>
__global__ void k_check_labels(const TM* __restrict__ b, int64_t m, int K, int* err) {
  for (int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; r < m;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const TM y = b[r];
    if (!(y >= TM(0) && y < TM(K) && y == floor(y))) set_err(err, DEV_BAD_LABEL);
  }
}

// ------------------------------------------------------------------------------ k_xupd_k
// Grid (row tiles of ROWS, M, N), XT threads, a warp on RB rows of P_ij at a time.  R_ij (n_j x K) is
// read in its own (column-major-in-K) order and staged transposed in shared memory,
// [KC][ldp + 4] (zero padded; the 4-element pad spreads the transposing stores over the
// banks), so a lane reads the K values of its VE consecutive columns as K 16-byte loads;
// the rows of P_ij are read in 16-byte vectors too.  The K dot products of a row are
// reduced with one warp reduce-scatter.
template <typename TP, int KC, int XT, int ROWS>
__global__ void __launch_bounds__(XT)
k_xupd_k(const TP* __restrict__ P, const int64_t* __restrict__ P_off,
         const int* __restrict__ blk_col0, const int* __restrict__ blk_ldp,
         const double* __restrict__ r, double* __restrict__ x, TP* __restrict__ xlo, int M,
         int64_t ldx, int K, unsigned char* __restrict__ wpk, int nslab) {
  using V = typename PVec<TP>::type;
  constexpr int VE = PVec<TP>::n;
  constexpr int C = ClassPad<KC>::C;
  extern __shared__ __align__(16) unsigned char rs_raw[];
  TP* rs = reinterpret_cast<TP*>(rs_raw);  // [KC][ldp + 4]
  const int i = blockIdx.z, j = blockIdx.y;
  const int col0 = blk_col0[j], nj = blk_col0[j + 1] - col0, ldp = blk_ldp[j];
  const int lds = ldp + 4;
  const int row_begin = blockIdx.x * ROWS;
  if (row_begin >= nj) return;
  for (int e = threadIdx.x; e < lds * KC; e += XT) rs[e] = TP(0);
  __syncthreads();
  const double* rsrc = r + i * ldx + static_cast<int64_t>(col0) * K;
  const int tot = nj * K;
  for (int e0 = threadIdx.x; e0 < tot; e0 += 4 * XT) {  // contiguous reads, four in flight
    double v4[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v4[u] = e0 + u * XT < tot ? rsrc[e0 + u * XT] : 0.0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = e0 + u * XT;
      if (e < tot) {
        const int bq = e / K, k = e - bq * K;
        rs[k * lds + bq] = static_cast<TP>(v4[u]);
      }
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const TP* Pb = P + P_off[i * M + j];
  const int nv = ldp / VE;
  // RB rows of P per warp pass: every R vector read from shared memory feeds RB rows (one
  // read per RB rows instead of per row, which made shared memory the bound)
  constexpr int RB = sizeof(TP) == 8 ? 2 : 4;
  for (int rb = row_begin + warp * RB; rb < row_begin + ROWS && rb < nj; rb += (XT / 32) * RB) {
    const V* pr[RB];
#pragma unroll
    for (int t = 0; t < RB; ++t)
      pr[t] = reinterpret_cast<const V*>(Pb + static_cast<int64_t>(rb + t < nj ? rb + t : rb) * ldp);
    TP accs[RB][C];
#pragma unroll
    for (int t = 0; t < RB; ++t)
#pragma unroll
      for (int k = 0; k < C; ++k) accs[t][k] = TP(0);
    for (int bv = lane; bv < nv; bv += 32) {
      V pv[RB];
#pragma unroll
      for (int t = 0; t < RB; ++t) pv[t] = pr[t][bv];
#pragma unroll
      for (int k = 0; k < KC; ++k) {
        const V rv = reinterpret_cast<const V*>(rs + k * lds)[bv];
        const TP* re = reinterpret_cast<const TP*>(&rv);
#pragma unroll
        for (int t = 0; t < RB; ++t) {
          const TP* pe = reinterpret_cast<const TP*>(&pv[t]);
#pragma unroll
          for (int e = 0; e < VE; ++e) accs[t][k] = fma(pe[e], re[e], accs[t][k]);
        }
      }
    }
#pragma unroll
    for (int tr = 0; tr < RB; ++tr) {
      const int row = rb + tr;
      if (row >= nj) break;  // warp-uniform
      const TP sum = warp_reduce_scatter<C>(accs[tr], lane);
      const int q = (lane >> (5 - (C == 4 ? 2 : (C == 8 ? 3 : 4)))) & (C - 1);
      if ((lane & ((32 / C) - 1)) == 0 && q < K) {
        const int64_t o = i * ldx + static_cast<int64_t>(col0 + row) * K + q;
        const double xn = x[o] + static_cast<double>(sum);
        x[o] = xn;
        xlo[o] = static_cast<TP>(xn);
        if (wpk) {
          // the same entry as BF16 hi/lo in the tensor-core pass's W tiles: per shard, per
          // 64-column box a 32 x 64 tile (rows 0-15 hi of the classes, 16-31 lo), 128-byte
          // swizzle; boxes in column order (two per 128-column slab)
          const int col = col0 + row;
          const float v = static_cast<float>(xn);
          const __nv_bfloat16 hi = __float2bfloat16_rn(v);
          const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
          unsigned char* t = wpk + (static_cast<int64_t>(i) * nslab * 2 + (col >> 6)) * 4096;
          *reinterpret_cast<__nv_bfloat16*>(t + sw128_off(q, col & 63)) = hi;
          *reinterpret_cast<__nv_bfloat16*>(t + sw128_off(q + 16, col & 63)) = lo;
        }
      }
    }
  }
}

// ------------------------------------------------------------------------ softmax prox
// Softmax omega-bar prox of eq. (p:GPU;omega) for one row on a half-warp (16 lanes; lane
// k < K holds class k):
//   argmin_w  CE(M w; y) + (M rho_l / 2) ||w - a||^2,   CE(q; y) = logsumexp(q) - q_y.
// Newton from w0 (the row's previous omega).  With p = softmax(M w), the Hessian is
// diag(D) - M^2 p p', D_k = M^2 p_k + M rho_l, and the Newton step follows from the
// Sherman-Morrison formula:
//   delta_k = (g_k + M^2 p_k t / den) / D_k,  t = sum p g / D,  den = M rho_l sum p / D
// (den written without the cancellation of 1 - M^2 sum p^2 / D, since sum p = 1).  Steps
// are damped by halving until ||g|| decreases (the Newton direction decreases ||g||^2);
// the loop ends when every |delta_k| is within a few ulps of w_k.  All lanes of the
// half-warp run the loop together: every branch depends only on half-warp reductions.
template <typename T>
struct HalfWarp {
  unsigned mask;
  __device__ __forceinline__ T sum(T v) const {
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, 16);
    return v;
  }
  __device__ __forceinline__ T max(T v) const {
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
      const T u = __shfl_xor_sync(mask, v, o, 16);
      v = u > v ? u : v;
    }
    return v;
  }
};

template <typename T>
__device__ __forceinline__ T softmax_prox(const HalfWarp<T>& hw, bool act, bool is_y, T a, T M,
                                          T rho_l, int newton_iters, T w0) {
  const T Mr = M * rho_l, M2 = M * M;
  T w = act ? w0 : T(0);
  T p, g, gn2;
  auto grad = [&](T wv, T& pk, T& gk) {
    const T q = M * wv;
    const T mx = hw.max(act ? q : -FpLim<T>::big);
    const T e = act ? dev_exp<T>(q - mx) : T(0);
    const T S = hw.sum(e);
    pk = e / S;
    gk = act ? M * (pk - (is_y ? T(1) : T(0))) + Mr * (wv - a) : T(0);
  };
  grad(w, p, g);
  gn2 = hw.sum(g * g);
  for (int it = 0; it < newton_iters; ++it) {
    const T D = M2 * p + Mr;
    const T t = hw.sum(act ? p * g / D : T(0));
    const T den = Mr * hw.sum(act ? p / D : T(0));
    const T delta = act ? (g + M2 * p * t / den) / D : T(0);
    const T aw = w < T(0) ? -w : w;
    const T ad = delta < T(0) ? -delta : delta;
    const bool small = ad <= T(4) * FpLim<T>::eps * (aw > T(1) ? aw : T(1));
    if (__all_sync(hw.mask, small)) break;
    T alpha = T(1), wt = w, pt = p, gt = g, gt2 = gn2;
    for (int bt = 0; bt < 40; ++bt) {
      wt = w - alpha * delta;
      grad(wt, pt, gt);
      gt2 = hw.sum(gt * gt);
      const T shrink = T(1) - T(1e-4) * alpha;
      if (gt2 <= shrink * shrink * gn2) break;
      alpha *= T(0.5);
    }
    w = wt;
    p = pt;
    g = gt;
    gn2 = gt2;
  }
  return w;
}

// ------------------------------------------------------------------------ k_fused_pass_k
// Same structure as k_fused_pass (persistent CTAs over contiguous panel ranges, one bulk
// TMA copy per panel into an S-stage mbarrier ring, slots flushed per shard, consensus in
// an extra CTA on the last sweep).  Thread tid owns the 16-byte vectors tid + kk*NT of a
// row (VE columns each) and holds W_i and the Q_i accumulators of those columns for all
// KC classes in registers.  Per panel row: KC partial dots, one warp reduce-scatter, the
// per-warp sums to shared memory; the epilogue (half-warp per row, lane per class) forms
// the row's K-vector, runs the softmax prox and writes d_r; the backward adds a_r d_r'.
template <typename TA, typename TM, int R, int VPT, int NT, int KC>
__global__ void __launch_bounds__(NT, 1)
k_fused_pass_k(const TA* __restrict__ A, int64_t lda, const TM* __restrict__ xlo, int64_t ldx,
               int K, const TM* __restrict__ b, TM* __restrict__ omega, TM* __restrict__ nu,
               TM* __restrict__ slots, double* __restrict__ cta_stats, PassGeometry geo, int S,
               TM Mf, TM rho_l, int newton_iters, int* __restrict__ err, long long wait_limit,
               ConsensusArgs cons, int path_loss) {
  static_assert(R <= NT / 16, "one half-warp per panel row in the epilogue");
  constexpr int C = ClassPad<KC>::C;
  constexpr int LOGC = C == 4 ? 2 : (C == 8 ? 3 : 4);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // the last consensus_ctas(cons) CTAs run the global step (one per instance of a path)
  if (cons.enabled && blockIdx.x >= gridDim.x - consensus_ctas(cons)) {
    const int q = blockIdx.x - (gridDim.x - consensus_ctas(cons));
    consensus_block<NT, kConsMW, true>(consensus_instance(cons, q), smem_raw);  // its dynamic smem holds the top-kappa candidates
    return;
  }
  using V = typename Vec16<TA>::type;
  constexpr int VE = Vec16<TA>::n;
  constexpr int NW = NT / 32;

  const int64_t nvec = lda / VE;
  const size_t stage_elems = static_cast<size_t>(R) * lda;
  TA* stages = reinterpret_cast<TA*>(smem_raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + S * stage_elems * sizeof(TA));
  TM* red = reinterpret_cast<TM*>(bars + S);  // [R][NW][C]
  TM* d_s = red + R * NW * C;                  // [R][C]

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

  int64_t n_issued = 0;
  int issue_shard = 0;
  auto issue = [&](int64_t k) {
    int64_t row0;
    int nrows;
    locate_panel<R>(geo, p_begin + k, issue_shard, row0, nrows);
    const int st = static_cast<int>(k % S);
    const uint32_t bytes = static_cast<uint32_t>(nrows * lda * sizeof(TA));
    mbar_arrive_expect_tx(&bars[st], bytes);
    bulk_copy_g2s(stages + st * stage_elems, A + row0 * lda, bytes, &bars[st]);
  };
  if (tid == 0) {
    for (; n_issued < np && n_issued < S; ++n_issued) issue(n_issued);
  }

  TM xr[VPT][VE][KC];
  TM acc[VPT][VE][KC];
  int cur = -1, shard = 0;
  TM st_res = TM(0), st_om = TM(0), st_ax = TM(0);

  auto flush = [&](int i) {
    TM* dst = slots + static_cast<int64_t>(c + i) * ldx;
#pragma unroll
    for (int kk = 0; kk < VPT; ++kk) {
      const int64_t v = tid + static_cast<int64_t>(kk) * NT;
      if (v < nvec) {
#pragma unroll
        for (int e = 0; e < VE; ++e)
#pragma unroll
          for (int k = 0; k < KC; ++k)
            if (k < K) dst[(v * VE + e) * K + k] = acc[kk][e][k];
      }
    }
  };

  // epilogue lane roles: half-warp hrow = tid / 16 takes row hrow, lane16 = class
  const int hrow = tid >> 4, cls = tid & 15;
  const HalfWarp<TM> hw{0xFFFFu << (lane & 16)};

  for (int64_t k = 0; k < np; ++k) {
    int64_t row0;
    int nrows;
    locate_panel<R>(geo, p_begin + k, shard, row0, nrows);
    if (shard != cur) {
      if (cur >= 0) flush(cur);
      cur = shard;
      const TM* xs = xlo + static_cast<int64_t>(shard) * ldx;
#pragma unroll
      for (int kk = 0; kk < VPT; ++kk) {
        const int64_t v = tid + static_cast<int64_t>(kk) * NT;
#pragma unroll
        for (int e = 0; e < VE; ++e)
#pragma unroll
          for (int q = 0; q < KC; ++q) {
            xr[kk][e][q] = (v < nvec && q < K) ? xs[(v * VE + e) * K + q] : TM(0);
            acc[kk][e][q] = TM(0);
          }
      }
    }
    // per-row scalars of the epilogue lane (previous omega warm-starts the prox)
    const bool erow = hrow < nrows;
    const bool act = erow && cls < K;
    TM y_r = TM(0), nu_r = TM(0), om_r = TM(0);
    if (erow) y_r = b[row0 + hrow];
    if (act) {
      nu_r = nu[(row0 + hrow) * K + cls];
      om_r = omega[(row0 + hrow) * K + cls];
    }
    const int st = static_cast<int>(k % S);
    const uint32_t parity = static_cast<uint32_t>((k / S) & 1);
    const bool ok = mbar_wait_bounded(&bars[st], parity, wait_limit);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        set_err(err, DEV_TIMEOUT_PASS);
        for (int64_t q = k; q < n_issued; ++q)
          mbar_wait_bounded(&bars[q % S], static_cast<uint32_t>((q / S) & 1), wait_limit);
      }
      return;
    }
    const V* sv = reinterpret_cast<const V*>(stages + st * stage_elems);

    // Forward: K partial dots per row, reduce-scattered across the warp.
#pragma unroll 1
    for (int r = 0; r < nrows; ++r) {
      TM part[C];
#pragma unroll
      for (int q = 0; q < C; ++q) part[q] = TM(0);
#pragma unroll
      for (int kk = 0; kk < VPT; ++kk) {
        const int64_t v = tid + static_cast<int64_t>(kk) * NT;
        if (v < nvec) {
          const V a = sv[r * nvec + v];
          const TA* ae = reinterpret_cast<const TA*>(&a);
#pragma unroll
          for (int e = 0; e < VE; ++e) {
            const TM av = conv<TM>(ae[e]);
#pragma unroll
            for (int q = 0; q < KC; ++q) part[q] = fma(av, xr[kk][e][q], part[q]);
          }
        }
      }
      const TM s = warp_reduce_scatter<C>(part, lane);
      if ((lane & ((32 >> LOGC) - 1)) == 0) red[(r * NW + warp) * C + (lane >> (5 - LOGC))] = s;
    }
    __syncthreads();

    // Epilogue: half-warp per row, lane per class (a half-warp is uniform in hrow).
    if (hrow < nrows) {
      TM tot = TM(0);
      if (act) {
#pragma unroll
        for (int w = 0; w < NW; ++w) tot += red[(hrow * NW + w) * C + cls];
      }
      const TM Axb = tot / Mf;
      const int y = static_cast<int>(y_r);
      // softmax: the row's K-vector prox; a path (path_loss >= 0): K instances, each lane's
      // column its own scalar prox on the row's target (path_loss is uniform: no divergence)
      const TM om = path_loss < 0
                        ? softmax_prox<TM>(hw, act, cls == y, Axb + nu_r, Mf, rho_l, newton_iters, om_r)
                        : (act ? omega_prox<TM>(path_loss, Axb + nu_r, y_r, Mf, rho_l, newton_iters, om_r) : TM(0));
      TM dval = TM(0);
      if (act) {
        const TM nun = nu_r + Axb - om;
        omega[(row0 + hrow) * K + cls] = om;
        nu[(row0 + hrow) * K + cls] = nun;
        dval = om - Axb - nun;
        const TM rr = Axb - om;
        st_res = fma(rr, rr, st_res);
        st_om = fma(om, om, st_om);
        st_ax = fma(Axb, Axb, st_ax);
      }
      if (cls < C) d_s[hrow * C + cls] = dval;  // C <= 16 entries per row
    }
    __syncthreads();

    // Backward: Q_i += A_panel' d (n x K).
#pragma unroll 1
    for (int r = 0; r < nrows; ++r) {
      TM dr[KC];
#pragma unroll
      for (int q = 0; q < KC; ++q) dr[q] = d_s[r * C + q];
#pragma unroll
      for (int kk = 0; kk < VPT; ++kk) {
        const int64_t v = tid + static_cast<int64_t>(kk) * NT;
        if (v < nvec) {
          const V a = sv[r * nvec + v];
          const TA* ae = reinterpret_cast<const TA*>(&a);
#pragma unroll
          for (int e = 0; e < VE; ++e) {
            const TM av = conv<TM>(ae[e]);
#pragma unroll
            for (int q = 0; q < KC; ++q) acc[kk][e][q] = fma(av, dr[q], acc[kk][e][q]);
          }
        }
      }
    }
    __syncthreads();  // every thread is done with this stage
    if (tid == 0 && n_issued < np) {
      issue(n_issued);
      ++n_issued;
    }
  }
  if (cur >= 0) flush(cur);

  st_res = warp_sum(st_res);
  st_om = warp_sum(st_om);
  st_ax = warp_sum(st_ax);
  __syncthreads();
  if (lane == 0) {
    red[warp * 3 + 0] = st_res;
    red[warp * 3 + 1] = st_om;
    red[warp * 3 + 2] = st_ax;
  }
  __syncthreads();
  if (tid == 0) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int w = 0; w < NW; ++w) {
      s0 += static_cast<double>(red[w * 3 + 0]);
      s1 += static_cast<double>(red[w * 3 + 1]);
      s2 += static_cast<double>(red[w * 3 + 2]);
    }
    cta_stats[c * 4 + 0] = s0;
    cta_stats[c * 4 + 1] = s1;
    cta_stats[c * 4 + 2] = s2;
    cta_stats[c * 4 + 3] = 0.0;
  }
}

// Shared-memory bytes of one k_fused_pass_k launch.
template <typename TA, typename TM>
inline size_t fused_pass_k_smem(int R, int S, int64_t lda, int NT, int C) {
  return static_cast<size_t>(S) * R * lda * sizeof(TA) + S * sizeof(uint64_t) +
         static_cast<size_t>(R) * (NT / 32 + 1) * C * sizeof(TM) + 16;
}

}  // namespace bic
