// Polish (not part of the paper's algorithm): after the iterations, the model restricted to
// the support S = the kappa largest |z_r| (ties to the lowest index) is re-fitted in FP64,
//
//     minimise_{supp x in S}  sum_r l(a_r x; b_r) + ||x||^2 / (2 gamma),
//
// by damped Newton: H = A_S' diag(l'') A_S + I/gamma, g = A_S' l' + x/gamma, step = H^-1 g,
// backtracking on the objective.  The squared loss is quadratic, so its first full step is
// exact.  A_S is gathered once into a column-major FP64 buffer (kappa x m).
#pragma once

#include "common.cuh"
#include "nspace.cuh"

namespace bic {

// Loss value and first/second derivatives of l(q; b) for one row.
__device__ __forceinline__ void row_loss(int loss, double q, double b, double& f, double& d1,
                                         double& d2) {
  if (loss == 0) {  // squared (q - b)^2
    const double r = q - b;
    f = r * r;
    d1 = 2.0 * r;
    d2 = 2.0;
  } else if (loss == 1) {  // logistic log(1 + exp(-b q))
    const double y = -b * q;
    const double sg = 1.0 / (1.0 + exp(-y));           // sigma(-b q)
    f = y > 0.0 ? y + log1p(exp(-y)) : log1p(exp(y));  // softplus(y)
    d1 = -b * sg;
    d2 = sg * (1.0 - sg);
  } else {  // squared hinge max(0, 1 - b q)^2
    const double t = 1.0 - b * q;
    f = t > 0.0 ? t * t : 0.0;
    d1 = t > 0.0 ? -2.0 * b * t : 0.0;
    d2 = t > 0.0 ? 2.0 : 0.0;
  }
}

// The kappa-support of z, ascending, into supp[kappa] (one CTA of GT threads).
template <int GT, int MW>
__global__ void __launch_bounds__(GT, 1)
k_support(const double* __restrict__ z, uint64_t* __restrict__ key, int64_t n, int64_t kappa,
          int64_t* __restrict__ supp) {
  __shared__ unsigned int wsum2[32];
  int64_t cb;
  int cl;
  uint32_t sel[MW];
  block_topk_select<GT, MW>(z, key, n, kappa, sel, cb, cl);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned int cnt = 0;
  for (int q = 0; q < cl; ++q) cnt += sel[q >> 5] >> (q & 31) & 1u;
  unsigned int incl = cnt;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned int y = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += y;
  }
  if (lane == 31) wsum2[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const unsigned int v = lane < GT / 32 ? wsum2[lane] : 0u;
    unsigned int inc = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += y;
    }
    wsum2[lane] = inc - v;
  }
  __syncthreads();
  unsigned int pos = wsum2[warp] + incl - cnt;
  for (int q = 0; q < cl; ++q)
    if (sel[q >> 5] >> (q & 31) & 1u) supp[pos++] = cb + q;
}

// AS[k*m + r] = A[r, supp[k] / K] in FP64 (K = 1: the support's columns; softmax: the
// feature of each support entry (c, class) = c K + class).  Grid (row chunks, kappa).
template <typename TA>
__global__ void k_gather_support(const TA* __restrict__ A, int64_t lda, const int64_t* __restrict__ supp,
                                 int64_t m, double* __restrict__ AS, int K = 1) {
  const int k = blockIdx.y;
  const int64_t col = supp[k] / K;
  for (int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; r < m;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x)
    AS[k * m + r] = conv<double>(A[r * lda + col]);
}

// Per row: q = a_S . x (x: kappa doubles), loss derivatives; per-CTA partial objective.
// With alpha != 0 evaluates the trial point instead: q - alpha p (p = A_S step), objective only.
template <typename TM, int T>
__global__ void __launch_bounds__(T)
k_polish_rows(const double* __restrict__ AS, const double* __restrict__ x, int kappa, int64_t m,
              const TM* __restrict__ b, int loss, double* __restrict__ q, double* __restrict__ d1,
              double* __restrict__ d2, const double* __restrict__ p, double alpha,
              double* __restrict__ fpart) {
  __shared__ double red[32];
  extern __shared__ double xs[];
  for (int k = threadIdx.x; k < kappa; k += T) xs[k] = x[k];
  __syncthreads();
  double facc = 0.0;
  for (int64_t r = static_cast<int64_t>(blockIdx.x) * T + threadIdx.x; r < m;
       r += static_cast<int64_t>(gridDim.x) * T) {
    double qr;
    if (alpha != 0.0) {
      qr = q[r] - alpha * p[r];
    } else {
      qr = 0.0;
      for (int k = 0; k < kappa; ++k) qr = fma(AS[k * m + r], xs[k], qr);
      q[r] = qr;
    }
    double f, g1, g2;
    row_loss(loss, qr, static_cast<double>(b[r]), f, g1, g2);
    if (alpha == 0.0) {
      d1[r] = g1;
      d2[r] = g2;
    }
    facc += f;
  }
  double v[1] = {facc};
  block_sum<1>(v, red);
  if (threadIdx.x == 0) fpart[blockIdx.x] = v[0];
}

// p = A_S step (m).
template <int T>
__global__ void k_polish_dir(const double* __restrict__ AS, const double* __restrict__ step,
                             int kappa, int64_t m, double* __restrict__ p) {
  extern __shared__ double ss[];
  for (int k = threadIdx.x; k < kappa; k += T) ss[k] = step[k];
  __syncthreads();
  for (int64_t r = static_cast<int64_t>(blockIdx.x) * T + threadIdx.x; r < m;
       r += static_cast<int64_t>(gridDim.x) * T) {
    double acc = 0.0;
    for (int k = 0; k < kappa; ++k) acc = fma(AS[k * m + r], ss[k], acc);
    p[r] = acc;
  }
}

// Partial gradient: gpart[c*kappa + k] = sum over rows of chunk c of AS[k, r] d1[r].
// Grid (chunks, kappa), T threads.
template <int T>
__global__ void k_polish_grad(const double* __restrict__ AS, const double* __restrict__ d1,
                              int kappa, int64_t m, int64_t chunk, double* __restrict__ gpart) {
  __shared__ double red[32];
  const int k = blockIdx.y, c = blockIdx.x;
  const int64_t r0 = c * chunk, r1 = r0 + chunk < m ? r0 + chunk : m;
  double acc = 0.0;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += T) acc = fma(AS[k * m + r], d1[r], acc);
  double v[1] = {acc};
  block_sum<1>(v, red);
  if (threadIdx.x == 0) gpart[static_cast<int64_t>(c) * kappa + k] = v[0];
}

// Partial weighted Gram: Hpart[c] (kappa x kappa, upper tiles) = sum over rows of chunk c of
// d2[r] a_S(r) a_S(r)'.  Grid (tile pairs, chunks), 256 threads, 32 x 32 tiles, 2 x 2 each.
__global__ void __launch_bounds__(256)
k_polish_hess(const double* __restrict__ AS, const double* __restrict__ d2, int kappa, int64_t m,
              int64_t chunk, double* __restrict__ Hpart) {
  constexpr int TL = 32, KC = 32;
  __shared__ double Ps[KC][TL + 1];
  __shared__ double Qs[KC][TL + 1];
  const int T = (kappa + TL - 1) / TL;
  int qq = blockIdx.x, ti = 0;
  while (qq >= T - ti) { qq -= T - ti; ++ti; if (ti >= T) return; }
  const int tj = ti + qq;
  const int c = blockIdx.y;
  const int64_t r0 = c * chunk, r1 = r0 + chunk < m ? r0 + chunk : m;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int64_t rb = r0; rb < r1; rb += KC) {
    for (int e = threadIdx.x; e < KC * TL; e += 256) {
      const int cc = e / KC, rr = e - cc * KC;  // consecutive threads: consecutive rows
      const int64_t r = rb + rr;
      const int pi = ti * TL + cc, qi = tj * TL + cc;
      const double w = r < r1 ? d2[r] : 0.0;
      Ps[rr][cc] = (r < r1 && pi < kappa) ? AS[pi * m + r] * w : 0.0;
      Qs[rr][cc] = (r < r1 && qi < kappa) ? AS[qi * m + r] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < KC; ++rr) {
      const double a0 = Ps[rr][ty * 2], a1 = Ps[rr][ty * 2 + 1];
      const double b0 = Qs[rr][tx * 2], b1 = Qs[rr][tx * 2 + 1];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
  double* H = Hpart + static_cast<int64_t>(c) * kappa * kappa;
  for (int a = 0; a < 2; ++a)
    for (int bq = 0; bq < 2; ++bq) {
      const int pi = ti * TL + ty * 2 + a, qi = tj * TL + tx * 2 + bq;
      if (pi < kappa && qi < kappa) {
        H[static_cast<int64_t>(pi) * kappa + qi] = acc[a][bq];
        H[static_cast<int64_t>(qi) * kappa + pi] = acc[a][bq];
      }
    }
}

// One CTA: H = sum_c Hpart[c] + I/gamma, g = sum_c gpart[c] + x/gamma (fixed order), then
// Cholesky H = L L' in place and step = H^-1 g (forward + back substitution, one thread per
// row segment).  Results: step[kappa]; flag[0] = 1 on a non-positive pivot.
template <int CT>
__global__ void __launch_bounds__(CT)
k_polish_solve(const double* __restrict__ Hpart, const double* __restrict__ gpart, int nchunks,
               const double* __restrict__ x, int kappa, double gamma, double* __restrict__ H,
               double* __restrict__ step, int* __restrict__ flag) {
  extern __shared__ double sm[];  // colk[kappa], y[kappa]
  double* colk = sm;
  double* y = sm + kappa;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NWP = CT / 32;
  const int64_t kk = static_cast<int64_t>(kappa) * kappa;
  for (int64_t e = tid; e < kk; e += CT) {
    double a = 0.0;
    for (int c = 0; c < nchunks; ++c) a += Hpart[c * kk + e];
    const int i = static_cast<int>(e / kappa), j = static_cast<int>(e - static_cast<int64_t>(i) * kappa);
    H[e] = a + (i == j ? 1.0 / gamma : 0.0);
  }
  for (int k = tid; k < kappa; k += CT) {
    double a = 0.0;
    for (int c = 0; c < nchunks; ++c) a += gpart[static_cast<int64_t>(c) * kappa + k];
    y[k] = a + x[k] / gamma;
  }
  __shared__ int bad;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < kappa; ++k) {
    if (tid == 0) {
      const double d = H[static_cast<int64_t>(k) * kappa + k];
      if (!(d > 0.0)) bad = 1;
      H[static_cast<int64_t>(k) * kappa + k] = d > 0.0 ? sqrt(d) : 1.0;
    }
    __syncthreads();
    const double dk = H[static_cast<int64_t>(k) * kappa + k];
    for (int a = k + 1 + tid; a < kappa; a += CT) {
      const double l = H[static_cast<int64_t>(a) * kappa + k] / dk;
      H[static_cast<int64_t>(a) * kappa + k] = l;
      colk[a] = l;
    }
    __syncthreads();
    for (int a = k + 1 + warp; a < kappa; a += NWP) {
      const double lak = colk[a];
      double* Ha = H + static_cast<int64_t>(a) * kappa;
      for (int bq = k + 1 + lane; bq <= a; bq += 32) Ha[bq] -= lak * colk[bq];
    }
    __syncthreads();
  }
  if (tid == 0) {
    flag[0] = bad;
    // L v = g, then L' step = v (sequential; kappa is small)
    for (int a = 0; a < kappa; ++a) {
      double sacc = y[a];
      const double* La = H + static_cast<int64_t>(a) * kappa;
      for (int bq = 0; bq < a; ++bq) sacc -= La[bq] * y[bq];
      y[a] = sacc / La[a];
    }
    for (int a = kappa - 1; a >= 0; --a) {
      double sacc = y[a];
      for (int bq = a + 1; bq < kappa; ++bq) sacc -= H[static_cast<int64_t>(bq) * kappa + a] * step[bq];
      step[a] = sacc / H[static_cast<int64_t>(a) * kappa + a];
    }
  }
}

// ---------------------------------------------------------------- softmax polish
// Restricted softmax problem on the support entries e = (c_e, k_e) of W (flattened c K + k),
// with the entries ordered by class (class k owns entries kb[k] .. kb[k+1]-1) and x_e their
// values:  minimise sum_r CE(q_r; y_r) + ||x||^2 / (2 gamma),  q_rk = sum_{e in k} a_{r c_e} x_e.
// Gradient g_e = sum_r a_{r c_e} (p_{r k_e} - [y_r = k_e]) + x_e / gamma; Hessian
// H_ee' = sum_r a_{r c_e} a_{r c_e'} p_{r k_e} ([k_e = k_e'] - p_{r k_e'}) + [e = e'] / gamma
//       = [k_e = k_e'] (U' A_S)_ee' - (U' U)_ee',   U_e = a_{c_e} * p_{k_e} (row-wise).

// Per row: q (K scores) from A_S and x (or q - alpha P for a trial point), softmax p, the
// loss; stores q, p and d1 = p - onehot(y) when alpha = 0; per-CTA partial objective.
template <typename TM, int KC, int T>
__global__ void __launch_bounds__(T)
k_polish_rows_sm(const double* __restrict__ AS, const double* __restrict__ x,
                 const int* __restrict__ kb, int K, int64_t m, const TM* __restrict__ b,
                 double* __restrict__ q, double* __restrict__ pr, double* __restrict__ d1,
                 const double* __restrict__ P, double alpha, double* __restrict__ fpart, int kappa) {
  __shared__ double red[32];
  extern __shared__ double xs[];
  for (int k = threadIdx.x; k < kappa; k += T) xs[k] = x[k];
  __shared__ int kbs[KC + 1];
  for (int k = threadIdx.x; k <= K; k += T) kbs[k] = kb[k];
  __syncthreads();
  double facc = 0.0;
  for (int64_t r = static_cast<int64_t>(blockIdx.x) * T + threadIdx.x; r < m;
       r += static_cast<int64_t>(gridDim.x) * T) {
    double qr[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      double acc = 0.0;
      if (k < K) {
        if (alpha != 0.0) {
          acc = q[r * K + k] - alpha * P[r * K + k];
        } else {
          for (int e = kbs[k]; e < kbs[k + 1]; ++e) acc = fma(AS[e * m + r], xs[e], acc);
          q[r * K + k] = acc;
        }
      }
      qr[k] = acc;
    }
    double mx = -HUGE_VAL;
#pragma unroll
    for (int k = 0; k < KC; ++k) if (k < K) mx = fmax(mx, qr[k]);
    double ssum = 0.0, ex[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) { ex[k] = k < K ? exp(qr[k] - mx) : 0.0; ssum += ex[k]; }
    const int y = static_cast<int>(b[r]);
    double qy = 0.0;
#pragma unroll
    for (int k = 0; k < KC; ++k) if (k == y) qy = qr[k];
    facc += mx + log(ssum) - qy;
    if (alpha == 0.0) {
#pragma unroll
      for (int k = 0; k < KC; ++k) {
        if (k < K) {
          const double pk = ex[k] / ssum;
          pr[r * K + k] = pk;
          d1[r * K + k] = pk - (k == y ? 1.0 : 0.0);
        }
      }
    }
  }
  double v[1] = {facc};
  block_sum<1>(v, red);
  if (threadIdx.x == 0) fpart[blockIdx.x] = v[0];
}

// Partial gradient of the softmax polish: gpart[c*kappa + e] = sum over rows of chunk c of
// AS[e, r] d1[r, k_e].  Grid (chunks, kappa).
template <int T>
__global__ void k_polish_grad_sm(const double* __restrict__ AS, const double* __restrict__ d1,
                                 const int* __restrict__ cls, int K, int kappa, int64_t m,
                                 int64_t chunk, double* __restrict__ gpart) {
  __shared__ double red[32];
  const int e = blockIdx.y, c = blockIdx.x, ke = cls[e];
  const int64_t r0 = c * chunk, r1 = r0 + chunk < m ? r0 + chunk : m;
  double acc = 0.0;
  for (int64_t r = r0 + threadIdx.x; r < r1; r += T) acc = fma(AS[e * m + r], d1[r * K + ke], acc);
  double v[1] = {acc};
  block_sum<1>(v, red);
  if (threadIdx.x == 0) gpart[static_cast<int64_t>(c) * kappa + e] = v[0];
}

// U[e, r] = AS[e, r] p[r, k_e].
__global__ void k_polish_u_sm(const double* __restrict__ AS, const double* __restrict__ pr,
                              const int* __restrict__ cls, int K, int kappa, int64_t m,
                              double* __restrict__ U) {
  const int e = blockIdx.y, ke = cls[e];
  for (int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; r < m;
       r += static_cast<int64_t>(gridDim.x) * blockDim.x)
    U[e * m + r] = AS[e * m + r] * pr[r * K + ke];
}

// Partial Hessian of the softmax polish, Hpart[c] = [k_e = k_e'] (U' A_S) - U' U over the rows
// of chunk c (upper tiles, mirrored).  Grid (tile pairs, chunks), 256 threads, 32 x 32 tiles.
__global__ void __launch_bounds__(256)
k_polish_hess_sm(const double* __restrict__ AS, const double* __restrict__ U,
                 const int* __restrict__ cls, int kappa, int64_t m, int64_t chunk,
                 double* __restrict__ Hpart) {
  constexpr int TL = 32, KC = 16;
  __shared__ double Us[KC][TL + 1];
  __shared__ double As_[KC][TL + 1];
  __shared__ double Uq[KC][TL + 1];
  const int T = (kappa + TL - 1) / TL;
  int qq = blockIdx.x, ti = 0;
  while (qq >= T - ti) { qq -= T - ti; ++ti; if (ti >= T) return; }
  const int tj = ti + qq;
  const int c = blockIdx.y;
  const int64_t r0 = c * chunk, r1 = r0 + chunk < m ? r0 + chunk : m;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double aA[2][2] = {{0.0, 0.0}, {0.0, 0.0}}, aU[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int64_t rb = r0; rb < r1; rb += KC) {
    for (int e = threadIdx.x; e < KC * TL; e += 256) {
      const int cc = e / KC, rr = e - cc * KC;
      const int64_t r = rb + rr;
      const int pi = ti * TL + cc, qi = tj * TL + cc;
      const bool okr = r < r1;
      Us[rr][cc] = (okr && pi < kappa) ? U[pi * m + r] : 0.0;
      As_[rr][cc] = (okr && qi < kappa) ? AS[qi * m + r] : 0.0;
      Uq[rr][cc] = (okr && qi < kappa) ? U[qi * m + r] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < KC; ++rr) {
      const double u0 = Us[rr][ty * 2], u1 = Us[rr][ty * 2 + 1];
      const double a0 = As_[rr][tx * 2], a1 = As_[rr][tx * 2 + 1];
      const double v0 = Uq[rr][tx * 2], v1 = Uq[rr][tx * 2 + 1];
      aA[0][0] = fma(u0, a0, aA[0][0]); aA[0][1] = fma(u0, a1, aA[0][1]);
      aA[1][0] = fma(u1, a0, aA[1][0]); aA[1][1] = fma(u1, a1, aA[1][1]);
      aU[0][0] = fma(u0, v0, aU[0][0]); aU[0][1] = fma(u0, v1, aU[0][1]);
      aU[1][0] = fma(u1, v0, aU[1][0]); aU[1][1] = fma(u1, v1, aU[1][1]);
    }
    __syncthreads();
  }
  double* H = Hpart + static_cast<int64_t>(c) * kappa * kappa;
  for (int a = 0; a < 2; ++a)
    for (int bq = 0; bq < 2; ++bq) {
      const int pi = ti * TL + ty * 2 + a, qi = tj * TL + tx * 2 + bq;
      if (pi < kappa && qi < kappa) {
        const double v = (cls[pi] == cls[qi] ? aA[a][bq] : 0.0) - aU[a][bq];
        H[static_cast<int64_t>(pi) * kappa + qi] = v;
        H[static_cast<int64_t>(qi) * kappa + pi] = v;
      }
    }
}

// P[r, k] = sum_{e in class k} AS[e, r] step[e].
template <int KC, int T>
__global__ void k_polish_dir_sm(const double* __restrict__ AS, const double* __restrict__ step,
                                const int* __restrict__ kb, int K, int kappa, int64_t m,
                                double* __restrict__ P) {
  extern __shared__ double ss[];
  __shared__ int kbs[KC + 1];
  for (int k = threadIdx.x; k < kappa; k += T) ss[k] = step[k];
  for (int k = threadIdx.x; k <= K; k += T) kbs[k] = kb[k];
  __syncthreads();
  for (int64_t r = static_cast<int64_t>(blockIdx.x) * T + threadIdx.x; r < m;
       r += static_cast<int64_t>(gridDim.x) * T) {
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      if (k < K) {
        double acc = 0.0;
        for (int e = kbs[k]; e < kbs[k + 1]; ++e) acc = fma(AS[e * m + r], ss[e], acc);
        P[r * K + k] = acc;
      }
    }
  }
}

}  // namespace bic
