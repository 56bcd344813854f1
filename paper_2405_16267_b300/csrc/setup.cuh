// Setup kernels: input conversion into the padded device layout, the per-block Gram
// matrices G_ij = A_ij' A_ij, and the FP64 Cholesky factorisation and inverse of
// rho_l G_ij + c0 I (the system matrix of the x_ij solve of eq. (p:GPU;x)).
#pragma once

#include "common.cuh"

namespace bic {

// dst[r, c] = src[r, c] for c < n, 0 for n <= c < lda_dst.
template <typename TIN, typename TOUT>
__global__ void k_convert_rows(const TIN* __restrict__ src, int64_t lda_src,
                               TOUT* __restrict__ dst, int64_t lda_dst, int64_t rows, int64_t n) {
  const int64_t total = rows * lda_dst;
  for (int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
       idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = idx / lda_dst, c = idx - r * lda_dst;
    dst[idx] = c < n ? conv<TOUT>(src[r * lda_src + c]) : conv<TOUT>(0.0f);
  }
}

// G_ij = A_ij' A_ij for every shard i and block j, FP64 output (row stride n_j).
// Grid (upper-triangle tile pairs, M, shards from shard0); 256 threads compute a 64 x 64
// tile, 4 x 4 each.
// TC is the multiply type; with TC = float the running sums are moved into FP64 every
// 256 rows to bound the FP32 accumulation error.
template <typename TA, typename TC>
__global__ void __launch_bounds__(256)
k_gram(const TA* __restrict__ A, int64_t lda, const int64_t* __restrict__ shard_row0,
       const int* __restrict__ blk_col0, double* __restrict__ G, const int64_t* __restrict__ G_off,
       int M, int shard0) {
  constexpr int TILE = 64, KC = 32;
  __shared__ TC As[KC][TILE + 1];
  __shared__ TC Bs[KC][TILE + 1];
  const int i = shard0 + blockIdx.z, j = blockIdx.y;
  const int col0 = blk_col0[j], nj = blk_col0[j + 1] - col0;
  const int T = (nj + TILE - 1) / TILE;
  int q = blockIdx.x, ti = 0;
  while (q >= T - ti) { q -= T - ti; ++ti; if (ti >= T) return; }
  const int tj = ti + q;  // ti <= tj
  const int64_t r_begin = shard_row0[i], r_end = shard_row0[i + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  TC acc[4][4];
  double acc2[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int bq = 0; bq < 4; ++bq) { acc[a][bq] = TC(0); acc2[a][bq] = 0.0; }
  int since_flush = 0;
  for (int64_t r0 = r_begin; r0 < r_end; r0 += KC) {
    for (int e = threadIdx.x; e < KC * TILE; e += 256) {
      const int k = e / TILE, cc = e - k * TILE;
      const int64_t row = r0 + k;
      const int ca = ti * TILE + cc, cb = tj * TILE + cc;
      As[k][cc] = (row < r_end && ca < nj) ? conv<TC>(A[row * lda + col0 + ca]) : TC(0);
      Bs[k][cc] = (row < r_end && cb < nj) ? conv<TC>(A[row * lda + col0 + cb]) : TC(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < KC; ++k) {
      TC av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) { av[a] = As[k][ty * 4 + a]; bv[a] = Bs[k][tx * 4 + a]; }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int bq = 0; bq < 4; ++bq) acc[a][bq] = fma(av[a], bv[bq], acc[a][bq]);
    }
    __syncthreads();
    if (++since_flush == 8) {
      since_flush = 0;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int bq = 0; bq < 4; ++bq) { acc2[a][bq] += static_cast<double>(acc[a][bq]); acc[a][bq] = TC(0); }
    }
  }
  double* Gb = G + G_off[i * M + j];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int bq = 0; bq < 4; ++bq) {
      const int ra = ti * TILE + ty * 4 + a, cb = tj * TILE + tx * 4 + bq;
      if (ra < nj && cb < nj) {
        const double val = acc2[a][bq] + static_cast<double>(acc[a][bq]);
        Gb[static_cast<int64_t>(ra) * nj + cb] = val;
        Gb[static_cast<int64_t>(cb) * nj + ra] = val;
      }
    }
}

// One CTA per block (i, j): K = rho_l G + c0 I (in place in G), Cholesky K = L L' in place in
// the lower triangle (right-looking, column k cached in shared memory), then L' is copied
// into the strict upper triangle so that both triangular solves read rows.
template <int CT>
__global__ void __launch_bounds__(CT)
k_chol(double* __restrict__ G, const int64_t* __restrict__ G_off, const int* __restrict__ blk_col0,
       int M, double rho_l, double c0, int* __restrict__ err) {
  extern __shared__ double colk[];
  const int blk = blockIdx.x, j = blk % M;
  const int nj = blk_col0[j + 1] - blk_col0[j];
  double* K = G + G_off[blk];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NWP = CT / 32;
  for (int64_t e = tid; e < static_cast<int64_t>(nj) * nj; e += CT) {
    const int a = static_cast<int>(e / nj), bq = static_cast<int>(e - static_cast<int64_t>(a) * nj);
    K[e] = rho_l * K[e] + (a == bq ? c0 : 0.0);
  }
  __syncthreads();
  for (int k = 0; k < nj; ++k) {
    if (tid == 0) {
      const double dkk = K[static_cast<int64_t>(k) * nj + k];
      if (!(dkk > 0.0)) set_err(err, DEV_NONPOS_PIVOT);
      K[static_cast<int64_t>(k) * nj + k] = dkk > 0.0 ? sqrt(dkk) : 1.0;
    }
    __syncthreads();
    const double dk = K[static_cast<int64_t>(k) * nj + k];
    for (int a = k + 1 + tid; a < nj; a += CT) {
      const double l = K[static_cast<int64_t>(a) * nj + k] / dk;
      K[static_cast<int64_t>(a) * nj + k] = l;
      colk[a] = l;
    }
    __syncthreads();
    for (int a = k + 1 + warp; a < nj; a += NWP) {
      const double lak = colk[a];
      double* Ka = K + static_cast<int64_t>(a) * nj;
      for (int bq = k + 1 + lane; bq <= a; bq += 32) Ka[bq] -= lak * colk[bq];
    }
    __syncthreads();
  }
  // upper triangle <- L'
  for (int64_t e = tid; e < static_cast<int64_t>(nj) * nj; e += CT) {
    const int a = static_cast<int>(e / nj), bq = static_cast<int>(e - static_cast<int64_t>(a) * nj);
    if (bq > a) K[e] = K[static_cast<int64_t>(bq) * nj + a];
  }
}

// One CTA per block (i, j): K = rho_l G + c0 I, then the Cholesky factor K = L L' in place
// in the lower triangle, right-looking with NB-column panels: the panel (rows kb.., columns
// kb..kb+NB) is held column-major in shared memory; one warp factors its diagonal block,
// every thread solves some of the rows below against it, and the trailing lower triangle
// is updated in 64 x 64 tiles (4 x 4 per thread, rows ty + 16 a, columns tx + 16 b) from
// the panel.  The entries above the diagonal are left as they were.
template <int CT, int NB>
__global__ void __launch_bounds__(CT)
k_chol_blk(double* __restrict__ G, const int64_t* __restrict__ G_off, const int* __restrict__ blk_col0,
           int M, double rho_l, double c0, int* __restrict__ err) {
  static_assert(CT == 256 && NB <= 32, "16 x 16 threads; one lane per diagonal-block row");
  extern __shared__ double panT[];  // [NB][ldpan]
  const int blk = blockIdx.x, j = blk % M;
  const int nj = blk_col0[j + 1] - blk_col0[j];
  const int ldpan = nj + 1;
  double* K = G + G_off[blk];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, tx = tid & 15, ty = tid >> 4;
  for (int64_t e = tid; e < static_cast<int64_t>(nj) * nj; e += CT) {
    const int a = static_cast<int>(e / nj), bq = static_cast<int>(e - static_cast<int64_t>(a) * nj);
    K[e] = rho_l * K[e] + (a == bq ? c0 : 0.0);
  }
  __syncthreads();
  for (int kb = 0; kb < nj; kb += NB) {
    const int nb = nj - kb < NB ? nj - kb : NB, nr = nj - kb;
    for (int e = tid; e < nr * nb; e += CT) {
      const int r = e / nb, k = e - r * nb;
      panT[k * ldpan + r] = r >= k ? K[static_cast<int64_t>(kb + r) * nj + kb + k] : 0.0;
    }
    __syncthreads();
    if (warp == 0) {  // diagonal block: lane = row
      for (int c = 0; c < nb; ++c) {
        double d = panT[c * ldpan + c];
        if (lane == 0 && !(d > 0.0)) set_err(err, DEV_NONPOS_PIVOT);
        d = d > 0.0 ? sqrt(d) : 1.0;
        __syncwarp();
        if (lane > c && lane < nb) panT[c * ldpan + lane] /= d;
        if (lane == c) panT[c * ldpan + c] = d;
        __syncwarp();
        if (lane > c && lane < nb) {
          const double lr = panT[c * ldpan + lane];
          for (int k = c + 1; k <= lane; ++k) panT[k * ldpan + lane] -= lr * panT[c * ldpan + k];
        }
        __syncwarp();
      }
    }
    __syncthreads();
    // rows below the diagonal block: x L11' = a, i.e. x_k = (a_k - sum_{q<k} x_q L11[k][q]) / L11[k][k]
    for (int r = nb + tid; r < nr; r += CT) {
      double x[NB];
#pragma unroll
      for (int k = 0; k < NB; ++k) x[k] = k < nb ? panT[k * ldpan + r] : 0.0;
#pragma unroll
      for (int k = 0; k < NB; ++k) {
        if (k < nb) {
          double sum = x[k];
#pragma unroll
          for (int q = 0; q < k; ++q) sum = fma(-x[q], panT[q * ldpan + k], sum);
          x[k] = sum / panT[k * ldpan + k];
        }
      }
#pragma unroll
      for (int k = 0; k < NB; ++k)
        if (k < nb) panT[k * ldpan + r] = x[k];
    }
    __syncthreads();
    for (int e = tid; e < nr * nb; e += CT) {
      const int r = e / nb, k = e - r * nb;
      if (r >= k) K[static_cast<int64_t>(kb + r) * nj + kb + k] = panT[k * ldpan + r];
    }
    // trailing lower triangle: K[r][c] -= sum_k L[r][k] L[c][k] for nb <= c <= r < nr
    const int nt = nr - nb, T = (nt + 63) / 64;
    for (int tile = 0; tile < T * (T + 1) / 2; ++tile) {
      int ti = 0, q = tile;
      while (q > ti) { q -= ti + 1; ++ti; }
      const int tj = q;  // tj <= ti
      const int r0 = nb + ti * 64, c0t = nb + tj * 64;
      double acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int bq = 0; bq < 4; ++bq) acc[a][bq] = 0.0;
      for (int k = 0; k < nb; ++k) {
        double av[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const int r = r0 + ty + 16 * a, c = c0t + tx + 16 * a;
          av[a] = r < nr ? panT[k * ldpan + r] : 0.0;
          bv[a] = c < nr ? panT[k * ldpan + c] : 0.0;
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int bq = 0; bq < 4; ++bq) acc[a][bq] = fma(av[a], bv[bq], acc[a][bq]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int bq = 0; bq < 4; ++bq) {
          const int r = r0 + ty + 16 * a, c = c0t + tx + 16 * bq;
          if (r < nr && c <= r) K[static_cast<int64_t>(kb + r) * nj + kb + c] -= acc[a][bq];
        }
    }
    __syncthreads();
  }
}

// Cholesky factor K = L L' (K = rho_l G + c0 I) of every block, in place in the lower
// triangle (the entries above the diagonal are left as they were), right-looking with
// NB-column panels and spread over the GPU: the host launches, per panel, one CTA per block
// for the panel (its NB x NB diagonal block factored by one warp, the rows below solved
// against it by every thread, the panel held column-major in shared memory) and then one
// CTA per 64 x 64 tile of every block's trailing lower triangle (4 x 4 entries per thread,
// summed over the panel's columns in order).  One CTA per block for the whole factorisation
// took about 17 ms for 625 columns at one SM's FP64 rate (k_chol_blk above, kept for blocks
// under 256 columns, where this form's launches would cost more than they save; its results
// agree with this form's to rounding).
// K = rho_l G + c0 I for every block.  Grid (blocks, chunks).
template <int CT>
__global__ void __launch_bounds__(CT)
k_chol_scale(double* __restrict__ G, const int64_t* __restrict__ G_off, const int* __restrict__ blk_col0,
             int M, double rho_l, double c0) {
  const int blk = blockIdx.x, j = blk % M;
  const int nj = blk_col0[j + 1] - blk_col0[j];
  double* K = G + G_off[blk];
  const int64_t tot = static_cast<int64_t>(nj) * nj;
  for (int64_t e = static_cast<int64_t>(blockIdx.y) * CT + threadIdx.x; e < tot;
       e += static_cast<int64_t>(gridDim.y) * CT) {
    const int a = static_cast<int>(e / nj), bq = static_cast<int>(e - static_cast<int64_t>(a) * nj);
    K[e] = rho_l * K[e] + (a == bq ? c0 : 0.0);
  }
}

// Panel kb of every block, grid (blocks, row chunks of RC rows): each CTA factors the
// diagonal NB x NB block (warp 0; every CTA of a block gets the same factor) and solves its
// chunk of the rows below against it.  The factored diagonal block is written by the last
// of the block's CTAs to finish (a ticket on tick[block], reset by that CTA), so that no CTA
// reads it from K after it was overwritten; no CTA waits for another.  Divisions by
// the diagonal are multiplications by its reciprocals, formed once per panel (on this part
// an FP64 division costs a dozen FP64 instructions, and a row's solve had one per column).
// Blocks with nj <= kb return.
template <int CT, int NB, int RC>
__global__ void __launch_bounds__(CT)
k_chol_panel(double* __restrict__ G, const int64_t* __restrict__ G_off, const int* __restrict__ blk_col0,
             int M, int kb, int* __restrict__ err, int* __restrict__ tick) {
  static_assert(CT == 256 && NB <= 32 && RC <= CT, "one lane per diagonal-block row, a row per thread");
  constexpr int LD = NB + RC + 1;    // rows held: the diagonal block, then the chunk
  __shared__ double panT[NB * LD];   // [k][row]
  __shared__ double rinv[NB];
  __shared__ bool last;
  const int blk = blockIdx.x, j = blk % M;
  const int nj = blk_col0[j + 1] - blk_col0[j];
  if (kb >= nj) return;
  double* K = G + G_off[blk];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = nj - kb < NB ? nj - kb : NB, nr = nj - kb;
  const int r_lo = nb + static_cast<int>(blockIdx.y) * RC;  // first chunk row (relative to kb)
  if (blockIdx.y > 0 && r_lo >= nr) return;
  const int nc = nr - r_lo < RC ? (nr - r_lo > 0 ? nr - r_lo : 0) : RC;  // chunk rows
  // local row i: i < nb the diagonal block's row i, i >= nb chunk row r_lo + i - nb
  for (int e = tid; e < (nb + nc) * nb; e += CT) {
    const int i = e / nb, k = e - i * nb;
    const int r = i < nb ? i : r_lo + i - nb;
    panT[k * LD + i] = r >= k ? K[static_cast<int64_t>(kb + r) * nj + kb + k] : 0.0;
  }
  __syncthreads();
  if (warp == 0) {  // diagonal block: lane = row
    for (int c = 0; c < nb; ++c) {
      double d = panT[c * LD + c];
      if (lane == 0 && blockIdx.y == 0 && !(d > 0.0)) set_err(err, DEV_NONPOS_PIVOT);
      d = d > 0.0 ? sqrt(d) : 1.0;
      const double di = 1.0 / d;
      __syncwarp();
      if (lane > c && lane < nb) panT[c * LD + lane] *= di;
      if (lane == c) {
        panT[c * LD + c] = d;
        rinv[c] = di;
      }
      __syncwarp();
      if (lane > c && lane < nb) {
        const double lr = panT[c * LD + lane];
        for (int k = c + 1; k <= lane; ++k) panT[k * LD + lane] -= lr * panT[c * LD + k];
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // chunk rows: x L11' = a, i.e. x_k = (a_k - sum_{q<k} x_q L11[k][q]) / L11[k][k]
  if (tid < nc) {
    const int i = nb + tid;
    double x[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) x[k] = k < nb ? panT[k * LD + i] : 0.0;
#pragma unroll
    for (int k = 0; k < NB; ++k) {
      if (k < nb) {
        double sum = x[k];
#pragma unroll
        for (int q = 0; q < k; ++q) sum = fma(-x[q], panT[q * LD + k], sum);
        x[k] = sum * rinv[k];
      }
    }
#pragma unroll
    for (int k = 0; k < NB; ++k)
      if (k < nb) panT[k * LD + i] = x[k];
  }
  __syncthreads();
  for (int e = tid; e < nc * nb; e += CT) {
    const int i = nb + e / nb, k = e % nb;
    K[static_cast<int64_t>(kb + r_lo + i - nb) * nj + kb + k] = panT[k * LD + i];
  }
  // the block's CTAs: chunk 0 and every chunk that starts above nr
  const int nact = nr - nb > RC ? (nr - nb + RC - 1) / RC : 1;
  __syncthreads();  // this CTA's reads of the diagonal block are done
  if (tid == 0) {
    __threadfence();
    last = atomicAdd(&tick[blk], 1) == nact - 1;
  }
  __syncthreads();
  if (last) {
    for (int e = tid; e < nb * nb; e += CT) {
      const int i = e / nb, k = e % nb;
      if (i >= k) K[static_cast<int64_t>(kb + i) * nj + kb + k] = panT[k * LD + i];
    }
    if (tid == 0) tick[blk] = 0;
  }
}

// Trailing update after panel kb: grid (64 x 64 tiles of the widest block's trailing lower
// triangle, blocks); tile (ti, tj), tj <= ti, of block b: K[r][c] -= sum_k L[r][k] L[c][k]
// over the panel's NB columns (rows of L read from K, staged in shared memory).
template <int CT, int NB>
__global__ void __launch_bounds__(CT)
k_chol_update(double* __restrict__ G, const int64_t* __restrict__ G_off, const int* __restrict__ blk_col0,
              int M, int kb) {
  __shared__ double La[NB][64], Lb[NB][64];
  const int blk = blockIdx.y, j = blk % M;
  const int nj = blk_col0[j + 1] - blk_col0[j];
  if (nj - kb <= NB) return;  // no trailing part
  const int nb = NB, nr = nj - kb, nt = nr - nb, T = (nt + 63) / 64;
  const int tile = blockIdx.x;
  if (tile >= T * (T + 1) / 2) return;
  int ti = 0, q = tile;
  while (q > ti) { q -= ti + 1; ++ti; }
  const int tj = q;
  const int r0 = nb + ti * 64, c0t = nb + tj * 64;
  double* K = G + G_off[blk];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int e = tid; e < NB * 64; e += CT) {
    const int k = e / 64, i = e - k * 64;
    const int r = r0 + i, c = c0t + i;
    La[k][i] = r < nr ? K[static_cast<int64_t>(kb + r) * nj + kb + k] : 0.0;
    Lb[k][i] = c < nr ? K[static_cast<int64_t>(kb + c) * nj + kb + k] : 0.0;
  }
  __syncthreads();
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int bq = 0; bq < 4; ++bq) acc[a][bq] = 0.0;
  for (int k = 0; k < nb; ++k) {
    double av[4], bv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      av[a] = La[k][ty + 16 * a];
      bv[a] = Lb[k][tx + 16 * a];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int bq = 0; bq < 4; ++bq) acc[a][bq] = fma(av[a], bv[bq], acc[a][bq]);
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int bq = 0; bq < 4; ++bq) {
      const int r = r0 + ty + 16 * a, c = c0t + tx + 16 * bq;
      if (r < nr && c <= r) K[static_cast<int64_t>(kb + r) * nj + kb + c] -= acc[a][bq];
    }
}

// Y = L^-1 column by column (one warp per column c: forward substitution L y = e_c, y in
// shared memory), stored transposed: YT row c = column c of Y (zero before c).  Rows go 32
// at a time: lane l adds L[a0 + r][k] y[k] for the known entries k = c + l, c + l + 32, ...
// into 32 row accumulators (coalesced reads of L), one warp reduce-scatter gives lane r the
// sum of row a0 + r, and the 32 x 32 diagonal block is solved in the warp with reciprocals
// of its diagonal formed in parallel.  On this part's FP64 pipe a per-row warp reduction
// and division cost more than the row's multiply-adds; this form spends one reduction and
// one division instruction per 32 rows.
__global__ void k_inv_fwd(const double* __restrict__ G, const int64_t* __restrict__ G_off,
                          const int* __restrict__ blk_col0, int M, double* __restrict__ YT) {
  extern __shared__ double ycol[];  // [warps][nj]
  const int blk = blockIdx.x, j = blk % M;
  const int nj = blk_col0[j + 1] - blk_col0[j];
  const int nw = blockDim.x >> 5, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.y * nw + warp;
  if (c >= nj) return;
  const double* K = G + G_off[blk];
  double* y = ycol + static_cast<int64_t>(warp) * nj;
  for (int a0 = c; a0 < nj; a0 += 32) {
    const int nr = nj - a0 < 32 ? nj - a0 : 32;
    double acc[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) acc[r] = 0.0;
    for (int k = c + lane; k < a0; k += 32) {
      const double yk = y[k];
#pragma unroll
      for (int r = 0; r < 32; ++r)
        if (r < nr) acc[r] = fma(K[static_cast<int64_t>(a0 + r) * nj + k], yk, acc[r]);
    }
    const double sum = warp_reduce_scatter<32>(acc, lane);  // lane r: row a0 + r
    const bool mine = lane < nr;
    const int64_t rowo = static_cast<int64_t>(a0 + (mine ? lane : 0)) * nj;
    const double dinv = mine ? 1.0 / K[rowo + a0 + lane] : 0.0;
    double x = (a0 + lane == c ? 1.0 : 0.0) - sum;
    double yme = 0.0;
    for (int t = 0; t < nr; ++t) {
      const double yt = __shfl_sync(0xffffffffu, x * dinv, t);
      if (lane == t) yme = yt;
      if (lane > t && mine) x = fma(-K[rowo + a0 + t], yt, x);
    }
    if (mine) y[a0 + lane] = yme;
    __syncwarp();
  }
  double* Yr = YT + G_off[blk] + static_cast<int64_t>(c) * nj;
  for (int a = lane; a < nj; a += 32) Yr[a] = a < c ? 0.0 : y[a];
}

// P_ij = K^-1 = L^-T L^-1 = Y' Y: P[a][b] = sum_{k >= max(a, b)} YT[a][k] YT[b][k], FP64
// sums, written in TP with row stride ldp (both triangles; the item (0, 0) of a block also
// zeroes the padding columns).  Grid (items, 1, shards), 4 x 4 per thread.  An item is the
// 64 x 64 tile pair (ti, tj), ti <= tj, of block j over k in [tj 64, nj), or one part of
// that range: the sum of a tile far from the diagonal is several times that of one near
// it, and one CTA per tile left most SMs idle behind the longest.  A part writes its partial
// tile to scratch (the block's region of G, free once the inverse has read L) and the last
// part of a tile (a ticket) adds the partials in part order.
struct YtyItem {
  int j, ti, tj;
  int part, nparts;
  int tick;  // the tile's ticket within a shard's tiles
  int scr;   // its first partial tile (of 64 x 64 doubles) within the block's scratch
  int pad;
};

template <typename TP>
__global__ void __launch_bounds__(256)
k_yty(const double* __restrict__ YT, const int64_t* __restrict__ G_off, const int* __restrict__ blk_col0,
      const int* __restrict__ blk_ldp, int M, TP* __restrict__ P, const int64_t* __restrict__ P_off,
      const YtyItem* __restrict__ items, int kspan, double* __restrict__ G, int* __restrict__ tick,
      int ntiles) {
  constexpr int TILE = 64, KC = 32;
  __shared__ double As[KC][TILE + 1];
  __shared__ double Bs[KC][TILE + 1];
  __shared__ int last_part;
  const YtyItem it = items[blockIdx.x];
  const int i = blockIdx.z, j = it.j, blk = i * M + j;
  const int nj = blk_col0[j + 1] - blk_col0[j], ldp = blk_ldp[j];
  const int ti = it.ti, tj = it.tj;
  const double* Y = YT + G_off[blk];
  TP* Pb = P + P_off[blk];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  if (ti == 0 && tj == 0 && it.part == 0 && ldp > nj) {
    for (int64_t e = threadIdx.x; e < static_cast<int64_t>(nj) * (ldp - nj); e += 256) {
      const int a = static_cast<int>(e / (ldp - nj)), cc = nj + static_cast<int>(e - static_cast<int64_t>(a) * (ldp - nj));
      Pb[static_cast<int64_t>(a) * ldp + cc] = TP(0);
    }
  }
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int bq = 0; bq < 4; ++bq) acc[a][bq] = 0.0;
  // YT[a][k] = 0 for k < a, so the sum starts at the column tile's first index
  const int k_lo = tj * TILE + it.part * kspan;
  const int k_hi = it.part + 1 == it.nparts ? nj : tj * TILE + (it.part + 1) * kspan;
  for (int k0 = k_lo; k0 < k_hi; k0 += KC) {
    for (int e = threadIdx.x; e < KC * TILE; e += 256) {
      const int r = e / KC, k = e - r * KC;
      const int ra = ti * TILE + r, rb = tj * TILE + r, kk = k0 + k;
      As[k][r] = (ra < nj && kk < k_hi) ? Y[static_cast<int64_t>(ra) * nj + kk] : 0.0;
      Bs[k][r] = (rb < nj && kk < k_hi) ? Y[static_cast<int64_t>(rb) * nj + kk] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < KC; ++k) {
      double av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) { av[a] = As[k][ty + 16 * a]; bv[a] = Bs[k][tx + 16 * a]; }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int bq = 0; bq < 4; ++bq) acc[a][bq] = fma(av[a], bv[bq], acc[a][bq]);
    }
    __syncthreads();
  }
  if (it.nparts > 1) {
    double* scr = G + G_off[blk] + static_cast<int64_t>(it.scr) * (TILE * TILE);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int bq = 0; bq < 4; ++bq)
        scr[static_cast<int64_t>(it.part) * (TILE * TILE) + (ty + 16 * a) * TILE + tx + 16 * bq] = acc[a][bq];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0)
      last_part = atomicAdd(&tick[static_cast<int64_t>(i) * ntiles + it.tick], 1) == it.nparts - 1;
    __syncthreads();
    if (!last_part) return;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int bq = 0; bq < 4; ++bq) {
        double v = 0.0;
        for (int p = 0; p < it.nparts; ++p)
          v += __ldcg(&scr[static_cast<int64_t>(p) * (TILE * TILE) + (ty + 16 * a) * TILE + tx + 16 * bq]);
        acc[a][bq] = v;
      }
    if (threadIdx.x == 0) tick[static_cast<int64_t>(i) * ntiles + it.tick] = 0;
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int bq = 0; bq < 4; ++bq) {
      const int ra = ti * TILE + ty + 16 * a, cb = tj * TILE + tx + 16 * bq;
      if (ra < nj && cb < nj) {
        Pb[static_cast<int64_t>(ra) * ldp + cb] = static_cast<TP>(acc[a][bq]);
        Pb[static_cast<int64_t>(cb) * ldp + ra] = static_cast<TP>(acc[a][bq]);
      }
    }
}

// Columns of K^-1 = L^-T L^-1: grid (blocks, column groups), one warp per column c:
// forward L y = e_c then back L' p = y, the column held in shared memory; P is written in
// TP with row stride ldp (P is symmetric, so column c is written as row c, its padding
// entries zeroed).
template <typename TP>
__global__ void k_inv_cols(const double* __restrict__ G, const int64_t* __restrict__ G_off,
                           const int* __restrict__ blk_col0, const int* __restrict__ blk_ldp,
                           int M, TP* __restrict__ P, const int64_t* __restrict__ P_off) {
  extern __shared__ double ycol[];  // [warps][nj]
  const int blk = blockIdx.x, j = blk % M;
  const int nj = blk_col0[j + 1] - blk_col0[j], ldp = blk_ldp[j];
  const int nw = blockDim.x >> 5, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.y * nw + warp;
  if (c >= nj) return;
  const double* K = G + G_off[blk];
  double* y = ycol + static_cast<int64_t>(warp) * nj;
  for (int a = lane; a < nj; a += 32) y[a] = 0.0;
  __syncwarp();
  // forward: y_a = (delta_ac - sum_{b<a} L[a,b] y_b) / L[a,a], zero for a < c
  for (int a = c; a < nj; ++a) {
    const double* La = K + static_cast<int64_t>(a) * nj;
    double part = 0.0;
    for (int bq = c + lane; bq < a; bq += 32) part = fma(La[bq], y[bq], part);
    part = warp_sum(part);
    if (lane == 0) y[a] = ((a == c ? 1.0 : 0.0) - part) / La[a];
    __syncwarp();
  }
  // back: p_a = (y_a - sum_{b>a} L[b,a] p_b) / L[a,a]; row a of the upper triangle is L[., a]
  for (int a = nj - 1; a >= 0; --a) {
    const double* Ua = K + static_cast<int64_t>(a) * nj;
    double part = 0.0;
    for (int bq = a + 1 + lane; bq < nj; bq += 32) part = fma(Ua[bq], y[bq], part);
    part = warp_sum(part);
    if (lane == 0) y[a] = (y[a] - part) / Ua[a];
    __syncwarp();
  }
  TP* Pr = P + P_off[blk] + static_cast<int64_t>(c) * ldp;
  for (int a = lane; a < ldp; a += 32) Pr[a] = a < nj ? static_cast<TP>(y[a]) : TP(0);
}

}  // namespace bic
