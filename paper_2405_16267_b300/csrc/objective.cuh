// Objective of problem (p:SML) (Sec. 2) at the consensus iterate z, in FP64:
//
//     F(z) = sum_r l(a_r z; b_r) + ||z||^2 / (2 gamma),
//
// with the stored A (rounded to the handle's precision) and every product, loss and sum in
// FP64.  Only the features where z is nonzero contribute to a_r z, so the row products run
// over a compacted list of those columns (all columns while z is dense, a few after the
// l1 projection has thresholded it).  Sums are taken in a fixed order: the result is
// bit-for-bit repeatable.  Three launches: k_obj_compact (one CTA), k_obj_rows (a warp per
// row), k_obj_final (one CTA).
#pragma once

#include "common.cuh"
#include "polish.cuh"

namespace bic {

constexpr int kObjThreads = 256;

// idx[0..cnt) = the features c (ascending) with z[c K + k] != 0 for some class k;
// out[1] = ||z||^2.  One CTA of GT threads; thread t owns features t, t + GT, ...
template <int GT>
__global__ void __launch_bounds__(GT, 1)
k_obj_compact(const double* __restrict__ z, int64_t n, int K, int* __restrict__ idx,
              int* __restrict__ cnt, double* __restrict__ out) {
  __shared__ int warp_cnt[GT / 32];
  __shared__ int base_s;
  __shared__ double red[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) base_s = 0;
  double zsq = 0.0;
  for (int64_t c0 = 0; c0 < n; c0 += GT) {
    const int64_t c = c0 + tid;
    bool nz = false;
    if (c < n) {
      for (int k = 0; k < K; ++k) {
        const double v = z[c * K + k];
        zsq = fma(v, v, zsq);
        nz |= v != 0.0;
      }
    }
    const unsigned int ball = __ballot_sync(0xffffffffu, nz);
    if (lane == 0) warp_cnt[warp] = __popc(ball);
    __syncthreads();
    int before = base_s;
    for (int w2 = 0; w2 < warp; ++w2) before += warp_cnt[w2];
    if (nz) idx[before + __popc(ball & ((1u << lane) - 1u))] = static_cast<int>(c);
    __syncthreads();
    if (tid == 0) {
      int tot = 0;
      for (int w2 = 0; w2 < GT / 32; ++w2) tot += warp_cnt[w2];
      base_s += tot;
    }
    __syncthreads();
  }
  double v[1] = {zsq};
  block_sum<1>(v, red);
  if (tid == 0) {
    *cnt = base_s;
    out[1] = v[0];
  }
}

// Row losses at q_r = a_r Z over the compacted features; part[blockIdx.x] = the CTA's sum.
// Warp w of the grid takes rows w, w + W, ... (W = warps in the grid); lanes split the
// features.  KC >= K classes (1 for the scalar losses).
template <typename TA, typename TM, int KC>
__global__ void __launch_bounds__(kObjThreads)
k_obj_rows(const TA* __restrict__ A, int64_t lda, const TM* __restrict__ b,
           const double* __restrict__ z, const int* __restrict__ idx, const int* __restrict__ cnt,
           int64_t m, int K, int loss, double* __restrict__ part) {
  __shared__ double red[32];
  const int lane = threadIdx.x & 31;
  const int64_t W = static_cast<int64_t>(gridDim.x) * (kObjThreads / 32);
  const int nnz = *cnt;
  double acc = 0.0;
  for (int64_t r = static_cast<int64_t>(blockIdx.x) * (kObjThreads / 32) + (threadIdx.x >> 5); r < m;
       r += W) {
    const TA* row = A + r * lda;
    double q[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) q[k] = 0.0;
    for (int e = lane; e < nnz; e += 32) {
      const int c = idx[e];
      const double a = conv<double>(row[c]);
#pragma unroll
      for (int k = 0; k < KC; ++k)
        if (k < K) q[k] = fma(a, z[static_cast<int64_t>(c) * K + k], q[k]);
    }
#pragma unroll
    for (int k = 0; k < KC; ++k) q[k] = warp_sum(q[k]);
    if (lane == 0) {
      const double br = static_cast<double>(b[r]);
      double f;
      if (KC == 1) {
        double d1, d2;
        row_loss(loss, q[0], br, f, d1, d2);
      } else {  // softmax cross-entropy logsumexp(q) - q_y
        double qm = q[0];
#pragma unroll
        for (int k = 1; k < KC; ++k)
          if (k < K) qm = fmax(qm, q[k]);
        double se = 0.0, qy = 0.0;
        const int y = static_cast<int>(br);
#pragma unroll
        for (int k = 0; k < KC; ++k)
          if (k < K) {
            se += exp(q[k] - qm);
            if (k == y) qy = q[k];
          }
        f = qm + log(se) - qy;
      }
      acc += f;
    }
  }
  double v[1] = {acc};
  block_sum<1>(v, red);
  if (threadIdx.x == 0) part[blockIdx.x] = v[0];
}

// out[0] = sum of the G partial sums (fixed order) + out[1] / (2 gamma).
template <int GT>
__global__ void __launch_bounds__(GT, 1)
k_obj_final(const double* __restrict__ part, int G, double gamma, double* __restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int g = threadIdx.x; g < G; g += GT) s += part[g];
  double v[1] = {s};
  block_sum<1>(v, red);
  if (threadIdx.x == 0) out[0] = v[0] + out[1] / (2.0 * gamma);
}

}  // namespace bic
