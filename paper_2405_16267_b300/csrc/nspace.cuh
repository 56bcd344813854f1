// n-space kernels of one Bi-cADMM outer iteration (everything except the A pass).
//
//   k_rhs       r_i = rho_l q_i + rho_c (z - u_i) - c0 x_i, q_i = sum of the pass slots of
//               shard i (fixed order)                              eq. (p:GPU;x) right side
//   k_xupd      x_ij += P_ij r_ij   (block-diagonal explicit inverse, one warp per row)
//   consensus   w = (1/N) sum_i (x_i + u_i), (z, t) root solve,    eqs. (global-z-t-updae),
//               top-kappa s, v, d_r, b_r (one CTA; run by the      (s-update-final), (v-update)
//               fused pass's spare CTA or by k_global)
//   k_dual      u_i += x_i - z, p_r, inner residual, next r_i      eq. (u-update), Termination
#pragma once

#include "common.cuh"

namespace bic {

// Records kept in a handle's residual trace ring.
constexpr int kTraceCapacity = 4096;

// Per-iteration residual record (mirrored by the host).
struct Resid {
  double p_r, d_r, b_r, i_r;
  double p_rel, d_rel, b_rel, i_rel;
  double t, v, tau, znorm;
  int64_t iter;
  int64_t zt_steps;
  int64_t zt_lists;  // 1: the step visited only the prep kernel's entry lists
};

// Device-resident scalars of the global step.
struct GlobalState {
  double t, v, tau;
  int64_t iter;         // outer iterations completed
  unsigned int ticket;  // arrival counter of k_dual's last-CTA reduction
  unsigned int pad;
};

// ------------------------------------------------------------------------------ k_rhs
template <typename TM>
__global__ void k_rhs(const TM* __restrict__ slots, const int* __restrict__ slot_lo,
                      const int* __restrict__ slot_hi, const double* __restrict__ x,
                      const double* __restrict__ u, const double* __restrict__ z,
                      double* __restrict__ r, int64_t lda, double rho_l, double rho_c,
                      double c0) {
  const int i = blockIdx.y;
  const int64_t col = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (col >= lda) return;
  double q = 0.0;
  for (int sl = slot_lo[i]; sl <= slot_hi[i]; ++sl) q += static_cast<double>(slots[sl * lda + col]);
  const int64_t o = i * lda + col;
  r[o] = rho_l * q + rho_c * (z[col] - u[o]) - c0 * x[o];
}

// ------------------------------------------------------------------------------ k_xupd
// Grid (row tiles, M, N), XT threads.  P_ij is stored row-major with row stride ldp_j
// (a multiple of 32, zero padded) at P_off[i*M + j].
template <typename TP> struct PVec;
template <> struct PVec<float> { using type = float4; static constexpr int n = 4; };
template <> struct PVec<double> { using type = double2; static constexpr int n = 2; };

// FP32: at most 32 registers, so that a full SM's worth of warps keeps P loads in flight.
template <typename TP, typename TX, int XT, int ROWS>
__global__ void __launch_bounds__(XT, sizeof(TP) == 4 ? 2048 / XT : 1)
k_xupd(const TP* __restrict__ P, const int64_t* __restrict__ P_off,
       const int* __restrict__ blk_col0, const int* __restrict__ blk_ldp,
       const double* __restrict__ r, double* __restrict__ x, TX* __restrict__ xlo, int M,
       int64_t lda) {
  using V = typename PVec<TP>::type;
  constexpr int VE = PVec<TP>::n;
  extern __shared__ __align__(16) unsigned char xs_raw[];
  TP* rs = reinterpret_cast<TP*>(xs_raw);
  const int i = blockIdx.z, j = blockIdx.y;
  const int col0 = blk_col0[j], nj = blk_col0[j + 1] - col0, ldp = blk_ldp[j];
  const int row_begin = blockIdx.x * ROWS;
  if (row_begin >= nj) return;
  for (int k = threadIdx.x; k < ldp; k += XT)
    rs[k] = k < nj ? static_cast<TP>(r[i * lda + col0 + k]) : TP(0);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const TP* Pb = P + P_off[i * M + j];
  const V* rv = reinterpret_cast<const V*>(rs);
  const int nv = ldp / VE;
  constexpr int U = 8;  // 16-byte loads in flight per lane
  for (int row = row_begin + warp; row < row_begin + ROWS && row < nj; row += XT / 32) {
    const V* pr = reinterpret_cast<const V*>(Pb + static_cast<int64_t>(row) * ldp);
    TP acc = TP(0);
    for (int k0 = 0; k0 < nv; k0 += 32 * U) {
      V a[U];
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int k = k0 + q * 32 + lane;
        if (k < nv) a[q] = pr[k]; else a[q] = V{};
      }
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int k = k0 + q * 32 + lane;
        if (k < nv) {
          const V bb = rv[k];
          const TP* ae = reinterpret_cast<const TP*>(&a[q]);
          const TP* be = reinterpret_cast<const TP*>(&bb);
#pragma unroll
          for (int e = 0; e < VE; ++e) acc = fma(ae[e], be[e], acc);
        }
      }
    }
    acc = warp_sum(acc);
    if (lane == 0) {
      const int64_t o = i * lda + col0 + row;
      const double xn = x[o] + static_cast<double>(acc);
      x[o] = xn;
      xlo[o] = static_cast<TX>(xn);
    }
  }
}

// ------------------------------------------------------------------------------ top-kappa
// Select the kappa largest |z_r| (ties: lowest index) inside one CTA of GT threads by an
// MSB-first radix select on the IEEE bit patterns of |z_r| (non-negative doubles order as
// unsigned integers), then rank the entries equal to the threshold by index with a
// block-wide scan.  Each thread owns a contiguous chunk of at most 32*MW indices and gets
// its selection as a bit mask.  key[] is global scratch of n entries.
// With ccap > 0, ckey is shared memory for ccap keys: the nonzero keys are gathered there
// (in any order: the digit counts do not depend on it) and, when they fit, the radix passes
// count only them.  A zero key is selected only when fewer than kappa keys are nonzero, and
// then it is the threshold itself (the first kappa - nnz zeros by index); z after the l1
// projection is mostly zero, so the passes touch a small fraction of the entries.
template <int GT, int MW>
__device__ void block_topk_select(const double* __restrict__ z, uint64_t* __restrict__ key,
                                  int64_t n, int64_t kappa, uint32_t (&sel)[MW],
                                  int64_t& chunk_begin, int& chunk_len,
                                  uint64_t* ckey = nullptr, int64_t ccap = 0) {
  __shared__ unsigned int hist[256];
  __shared__ long long sh[2];
  __shared__ unsigned int wsum[32];
  __shared__ unsigned int ncand_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) ncand_s = 0u;
  __syncthreads();
  for (int64_t r = tid; r < n; r += GT) {
    const uint64_t k = __double_as_longlong(fabs(z[r]));
    key[r] = k;
    if (ccap > 0 && k != 0) {
      const unsigned int pos = atomicAdd(&ncand_s, 1u);
      if (pos < ccap) ckey[pos] = k;
    }
  }
  __syncthreads();
  const int64_t ncand = ncand_s;
  const bool compact = ccap > 0 && ncand <= ccap;
  uint64_t prefix = 0, mask = 0;
  int64_t remaining = kappa;
  // fewer nonzero keys than kappa: every one of them is taken, and the threshold is 0
  const bool all_nonzero = compact && ncand < kappa;
  if (all_nonzero) remaining = kappa - ncand;
  for (int shift = 56; shift >= 0 && !all_nonzero; shift -= 8) {
    for (int b = tid; b < 256; b += GT) hist[b] = 0;
    __syncthreads();
    if (compact) {
      for (int64_t r = tid; r < ncand; r += GT) {
        const uint64_t k = ckey[r];
        if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & 255u], 1u);
      }
    } else {
      for (int64_t r = tid; r < n; r += GT) {
        const uint64_t k = key[r];
        if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & 255u], 1u);
      }
    }
    __syncthreads();
    if (warp == 0) {
      // lane l owns bins 255-8l .. 248-8l (descending); counts accumulate from the top.
      unsigned int cnt[8], tot = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) { cnt[q] = hist[255 - 8 * lane - q]; tot += cnt[q]; }
      unsigned int incl = tot;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const unsigned int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
      }
      const unsigned int excl = incl - tot;
      // the threshold digit is in the first lane whose inclusive count reaches remaining
      const bool here = static_cast<int64_t>(excl) < remaining &&
                        static_cast<int64_t>(incl) >= remaining;
      if (here) {
        unsigned int run = excl;
        for (int q = 0; q < 8; ++q) {
          if (static_cast<int64_t>(run + cnt[q]) >= remaining) {
            sh[0] = 255 - 8 * lane - q;
            sh[1] = remaining - run;
            break;
          }
          run += cnt[q];
        }
      }
    }
    __syncthreads();
    prefix |= static_cast<uint64_t>(sh[0]) << shift;
    mask |= static_cast<uint64_t>(255) << shift;
    remaining = sh[1];
    __syncthreads();
  }
  // prefix = threshold key; take every key above it and the first `remaining` equal ones.
  const int64_t ch = (n + GT - 1) / GT;
  chunk_begin = tid * ch;
  const int64_t cend = chunk_begin + ch < n ? chunk_begin + ch : n;
  chunk_len = chunk_begin < cend ? static_cast<int>(cend - chunk_begin) : 0;
  unsigned int eq = 0;
  for (int q = 0; q < chunk_len; ++q) eq += key[chunk_begin + q] == prefix;
  unsigned int incl = eq;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned int y = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const unsigned int v = lane < GT / 32 ? wsum[lane] : 0u;
    unsigned int inc = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned int y = __shfl_up_sync(0xffffffffu, inc, off);
      if (lane >= off) inc += y;
    }
    wsum[lane] = inc - v;
  }
  __syncthreads();
  unsigned int rank = wsum[warp] + incl - eq;
#pragma unroll
  for (int q = 0; q < MW; ++q) sel[q] = 0u;
  for (int q = 0; q < chunk_len; ++q) {
    const uint64_t k = key[chunk_begin + q];
    bool take = k > prefix;
    if (k == prefix) { take = static_cast<int64_t>(rank) < remaining; ++rank; }
    if (take) sel[q >> 5] |= 1u << (q & 31);
  }
  __syncthreads();
}

// ------------------------------------------------------------------------------ consensus
// The global step of one outer iteration, executed by one CTA:
//   w = (1/N) sum_i (x_i + u_i)              (or taken from the caller)
//   (z, t) of eq. (global-z-t-updae), s of eq. (s-update-final), v of eq. (v-update)
//   and the d_r / b_r part of the residual record.
// The (z,t) root: h(tau) = v + beta tau + sum_{r: tau_r > tau} (c_r + e_r tau) is concave,
// increasing and piecewise linear (c_r = s_r w_r - |w_r|, e_r = (s_r - sign w_r)^2,
// tau_r = |w_r| / (1 - sign(w_r) s_r) the point where z_r reaches 0).  Newton from the left
// never overshoots the root and the active set only shrinks, so the iteration ends, exactly,
// when the active set stops changing.  It starts from the previous iteration's tau when
// h is still non-positive there, else from 0.
struct ConsensusArgs {
  const double* x;   // N x lda, or nullptr when w is given
  const double* u;   // N x lda
  double* w;         // n: written when x is given, read otherwise
  double* z;         // n: in z^k (dual residual), out z^{k+1}
  double* s;         // n: in s^k, out s^{k+1}
  double* tau_r;     // n scratch
  double* c_arr;     // n scratch
  double* e_arr;     // n scratch
  uint64_t* key;     // n scratch
  GlobalState* gs;
  Resid* trace;
  int trace_cap;
  int N;
  int64_t n, kappa, lda;
  double rho_c, rho_b;
  int* err;
  int enabled;       // used by the fused pass: 1 = its last CTA runs this step
  int prepared;      // 1: w, tau_r, c_arr, e_arr were formed by k_consensus_prep
  int64_t cand_bytes;  // dynamic shared memory the running CTA may use for top-kappa
                       // candidates (0: none; the select then reads every key each pass)
  // Several instances on one A (a sparsity path, see bicadmm_create_path): ninst > 1
  // consensus CTAs, instance q working on w, z, s, tau_r, c_arr, e_arr, key + q * inst_n
  // (instance-major slices of n entries), its own kappas[q], gs + q and trace + q * trace_cap.
  int ninst;           // 0 or 1: one instance (the fields above as they are)
  int64_t inst_n;
  const int64_t* kappas;
  // Entry lists of k_consensus_prep (nullptr: none): for each block of kPrepBlock entries,
  // u_cnt[b] entries of U = {r : tau_r > tau_prev or z_r != 0 or s_r != 0} at
  // u_idx[b kPrepBlock ...] in index order; u_nb blocks per instance.
  const int* u_idx;
  const int* u_cnt;
  int u_nb;
};

// The consensus arguments of instance q of a path (q = 0 and a single instance: unchanged).
__device__ __forceinline__ ConsensusArgs consensus_instance(const ConsensusArgs& c, int q) {
  ConsensusArgs a = c;
  if (c.ninst > 1) {
    const int64_t o = static_cast<int64_t>(q) * c.inst_n;
    a.w += o; a.z += o; a.s += o; a.tau_r += o; a.c_arr += o; a.e_arr += o; a.key += o;
    a.gs += q;
    a.trace += static_cast<int64_t>(q) * c.trace_cap;
    a.kappa = c.kappas[q];
    if (c.u_idx) {
      a.u_idx += o;
      a.u_cnt += static_cast<int64_t>(q) * c.u_nb;
    }
  }
  return a;
}
__device__ __forceinline__ int consensus_ctas(const ConsensusArgs& c) {
  return c.enabled ? (c.ninst > 1 ? c.ninst : 1) : 0;
}

// Entries per block of k_consensus_prep (its lists are per block of this many entries).
constexpr int kPrepBlock = 256;

// Exclusive prefix of x over the CTA's GT threads in thread order; *total gets the sum.
// wtot: GT / 32 + 1 ints of shared memory.
template <int GT>
__device__ __forceinline__ int block_excl_scan(int x, int* wtot, int* total) {
  constexpr int NW = GT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = x;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += y;
  }
  if (lane == 31) wtot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int t = lane < NW ? wtot[lane] : 0;
    int ti = t;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, ti, off);
      if (lane >= off) ti += y;
    }
    __syncwarp();
    if (lane < NW) wtot[lane] = ti - t;
    if (lane == 31) wtot[NW] = ti;
  }
  __syncthreads();
  const int res = wtot[warp] + incl - x;
  *total = wtot[NW];
  __syncthreads();
  return res;
}

// The record of the step (residual trace, t, v, tau) written by thread 0.
__device__ __forceinline__ void consensus_record(const ConsensusArgs& a, double v, double t, double g,
                                                 double tau, const double (&a4)[4], int64_t steps,
                                                 int lists) {
  const double vn = v + g;
  Resid& rec = a.trace[a.gs->iter % a.trace_cap];
  const double dz = sqrt(a4[2]), zn = sqrt(a4[3]);
  rec.d_r = sqrt(static_cast<double>(a.N)) * a.rho_c * dz;
  rec.b_r = fabs(g);
  rec.d_rel = dz / fmax(zn, 1e-30);
  rec.b_rel = fabs(g) / fmax(t, 1e-30);
  rec.t = t;
  rec.v = vn;
  rec.tau = tau;
  rec.znorm = zn;
  rec.iter = a.gs->iter + 1;
  rec.zt_steps = steps;
  rec.zt_lists = lists;
  a.gs->t = t;
  a.gs->v = vn;
  a.gs->tau = tau;
}

// The consensus step on the entry lists of k_consensus_prep.  With the previous root
// tau_prev > 0, every entry outside U has s_r = 0, z_r = 0 and tau_r = |w_r| <= tau_prev; a
// warm start from tau_prev (h(tau_prev) <= 0) only moves tau up, so such an entry stays at
// z_r = S_tau(w_r) = 0 and s_r = 0 and adds nothing to any sum.  The step therefore visits U
// alone: the root's sums over {tau_r > tau} (a subset of U), z and the norms on U, the
// top-kappa select over U's nonzero z (ties by index: U is in index order), s on U.  Every
// O(n) scan ran on all SMs in the prep kernel; here U (about the support size) is gathered
// into shared memory with independent loads.  Returns false, having written nothing, when U
// does not fit in `bytes` of shared memory or h(tau_prev) > 0; the caller then runs the
// full-length step.  The arithmetic per entry is that of the full-length step.
template <int GT>
__device__ bool consensus_lists(const ConsensusArgs& a, unsigned char* smem, int64_t bytes,
                                double v, double tau_prev, double beta, double* red) {
  constexpr int NW = GT / 32;
  __shared__ unsigned int hist[256];
  __shared__ long long sh[2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = a.u_nb;
  if (nb <= 0 || nb > GT) return false;
  int* pref = reinterpret_cast<int*>(smem);  // nb + 1 list offsets
  int* wtot = pref + GT + 1;                 // NW + 1
  const int64_t head = (static_cast<int64_t>(GT + 1 + NW + 1) * 4 + 15) & ~15ll;
  const int64_t cap = (bytes - head) / 60;   // 7 doubles and an index per entry
  if (cap <= 0) return false;
  int total = 0;
  const int off = block_excl_scan<GT>(tid < nb ? a.u_cnt[tid] : 0, wtot, &total);
  if (total > cap) return false;  // total is the same in every thread
  if (tid < nb) pref[tid] = off;
  if (tid == 0) pref[nb] = total;
  __syncthreads();
  double* U_tau = reinterpret_cast<double*>(smem + head);
  double* U_c = U_tau + cap;   // c_r; after the root: 1.0 for a selected entry
  double* U_e = U_c + cap;     // e_r
  double* U_w = U_e + cap;
  double* U_s = U_w + cap;
  double* U_zo = U_s + cap;
  double* U_zn = U_zo + cap;
  int* U_idx = reinterpret_cast<int*>(U_zn + cap);
  for (int b = warp; b < nb; b += NW) {
    const int p0 = pref[b], cb = pref[b + 1] - p0;
    const int* src = a.u_idx + static_cast<int64_t>(b) * kPrepBlock;
    for (int j = lane; j < cb; j += 32) U_idx[p0 + j] = src[j];
  }
  __syncthreads();
  // six independent gathers per entry, four entries per thread in flight
  for (int i0 = tid; i0 < total; i0 += 4 * GT) {
    int r[4];
    double t4[4], c4[4], e4[4], w4[4], s4[4], z4[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) r[k] = i0 + k * GT < total ? U_idx[i0 + k * GT] : -1;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (r[k] >= 0) {
        t4[k] = a.tau_r[r[k]];
        c4[k] = a.c_arr[r[k]];
        e4[k] = a.e_arr[r[k]];
        w4[k] = a.w[r[k]];
        s4[k] = a.s[r[k]];
        z4[k] = a.z[r[k]];
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (r[k] >= 0) {
        const int i = i0 + k * GT;
        U_tau[i] = t4[k];
        U_c[i] = c4[k];
        U_e[i] = e4[k];
        U_w[i] = w4[k];
        U_s[i] = s4[k];
        U_zo[i] = z4[k];
      }
    }
  }
  __syncthreads();

  // the root: sums of c_r, e_r and the count over {tau_r > at} (all in U for at >= tau_prev)
  auto active_sums = [&](double at, double (&o)[3]) {
    o[0] = o[1] = 0.0;
    int cnt = 0;
    const long long atb = __double_as_longlong(at);
    for (int i = tid; i < total; i += GT) {
      if (__double_as_longlong(U_tau[i]) > atb) {
        o[0] += U_c[i];
        o[1] += U_e[i];
        ++cnt;
      }
    }
    o[2] = static_cast<double>(cnt);
    block_sum<3>(o, red);
  };
  double cur[3];
  active_sums(tau_prev, cur);
  if (!(v + cur[0] + (beta + cur[1]) * tau_prev <= 0.0)) return false;  // h(tau_prev) > 0
  double tau = tau_prev;
  int64_t steps = 0;
  const int64_t max_steps = a.n + 2;
  for (;;) {
    const double tn = -(v + cur[0]) / (beta + cur[1]);
    double nxt[3];
    active_sums(tn, nxt);
    ++steps;
    tau = tn;
    if (nxt[2] >= cur[2]) break;
    cur[0] = nxt[0]; cur[1] = nxt[1]; cur[2] = nxt[2];
    if (steps > max_steps) {
      if (tid == 0) set_err(a.err, DEV_ZT_NOCONV);
      break;
    }
  }

  // z = S_tau(w + tau s) on U (tau >= tau_prev > 0); norms; nonzero keys counted
  double a4[4] = {0.0, 0.0, 0.0, 0.0};  // ||z||_1, (unused), ||z - z_prev||^2, ||z||^2
  const long long taub = __double_as_longlong(tau);
  int ncl = 0;
  for (int i = tid; i < total; i += GT) {
    const double wr = U_w[i], sr = U_s[i], zo = U_zo[i];
    const bool s_zero = (__double_as_longlong(sr) << 1) == 0;
    double zn = 0.0;
    if (!(s_zero && (__double_as_longlong(wr) & 0x7FFFFFFFFFFFFFFFll) <= taub)) {
      const double y = wr + tau * sr;
      const double mg = fabs(y) - tau;
      zn = mg > 0.0 ? dsign(y) * mg : 0.0;
    }
    U_zn[i] = zn;
    ncl += (__double_as_longlong(zn) << 1) != 0;
    if (((__double_as_longlong(zn) | __double_as_longlong(zo)) << 1) != 0) {
      a4[0] += fabs(zn);
      a4[2] += (zn - zo) * (zn - zo);
      a4[3] += zn * zn;
      a.z[U_idx[i]] = zn;
    }
  }
  block_sum<4>(a4, red);
  const double t = a4[0];
  int ncand = 0;
  block_excl_scan<GT>(ncl, wtot, &ncand);

  // top-kappa of |z| over the nonzero keys of U (a zero z_r gets s_r = 0 whether or not it
  // is counted among the kappa); ties at the threshold by index, i.e. by position in U
  const bool take_all = ncand <= a.kappa;
  uint64_t prefix = 0, mask = 0;
  int64_t remaining = a.kappa;
  for (int shift = 56; shift >= 0 && !take_all; shift -= 8) {
    for (int b = tid; b < 256; b += GT) hist[b] = 0;
    __syncthreads();
    for (int i = tid; i < total; i += GT) {
      const uint64_t k = __double_as_longlong(fabs(U_zn[i]));
      if (k != 0 && (k & mask) == prefix) atomicAdd(&hist[(k >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (warp == 0) {
      unsigned int cnt[8], tot = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) { cnt[q] = hist[255 - 8 * lane - q]; tot += cnt[q]; }
      unsigned int incl = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const unsigned int excl = incl - tot;
      if (static_cast<int64_t>(excl) < remaining && static_cast<int64_t>(incl) >= remaining) {
        unsigned int run = excl;
        for (int q = 0; q < 8; ++q) {
          if (static_cast<int64_t>(run + cnt[q]) >= remaining) {
            sh[0] = 255 - 8 * lane - q;
            sh[1] = remaining - run;
            break;
          }
          run += cnt[q];
        }
      }
    }
    __syncthreads();
    prefix |= static_cast<uint64_t>(sh[0]) << shift;
    mask |= static_cast<uint64_t>(255) << shift;
    remaining = sh[1];
    __syncthreads();
  }
  // selection flags: above the threshold, or equal to it and among the first `remaining`
  // equal ones in U order (each thread ranks a contiguous segment of U)
  const int seg = (total + GT - 1) / GT;
  const int s0 = tid * seg < total ? tid * seg : total;
  const int s1 = s0 + seg < total ? s0 + seg : total;
  int eq = 0;
  if (!take_all)
    for (int i = s0; i < s1; ++i) eq += static_cast<uint64_t>(__double_as_longlong(fabs(U_zn[i]))) == prefix;
  int eqt = 0;
  int rank = block_excl_scan<GT>(eq, wtot, &eqt);
  double a1b[1] = {0.0};
  for (int i = s0; i < s1; ++i) {
    const uint64_t k = __double_as_longlong(fabs(U_zn[i]));
    bool take;
    if (take_all) {
      take = k != 0;
    } else {
      take = k > prefix;
      if (k == prefix) { take = rank < remaining; ++rank; }
    }
    U_c[i] = take ? 1.0 : 0.0;
    if (take) a1b[0] += fabs(U_zn[i]);
  }
  block_sum<1>(a1b, red);
  const double T = a1b[0];
  double scale = 0.0;
  if (T > 0.0) {
    scale = (t - v) / T;
    scale = scale > 1.0 ? 1.0 : (scale < -1.0 ? -1.0 : scale);
  }
  double a1c[1] = {0.0};
  for (int i = s0; i < s1; ++i) {
    double sn = 0.0;
    if (U_c[i] != 0.0) {
      const double zr = U_zn[i];
      sn = scale * dsign(zr);
      a1c[0] += zr * sn;
    }
    if ((__double_as_longlong(sn) | __double_as_longlong(U_s[i])) != 0) a.s[U_idx[i]] = sn;
  }
  block_sum<1>(a1c, red);
  if (tid == 0) consensus_record(a, v, t, a1c[0] - t, tau, a4, steps, 1);
  return true;
}

// LISTS: compile the list form in (the multi-column passes, whose consensus is prepared).
template <int GT, int MW, bool LISTS = false>
__device__ void consensus_block(const ConsensusArgs& a, unsigned char* dyn_smem = nullptr) {
  __shared__ double red[32 * 4];
  const int tid = threadIdx.x;
  const int64_t n = a.n;
  const double v = a.gs->v, tau_prev = a.gs->tau;
  const double beta = a.N * a.rho_c / a.rho_b;
  if constexpr (LISTS) {
    if (a.prepared && a.u_idx && dyn_smem && tau_prev > 0.0 &&
        consensus_lists<GT>(a, dyn_smem, a.cand_bytes, v, tau_prev, beta, red))
      return;
  }

  for (int64_t r = a.prepared ? n : tid; r < n; r += GT) {
    double wr;
    if (a.x) {
      double acc = 0.0;
      for (int i = 0; i < a.N; ++i) acc += a.x[i * a.lda + r] + a.u[i * a.lda + r];
      wr = acc / a.N;
      a.w[r] = wr;
    } else {
      wr = a.w[r];
    }
    const double sr = a.s[r], sg = dsign(wr);
    a.c_arr[r] = sr * wr - fabs(wr);
    a.e_arr[r] = (sr - sg) * (sr - sg);
    // w_r = 0: z_r stays 0 for every tau >= 0 (never active).  sign(w_r) s_r = 1: never
    // zeroed, and contributes c_r = e_r = 0.
    a.tau_r[r] = wr == 0.0 ? 0.0 : (sg * sr < 1.0 ? fabs(wr) / (1.0 - sg * sr) : HUGE_VAL);
  }
  __syncthreads();

  // sums of c_r, e_r and the count over the active set {r : tau_r > at}; breakpoints are
  // non-negative, so they compare as their bit patterns.
  auto active_sums = [&](double at, double (&o)[3]) {
    o[0] = o[1] = 0.0;
    int cnt = 0;
    const long long atb = __double_as_longlong(at);
    for (int64_t r = tid; r < n; r += GT) {
      if (__double_as_longlong(a.tau_r[r]) > atb) {
        o[0] += a.c_arr[r];
        o[1] += a.e_arr[r];
        ++cnt;
      }
    }
    o[2] = static_cast<double>(cnt);
    block_sum<3>(o, red);
  };

  double cur[3];
  double tau = 0.0, tstart = 0.0;
  bool active = true;
  bool warm = false;
  if (tau_prev > 0.0) {
    active_sums(tau_prev, cur);
    warm = v + cur[0] + (beta + cur[1]) * tau_prev <= 0.0;  // h(tau_prev) <= 0
  }
  if (warm) {
    tstart = tau_prev;
  } else {
    active_sums(0.0, cur);
    active = v + cur[0] < 0.0;  // h(0) < 0: the l1 constraint binds
  }
  int64_t steps = 0;
  if (active) {
    tau = tstart;
    const int64_t max_steps = n + 2;
    for (;;) {
      const double tn = -(v + cur[0]) / (beta + cur[1]);
      double nxt[3];
      active_sums(tn, nxt);
      ++steps;
      tau = tn;
      if (nxt[2] >= cur[2]) break;
      cur[0] = nxt[0]; cur[1] = nxt[1]; cur[2] = nxt[2];
      if (steps > max_steps) {
        if (tid == 0) set_err(a.err, DEV_ZT_NOCONV);
        break;
      }
    }
  }

  // z = S_tau(w + tau s) (z = w when the constraint is inactive); norms for t and d_r.
  double a4[4] = {0.0, 0.0, 0.0, 0.0};  // ||z||_1, s'w, ||z - z_prev||^2, ||z||^2
  // FP64 instructions are the scarce resource of this single CTA (each occupies the SM's
  // FP64 pipe for many cycles), and after the projection most entries stay zero: an entry
  // with s_r = 0 and |w_r| <= tau is zero without arithmetic (an integer compare of bit
  // patterns), and entries zero before and after add exact zeros to every sum (skipped, so
  // the sums are those of the full loop).
  const long long taub = __double_as_longlong(tau);
  const bool tpos = tau > 0.0;
  for (int64_t r = tid; r < n; r += GT) {
    const double wr = a.w[r], sr = a.s[r];
    const double zo = a.z[r];
    const bool s_zero = (__double_as_longlong(sr) << 1) == 0;
    double zn = 0.0;
    if (tpos) {
      if (!(s_zero && (__double_as_longlong(wr) & 0x7FFFFFFFFFFFFFFFll) <= taub)) {
        const double y = wr + tau * sr;
        const double mg = fabs(y) - tau;
        zn = mg > 0.0 ? dsign(y) * mg : 0.0;
      }
    } else {
      zn = wr;
      if (!s_zero) a4[1] += sr * wr;
    }
    if (((__double_as_longlong(zn) | __double_as_longlong(zo)) << 1) != 0) {
      a4[0] += fabs(zn);
      a4[2] += (zn - zo) * (zn - zo);
      a4[3] += zn * zn;
      a.z[r] = zn;
    }
  }
  block_sum<4>(a4, red);
  const double t = tau > 0.0 ? a4[0] : a4[1] + v;

  // s: top-kappa signs of z scaled by clamp((t - v)/T, -1, 1).
  int64_t cb;
  int cl;
  uint32_t sel[MW];
  block_topk_select<GT, MW>(a.z, a.key, n, a.kappa, sel, cb, cl,
                            reinterpret_cast<uint64_t*>(dyn_smem),
                            dyn_smem ? a.cand_bytes / static_cast<int64_t>(sizeof(uint64_t)) : 0);
  double a1b[1] = {0.0};
  for (int q = 0; q < cl; ++q)
    if (sel[q >> 5] >> (q & 31) & 1u) a1b[0] += fabs(a.z[cb + q]);
  block_sum<1>(a1b, red);
  const double T = a1b[0];
  double scale = 0.0;
  if (T > 0.0) {
    scale = (t - v) / T;
    scale = scale > 1.0 ? 1.0 : (scale < -1.0 ? -1.0 : scale);
  }
  double a1c[1] = {0.0};
  for (int q = 0; q < cl; ++q) {
    if (sel[q >> 5] >> (q & 31) & 1u) {
      const double zr = a.z[cb + q];
      const double sn = scale * dsign(zr);
      a.s[cb + q] = sn;
      a1c[0] += zr * sn;
    } else {
      a.s[cb + q] = 0.0;  // an unselected entry adds an exact zero to z's
    }
  }
  block_sum<1>(a1c, red);
  const double g = a1c[0] - t;
  if (tid == 0) consensus_record(a, v, t, g, tau, a4, steps, 0);
}

// Standalone single-CTA consensus step (n <= 32 * MW * GT).
template <int GT, int MW>
__global__ void __launch_bounds__(GT, 1) k_global(ConsensusArgs a) {
  consensus_block<GT, MW>(a);
}

// ------------------------------------------------------------------------------ k_consensus_prep
// The per-entry part of the (z,t) step, on every SM: w = (1/N) sum_i (x_i + u_i) (shards
// in index order, deterministic) and, with the current s, the breakpoint tau_r and the
// coefficients c_r, e_r of h (the same formulas as the consensus block).  Run before the
// pass that carries the consensus CTA (ConsensusArgs::prepared = 1), which then starts at
// the root search; on B300 FP64 runs at a small fraction of FP32, so this per-entry work
// (a division per entry) is what one SM should not do for large n.  Each block of
// kPrepBlock entries also lists, in index order, its entries of
// U = {r : tau_r > tau_prev or z_r != 0 or s_r != 0} (tau_prev = gs->tau, the root of the
// previous step): the consensus CTA's warm-started step visits only those.

// Appends `value` for every thread with `flag` to dst in thread order; *cnt = their number.
// One block of kPrepBlock threads.
__device__ __forceinline__ void block_list_append(bool flag, int value, int* __restrict__ dst,
                                                  int* __restrict__ cnt) {
  __shared__ int wc[kPrepBlock / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned int m = __ballot_sync(0xffffffffu, flag);
  if (lane == 0) wc[warp] = __popc(m);
  __syncthreads();
  int base = 0;
  for (int k = 0; k < warp; ++k) base += wc[k];
  if (flag) dst[base + __popc(m & ((1u << lane) - 1u))] = value;
  if (threadIdx.x == 0) {
    int t = 0;
    for (int k = 0; k < kPrepBlock / 32; ++k) t += wc[k];
    *cnt = t;
  }
}

__device__ __forceinline__ bool prep_entry(const double* __restrict__ x, const double* __restrict__ u,
                                           int64_t xo, int64_t ld, int N, double sr, double zr,
                                           long long tau_prev_bits, double& wr, double& c, double& e,
                                           double& tr) {
  double acc = 0.0;
  for (int i = 0; i < N; ++i) acc += x[i * ld + xo] + u[i * ld + xo];
  wr = acc / N;
  const double sg = dsign(wr);
  c = sr * wr - fabs(wr);
  e = (sr - sg) * (sr - sg);
  tr = wr == 0.0 ? 0.0 : (sg * sr < 1.0 ? fabs(wr) / (1.0 - sg * sr) : HUGE_VAL);
  return __double_as_longlong(tr) > tau_prev_bits ||
         ((__double_as_longlong(zr) | __double_as_longlong(sr)) << 1) != 0;
}

static __global__ void __launch_bounds__(kPrepBlock)
k_consensus_prep(const double* __restrict__ x, const double* __restrict__ u,
                 const double* __restrict__ s, const double* __restrict__ z,
                 double* __restrict__ w, double* __restrict__ tau_r, double* __restrict__ c_arr,
                 double* __restrict__ e_arr, const GlobalState* __restrict__ gs,
                 int* __restrict__ u_idx, int* __restrict__ u_cnt, int N, int64_t n, int64_t lda) {
  const int64_t r = static_cast<int64_t>(blockIdx.x) * kPrepBlock + threadIdx.x;
  bool in_u = false;
  if (r < n) {
    double wr, c, e, tr;
    in_u = prep_entry(x, u, r, lda, N, s[r], z[r], __double_as_longlong(gs->tau), wr, c, e, tr);
    w[r] = wr;
    c_arr[r] = c;
    e_arr[r] = e;
    tau_r[r] = tr;
  }
  block_list_append(in_u, static_cast<int>(r), u_idx + static_cast<int64_t>(blockIdx.x) * kPrepBlock,
                    u_cnt + blockIdx.x);
}

// A path (several instances on one A, K = their count): the same per-entry work, written
// instance-major (instance q's n entries contiguous, from q n), which is the layout its
// consensus CTAs work on; x and u are feature-major (entry (c, q) at c K + q), s and z
// instance-major.  Grid (blocks per instance, K); instance q's lists hold indices within
// the instance, from q n (u_idx) and q gridDim.x (u_cnt).
static __global__ void __launch_bounds__(kPrepBlock)
k_consensus_prep_path(const double* __restrict__ x, const double* __restrict__ u,
                      const double* __restrict__ s_cm, const double* __restrict__ z_cm,
                      double* __restrict__ w_cm, double* __restrict__ tau_r,
                      double* __restrict__ c_arr, double* __restrict__ e_arr,
                      const GlobalState* __restrict__ gs, int* __restrict__ u_idx,
                      int* __restrict__ u_cnt, int N, int64_t n, int K, int64_t ldx) {
  const int q = blockIdx.y;
  const int64_t c = static_cast<int64_t>(blockIdx.x) * kPrepBlock + threadIdx.x;
  const int64_t r = static_cast<int64_t>(q) * n + c;
  bool in_u = false;
  if (c < n) {
    double wr, cc, e, tr;
    in_u = prep_entry(x, u, c * K + q, ldx, N, s_cm[r], z_cm[r], __double_as_longlong(gs[q].tau),
                      wr, cc, e, tr);
    w_cm[r] = wr;
    c_arr[r] = cc;
    e_arr[r] = e;
    tau_r[r] = tr;
  }
  block_list_append(in_u, static_cast<int>(c),
                    u_idx + static_cast<int64_t>(q) * n + static_cast<int64_t>(blockIdx.x) * kPrepBlock,
                    u_cnt + static_cast<int64_t>(q) * gridDim.x + blockIdx.x);
}

// A path: the consensus CTAs' z and s (instance-major) to the feature-major layout the
// x-update and the duals read.
static __global__ void k_path_to_feature_major(const double* __restrict__ z_cm,
                                               const double* __restrict__ s_cm, double* __restrict__ z,
                                               double* __restrict__ s, int64_t n, int K) {
  const int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (r >= n * K) return;
  const int64_t q = r / n, c = r - q * n;
  z[c * K + q] = z_cm[r];
  s[c * K + q] = s_cm[r];
}

// ------------------------------------------------------------------------------ k_dual
// Grid (chunks, N), DT threads.  End of an outer iteration: u_i += x_i - z (eq. u-update),
// per-(shard, chunk) sums of ||x_i - z||^2 and ||x_i||^2, and the right-hand side of the next
// iteration's first x-block solve, r_i = rho_l q_i + rho_c (z - u_i) - c0 x_i with q_i the
// fixed-order sum of the last pass's slots of shard i.  The last CTA to finish reduces the
// sums (fixed order) with the pass's inner-residual sums into the residual record and
// advances the iteration counter.
// The last CTA's sums in k_dual / k_dual_batch, in a fixed order with the whole CTA: warp w
// takes shards w, w + NW, ... and its lanes the chunks lane, lane + 32, ... of each (one
// warp_sum per shard), every thread a strided share of the pass CTAs' statistics; per-warp
// results are added in warp order by thread 0, which receives pr = sum_i ||x_i - z||,
// nx = sum_i ||x_i|| and the three inner-residual sums.
template <int DT>
__device__ __forceinline__ void dual_final_sums(const double* __restrict__ part, int N, int nch,
                                                const double* __restrict__ cta_stats, int G,
                                                double (&out)[5]) {
  constexpr int NW = DT / 32;
  constexpr int U = 4;  // shards of a warp whose partial sums are loaded together
  __shared__ double fin[NW * 5];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double w[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  // The pass CTAs' statistics, two strided entries per thread in flight at once (the same
  // order of additions as one entry at a time).
  double g[3] = {0.0, 0.0, 0.0};
  for (int q0 = threadIdx.x; q0 < G; q0 += 2 * DT) {
    double v[2][3];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = q0 + h * DT;
#pragma unroll
      for (int k = 0; k < 3; ++k) v[h][k] = q < G ? cta_stats[q * 4 + k] : 0.0;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int k = 0; k < 3; ++k) g[k] += v[h][k];
  }
  // The shard sums: U shards of a warp at a time (w, w + NW, ...), all their loads issued
  // before the first warp sum; the square roots are added in shard order as before.
  for (int ii0 = warp; ii0 < N; ii0 += U * NW) {
    double s0[U], s1[U];
#pragma unroll
    for (int u = 0; u < U; ++u) s0[u] = s1[u] = 0.0;
    for (int c = lane; c < nch; c += 32) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int ii = ii0 + u * NW;
        if (ii < N) {
          s0[u] += part[(static_cast<int64_t>(ii) * nch + c) * 2 + 0];
          s1[u] += part[(static_cast<int64_t>(ii) * nch + c) * 2 + 1];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const double a0 = warp_sum(s0[u]), a1 = warp_sum(s1[u]);
      if (ii0 + u * NW < N) {
        w[0] += sqrt(a0);
        w[1] += sqrt(a1);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) w[2 + k] = warp_sum(g[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 5; ++k) fin[warp * 5 + k] = w[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 5; ++k) out[k] = 0.0;
  if (threadIdx.x == 0) {
    for (int ww = 0; ww < NW; ++ww)
#pragma unroll
      for (int k = 0; k < 5; ++k) out[k] += fin[ww * 5 + k];
  }
}

template <typename TM, int DT>
__global__ void __launch_bounds__(DT)
k_dual(double* __restrict__ u, const double* __restrict__ x, const double* __restrict__ z,
       const TM* __restrict__ slots, const int* __restrict__ slot_lo,
       const int* __restrict__ slot_hi, double* __restrict__ r, double rho_l, double c0,
       double* __restrict__ part, const double* __restrict__ cta_stats, int G, GlobalState* gs,
       Resid* trace, int trace_cap, int N, int64_t n, int64_t lda, double rho_c, int* err,
       int ninst) {
  __shared__ double red[32 * 2];
  __shared__ bool last;
  const int i = blockIdx.y, nch = gridDim.x;
  double a[2] = {0.0, 0.0};
  // each CTA takes the columns blockIdx.x * DT + tid + k * nch * DT of its shard, two per
  // step with all their loads issued before use (the loop is latency-bound)
  const int s_lo = slot_lo[i], s_hi = slot_hi[i];
  const int64_t stride = static_cast<int64_t>(nch) * DT;
  for (int64_t c0l = static_cast<int64_t>(blockIdx.x) * DT + threadIdx.x; c0l < lda; c0l += 2 * stride) {
    double xv[2], zv[2], uv[2];
    TM q[2] = {TM(0), TM(0)};  // the slots are partial sums in the arithmetic type of the pass
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t col = c0l + h * stride;
      const bool ok = col < lda;
      const int64_t o = i * lda + (ok ? col : 0);
      xv[h] = ok ? x[o] : 0.0;
      zv[h] = ok ? z[col] : 0.0;
      uv[h] = ok ? u[o] : 0.0;
      if (ok)
        for (int sl = s_lo; sl <= s_hi; ++sl) q[h] += slots[sl * lda + col];
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t col = c0l + h * stride;
      if (col < lda) {
        const int64_t o = i * lda + col;
        const double dv = xv[h] - zv[h];
        const double un = uv[h] + dv;
        u[o] = un;
        r[o] = rho_l * static_cast<double>(q[h]) + rho_c * (zv[h] - un) - c0 * xv[h];
        a[0] += dv * dv;  // padding columns hold zeros
        a[1] += xv[h] * xv[h];
      }
    }
  }
  block_sum<2>(a, red);
  if (threadIdx.x == 0) {
    part[(static_cast<int64_t>(i) * nch + blockIdx.x) * 2 + 0] = a[0];
    part[(static_cast<int64_t>(i) * nch + blockIdx.x) * 2 + 1] = a[1];
    __threadfence();
    const unsigned int total = gridDim.x * gridDim.y;
    last = atomicAdd(&gs->ticket, 1u) == total - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // thread 0 reads the iteration counter and the record's ||z|| (from earlier launches)
  // before the sums, so that their latency overlaps the sums'
  double zn0 = 0.0;
  if (threadIdx.x == 0) zn0 = trace[gs->iter % trace_cap].znorm;
  double fs[5];
  dual_final_sums<DT>(part, N, nch, cta_stats, G, fs);
  {
    const double pr = fs[0], nx = fs[1], q0 = fs[2], q1 = fs[3], q2 = fs[4];
    if (threadIdx.x == 0) {
      // A path (ninst > 1): the shard sums and the inner residual cover every instance's
      // column (one record each gets them, with ||z|| over all instances); one instance:
      // its own record.
      const int nq = ninst > 1 ? ninst : 1;
      double zn = zn0;
      if (nq > 1) {
        double zn2 = 0.0;
        for (int q = 0; q < nq; ++q) {
          const double zq = trace[static_cast<int64_t>(q) * trace_cap + gs[q].iter % trace_cap].znorm;
          zn2 += zq * zq;
        }
        zn = sqrt(zn2);
      }
      for (int q = 0; q < nq; ++q) {
        GlobalState* g = gs + q;
        Resid& rec = trace[static_cast<int64_t>(q) * trace_cap + g->iter % trace_cap];
        rec.p_r = pr;
        rec.p_rel = pr / fmax(fmax(nx, N * zn), 1e-30);
        rec.i_r = sqrt(q0);
        rec.i_rel = sqrt(q0) / fmax(fmax(sqrt(q1), sqrt(q2)), 1e-30);
        const double chk = rec.p_r + rec.d_r + rec.b_r + rec.i_r + rec.t + rec.v;
        if (!isfinite(chk)) set_err(err, DEV_NONFINITE);
        g->iter += 1;
      }
      gs->ticket = 0;
    }
  }
}

}  // namespace bic
