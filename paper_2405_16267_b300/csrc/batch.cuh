// Batched execution: many independent Bi-cADMM instances advanced together, one launch per
// kernel kind per outer iteration.  Every instance keeps its own buffers (those of its
// handle); the batch adds device tables that describe them.
//
// The pass runs over a global panel list: the rows of every (instance, shard) pair form a
// "segment", segments are laid end to end, and each persistent CTA takes a contiguous range
// of panels exactly as the single-instance pass does over shards.  Crossing a segment
// boundary reloads x, flushes the A'd accumulators to the instance's slot
// (cta - first CTA of the instance) + shard, and, crossing an instance boundary, flushes the
// inner-residual sums.  The instance's slot ranges for this partition are kept by the batch
// so the dual kernel sums the right slots.
//
// Narrow instances (a row of at most NT/2 16-byte vectors) go through a second pass kernel
// over their own panel list, which splits the CTA into RP row groups of L = NT/RP threads:
// each group takes every RP-th row of the panel, so a panel holds up to R * RP rows and
// every thread has work; the groups' A'd partial sums are added in shared memory when the
// segment is flushed.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "nspace.cuh"
#include "pass.cuh"

namespace bic {

// Per-instance constants and pointers used by the batched kernels.
struct BatchInst {
  // pass
  const void* A;
  int64_t lda;
  const void* xlo;
  const void* b;
  void* omega;
  void* nu;
  void* slots;
  double* cta_stats;
  int c_lo;          // first panel CTA of the batch partition touching this instance
  int G_inst;        // panel CTAs touching it
  int loss, newton_iters;
  int lsh;           // log2 of the threads per row group (log2 NT for wide instances)
  double M, rho_l;
  // x-update and dual
  const void* P;
  const int64_t* P_off;
  const int* blk_col0;
  const int* blk_ldp;
  int M_blocks, N;
  double* x;
  double* u;
  double* r;
  const double* z;
  double rho_c, c0;
  const int* slot_lo;  // per shard, for this batch partition
  const int* slot_hi;
  double* dual_part;
  int dual_chunks;
  int64_t n;
  GlobalState* gs;
  Resid* trace;
  int* err;
};

// Panels in flight per CTA of the wide-row pass at most (its mbarrier slots).
constexpr int kBatchSlots = 16;

// The copy issuer's view of the segment of the next panel it copies (shared memory).
struct BatchCursor {
  const void* A;
  int64_t lda, first, next_first, row0, end;
  int s, rpp;
};

// One segment: the rows of shard `shard` of instance `inst`, cut into panels of `rpp` rows
// (rpp * row bytes <= the stage size, rpp <= R of the kernel).
struct BatchSeg {
  int inst, shard;
  int64_t first_panel;  // global index of its first panel
  int64_t row0;         // first row within the instance
  int64_t rows;
  int rpp;
  int pad;
};

template <typename TA, typename TM, int R, int VPT, int NT>
__global__ void __launch_bounds__(NT, 1)
k_fused_pass_batch(const BatchInst* __restrict__ inst, const BatchSeg* __restrict__ seg, int nseg,
                   int64_t P, int S, size_t stage_bytes, long long wait_limit) {
  using V = typename Vec16<TA>::type;
  constexpr int VE = Vec16<TA>::n;
  constexpr int NW = NT / 32;
  extern __shared__ __align__(128) unsigned char smem_raw[];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c = blockIdx.x, G = gridDim.x;
  const int64_t p_begin = static_cast<int64_t>(c) * P / G;
  const int64_t p_end = static_cast<int64_t>(c + 1) * P / G;
  const int64_t np = p_end - p_begin;

  // layout: a ring of S * stage_bytes | kBatchSlots mbarriers | the panels' ring offsets |
  // the issuer's segment cursor | red[R][NW] | d[R].  Panels (at most stage_bytes each) are placed end to end in the ring,
  // so an instance with short panels keeps several of them in flight; panel k waits on
  // barrier k % kBatchSlots.
  const uint32_t ring = static_cast<uint32_t>(S * stage_bytes);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + ring);
  uint32_t* poff = reinterpret_cast<uint32_t*>(bars + kBatchSlots);
  BatchCursor* icur = reinterpret_cast<BatchCursor*>(poff + kBatchSlots);
  TM* red = reinterpret_cast<TM*>(icur + 1);
  TM* d_s = red + R * NW;

  if (tid == 0) {
    for (int st = 0; st < kBatchSlots; ++st) mbar_init(&bars[st], 1);
    fence_barrier_init();
  }
  __syncthreads();

  auto locate = [&](int64_t p, int& s, int64_t& row0, int& nrows) {
    while (s + 1 < nseg && seg[s + 1].first_panel <= p) ++s;
    const BatchSeg& g = seg[s];
    row0 = g.row0 + (p - g.first_panel) * g.rpp;
    const int64_t rem = g.row0 + g.rows - row0;
    nrows = rem < g.rpp ? static_cast<int>(rem) : g.rpp;
  };

  // segment holding this CTA's first panel (binary search; later lookups walk forward)
  int seg0 = 0;
  {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (seg[mid].first_panel <= p_begin) lo = mid; else hi = mid - 1;
    }
    seg0 = lo;
  }

  // Thread 0 issues the copies.  Panels [done, n_issued) are in flight and occupy the ring
  // from poff[done % kBatchSlots] up to `head`, wrapping at most once; a panel is placed at
  // `head` when it fits before the ring's end, else at 0 when it fits before the oldest one.
  // Every size and offset is a multiple of 16 bytes (rows are padded to 16-byte vectors).
  // Its segment cursor (the current segment's rows, its instance's A and lda, and where the
  // next segment starts) sits in shared memory, so that an issue reads the tables only when
  // it crosses into a later segment.
  int64_t n_issued = 0;
  uint32_t head = 0;
  auto icur_load = [&](int s) {
    const BatchSeg& g = seg[s];
    const BatchInst& I = inst[g.inst];
    icur->A = I.A;
    icur->lda = I.lda;
    icur->first = g.first_panel;
    icur->next_first = s + 1 < nseg ? seg[s + 1].first_panel : static_cast<int64_t>(0x7fffffffffffffffLL);
    icur->row0 = g.row0;
    icur->end = g.row0 + g.rows;
    icur->s = s;
    icur->rpp = g.rpp;
  };
  if (tid == 0) icur_load(seg0);
  auto try_issue = [&](int64_t done) -> bool {
    if (n_issued >= np || n_issued - done >= kBatchSlots) return false;
    const int64_t p = p_begin + n_issued;
    while (p >= icur->next_first) icur_load(icur->s + 1);
    const int64_t row0 = icur->row0 + (p - icur->first) * icur->rpp;
    const int64_t lda_i = icur->lda;
    const int nrows = static_cast<int>(icur->end - row0 < icur->rpp ? icur->end - row0 : icur->rpp);
    const uint32_t bytes = static_cast<uint32_t>(nrows * lda_i * sizeof(TA));
    uint32_t at = 0;
    if (n_issued > done) {
      const uint32_t tail = poff[done % kBatchSlots];
      if (head > tail) {
        if (head + bytes <= ring) at = head;
        else if (bytes <= tail) at = 0;
        else return false;
      } else if (head + bytes <= tail) {
        at = head;
      } else {
        return false;
      }
    }
    const int sl = static_cast<int>(n_issued % kBatchSlots);
    poff[sl] = at;
    head = at + bytes;
    mbar_arrive_expect_tx(&bars[sl], bytes);
    bulk_copy_g2s(smem_raw + at, static_cast<const TA*>(icur->A) + row0 * lda_i, bytes, &bars[sl]);
    ++n_issued;
    return true;
  };
  if (tid == 0) {
    while (try_issue(0)) {
    }
  }

  // x_i in the storage type when it is the arithmetic type, else (BF16) in the arithmetic type
  using XT = typename std::conditional<std::is_same<TA, __nv_bfloat16>::value, TM, TA>::type;
  XT xr[VPT][VE];
  TM acc[VPT][VE];
  int cur_seg = -1, cur_inst = -1, sidx = seg0;
  int64_t nvec = 0, lda = 0;
  int loss = 0, newton_iters = 0;
  TM Mf = TM(1), rho_l = TM(1);
  TM st_res = TM(0), st_om = TM(0), st_ax = TM(0);

  auto flush_acc = [&](int s) {
    const BatchSeg& g = seg[s];
    const BatchInst& I = inst[g.inst];
    TM* dst = static_cast<TM*>(I.slots) + static_cast<int64_t>(c - I.c_lo + g.shard) * I.lda;
#pragma unroll
    for (int kk = 0; kk < VPT; ++kk) {
      const int64_t v = tid + static_cast<int64_t>(kk) * NT;
      if (v < nvec) {
#pragma unroll
        for (int e = 0; e < VE; ++e) dst[v * VE + e] = acc[kk][e];
      }
    }
  };
  auto flush_stats = [&](int ii) {
    if (warp == 0) {
      const TM a0 = warp_sum(st_res), a1 = warp_sum(st_om), a2 = warp_sum(st_ax);
      if (lane == 0) {
        const BatchInst& I = inst[ii];
        double* cs = I.cta_stats + (c - I.c_lo) * 4;
        cs[0] = static_cast<double>(a0);
        cs[1] = static_cast<double>(a1);
        cs[2] = static_cast<double>(a2);
        cs[3] = 0.0;
      }
    }
    st_res = st_om = st_ax = TM(0);
  };

  for (int64_t k = 0; k < np; ++k) {
    int64_t row0;
    int nrows;
    locate(p_begin + k, sidx, row0, nrows);
    if (sidx != cur_seg) {
      if (cur_seg >= 0) flush_acc(cur_seg);
      const int ni = seg[sidx].inst;
      if (ni != cur_inst) {
        if (cur_inst >= 0) flush_stats(cur_inst);
        const BatchInst& I = inst[ni];
        lda = I.lda;
        nvec = lda / VE;
        loss = I.loss;
        newton_iters = I.newton_iters;
        Mf = static_cast<TM>(I.M);
        rho_l = static_cast<TM>(I.rho_l);
        cur_inst = ni;
      }
      cur_seg = sidx;
      if constexpr (std::is_same<XT, TA>::value) {  // one 16-byte load per vector
        const V* xv = reinterpret_cast<const V*>(static_cast<const TA*>(inst[ni].xlo) +
                                                 static_cast<int64_t>(seg[sidx].shard) * lda);
#pragma unroll
        for (int kk = 0; kk < VPT; ++kk) {
          const int64_t v = tid + static_cast<int64_t>(kk) * NT;
          V t;
          if (v < nvec) t = xv[v]; else t = V{};
          const TA* te = reinterpret_cast<const TA*>(&t);
#pragma unroll
          for (int e = 0; e < VE; ++e) { xr[kk][e] = te[e]; acc[kk][e] = TM(0); }
        }
      } else {
        const XT* xsrc = static_cast<const XT*>(inst[ni].xlo) + static_cast<int64_t>(seg[sidx].shard) * lda;
#pragma unroll
        for (int kk = 0; kk < VPT; ++kk) {
          const int64_t v = tid + static_cast<int64_t>(kk) * NT;
#pragma unroll
          for (int e = 0; e < VE; ++e) {
            xr[kk][e] = v < nvec ? xsrc[v * VE + e] : XT(0);
            acc[kk][e] = TM(0);
          }
        }
      }
    }
    const BatchInst& I = inst[cur_inst];
    TM b_r = TM(0), nu_r = TM(0), om_r = TM(0);
    if (warp == 0 && lane < nrows) {
      b_r = static_cast<const TM*>(I.b)[row0 + lane];
      nu_r = static_cast<const TM*>(I.nu)[row0 + lane];
      om_r = static_cast<const TM*>(I.omega)[row0 + lane];
    }
    const int sl = static_cast<int>(k % kBatchSlots);
    const uint32_t parity = static_cast<uint32_t>((k / kBatchSlots) & 1);
    const bool ok = mbar_wait_bounded(&bars[sl], parity, wait_limit);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        set_err(I.err, DEV_TIMEOUT_PASS);
        for (int64_t q = k; q < n_issued; ++q)
          mbar_wait_bounded(&bars[q % kBatchSlots], static_cast<uint32_t>((q / kBatchSlots) & 1), wait_limit);
      }
      return;
    }
    // poff[sl] was written before the barrier above
    const V* sv = reinterpret_cast<const V*>(smem_raw + poff[sl]);

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
            const TA* ae = reinterpret_cast<const TA*>(&a);
#pragma unroll
            for (int e = 0; e < VE; ++e) dot[r] = fma(conv<TM>(ae[e]), conv<TM>(xr[kk][e]), dot[r]);
          }
        }
      }
    }
    {
      // the warp's R row sums in one reduce-scatter (R - 1 + 5 - log2 R shuffles instead of
      // 5 R): lane r (32 / R) holds row r's
      const TM dsum = warp_reduce_scatter<R>(dot, lane);
      if ((lane & (32 / R - 1)) == 0) red[(lane / (32 / R)) * NW + warp] = dsum;
    }
    __syncthreads();

    if (warp == 0) {
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
        static_cast<TM*>(I.omega)[row0 + lane] = om;
        static_cast<TM*>(I.nu)[row0 + lane] = nun;
        d_s[lane] = om - Axb - nun;
        const TM rr = Axb - om;
        st_res = fma(rr, rr, st_res);
        st_om = fma(om, om, st_om);
        st_ax = fma(Axb, Axb, st_ax);
      }
    }
    __syncthreads();

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
            const V a = sv[r * nvec + v];
            const TA* ae = reinterpret_cast<const TA*>(&a);
#pragma unroll
            for (int e = 0; e < VE; ++e) acc[kk][e] = fma(dr[r], conv<TM>(ae[e]), acc[kk][e]);
          }
        }
      }
    }
    __syncthreads();
    if (tid == 0) {
      while (try_issue(k + 1)) {
      }
    }
  }
  if (cur_seg >= 0) flush_acc(cur_seg);
  if (cur_inst >= 0) flush_stats(cur_inst);
}

// The pass over narrow instances (rows of at most NT/2 vectors): row groups of L = 2^lsh
// threads (8 <= L <= NT/2), one vector per thread, RP = NT/L rows in flight per step.
template <typename TA, typename TM, int R, int NT>
__global__ void __launch_bounds__(NT, 2)
k_fused_pass_batch_narrow(const BatchInst* __restrict__ inst, const BatchSeg* __restrict__ seg, int nseg,
                   int64_t P, int S, size_t stage_bytes, long long wait_limit) {
  using V = typename Vec16<TA>::type;
  constexpr int VE = Vec16<TA>::n;
  constexpr int NW = NT / 32;
  constexpr int kMaxRows = R * 32;  // rows per panel at most (row groups of >= 8 threads)
  extern __shared__ __align__(128) unsigned char smem_raw[];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c = blockIdx.x, G = gridDim.x;
  const int64_t p_begin = static_cast<int64_t>(c) * P / G;
  const int64_t p_end = static_cast<int64_t>(c + 1) * P / G;
  const int64_t np = p_end - p_begin;

  // layout: S stages of stage_bytes | S mbarriers | red[kMaxRows] | d[kMaxRows] |
  //         racc[NT * VE] | stat[3 * NW]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + S * stage_bytes);
  TM* red = reinterpret_cast<TM*>(bars + S);
  TM* d_s = red + kMaxRows;
  TM* racc = d_s + kMaxRows;
  TM* stat = racc + NT * VE;

  if (tid == 0) {
    for (int st = 0; st < S; ++st) mbar_init(&bars[st], 1);
    fence_barrier_init();
  }
  __syncthreads();

  auto locate = [&](int64_t p, int& s, int64_t& row0, int& nrows) {
    while (s + 1 < nseg && seg[s + 1].first_panel <= p) ++s;
    const BatchSeg& g = seg[s];
    row0 = g.row0 + (p - g.first_panel) * g.rpp;
    const int64_t rem = g.row0 + g.rows - row0;
    nrows = rem < g.rpp ? static_cast<int>(rem) : g.rpp;
  };

  // segment holding this CTA's first panel (binary search; later lookups walk forward)
  int seg0 = 0;
  {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (seg[mid].first_panel <= p_begin) lo = mid; else hi = mid - 1;
    }
    seg0 = lo;
  }

  int64_t n_issued = 0;
  int issue_seg = seg0;
  auto issue = [&](int64_t k) {
    int64_t row0;
    int nrows;
    locate(p_begin + k, issue_seg, row0, nrows);
    const BatchInst& I = inst[seg[issue_seg].inst];
    const int st = static_cast<int>(k % S);
    const uint32_t bytes = static_cast<uint32_t>(nrows * I.lda * sizeof(TA));
    mbar_arrive_expect_tx(&bars[st], bytes);
    bulk_copy_g2s(smem_raw + st * stage_bytes, static_cast<const TA*>(I.A) + row0 * I.lda, bytes,
                  &bars[st]);
  };
  if (tid == 0) {
    for (; n_issued < np && n_issued < S; ++n_issued) issue(n_issued);
  }

  // x_i in the storage type when it is the arithmetic type, else (BF16) in the arithmetic type
  using XT = typename std::conditional<std::is_same<TA, __nv_bfloat16>::value, TM, TA>::type;
  XT xr[VE];
  TM acc[VE];
  int cur_seg = -1, cur_inst = -1, sidx = seg0;
  int64_t nvec = 0, lda = 0;
  int loss = 0, newton_iters = 0;
  // row groups of the current instance: L threads each, RP of them, wpg warps per group
  int L = NT / 2, RP = 2, wpg = 1, vl = 0, rp = 0;
  TM Mf = TM(1), rho_l = TM(1);
  TM st_res = TM(0), st_om = TM(0), st_ax = TM(0);

  auto flush_acc = [&](int s) {
    const BatchSeg& g = seg[s];
    const BatchInst& I = inst[g.inst];
    TM* dst = static_cast<TM*>(I.slots) + static_cast<int64_t>(c - I.c_lo + g.shard) * I.lda;
    // add the RP groups' partial sums
#pragma unroll
    for (int e = 0; e < VE; ++e) racc[tid * VE + e] = acc[e];
    __syncthreads();
    const int span = L * VE;
    for (int idx = tid; idx < nvec * VE; idx += NT) {
      TM sum = TM(0);
      for (int q = 0; q < RP; ++q) sum += racc[q * span + idx];
      dst[idx] = sum;
    }
    __syncthreads();
  };
  auto flush_stats = [&](int ii) {
    const TM a0 = warp_sum(st_res), a1 = warp_sum(st_om), a2 = warp_sum(st_ax);
    if (lane == 0) {
      stat[warp * 3 + 0] = a0;
      stat[warp * 3 + 1] = a1;
      stat[warp * 3 + 2] = a2;
    }
    __syncthreads();
    if (tid == 0) {
      TM s0 = TM(0), s1 = TM(0), s2 = TM(0);
      for (int w = 0; w < NW; ++w) {
        s0 += stat[w * 3 + 0];
        s1 += stat[w * 3 + 1];
        s2 += stat[w * 3 + 2];
      }
      const BatchInst& I = inst[ii];
      double* cs = I.cta_stats + (c - I.c_lo) * 4;
      cs[0] = static_cast<double>(s0);
      cs[1] = static_cast<double>(s1);
      cs[2] = static_cast<double>(s2);
      cs[3] = 0.0;
    }
    __syncthreads();
    st_res = st_om = st_ax = TM(0);
  };

  for (int64_t k = 0; k < np; ++k) {
    int64_t row0;
    int nrows;
    locate(p_begin + k, sidx, row0, nrows);
    if (sidx != cur_seg) {
      if (cur_seg >= 0) flush_acc(cur_seg);
      const int ni = seg[sidx].inst;
      if (ni != cur_inst) {
        if (cur_inst >= 0) flush_stats(cur_inst);
        const BatchInst& I = inst[ni];
        lda = I.lda;
        nvec = lda / VE;
        loss = I.loss;
        newton_iters = I.newton_iters;
        Mf = static_cast<TM>(I.M);
        rho_l = static_cast<TM>(I.rho_l);
        L = 1 << I.lsh;
        RP = NT >> I.lsh;
        wpg = L >= 32 ? L >> 5 : 1;
        vl = tid & (L - 1);
        rp = tid >> I.lsh;
        cur_inst = ni;
      }
      cur_seg = sidx;
      if constexpr (std::is_same<XT, TA>::value) {  // one 16-byte load per vector
        const V* xv = reinterpret_cast<const V*>(static_cast<const TA*>(inst[ni].xlo) +
                                                 static_cast<int64_t>(seg[sidx].shard) * lda);
        V t;
        if (vl < nvec) t = xv[vl]; else t = V{};
        const TA* te = reinterpret_cast<const TA*>(&t);
#pragma unroll
        for (int e = 0; e < VE; ++e) { xr[e] = te[e]; acc[e] = TM(0); }
      } else {
        const XT* xsrc = static_cast<const XT*>(inst[ni].xlo) + static_cast<int64_t>(seg[sidx].shard) * lda;
#pragma unroll
        for (int e = 0; e < VE; ++e) {
          xr[e] = vl < nvec ? xsrc[vl * VE + e] : XT(0);
          acc[e] = TM(0);
        }
      }
    }
    const BatchInst& I = inst[cur_inst];
    // row `tid` of the panel: its label and duals, fetched before the wait
    TM b_r = TM(0), nu_r = TM(0), om_r = TM(0);
    if (tid < nrows) {
      b_r = static_cast<const TM*>(I.b)[row0 + tid];
      nu_r = static_cast<const TM*>(I.nu)[row0 + tid];
      om_r = static_cast<const TM*>(I.omega)[row0 + tid];
    }
    const int st = static_cast<int>(k % S);
    const uint32_t parity = static_cast<uint32_t>((k / S) & 1);
    const bool ok = mbar_wait_bounded(&bars[st], parity, wait_limit);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        set_err(I.err, DEV_TIMEOUT_PASS);
        for (int64_t q = k; q < n_issued; ++q)
          mbar_wait_bounded(&bars[q % S], static_cast<uint32_t>((q / S) & 1), wait_limit);
      }
      return;
    }
    const V* sv = reinterpret_cast<const V*>(smem_raw + st * stage_bytes);

    // forward: group rp takes rows rp, rp + RP, ...; thread vl of the group its vectors
    TM dot[R];
#pragma unroll
    for (int r = 0; r < R; ++r) dot[r] = TM(0);
    if (vl < nvec) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int row = r * RP + rp;
        if (row < nrows) {
          const V a = sv[row * nvec + vl];
          const TA* ae = reinterpret_cast<const TA*>(&a);
#pragma unroll
          for (int e = 0; e < VE; ++e) dot[r] = fma(conv<TM>(ae[e]), conv<TM>(xr[e]), dot[r]);
        }
      }
    }
    // sum over the group's lanes within each warp, then one partial per (row, warp of group)
    const int gl = L < 32 ? L : 32;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      for (int off = gl >> 1; off > 0; off >>= 1) dot[r] += __shfl_xor_sync(0xffffffffu, dot[r], off);
    }
    if ((vl & 31) == 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int row = r * RP + rp;
        if (row < nrows) red[row * wpg + (vl >> 5)] = dot[r];
      }
    }
    __syncthreads();

    // prox epilogue: thread t owns row t of the panel (nrows <= NT)
    if (tid < nrows) {
      TM tot = TM(0);
      for (int w = 0; w < wpg; ++w) tot += red[tid * wpg + w];
      const TM Axb = tot / Mf;
      const TM om = omega_prox<TM>(loss, Axb + nu_r, b_r, Mf, rho_l, newton_iters, om_r);
      const TM nun = nu_r + Axb - om;
      static_cast<TM*>(I.omega)[row0 + tid] = om;
      static_cast<TM*>(I.nu)[row0 + tid] = nun;
      d_s[tid] = om - Axb - nun;
      const TM rr = Axb - om;
      st_res = fma(rr, rr, st_res);
      st_om = fma(om, om, st_om);
      st_ax = fma(Axb, Axb, st_ax);
    }
    __syncthreads();

    TM dr[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int row = r * RP + rp;
      dr[r] = row < nrows ? d_s[row] : TM(0);
    }
    if (vl < nvec) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int row = r * RP + rp;
        if (row < nrows) {
          const V a = sv[row * nvec + vl];
          const TA* ae = reinterpret_cast<const TA*>(&a);
#pragma unroll
          for (int e = 0; e < VE; ++e) acc[e] = fma(dr[r], conv<TM>(ae[e]), acc[e]);
        }
      }
    }
    __syncthreads();
    if (tid == 0 && n_issued < np) {
      issue(n_issued);
      ++n_issued;
    }
  }
  if (cur_seg >= 0) flush_acc(cur_seg);
  if (cur_inst >= 0) flush_stats(cur_inst);
}

// x-update over a flattened list of (instance, shard, block, row tile) items.
struct XItem {
  int inst, shard, block, row_begin;
};

// FP32: at most 32 registers, so that a full SM's worth of warps keeps P loads in flight.
template <typename TP, int XT, int ROWS>
__global__ void __launch_bounds__(XT, sizeof(TP) == 4 ? 2048 / XT : 1)
k_xupd_batch(const BatchInst* __restrict__ inst, const XItem* __restrict__ items) {
  using V = typename PVec<TP>::type;
  constexpr int VE = PVec<TP>::n;
  extern __shared__ __align__(16) unsigned char xs_raw[];
  TP* rs = reinterpret_cast<TP*>(xs_raw);
  const XItem it = items[blockIdx.x];
  const BatchInst& I = inst[it.inst];
  const int i = it.shard, j = it.block;
  const int col0 = I.blk_col0[j], nj = I.blk_col0[j + 1] - col0, ldp = I.blk_ldp[j];
  const int64_t lda = I.lda;
  for (int k = threadIdx.x; k < ldp; k += XT)
    rs[k] = k < nj ? static_cast<TP>(I.r[i * lda + col0 + k]) : TP(0);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const TP* Pb = static_cast<const TP*>(I.P) + I.P_off[i * I.M_blocks + j];
  const V* rv = reinterpret_cast<const V*>(rs);
  const int nv = ldp / VE;
  constexpr int U = 4;  // 16-byte loads in flight per lane (64 warps per SM)
  for (int row = it.row_begin + warp; row < it.row_begin + ROWS && row < nj; row += XT / 32) {
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
      const double xn = I.x[o] + static_cast<double>(acc);
      I.x[o] = xn;
      static_cast<TP*>(const_cast<void*>(I.xlo))[o] = static_cast<TP>(xn);
    }
  }
}

// Consensus step, one CTA per instance.
template <int GT, int MW>
__global__ void __launch_bounds__(GT, 1) k_global_batch(const ConsensusArgs* __restrict__ args) {
  consensus_block<GT, MW>(args[blockIdx.x]);
}

// Dual update + next right-hand side over a flattened list of (instance, shard, chunk)
// items; per instance the last CTA reduces its residual record.
struct DItem {
  int inst, shard, chunk;
};

template <typename TM, int DT>
__global__ void __launch_bounds__(DT)
k_dual_batch(const BatchInst* __restrict__ inst, const DItem* __restrict__ items) {
  __shared__ double red[32 * 2];
  __shared__ bool last;
  const DItem it = items[blockIdx.x];
  const BatchInst& I = inst[it.inst];
  const int i = it.shard, nch = I.dual_chunks, N = I.N;
  const int64_t lda = I.lda, n = I.n;
  double a[2] = {0.0, 0.0};
  // each item takes the columns chunk * DT + tid + k * nch * DT of its shard
  for (int64_t col = static_cast<int64_t>(it.chunk) * DT + threadIdx.x; col < lda;
       col += static_cast<int64_t>(nch) * DT) {
    const int64_t o = i * lda + col;
    const double xv = I.x[o], zv = I.z[col], dv = xv - zv;
    const double un = I.u[o] + dv;
    I.u[o] = un;
    TM q = TM(0);
    const TM* slots = static_cast<const TM*>(I.slots);
    for (int sl = I.slot_lo[i]; sl <= I.slot_hi[i]; ++sl) q += slots[sl * lda + col];
    I.r[o] = I.rho_l * static_cast<double>(q) + I.rho_c * (zv - un) - I.c0 * xv;
    a[0] += dv * dv;
    a[1] += xv * xv;
  }
  block_sum<2>(a, red);
  if (threadIdx.x == 0) {
    I.dual_part[(static_cast<int64_t>(i) * nch + it.chunk) * 2 + 0] = a[0];
    I.dual_part[(static_cast<int64_t>(i) * nch + it.chunk) * 2 + 1] = a[1];
    __threadfence();
    last = atomicAdd(&I.gs->ticket, 1u) == static_cast<unsigned>(N * nch) - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double fs[5];
  dual_final_sums<DT>(I.dual_part, N, nch, I.cta_stats, I.G_inst, fs);
  {
    const double pr = fs[0], nx = fs[1], q0 = fs[2], q1 = fs[3], q2 = fs[4];
    if (threadIdx.x == 0) {
      GlobalState* gs = I.gs;
      Resid& rec = I.trace[gs->iter % kTraceCapacity];
      rec.p_r = pr;
      rec.p_rel = pr / fmax(fmax(nx, N * rec.znorm), 1e-30);
      rec.i_r = sqrt(q0);
      rec.i_rel = sqrt(q0) / fmax(fmax(sqrt(q1), sqrt(q2)), 1e-30);
      const double chk = rec.p_r + rec.d_r + rec.b_r + rec.i_r + rec.t + rec.v;
      if (!isfinite(chk)) set_err(I.err, DEV_NONFINITE);
      gs->iter += 1;
      gs->ticket = 0;
    }
  }
  (void)n;
}

}  // namespace bic
