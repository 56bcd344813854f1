// Tensor-core A pass of the multi-column case (softmax with K <= 16 classes, or a sparsity
// path of K instances) on pairs of SMs: a thread-block cluster of two CTAs shares each
// 128-row panel and splits its columns.  Same arithmetic as k_fused_pass_tc (Sec. 3.1 with K
// right-hand sides: eqs. p:GPU;x, p:GPU;omega, p:GPU;nu):
//
//   forward   P_r[128 x 32] = A_panel[:, half r] [W_hi | W_lo][half r]   (CTA r of the pair)
//             D1 = P_0 + P_1, exchanged through distributed shared memory
//   backward  D2_r[half r x 32] += A_panel[:, half r]' [d_hi | d_lo]      (A'd, own columns)
//
// Why pairs: one CTA per SM over whole rows spends its shared-memory bandwidth on W tiles
// and on reading each slab twice in the backward (d_hi and d_lo as two N = 16 products,
// because 16 slabs of N = 32 accumulators and the forward ones exceed the 512 TMEM columns).
// With the columns split, a CTA holds at most 8 slabs, so d_hi and d_lo go side by side into
// one N = 32 backward product (each slab read once), the forward has M = 128 (the W tile
// is read once per 128 rows instead of per 64), and every SM issues half the MMAs per row.
//
// Per CTA and panel: the producer (warp 4) loads, for each of its slabs, a 128 x 128 BF16
// slab by two 2D TMA boxes (128-byte swizzle) plus the slab's 8 KB W tile for the forward,
// and the slab again for the backward.  The MMA warp (warp 5) issues F(k) (8 MMAs per slab,
// M = 128, N = 32, K = 16) and B(k-1) (8 MMAs per slab, N = 32) in the order of
// k_fused_pass_tc.  The four epilogue warps own the 128 TMEM lanes = panel rows: they read
// their partial row dots, store them into the partner CTA's shared memory and arrive on its
// barrier, wait for the partner's partial, add the two in rank order (both CTAs get the same
// sums), run the prox for all 128 rows (both CTAs, identical results), write omega and nu for
// their half of the rows, and write d_hi / d_lo as the backward's B operand.  At a shard end
// they add D2's hi and lo columns into the pair's slot (CTA r its own columns).
//
// Every wait is bounded; an expired wait raises the abort flag, which the partner sees as its
// own expired wait.  Both CTAs of a pair always reach the final cluster barrier, so neither
// exits while the other may still write into its shared memory.
#pragma once

#include <cuda.h>

#include "common.cuh"
#include "mc_tc.cuh"
#include "nspace.cuh"
#include "pass.cuh"

namespace bic {

constexpr int kTc2Rows = 128;                       // panel rows (the forward's M)
constexpr int kTc2Threads = 256;
// ring stages: 4 of 40 KB, 3 for 16 classes (whose staged row data take 12 KB more)
template <int KC>
__host__ __device__ constexpr int tc2_stages() { return KC > 10 ? 3 : 4; }
// one panel's row data staged by the loader warps: nu and omega (KC floats a row) and b
__host__ __device__ constexpr int tc2_row_bytes(int KC) { return (2 * 128 * KC + 128) * 4; }
constexpr int kTc2BoxBytes = kTc2Rows * 128;        // a 64-column x 128-row BF16 box: 16 KB
constexpr int kTc2StageABytes = 2 * kTc2BoxBytes;   // one 128-column slab
constexpr int kTc2WBytes = 2 * 4096;                // its W tile: [box] 32 x 64 BF16 (hi | lo)
constexpr int kTc2StageBytes = kTc2StageABytes + kTc2WBytes;
constexpr int kTc2MaxSlabs = 8;                     // per CTA (lda <= 2048)
constexpr int kTc2DBytes = 2 * 4096;                // d tile: [row block][32 x 64 BF16]
constexpr int kTc2XBytes = kTc2Rows * 16 * 4;       // partial row dots: 128 rows x 16 floats
constexpr int kTc2TmemCols = 512;                   // D1 x2 at 0 / 32, D2 slab s at 64 + 32 s
constexpr int kTc2D2Col = 64;

inline size_t fused_pass_tc2_smem(int KC) {
  // alignment, ring, two d tiles, two exchange buffers, two row-data buffers, barriers and
  // scalars
  const int S = KC > 10 ? tc2_stages<16>() : tc2_stages<10>();
  return 1024 + static_cast<size_t>(S) * kTc2StageBytes + 2 * kTc2DBytes + 2 * kTc2XBytes +
         2 * static_cast<size_t>(tc2_row_bytes(KC)) + 512;
}

// ------------------------------------------------------------------ cluster PTX wrappers
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Every thread of both CTAs; orders shared-memory accesses across the cluster.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// The shared::cluster address of the same offset in CTA `rank`'s shared memory.
__device__ __forceinline__ uint32_t mapa_shared(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cluster_v4(uint32_t raddr, float a, float b, float c, float d) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(raddr), "f"(a), "f"(b),
               "f"(c), "f"(d)
               : "memory");
}
// Store 16 bytes into another CTA's shared memory, completing as 16 transaction bytes on that
// CTA's barrier at rbar (no fence: the barrier's phase carries the data).
__device__ __forceinline__ void st_async_v4(uint32_t raddr, float a, float b, float c, float d,
                                            uint32_t rbar) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
          raddr),
      "f"(a), "f"(b), "f"(c), "f"(d), "r"(rbar)
      : "memory");
}
__device__ __forceinline__ void st_cluster_f64(uint32_t raddr, double a) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(raddr), "d"(a) : "memory");
}
// Arrive on a barrier in another CTA of the cluster, releasing this thread's earlier writes.
__device__ __forceinline__ void mbar_arrive_remote(uint32_t raddr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(raddr) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_cluster_or_abort(uint64_t* bar, uint32_t parity,
                                                           long long limit, volatile int* abort) {
  if (mbar_try_wait_cluster(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait_cluster(bar, parity)) {
    if (*abort || clock64() - t0 > limit) return false;
  }
  return true;
}

// The shard table entries a CTA's panels need (first panel and first row of shards
// base .. base + count - 1), in shared memory when they fit: every panel lookup of the three
// roles then reads shared memory instead of chasing global loads.
constexpr int kTc2GeoCache = 66;
struct Tc2Geo {
  const int64_t* ps;  // panel_start[base ...]
  const int64_t* r0;  // shard_row0[base ...]
  int base, N;
  __device__ void locate(int64_t p, int& i, int64_t& row0, int& nrows) const {
    while (i + 1 < N && ps[i + 1 - base] <= p) ++i;
    row0 = r0[i - base] + (p - ps[i - base]) * kTc2Rows;
    const int64_t rem = r0[i + 1 - base] - row0;
    nrows = rem < kTc2Rows ? static_cast<int>(rem) : kTc2Rows;
  }
};

// Consensus CTAs of a launch at most: the instances of a path are spread over them and each
// runs its instances' steps one after another (the list-form step of one instance is short
// beside the pass), so that the other pairs stay on the panel stream.
constexpr int kTc2ConsCtas = 2;
__host__ __device__ constexpr int tc2_cons_ctas(int ninst) {
  return ninst < kTc2ConsCtas ? ninst : kTc2ConsCtas;
}

// ------------------------------------------------------------------ k_fused_pass_tc2
// Grid: 2 G panel CTAs (G pairs, a pair = one cluster) and, on the last sweep, the
// consensus CTAs (tc2_cons_ctas of the instances, their count rounded up to even; a spare
// one returns).
template <int KC>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kTc2Threads, 1)
k_fused_pass_tc2(const __grid_constant__ CUtensorMap tmap, int64_t lda,
                 const unsigned char* __restrict__ wpk, int nslab_all, int64_t ldx, int K,
                 const float* __restrict__ b, float* __restrict__ omega, float* __restrict__ nu,
                 float* __restrict__ slots, double* __restrict__ cta_stats, PassGeometry geo,
                 float Mf, float rho_l, int newton_iters, int* __restrict__ err,
                 long long wait_limit, ConsensusArgs cons, int path_loss) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int ninst_c = consensus_ctas(cons);
  const int nct = tc2_cons_ctas(ninst_c);
  const int npc = static_cast<int>(gridDim.x) - ((nct + 1) & ~1);  // panel CTAs
  if (static_cast<int>(blockIdx.x) >= npc) {
    // instances q0, q0 + nct, ... (nct >= 1 whenever q0 < ninst_c)
    const int q0 = static_cast<int>(blockIdx.x) - npc;
    for (int q = q0; q < ninst_c; q += nct) {
      if (q != q0) __syncthreads();  // the previous instance's shared memory is free
      consensus_block<kTc2Threads, kConsMW, true>(consensus_instance(cons, q), smem_raw);
    }
    return;
  }
  constexpr int S = tc2_stages<KC>();
  constexpr int RB = tc2_row_bytes(KC);
  constexpr uint32_t IDESC_FWD = idesc_bf16(128, 32, false, false);
  constexpr uint32_t IDESC_BWD = idesc_bf16(128, 32, true, false);
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  unsigned char* ring = base;
  unsigned char* ds = ring + S * kTc2StageBytes;   // [2] d tiles
  float* xbuf = reinterpret_cast<float*>(ds + 2 * kTc2DBytes);  // [2][128][16] partner's partials
  unsigned char* rows = reinterpret_cast<unsigned char*>(xbuf + 2 * kTc2Rows * 16);  // [2] row data
  uint64_t* full = reinterpret_cast<uint64_t*>(rows + 2 * RB);
  uint64_t* empty = full + S;
  uint64_t* d1full = empty + S;   // [2]
  uint64_t* dready = d1full + 2;  // [2]
  uint64_t* bwddone = dready + 2;
  uint64_t* flushed = bwddone + 1;
  uint64_t* drainbar = flushed + 1;
  uint64_t* xfull = drainbar + 1;  // [2] the partner's 128 rows of partials have arrived
  uint64_t* rowfull = xfull + 2;   // [2] a panel's row data are staged
  uint64_t* rowfree = rowfull + 2; // [2] the epilogue has read them
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(rowfree + 2);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  long long* counts = reinterpret_cast<long long*>(tmem_slot + 2);  // [0] issued, [1] consumed
  double* xstat = reinterpret_cast<double*>(counts + 2);            // [3] rank 1's row sums
  float* red = reinterpret_cast<float*>(xstat + 4);                 // [4 warps][3]

  __shared__ int64_t geo_ps[kTc2GeoCache], geo_r0[kTc2GeoCache];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t rank = cluster_ctarank(), partner = rank ^ 1u;
  const int pair = static_cast<int>(blockIdx.x) >> 1, G = npc >> 1;
  const int64_t p_begin = static_cast<int64_t>(pair) * geo.P / G;
  const int64_t p_end = static_cast<int64_t>(pair + 1) * geo.P / G;
  const int np = static_cast<int>(p_end - p_begin);
  // shards of this pair's first and last panels (binary search over the shards' first panels)
  auto shard_search = [&](int64_t p) {
    int lo = 0, hi = geo.N - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (geo.panel_start[mid] <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
  };
  const int shard0 = shard_search(p_begin);
  const int shard1 = np > 0 ? shard_search(p_end - 1) : shard0;
  const int ncache = shard1 - shard0 + 2;  // entries shard0 .. shard1 + 1 (<= N)
  const bool cached = ncache <= kTc2GeoCache;
  if (cached) {
    for (int i = tid; i < ncache; i += blockDim.x) {
      geo_ps[i] = geo.panel_start[shard0 + i];
      geo_r0[i] = geo.shard_row0[shard0 + i];
    }
  }
  const Tc2Geo gv{cached ? geo_ps : geo.panel_start, cached ? geo_r0 : geo.shard_row0,
                  cached ? shard0 : 0, geo.N};
  // this CTA's slabs: the first ceil(n/2) 128-column slabs for rank 0, the rest for rank 1
  const int nsl_all = static_cast<int>((lda + 127) / 128), h0 = (nsl_all + 1) / 2;
  const int sl0 = rank ? h0 : 0, nsl = rank ? nsl_all - h0 : h0;
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
    mbar_init(&xfull[0], 128);
    mbar_init(&xfull[1], 128);
    mbar_init(&rowfull[0], 64);
    mbar_init(&rowfull[1], 64);
    mbar_init(&rowfree[0], 128);
    mbar_init(&rowfree[1], 128);
    *abort_flag = 0;
    counts[0] = counts[1] = 0;
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, kTc2TmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  cluster_sync();  // both CTAs' barriers exist before any remote arrive
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  auto panel_at = [&](int k, int& hint, int64_t& row0, int& nrows) {
    gv.locate(p_begin + k, hint, row0, nrows);
  };
  auto shard_of = [&](int k) -> int {
    if (k < 0 || k >= np) return -1;
    int h = shard0, nr;
    int64_t r0;
    panel_at(k, h, r0, nr);
    return h;
  };
  // Step order shared by the producer and the MMA issuer: F(0); F(k), B(k-1) inside a shard,
  // B(k-1), F(k) when k starts a new shard; B(last).
  auto schedule = [&](auto&& fn) {
    int h = shard0, prev_shard = -1;
    for (int k = 0; k < np; ++k) {
      int64_t r0;
      int nr;
      panel_at(k, h, r0, nr);
      const bool boundary = h != prev_shard;
      if (k > 0 && boundary && !fn(false, k - 1)) return;
      if (!fn(true, k)) return;
      if (k > 0 && !boundary && !fn(false, k - 1)) return;
      prev_shard = h;
    }
    if (np > 0) fn(false, np - 1);
  };

  float st_res = 0.f, st_om = 0.f, st_ax = 0.f;

  if (warp == 4) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      long long j = 0;
      int hint = shard0;
      const uint64_t keep = l2_policy_evict_last(), drop = l2_policy_evict_first();
      schedule([&](bool fwd, int k) -> bool {
        int64_t row0;
        int nr;
        panel_at(k, hint, row0, nr);  // non-decreasing shard along the schedule
        const unsigned char* wsrc =
            wpk + (static_cast<int64_t>(hint) * nslab_all + sl0) * kTc2WBytes;
        for (int sg = 0; sg < nsl; ++sg, ++j) {
          const int st = static_cast<int>(j % S);
          if (j >= S && !mbar_wait_or_abort(&empty[st], static_cast<uint32_t>(((j / S) - 1) & 1), wait_limit, abort_v)) {
            *abort_v = 1;
            counts[0] = j;
            return false;
          }
          unsigned char* dst = ring + st * kTc2StageBytes;
          mbar_arrive_expect_tx(&full[st], kTc2StageABytes + (fwd ? kTc2WBytes : 0));
          // the backward takes its slabs newest first (the shortest reuse distances in L2)
          const int x0 = (sl0 + (fwd ? sg : nsl - 1 - sg)) * 128;
          tma_load_2d_hint(dst, &tmap, x0, static_cast<int>(row0), &full[st], fwd ? keep : drop);
          tma_load_2d_hint(dst + kTc2BoxBytes, &tmap, x0 + 64, static_cast<int>(row0), &full[st],
                           fwd ? keep : drop);
          if (fwd) bulk_copy_g2s(dst + kTc2StageABytes, wsrc + sg * kTc2WBytes, kTc2WBytes, &full[st]);
        }
        counts[0] = j;
        return true;
      });
    }
  } else if (warp == 5) {
    // ---------------------------------------------------------------- MMA issuer (whole warp)
    const uint64_t tk = sdesc_sw128(0, 16, 1024);            // K-major operands
    const uint64_t tm_ = sdesc_sw128(0, kTc2BoxBytes, 1024);  // MN-major slab (backward A)
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
      for (int sg = 0; sg < nsl; ++sg, ++j) {
        const int st = static_cast<int>(j % S);
        if (!mbar_wait_or_abort(&full[st], static_cast<uint32_t>((j / S) & 1), wait_limit, abort_v)) return false;
        const uint32_t sa = ring_a + st * kTc2StageBytes;
        if (fwd) {
          const uint32_t d1 = tmem + 32 * (k & 1);
#pragma unroll
          for (int bx = 0; bx < 2; ++bx)
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
              umma_bf16_warp(d1, dsc(tk, sa + bx * kTc2BoxBytes + ks * 32),
                             dsc(tk, sa + kTc2StageABytes + bx * 4096 + ks * 32), IDESC_FWD,
                             (sg | bx | ks) != 0 ? 1u : 0u);
        } else {
          const uint32_t d2 = tmem + kTc2D2Col + 32 * (nsl - 1 - sg);
          const uint32_t db = ds_a + (k & 1) * kTc2DBytes;
#pragma unroll
          for (int ks = 0; ks < 8; ++ks)
            umma_bf16_warp(d2, dsc(tm_, sa + ks * 2048), dsc(tk, db + (ks >> 2) * 4096 + (ks & 3) * 32),
                           IDESC_BWD, (first_bwd && ks == 0) ? 0u : 1u);
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
  } else if (warp >= 6) {
    // ---------------------------------------------------------------- row-data loaders
    // nu, omega (K floats a row, contiguous over the panel) and b of the panels ahead, into
    // two shared-memory buffers; the epilogue releases a buffer once it has read its row.
    const int lt = tid - 192;  // 0..63
    int hint = shard0;
    for (int k = 0; k < np; ++k) {
      const int buf = k & 1;
      if (k >= 2 && !mbar_wait_or_abort(&rowfree[buf], static_cast<uint32_t>(((k - 2) >> 1) & 1), wait_limit, abort_v)) {
        *abort_v = 1;
        break;
      }
      int64_t row0;
      int nr;
      panel_at(k, hint, row0, nr);
      float* rnu = reinterpret_cast<float*>(rows + buf * RB);
      float* rom = rnu + kTc2Rows * KC;
      float* rbv = rom + kTc2Rows * KC;
      const float* snu = nu + row0 * K;
      const float* som = omega + row0 * K;
      const int cnt = nr * K;
      for (int i0 = lt; i0 < cnt; i0 += 4 * 64) {
        float va[4], vb[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + 64 * u;
          va[u] = i < cnt ? snu[i] : 0.f;
          vb[u] = i < cnt ? som[i] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + 64 * u;
          if (i < cnt) {
            rnu[i] = va[u];
            rom[i] = vb[u];
          }
        }
      }
      for (int i = lt; i < nr; i += 64) rbv[i] = b[row0 + i];
      mbar_arrive(&rowfull[buf]);
    }
  } else if (warp < 4) {
    // ---------------------------------------------------------------- epilogue warps
    const uint32_t lane_base = static_cast<uint32_t>(warp * 32) << 16;
    const int r = tid;                       // panel row of this thread (TMEM lane)
    const bool own_row = (r >> 6) == static_cast<int>(rank);  // omega, nu and sums of this row
    const uint32_t x_remote0 = mapa_shared(smem_addr(xbuf + r * 16), partner);
    const uint32_t xfull_remote0 = mapa_shared(smem_addr(&xfull[0]), partner);
    const float invM = 1.f / Mf;
    int seg = 0;
    bool eok = true;
    int hint = shard0;
    for (int k = 0; k < np && eok; ++k) {
      int64_t row0;
      int nrows;
      panel_at(k, hint, row0, nrows);
      const int shard = hint;
      const int buf = k & 1;
      const uint32_t par = static_cast<uint32_t>((k >> 1) & 1);
      if (!mbar_wait_or_abort(&d1full[buf], par, wait_limit, abort_v)) { eok = false; break; }
      tc_fence_after();
      uint32_t v[16], vl[16];
      tmem_ld16(tmem + lane_base + 32 * buf, v);
      tmem_ld16(tmem + lane_base + 32 * buf + 16, vl);
      float part[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) part[q] = __uint_as_float(v[q]) + __uint_as_float(vl[q]);
      // expect the partner's 64 bytes for this row, then send ours (they complete on its barrier)
      mbar_arrive_expect_tx(&xfull[buf], 64);
      const uint32_t xr = x_remote0 + buf * kTc2XBytes, xb = xfull_remote0 + buf * 8;
#pragma unroll
      for (int q = 0; q < 16; q += 4) st_async_v4(xr + q * 4, part[q], part[q + 1], part[q + 2], part[q + 3], xb);
      // this panel's row data
      const bool valid = r < nrows;
      if (!mbar_wait_or_abort(&rowfull[buf], par, wait_limit, abort_v)) { eok = false; break; }
      float nk[KC], w[KC];
      int yk = 0;
      float ybk = 0.f;
      {
        const float* rnu = reinterpret_cast<const float*>(rows + buf * RB);
        const float* rom = rnu + kTc2Rows * KC;
        const float* rbv = rom + kTc2Rows * KC;
#pragma unroll
        for (int q = 0; q < KC; ++q) {
          nk[q] = (valid && q < K) ? rnu[r * K + q] : 0.f;
          w[q] = (valid && q < K) ? rom[r * K + q] : 0.f;
        }
        ybk = valid ? rbv[r] : 0.f;
        yk = static_cast<int>(ybk);
      }
      mbar_arrive(&rowfree[buf]);
      if (!mbar_wait_cluster_or_abort(&xfull[buf], par, wait_limit, abort_v)) { eok = false; break; }
      float other[16];
      {
        const float4* xp = reinterpret_cast<const float4*>(xbuf + buf * kTc2Rows * 16 + r * 16);
#pragma unroll
        for (int c4 = 0; c4 < 4; ++c4) {
          const float4 t4 = xp[c4];
          other[4 * c4 + 0] = t4.x;
          other[4 * c4 + 1] = t4.y;
          other[4 * c4 + 2] = t4.z;
          other[4 * c4 + 3] = t4.w;
        }
      }
      float Axb[KC], aa[KC];
#pragma unroll
      for (int q = 0; q < KC; ++q) {
        // rank order: both CTAs form the same sum
        Axb[q] = (rank == 0 ? part[q] + other[q] : other[q] + part[q]) * invM;
        aa[q] = Axb[q] + nk[q];
      }
      if (valid) {
        if (path_loss < 0) {
          softmax_prox_row<KC>(w, aa, yk, K, Mf, rho_l, newton_iters);
        } else {  // a path: K instances, each column its own scalar prox on target b_r
#pragma unroll
          for (int q = 0; q < KC; ++q)
            if (q < K) w[q] = omega_prox<float>(path_loss, aa[q], ybk, Mf, rho_l, newton_iters, w[q]);
        }
      }
      unsigned char* dbuf = ds + buf * kTc2DBytes + (r >> 6) * 4096;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        float dv = 0.f;
        if (q < KC && q < K && valid) {
          const float nun = nk[q] + Axb[q] - w[q];
          if (own_row) {
            omega[(row0 + r) * K + q] = w[q];
            nu[(row0 + r) * K + q] = nun;
            const float rr = Axb[q] - w[q];
            st_res = fmaf(rr, rr, st_res);
            st_om = fmaf(w[q], w[q], st_om);
            st_ax = fmaf(Axb[q], Axb[q], st_ax);
          }
          dv = w[q] - Axb[q] - nun;
        }
        const __nv_bfloat16 hi = __float2bfloat16_rn(dv);
        const __nv_bfloat16 lo = __float2bfloat16_rn(dv - __bfloat162float(hi));
        *reinterpret_cast<__nv_bfloat16*>(dbuf + sw128_off(q, r & 63)) = hi;
        *reinterpret_cast<__nv_bfloat16*>(dbuf + sw128_off(16 + q, r & 63)) = lo;
      }
      fence_async_smem();
      tc_fence_before();
      mbar_arrive(&dready[buf]);
      // end of a shard: this CTA's columns of the shard's A'd (hi + lo) into the pair's slot
      if (k + 1 >= np || shard_of(k + 1) != shard) {
        if (!mbar_wait_or_abort(bwddone, static_cast<uint32_t>(seg & 1), wait_limit, abort_v)) { eok = false; break; }
        ++seg;
        tc_fence_after();
        float* dst = slots + static_cast<int64_t>(pair + shard) * ldx;
        for (int sg = 0; sg < nsl; ++sg) {
          uint32_t u[16], ul[16];
          tmem_ld16(tmem + lane_base + kTc2D2Col + 32 * sg, u);
          tmem_ld16(tmem + lane_base + kTc2D2Col + 32 * sg + 16, ul);
          const int64_t col = static_cast<int64_t>(sl0 + sg) * 128 + r;
          if (col < lda) {
#pragma unroll
            for (int q = 0; q < KC; ++q)
              if (q < K) dst[col * K + q] = __uint_as_float(u[q]) + __uint_as_float(ul[q]);
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
  // the pair's row sums: rank 1 hands its three to rank 0, which adds them in rank order
  double s3[3] = {0.0, 0.0, 0.0};
  if (tid == 0) {
    for (int w = 0; w < 4; ++w) {
      s3[0] += static_cast<double>(red[w * 3 + 0]);
      s3[1] += static_cast<double>(red[w * 3 + 1]);
      s3[2] += static_cast<double>(red[w * 3 + 2]);
    }
    if (rank == 1) {
      const uint32_t xs = mapa_shared(smem_addr(xstat), partner);
      for (int i = 0; i < 3; ++i) st_cluster_f64(xs + 8 * i, s3[i]);
    }
  }
  tc_fence_before();
  cluster_sync();  // the partner's writes into this CTA's shared memory are complete
  tc_fence_after();
  if (tid == 0 && rank == 0) {
    cta_stats[pair * 4 + 0] = s3[0] + xstat[0];
    cta_stats[pair * 4 + 1] = s3[1] + xstat[1];
    cta_stats[pair * 4 + 2] = s3[2] + xstat[2];
    cta_stats[pair * 4 + 3] = 0.0;
  }
  if (warp == 0) tmem_dealloc(tmem, kTc2TmemCols);
}

}  // namespace bic
