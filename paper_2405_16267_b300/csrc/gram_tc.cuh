// Tensor-core (tcgen05) Gram matrices for BF16 storage: G_ij = A_ij' A_ij for every shard i
// and block j (the system matrix of the x_ij solve of eq. (p:GPU;x) is rho_l G_ij + c0 I).
// The products of BF16 values are exact in the FP32 accumulator, which runs over all rows
// of the shard in TMEM; the result is stored in FP64 like the CUDA-core kernel's.
//
// Work item (shard i, block j, strip a, chunk b) over the block's 64-aligned column window
// [s0, e0) (s0 = first column rounded down to 64, because a TMA box must start on a 16-byte
// boundary): D[128 x 256] = A[:, s0 + 128 a + (0..127)]' A[:, s0 + 256 b + (0..255)] summed
// over the shard's rows, kept for chunk/strip pairs that touch the upper triangle.  Entries
// whose two columns both lie in block j are written to G_ij (both triangles); the rest
// (columns of a neighbouring block or of the zero padding) are computed and dropped.
//
// Per 64-row stage: four 64 x 64 boxes of the chunk (the N operand) and, unless the strip
// lies inside the chunk, two boxes of the strip (the M operand), by 2D TMA with the 128-byte
// swizzle; both operands are MN-major (rows are the contraction), the 64-column boxes LBO
// apart.  Four MMAs M = 128, N = 256, K = 16 per stage.  Rows past the shard's end in its
// last stage (they belong to the next shard) are zeroed in shared memory before the MMAs.
//
// Warp roles (192 threads): warps 0-3 read the 128 accumulator lanes at the end, warp 4
// lane 0 issues the loads, warp 5 (whole warp, one elected lane) the MMAs.
#pragma once

#include "mc_tc.cuh"

namespace bic {

struct GramItem {
  int shard, block, a, b;
};

constexpr int kGramThreads = 192;
constexpr int kGramStages = 4;
constexpr int kGramStageBytes = 6 * kTcBoxBytes;  // 4 chunk boxes + 2 strip boxes (48 KB)
constexpr int kGramTmemCols = 256;

inline size_t gram_tc_smem() {
  return 1024 + static_cast<size_t>(kGramStages) * kGramStageBytes + 256;
}

__global__ void __launch_bounds__(kGramThreads, 1)
k_gram_tc(const __grid_constant__ CUtensorMap tmap, const GramItem* __restrict__ items,
          const int64_t* __restrict__ shard_row0, const int* __restrict__ blk_col0,
          double* __restrict__ G, const int64_t* __restrict__ G_off, int M, int* __restrict__ err,
          long long wait_limit) {
  constexpr int S = kGramStages;
  constexpr uint32_t IDESC = idesc_bf16(128, 256, true, true);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* ring = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + S * kGramStageBytes);
  uint64_t* empty = full + S;
  uint64_t* done = empty + S;
  uint64_t* drainbar = done + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drainbar + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  long long* counts = reinterpret_cast<long long*>(tmem_slot + 2);  // [0] issued, [1] consumed
  volatile int* abort_v = abort_flag;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const GramItem it = items[blockIdx.x];
  const int col0 = blk_col0[it.block], nj = blk_col0[it.block + 1] - col0;
  const int s0 = col0 & ~63;
  const int fa = s0 + 128 * it.a;            // first column of the strip (M operand)
  const int fb = s0 + 256 * it.b;            // first column of the chunk (N operand)
  const bool strip_in_chunk = (it.a >> 1) == it.b;
  const int64_t r_begin = shard_row0[it.shard], r_end = shard_row0[it.shard + 1];
  const int nstg = static_cast<int>((r_end - r_begin + kTcRows - 1) / kTcRows);
  const int nbox = strip_in_chunk ? 4 : 6;

  if (tid == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], 1);
    }
    mbar_init(done, 1);
    mbar_init(drainbar, 1);
    *abort_flag = 0;
    counts[0] = counts[1] = 0;
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, kGramTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 4) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      for (int s = 0; s < nstg; ++s) {
        const int st = s % S;
        if (s >= S && !mbar_wait_or_abort(&empty[st], static_cast<uint32_t>(((s / S) - 1) & 1), wait_limit, abort_v)) {
          *abort_v = 1;
          break;
        }
        unsigned char* dst = ring + st * kGramStageBytes;
        const int y = static_cast<int>(r_begin + static_cast<int64_t>(s) * kTcRows);
        mbar_arrive_expect_tx(&full[st], static_cast<uint32_t>(nbox * kTcBoxBytes));
#pragma unroll
        for (int bx = 0; bx < 4; ++bx) tma_load_2d(dst + bx * kTcBoxBytes, &tmap, fb + 64 * bx, y, &full[st]);
        if (!strip_in_chunk) {
#pragma unroll
          for (int bx = 0; bx < 2; ++bx)
            tma_load_2d(dst + (4 + bx) * kTcBoxBytes, &tmap, fa + 64 * bx, y, &full[st]);
        }
        counts[0] = s + 1;
      }
    }
  } else if (warp == 5) {
    // ---------------------------------------------------------------- MMA issuer (whole warp)
    const uint64_t tmn = sdesc_sw128(0, kTcBoxBytes, 1024);  // MN-major, 64-column boxes LBO apart
    const uint32_t ring_a = smem_addr(ring);
    auto dsc = [](uint64_t t, uint32_t addr) -> uint64_t { return t | ((addr >> 4) & 0x3FFFu); };
    bool ok = true;
    for (int s = 0; s < nstg; ++s) {
      const int st = s % S;
      if (!mbar_wait_or_abort(&full[st], static_cast<uint32_t>((s / S) & 1), wait_limit, abort_v)) {
        ok = false;
        break;
      }
      unsigned char* sp = ring + st * kGramStageBytes;
      const int64_t valid = r_end - (r_begin + static_cast<int64_t>(s) * kTcRows);
      if (valid < kTcRows) {
        // rows valid..63 of every box belong to the next shard: zero them (each row is 128
        // contiguous bytes whatever the swizzle), then hand the writes to the async proxy
        const int nrow = kTcRows - static_cast<int>(valid);
        for (int e = lane; e < nbox * nrow * 8; e += 32) {
          const int bx = e / (nrow * 8), rem = e - bx * nrow * 8;
          const int q = static_cast<int>(valid) + rem / 8, ch = rem & 7;
          *reinterpret_cast<uint4*>(sp + bx * kTcBoxBytes + (q >> 3) * 1024 + (q & 7) * 128 + ch * 16) =
              make_uint4(0u, 0u, 0u, 0u);
        }
        fence_async_smem();
        __syncwarp();
      }
      tc_fence_after();
      const uint32_t sa = ring_a + st * kGramStageBytes;
      const uint32_t ma = strip_in_chunk ? sa + (it.a & 1) * 2 * kTcBoxBytes : sa + 4 * kTcBoxBytes;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks)
        umma_bf16_warp(tmem, dsc(tmn, ma + ks * 2048), dsc(tmn, sa + ks * 2048), IDESC,
                       (s | ks) != 0 ? 1u : 0u);
      umma_commit_warp(&empty[st]);
      counts[1] = s + 1;
    }
    if (!ok) *abort_v = 1;
    umma_commit_warp(done);
  } else if (warp < 4) {
    // ---------------------------------------------------------------- epilogue warps
    if (mbar_wait_or_abort(done, 0u, wait_limit, abort_v) && !*abort_v) {
      tc_fence_after();
      double* Gb = G + G_off[it.shard * M + it.block];
      const int l1 = fa + warp * 32 + lane - col0;  // local column of this accumulator row
      const uint32_t lane_base = static_cast<uint32_t>(warp * 32) << 16;
      for (int cc = 0; cc < 16; ++cc) {
        uint32_t v[16];
        tmem_ld16(tmem + lane_base + cc * 16, v);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int l2 = fb + cc * 16 + q - col0;
          if (l1 >= 0 && l1 < nj && l2 >= l1 && l2 < nj) {
            const double val = static_cast<double>(__uint_as_float(v[q]));
            Gb[static_cast<int64_t>(l1) * nj + l2] = val;
            Gb[static_cast<int64_t>(l2) * nj + l1] = val;
          }
        }
      }
      tc_fence_before();
    } else {
      *abort_v = 1;
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
      umma_commit_warp(drainbar);
      mbar_wait_bounded(drainbar, 0, wait_limit);
    }
    __syncthreads();
  }
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kGramTmemCols);
  }
}

}  // namespace bic
