// Tensor-core (tcgen05, kind::tf32) Gram matrices G_ij = A_ij' A_ij for every shard i and
// block j (the system matrix of the x_ij solve of eq. (p:GPU;x) is rho_l G_ij + c0 I),
// stored in FP64, for every 16/32-bit storage of A.
//
// TF32 keeps 11 significant bits.  FP32 storage (TERMS = 3): every element is split as
// a = hi + lo with hi = tf32(a) and lo = tf32(a - hi) (both rounded to nearest even), and
// the product is accumulated as hi hi' (BIG) + hi lo' + lo hi' (SMALL; the lo lo' term,
// below 2^-22 of the product, is dropped), so G carries about 22 bits of A instead of 11.
// TF32 storage (A rounded to TF32 when it was loaded) and BF16 storage (BF16 values are
// exact in TF32) take one product per pair, exact in the FP32 accumulator (TERMS = 1).
//
// Accumulation chains are kept short.  The tensor cores' FP32 accumulation is biased toward
// zero (measured on this part: a 12500-row chain in one accumulator lost 5e-5 to 1.4e-4 of
// every diagonal entry, growing in proportion to the rows), so every F = 8 stages (256 rows)
// the staging warps fold the chain into a compensated sum kept
// in TMEM (S + C, Knuth's two-sum on the CUDA cores) and the MMA warp starts a fresh chain.
// The epilogue adds S, C and the last chain in FP64.
//
// Work item (shard i, block j, strip a, chunk b) over the block's own columns: the strip is
// columns 128 a .. 128 a + 127 (the M = 128 operand, rows of the accumulator), the chunk
// columns 128 b .. (the N operand, N = the chunk's columns in the block rounded up to 16);
// chunks b >= a are computed, which covers every (l1, l2 >= l1) pair once; the epilogue
// writes both triangles.  Columns outside the block and rows outside the shard are staged
// as zeros, so no TMA alignment rule constrains where a block starts.
//
// Both operands are K-major (the contraction runs over rows): each stage holds 32 rows of
// A, which the staging warps load with plain coalesced loads, split, and write transposed
// into 128-byte-swizzled tiles (one 128-byte row of 32 TF32 values per column, the 16-byte
// chunks XORed with the column index mod 8, exactly the TMA SWIZZLE_128B pattern).  Four
// K = 8 MMAs per term consume a stage.
//
// Warp roles (288 threads): warps 0-7 stage operands (the next stage's loads are issued
// before the current stage is written), fold chains and, at the end, read the accumulators
// (warp w: TMEM lanes 32 (w % 4).., columns 64 (w / 4)..); warp 8 issues the MMAs (one
// elected lane of a converged warp).  TMEM: BIG, SMALL, S, C, 128 columns each.  Every wait
// is bounded; on expiry the CTA records BICADMM_ERR_TIMEOUT, lets its issued MMAs complete
// and frees its TMEM.
#pragma once

#include "mc_tc.cuh"

namespace bic {

constexpr int kG32Threads = 288;
constexpr int kG32StageRows = 32;     // one 128-byte swizzle row of TF32 per column
constexpr int kG32MaxStages = 4;
constexpr int kG32SmemBudget = 200 * 1024;

// Bytes of one stage: chunk and strip tiles (hi, and lo when TERMS = 3).
__host__ __device__ constexpr int g32_stage_bytes(int cw, int terms) {
  return (cw + 128) * 128 * (terms == 3 ? 2 : 1);
}
__host__ __device__ constexpr int g32_stages(int cw, int terms) {
  return kG32SmemBudget / g32_stage_bytes(cw, terms) < kG32MaxStages
             ? kG32SmemBudget / g32_stage_bytes(cw, terms)
             : kG32MaxStages;
}
inline size_t gram_tf32_smem(int cw, int terms) {
  return 1024 + static_cast<size_t>(g32_stages(cw, terms)) * g32_stage_bytes(cw, terms) + 256;
}

// Round an FP32 bit pattern to TF32 (10 stored mantissa bits), to nearest, ties to even:
// add 0xFFF (half an ulp of the kept part, minus one) plus the kept part's lowest bit, so
// that only a dropped part above one half, or exactly one half next to an odd kept part,
// carries; then clear the 13 dropped bits.  Inf and NaN pass through unchanged.
__host__ __device__ __forceinline__ uint32_t tf32_rne_bits(uint32_t u) {
  if ((u & 0x7F800000u) == 0x7F800000u) return u;
  u += 0xFFFu + ((u >> 13) & 1u);
  return u & 0xFFFFE000u;
}
__device__ __forceinline__ float tf32_rne(float a) { return __uint_as_float(tf32_rne_bits(__float_as_uint(a))); }

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void umma_tf32_warp(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                               uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p, e;\n\tsetp.ne.b32 p, %4, 0;\n\telect.sync _|e, 0xffffffff;\n\t"
      "@e tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// In-place rounding of rows [r0, r1) of a 32-bit matrix to TF32 (TF32 storage).
__global__ void k_round_tf32(float* __restrict__ A, int64_t lda, int64_t r0, int64_t r1) {
  const int64_t total = (r1 - r0) * lda;
  float* base = A + r0 * lda;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    base[i] = tf32_rne(base[i]);
}

// tcgen05.st of 16 consecutive 32-bit columns of this warp's 32 TMEM lanes, and the wait for
// this thread's stores.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
      "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Work item of the TF32 Gram (one CTA): shard, block, strip a (128 columns), chunk b (128).
// A work item: the (a, b) 128 x 128 tile of block `block`'s Gram matrix over shard `shard`'s
// rows, or over part `part` of them (`nparts` contiguous pieces, each a CTA, for a shard's
// few tiles to fill the GPU): a part writes its partial tile to scratch tile
// `group * nparts + part`, and the last part to finish (a ticket per group) adds the
// partials in part order into G.
struct Gram32Item {
  int shard, block, a, b;
  int part, nparts, group;
};

// TMEM columns: the running products of the current chain (hi hi' in BIG; hi lo' + lo hi' in
// SMALL when TERMS = 3) and the compensated sum of the folded chains (SACC + CACC).
constexpr uint32_t kG32Big = 0, kG32Small = 128, kG32SAcc = 256, kG32CAcc = 384;
// stages per accumulation chain: 4 MMAs of K = 8 per stage, so a chain adds 32 F partial
// products into the FP32 accumulator
__host__ __device__ constexpr int g32_chain_stages(int) { return 8; }

template <int TERMS, typename TIN>
__global__ void __launch_bounds__(kG32Threads, 1)
k_gram_tf32(const TIN* __restrict__ A, int64_t lda, const Gram32Item* __restrict__ items,
            const int64_t* __restrict__ shard_row0, const int* __restrict__ blk_col0,
            double* __restrict__ G, const int64_t* __restrict__ G_off, int M,
            double* __restrict__ scratch, int* __restrict__ tick, int* __restrict__ err,
            long long wait_limit) {
  constexpr int CW = 128;
  constexpr int S = g32_stages(CW, TERMS);
  constexpr int SB = g32_stage_bytes(CW, TERMS);
  constexpr int F = g32_chain_stages(TERMS);
  constexpr int CHB = CW * 128;             // one chunk tile (hi or lo)
  constexpr int STB = 128 * 128;            // one strip tile
  constexpr int IT_C = CW * 8 / 256;        // chunk items per staging thread (4 rows x 1 col each)
  constexpr int IT = IT_C + 4;              // + strip items (128 x 8 / 256)
  static_assert(S >= 2, "at least two stages");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* ring = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + S * SB);
  uint64_t* empty = full + S;
  uint64_t* done = empty + S;
  uint64_t* drainbar = done + 1;
  uint64_t* accfree = drainbar + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accfree + 1);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  volatile int* abort_v = abort_flag;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const Gram32Item it = items[blockIdx.x];
  const int col0 = blk_col0[it.block], nj = blk_col0[it.block + 1] - col0;
  const int sa0 = 128 * it.a, cb0 = CW * it.b;                // local first columns
  const int cvalid = nj - cb0 < CW ? nj - cb0 : CW;            // chunk columns in the block
  const int N = (cvalid + 15) & ~15;                           // MMA N (multiple of 16)
  const bool sic = it.a == it.b;                               // strip = chunk
  const int cfill = sic ? CW : N;  // chunk tile rows holding data (all 128 when it is the strip too)
  // this item's rows: its part of the shard, cut at 32-row stage boundaries
  const int64_t rs0 = shard_row0[it.shard], rs1 = shard_row0[it.shard + 1];
  const int64_t nst_all = (rs1 - rs0 + kG32StageRows - 1) / kG32StageRows;
  const int64_t st_lo = nst_all * it.part / it.nparts, st_hi = nst_all * (it.part + 1) / it.nparts;
  const int64_t r_begin = rs0 + st_lo * kG32StageRows;
  const int64_t r_end = rs0 + st_hi * kG32StageRows < rs1 ? rs0 + st_hi * kG32StageRows : rs1;
  const int nstg = static_cast<int>(st_hi - st_lo);
  __shared__ int last_part;
  // a chain ends after stage s when (s + 1) % F == 0 and stage s + S exists (its staging is
  // where the fold happens); the last chain runs to the end and is folded in the epilogue
  auto chain_end = [&](int s) { return (s + 1) % F == 0 && s + S < nstg; };

  if (tid == 0) {
    for (int st = 0; st < S; ++st) {
      mbar_init(&full[st], 8);   // one arrival per staging warp
      mbar_init(&empty[st], 1);  // the MMA warp's commit
    }
    mbar_init(done, 1);
    mbar_init(drainbar, 1);
    mbar_init(accfree, 8);       // the staging warps, after folding a chain
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp < 8) {
    // ------------------------------------------------------------ staging warps
    const TIN* Ab = A + col0;
    float cur[IT][4], nxt[IT][4];
    // item e of this thread: t = tid + 256 e; chunk items first (column q = t % cfill,
    // 4-row group kc = t / cfill), then strip items (q = t % 128, kc = t / 128)
    auto load = [&](float (&v)[IT][4], int s) {
      const int64_t rb = r_begin + static_cast<int64_t>(s) * kG32StageRows;
#pragma unroll
      for (int e = 0; e < IT; ++e) {
        const bool strip = e >= IT_C;
        const int t = tid + 256 * (strip ? e - IT_C : e);
        const int W = strip ? 128 : cfill;
        const bool live = strip ? !sic : t < W * 8;
        const int q = t % W, kc = t / W;
        const int col = (strip ? sa0 : cb0) + q;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int64_t r = rb + 4 * kc + i;
          v[e][i] = (live && col < nj && r < r_end) ? conv<float>(Ab[r * lda + col]) : 0.0f;
        }
      }
    };
    auto store = [&](const float (&v)[IT][4], unsigned char* stage) {
#pragma unroll
      for (int e = 0; e < IT; ++e) {
        const bool strip = e >= IT_C;
        const int t = tid + 256 * (strip ? e - IT_C : e);
        const int W = strip ? 128 : cfill;
        if (strip ? sic : t >= W * 8) continue;
        const int q = t % W, kc = t / W;
        const uint32_t off = static_cast<uint32_t>(q) * 128u + ((static_cast<uint32_t>(kc ^ q) & 7u) << 4);
        // stage layout: chunk hi | chunk lo | strip hi | strip lo  (TERMS = 1: chunk | strip)
        unsigned char* hi_tile = strip ? stage + (TERMS == 3 ? 2 * CHB : CHB) : stage;
        float hv[4], lv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          hv[i] = tf32_rne(v[e][i]);
          lv[i] = tf32_rne(v[e][i] - hv[i]);
        }
        *reinterpret_cast<uint4*>(hi_tile + off) =
            make_uint4(__float_as_uint(hv[0]), __float_as_uint(hv[1]), __float_as_uint(hv[2]), __float_as_uint(hv[3]));
        if (TERMS == 3)
          *reinterpret_cast<uint4*>(hi_tile + (strip ? STB : CHB) + off) =
              make_uint4(__float_as_uint(lv[0]), __float_as_uint(lv[1]), __float_as_uint(lv[2]), __float_as_uint(lv[3]));
      }
    };
    // Fold the finished chain into (SACC, CACC) with Knuth's two-sum (rounding to nearest on
    // the CUDA cores), so the long sum carries no accumulator bias: S' = S + v exactly as
    // S' + e, e added to C.  Warp w owns lanes 32 (w % 4).. and columns 64 (w / 4)..
    const int lq = warp & 3, half = warp >> 2;
    const uint32_t lane_base = static_cast<uint32_t>(32 * lq) << 16;
    bool folded = false;
    auto fold = [&]() {
      for (int cc = 4 * half; cc < 4 * half + 4 && 16 * cc < N; ++cc) {
        const uint32_t col = lane_base + 16 * cc;
        uint32_t vb[16], vs[16], sa[16], ca[16];
        tmem_ld16(tmem + col + kG32Big, vb);
        if (TERMS == 3) tmem_ld16(tmem + col + kG32Small, vs);
        if (folded) {
          tmem_ld16(tmem + col + kG32SAcc, sa);
          tmem_ld16(tmem + col + kG32CAcc, ca);
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const float v = TERMS == 3 ? __uint_as_float(vb[q]) + __uint_as_float(vs[q]) : __uint_as_float(vb[q]);
          if (!folded) {
            sa[q] = __float_as_uint(v);
            ca[q] = 0u;
          } else {
            const float s0 = __uint_as_float(sa[q]);
            const float s1 = s0 + v;
            const float bp = s1 - s0;
            const float e = (s0 - (s1 - bp)) + (v - bp);
            sa[q] = __float_as_uint(s1);
            ca[q] = __float_as_uint(__uint_as_float(ca[q]) + e);
          }
        }
        tmem_st16(tmem + col + kG32SAcc, sa);
        tmem_st16(tmem + col + kG32CAcc, ca);
      }
      tmem_st_wait();
      folded = true;
    };
    bool ok = true;
    if (nstg > 0) load(cur, 0);
    for (int s = 0; s < nstg; ++s) {
      const int st = s % S;
      if (s + 1 < nstg) load(nxt, s + 1);
      if (s >= S) {
        if (!mbar_wait_or_abort(&empty[st], static_cast<uint32_t>(((s / S) - 1) & 1), wait_limit, abort_v)) {
          ok = false;
          break;
        }
        if (chain_end(s - S)) {  // the MMAs of stage s - S (the chain's last) have completed
          tc_fence_after();
          fold();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(accfree);
        }
      }
      store(cur, ring + st * SB);
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&full[st]);
#pragma unroll
      for (int e = 0; e < IT; ++e)
#pragma unroll
        for (int i = 0; i < 4; ++i) cur[e][i] = nxt[e][i];
    }
    if (!ok) *abort_v = 1;
    // ------------------------------------------------------------ epilogue
    if (ok && mbar_wait_or_abort(done, 0u, wait_limit, abort_v) && !*abort_v) {
      tc_fence_after();
      double* Gb = G + G_off[it.shard * M + it.block];
      const int l1 = sa0 + 32 * lq + lane;  // local column of this accumulator row
      for (int cc = 4 * half; cc < 4 * half + 4 && 16 * cc < N; ++cc) {
        const uint32_t col = lane_base + 16 * cc;
        uint32_t vb[16], vs[16], sa[16], ca[16];
        tmem_ld16(tmem + col + kG32Big, vb);
        if (TERMS == 3) tmem_ld16(tmem + col + kG32Small, vs);
        if (folded) {
          tmem_ld16(tmem + col + kG32SAcc, sa);
          tmem_ld16(tmem + col + kG32CAcc, ca);
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int l2 = cb0 + 16 * cc + q;
          if (l1 < nj && l2 >= l1 && l2 < nj) {
            double val = static_cast<double>(__uint_as_float(vb[q]));
            if (TERMS == 3) val += static_cast<double>(__uint_as_float(vs[q]));
            if (folded) val += static_cast<double>(__uint_as_float(sa[q])) + static_cast<double>(__uint_as_float(ca[q]));
            if (it.nparts == 1) {
              Gb[static_cast<int64_t>(l1) * nj + l2] = val;
              Gb[static_cast<int64_t>(l2) * nj + l1] = val;
            } else {
              scratch[(static_cast<int64_t>(it.group) * it.nparts + it.part) * (128 * 128) +
                      (32 * lq + lane) * 128 + 16 * cc + q] = val;
            }
          }
        }
      }
      if (it.nparts > 1) __threadfence();  // the partial tile before this CTA's ticket
      tc_fence_before();
    } else {
      *abort_v = 1;
    }
  } else {
    // ------------------------------------------------------------ MMA issuer (warp 8)
    const uint32_t idesc = idesc_tf32(128, N);
    const uint64_t tk = sdesc_sw128(0, 16, 1024);  // K-major, 8-row groups 1024 bytes apart
    auto dsc = [&](uint32_t addr) -> uint64_t { return tk | ((addr >> 4) & 0x3FFFu); };
    const uint32_t ring_a = smem_addr(ring);
    bool ok = true, fresh = true;
    int nfold = 0;
    for (int s = 0; s < nstg; ++s) {
      const int st = s % S;
      if (!mbar_wait_or_abort(&full[st], static_cast<uint32_t>((s / S) & 1), wait_limit, abort_v)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t sb = ring_a + st * SB;
      const uint32_t b_hi = sb, b_lo = sb + CHB;
      const uint32_t strip_base = TERMS == 3 ? sb + 2 * CHB : sb + CHB;
      const uint32_t a_hi = sic ? b_hi : strip_base;
      const uint32_t a_lo = sic ? b_lo : strip_base + STB;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const uint32_t acc = (fresh && ks == 0) ? 0u : 1u;
        umma_tf32_warp(tmem + kG32Big, dsc(a_hi + 32 * ks), dsc(b_hi + 32 * ks), idesc, acc);
        if (TERMS == 3) {
          umma_tf32_warp(tmem + kG32Small, dsc(a_hi + 32 * ks), dsc(b_lo + 32 * ks), idesc, acc);
          umma_tf32_warp(tmem + kG32Small, dsc(a_lo + 32 * ks), dsc(b_hi + 32 * ks), idesc, 1u);
        }
      }
      fresh = false;
      umma_commit_warp(&empty[st]);
      if (chain_end(s)) {  // wait until the staging warps have folded this chain
        if (!mbar_wait_or_abort(accfree, static_cast<uint32_t>(nfold & 1), wait_limit, abort_v)) {
          ok = false;
          break;
        }
        ++nfold;
        tc_fence_after();
        fresh = true;
      }
    }
    if (!ok) *abort_v = 1;
    umma_commit_warp(done);
  }
  __syncthreads();
  if (*abort_v) {
    if (tid == 0) set_err(err, DEV_TIMEOUT_PASS);
    // let every MMA this CTA issued complete before its TMEM is freed
    if (warp == 8) {
      umma_commit_warp(drainbar);
      mbar_wait_bounded(drainbar, 0, kWaitLimitCycles);
    }
    __syncthreads();
  }
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
  if (it.nparts > 1 && !*abort_v) {
    // the last part of the group adds the partials in part order and writes both triangles
    if (tid == 0) last_part = atomicAdd(&tick[it.group], 1) == it.nparts - 1;
    __syncthreads();
    if (last_part && warp < 8) {
      const int lq = warp & 3, half = warp >> 2;
      double* Gb = G + G_off[it.shard * M + it.block];
      const int l1 = sa0 + 32 * lq + lane;
      for (int cc = 4 * half; cc < 4 * half + 4 && 16 * cc < N; ++cc) {
        for (int q = 0; q < 16; ++q) {
          const int l2 = cb0 + 16 * cc + q;
          if (l1 < nj && l2 >= l1 && l2 < nj) {
            double val = 0.0;
            for (int p = 0; p < it.nparts; ++p)
              val += __ldcg(&scratch[(static_cast<int64_t>(it.group) * it.nparts + p) * (128 * 128) +
                                     (32 * lq + lane) * 128 + 16 * cc + q]);
            Gb[static_cast<int64_t>(l1) * nj + l2] = val;
            Gb[static_cast<int64_t>(l2) * nj + l1] = val;
          }
        }
      }
    }
    if (last_part && tid == 0) tick[it.group] = 0;
  }
}

}  // namespace bic
