// Device-side helpers shared by the Bi-cADMM kernels: vector types, warp/block
// reductions, and the PTX wrappers for mbarriers and bulk (TMA) copies.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace bic {

// Device error codes written to the handle's error word (first writer wins).
enum DevErr : int {
  DEV_OK = 0,
  DEV_TIMEOUT_PASS = 1,    // an mbarrier wait in the A pass hit its cycle limit
  DEV_NONPOS_PIVOT = 2,    // Cholesky met a non-positive pivot
  DEV_NONFINITE = 3,       // NaN/Inf in a residual
  DEV_ZT_NOCONV = 4,       // (z,t) root iteration exceeded its bound
  DEV_BAD_LABEL = 5,       // a softmax label is not an integer in [0, K)
};

// Upper bound on any single spin-wait, in SM clock cycles (about 2 s at 2 GHz).
constexpr long long kWaitLimitCycles = 4000000000LL;

__device__ __forceinline__ void set_err(int* err, int code) { atomicCAS(err, 0, code); }

// 16-byte vector of A elements.
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };
template <> struct Vec16<__nv_bfloat16> { using type = uint4; static constexpr int n = 8; };

// Element conversion between the stored A type and the arithmetic types (to BF16: round
// to nearest even).
template <typename TO, typename TI> __device__ __forceinline__ TO conv(TI v) { return static_cast<TO>(v); }
template <> __device__ __forceinline__ float conv<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ double conv<double, __nv_bfloat16>(__nv_bfloat16 v) { return static_cast<double>(__bfloat162float(v)); }
template <> __device__ __forceinline__ __nv_bfloat16 conv<__nv_bfloat16, double>(double v) { return __double2bfloat16(v); }
template <> __device__ __forceinline__ __nv_bfloat16 conv<__nv_bfloat16, float>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 conv<__nv_bfloat16, __nv_bfloat16>(__nv_bfloat16 v) { return v; }

// Reduce-scatter of C values (C a power of two <= 32) across a warp: on return lane l
// holds the warp-wide sum of v[(l >> (5 - log2 C)) & (C - 1)] (v is clobbered).  Costs
// C - 1 + 5 - log2 C shuffles instead of 5 C for C separate butterflies.
template <int C, typename T>
__device__ __forceinline__ T warp_reduce_scatter(T (&v)[C], int lane) {
#pragma unroll
  for (int c = C, o = 16; c > 1; c >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < c / 2; ++i) {
      const T send = up ? v[i] : v[i + c / 2];
      const T keep = up ? v[i + c / 2] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  T s = v[0];
#pragma unroll
  for (int o = 16 / C; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// Byte offset of element (row q, column c) inside a tile of rows of 64 BF16 (128 bytes)
// with the 128-byte swizzle: the 16-byte chunk index is XORed with the row index mod 8.
__host__ __device__ __forceinline__ uint32_t sw128_off(int q, int c) {
  return static_cast<uint32_t>((q >> 3) * 1024 + (q & 7) * 128 + ((((c >> 3) ^ q) & 7) << 4) + (c & 7) * 2);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Block-wide sum of NV doubles, result broadcast to every thread.  scratch holds at least
// 32 * NV doubles.  Fixed reduction order (deterministic).
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) scratch[k * 32 + warp] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double x = lane < nw ? scratch[k * 32 + lane] : 0.0;
      x = warp_sum(x);
      if (lane == 0) scratch[k * 32] = x;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = scratch[k * 32];
  __syncthreads();
}

// ----------------------------------------------------------------- mbarrier / bulk copy

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

// Make mbarrier initialisation visible to the async (bulk-copy) proxy.
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// One-dimensional bulk copy global -> shared through the TMA unit, completing as
// transaction bytes on *bar.  dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of *bar to complete, giving up after `limit` cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

__device__ __forceinline__ double dsign(double x) { return (x > 0.0) - (x < 0.0); }

}  // namespace bic
