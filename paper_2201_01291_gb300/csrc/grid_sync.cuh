// Deterministic block and grid reductions for persistent (cooperatively launched) kernels.
//
// The grid reduction doubles as the grid-wide barrier: every block publishes its partial
// sums, the last block to arrive adds all partials in block order (so the result does not
// depend on arrival order) and releases the others by bumping a generation counter.  Every
// wait is bounded: after kSpinLimitNs of polling a block raises `abort`, every waiter leaves,
// and the kernel reports AVIP_ETIMEOUT instead of hanging.
#pragma once
#include <cstdint>

#include "avip_internal.h"

namespace avip {

constexpr unsigned long long kSpinLimitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Sum NV values over the block; the result is valid in every thread.  Fixed shuffle/smem
// order, so identical inputs give identical bits.  smem must hold 32*NV doubles + NV.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* smem) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  }
  __syncthreads();  // smem may still be read by a previous call
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) smem[k * 32 + warp] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = lane < nw ? smem[k * 32 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) smem[32 * NV + k] = t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = smem[32 * NV + k];
}

// Grid-wide sum of NV (<= 8, <= warps per block) values; also a grid barrier.  Returns false
// if the wait was abandoned (timeout or another block aborted); the caller must then leave.
template <int NV>
__device__ __forceinline__ bool grid_sum(double (&v)[NV], double* partials, GridSync* gs,
                                         double* smem) {
  block_sum<NV>(v, smem);
  const int nb = gridDim.x;
  if (nb == 1) return true;
  __shared__ int s_last;
  __shared__ unsigned s_gen;
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) __stcg(partials + (size_t)blockIdx.x * NV + k, v[k]);
    unsigned g = ld_acquire_u32(&gs->gen);
    __threadfence();
    unsigned arrived = atomicAdd(&gs->count, 1u);
    __threadfence();
    s_last = (arrived == (unsigned)nb - 1);
    s_gen = g;
    s_ok = 1;
  }
  __syncthreads();
  if (s_last) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp < NV) {
      double t = 0.0;
      for (int b = lane; b < nb; b += 32) t += __ldcg(partials + (size_t)b * NV + warp);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) __stcg(&gs->red[warp], t);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      atomicExch(&gs->count, 0u);
      __threadfence();
      st_release_u32(&gs->gen, s_gen + 1);
    }
  } else if (threadIdx.x == 0) {
    const unsigned long long t0 = global_timer_ns();
    unsigned spins = 0;
    while (ld_acquire_u32(&gs->gen) == s_gen) {
      if ((++spins & 255u) == 0) {
        if (*((volatile int*)&gs->abort)) {
          s_ok = 0;
          break;
        }
        if (global_timer_ns() - t0 > kSpinLimitNs) {
          atomicExch(&gs->abort, 1);
          s_ok = 0;
          break;
        }
      }
    }
  }
  __syncthreads();
  if (!s_ok) return false;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = __ldcg(&gs->red[k]);
  return true;
}

}  // namespace avip
