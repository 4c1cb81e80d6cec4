// Deterministic block and grid reductions for persistent (cooperatively launched) kernels.
//
// Grid reduction = grid barrier: every block publishes its partial sums, every block reads all
// partials in block order once everybody has arrived, so every block obtains bit-identical
// totals (deterministic, independent of arrival order).  An optional epilogue derives scalars
// from the totals (e.g. the CG step alpha = r.r / p.q) once per block.
//
// Every wait is bounded: after FlagSync::spin_ns of polling (the handle's wait_timeout) a block
// raises `abort`, every waiter leaves, and the kernel reports a timeout instead of hanging.
//
// The blocks taking part are the whole grid, or one contiguous group of it (solves that run side
// by side in one launch, each with its own barrier state): FlagSync::nb blocks, this block being
// number FlagSync::rank among them.  The arrival counter is a 32-bit value that only grows
// (mod 2^32); a block waits for barrier seq until counter - seq * nb, taken as a signed
// difference, is no longer negative.  The counter never runs more than nb arrivals ahead of or
// behind the barrier a block waits for, so the test stays right when seq * nb wraps past 2^32 on
// very long solves.
#pragma once
#include <cstdint>

#include "avip_internal.h"

namespace avip {

constexpr unsigned long long kSpinLimitNs = 2000000000ull;  // default wait limit: 2 s
constexpr int kPollUnroll = 8;  // partial loads per lane kept in flight (grids up to 256 blocks)

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Sum NV values over the block; the result is valid in every thread.  Fixed shuffle/smem
// order, so identical inputs give identical bits.  smem must hold 32*NV + NV doubles.
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

// Barrier state of the blocks of one solve.  `flags[0]` (the arrival counter) must be zero at
// launch; `parts` holds 2 * nb * 4 doubles.
struct FlagSync {
  unsigned* flags;
  double* parts;  // [2][nb][4]
  GridSync* gs;   // abort flag
  unsigned seq;   // reductions passed so far (identical in every thread)
  unsigned long long spin_ns;  // give up a wait after this long (0: at the first unsatisfied poll)
  int nb;         // blocks taking part (gridDim.x for a whole-grid solve)
  int rank;       // this block's index among them (blockIdx.x for a whole-grid solve)
};

// True while the arrival counter has not reached `target` (wrap-safe, see above).
__device__ __forceinline__ bool arrivals_behind(const unsigned* counter, unsigned target) {
  return (int)(ld_acquire_u32(counter) - target) < 0;
}

// Bounded wait of one thread for `target` arrivals: false if the wait was abandoned (its time
// limit passed, or another block raised `abort`).  The limit and the abort flag are checked on
// the first poll and then every 64 polls.
__device__ __forceinline__ bool wait_arrivals(const FlagSync& fs, unsigned target) {
  const unsigned long long t0 = global_timer_ns();
  unsigned spins = 0;
  while (arrivals_behind(fs.flags, target)) {
    if ((spins++ & 63u) == 0) {
      if (*((volatile int*)&fs.gs->abort) || global_timer_ns() - t0 >= fs.spin_ns) return false;
    }
  }
  return true;
}

// Shared-memory scratch of grid_allsum.  A __shared__ variable declared inside a function
// template exists once per instantiation, so a kernel that reduces with several (NV, NE)
// combinations would reserve the scratch several times over (less L1 for the gathers, fewer
// co-resident blocks); declared in this one non-template function it exists once per kernel.
struct AllsumScratch {
  double thr[4 * 1024];  // per-thread values, [value k][thread]
  double res[8];         // totals, then epilogue results
  int ok;
};
__device__ __forceinline__ AllsumScratch& allsum_scratch() {
  __shared__ AllsumScratch s;
  return s;
}

struct NoEpilogue {
  __device__ void operator()(const double*, double*) const {}
};

__device__ __forceinline__ void red_add_release_u32(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Sum of NV (<= 4) values over the participating blocks; NE (<= 4) scalars are then derived from the totals by
// `epi` on one thread per block.  On return v[] holds the totals and out[] the epilogue
// results, identical in every thread of the grid.  Returns false if the wait was abandoned
// (timeout or another block aborted); the caller must leave.
//
// Protocol (measured fastest on GB300 among flag-per-block, last-block and counter schemes):
// warp sums -> shared memory -> warp 0 adds the block partial, stores it in the block's slot
// and announces it with one release reduction on a monotone arrival counter; every lane of
// warp 0 waits (acquire) until the counter reaches seq * nb and then reads all partials in
// block order.  Partials are double-buffered by the parity of seq because a fast
// block may publish reduction k+1 while a slow one is still reading reduction k.
template <int NV, int NE, typename Epi>
__device__ __forceinline__ bool grid_allsum(double (&v)[NV], double (&out)[NE > 0 ? NE : 1], FlagSync& fs,
                                            double* smem, Epi epi) {
  static_assert(NV <= 4 && NE <= 4, "grid_allsum: at most 4 sums and 4 derived scalars");
  const int nb = fs.nb;
  const unsigned seq = ++fs.seq;
  const int par = seq & 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  AllsumScratch& scr = allsum_scratch();
  double* s_res = scr.res;
  int& s_ok = scr.ok;
  double* s_thr = scr.thr;
  // Block partial: every thread stores its values, then warp 0 adds them (lane l takes
  // threads l, l+32, ...) and finishes with a shuffle tree.  On GB300 an FP64 add costs a
  // warp ~16 cycles of the SM's FP64 pipe, so this uses blockDim/32 + 5 warp-wide adds per
  // value instead of the 5 * blockDim/32 + 5 of a shuffle tree in every warp.
  (void)smem;
#pragma unroll
  for (int k = 0; k < NV; ++k) s_thr[k * 1024 + threadIdx.x] = v[k];
  __syncthreads();
  if (warp == 0) {
    double bt[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += s_thr[k * 1024 + w * 32 + lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      bt[k] = t;
    }
    int ok = 1;
    if (nb > 1) {
      if (lane == 0) {
        double* mine = fs.parts + ((size_t)par * nb + fs.rank) * 4;
#pragma unroll
        for (int k = 0; k < NV; ++k) __stcg(mine + k, bt[k]);
        red_add_release_u32(fs.flags, 1u);
      }
      if (!wait_arrivals(fs, seq * (unsigned)nb)) ok = 0;
      ok = __all_sync(0xffffffffu, ok);
      double acc[NV];
#pragma unroll
      for (int k = 0; k < NV; ++k) acc[k] = 0.0;
      if (ok) {
        if (nb <= 32 * kPollUnroll) {
          const int mine = (nb - lane + 31) / 32;
          double pv[kPollUnroll][NV];
#pragma unroll
          for (int q = 0; q < kPollUnroll; ++q) {
            const double* pb = fs.parts + ((size_t)par * nb + lane + 32 * q) * 4;
#pragma unroll
            for (int k = 0; k < NV; ++k) pv[q][k] = (q < mine) ? __ldcg(pb + k) : 0.0;
          }
#pragma unroll
          for (int q = 0; q < kPollUnroll; ++q)
#pragma unroll
            for (int k = 0; k < NV; ++k) acc[k] += pv[q][k];
        } else {
          for (int b = lane; b < nb; b += 32) {
            const double* pb = fs.parts + ((size_t)par * nb + b) * 4;
#pragma unroll
            for (int k = 0; k < NV; ++k) acc[k] += __ldcg(pb + k);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < NV; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
        bt[k] = acc[k];
      }
    }
    if (lane == 0) {
      s_ok = ok;
      if (!ok) atomicExch(&fs.gs->abort, 1);
#pragma unroll
      for (int k = 0; k < NV; ++k) s_res[k] = bt[k];
      double e[NE > 0 ? NE : 1];
      epi(s_res, e);
#pragma unroll
      for (int k = 0; k < NE; ++k) s_res[NV + k] = e[k];
    }
  }
  __syncthreads();
  if (!s_ok) return false;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = s_res[k];
#pragma unroll
  for (int k = 0; k < NE; ++k) out[k] = s_res[NV + k];
  return true;
}

template <int NV>
__device__ __forceinline__ bool grid_allsum(double (&v)[NV], FlagSync& fs, double* smem) {
  double dummy[1];
  return grid_allsum<NV, 0>(v, dummy, fs, smem, NoEpilogue());
}

// Grid barrier without a sum: the block's writes are ordered before one release increment of
// the same monotone arrival counter by thread 0, which then waits (acquire, bounded) for
// seq * nb arrivals.  It shares the counter and the sequence number with grid_allsum,
// whose partials it does not touch; a reduction k and the next one of the same buffer parity,
// k + 2, are then separated by this barrier k + 1, which no block passes before every block has
// finished reading reduction k.  Returns false if the wait was abandoned.
__device__ __forceinline__ bool grid_barrier(FlagSync& fs) {
  const unsigned seq = ++fs.seq;
  AllsumScratch& scr = allsum_scratch();
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const int nb = fs.nb;
    if (nb > 1) {
      red_add_release_u32(fs.flags, 1u);
      if (!wait_arrivals(fs, seq * (unsigned)nb)) ok = 0;
    }
    if (!ok) atomicExch(&fs.gs->abort, 1);
    scr.ok = ok;
  }
  __syncthreads();
  return scr.ok != 0;
}

}  // namespace avip
