// SELL-32 row product shared by the FP64 Krylov kernels.
#pragma once
#include "avip_internal.h"

namespace avip {

// One row of y = A v over the SELL-32 structure (diagonal first, then ascending columns).
// Slots are fetched in groups of 8 so that the column loads, the value loads and the
// dependent gathers of a group are all in flight together.
__device__ __forceinline__ double sell_row_dot(const SellView& A, int slice, int lane, int row,
                                               const double* __restrict__ v) {
  constexpr int U = 8;
  const int base = __ldg(A.sl_ptr + slice) + lane;
  const int w = __ldg(A.sl_w + slice);
  const int rl = __ldg(A.rlen + row);
  double acc = 0.0;
  for (int k0 = 0; k0 < w; k0 += U) {
    int c[U];
    double av[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u;
      c[u] = row;
      av[u] = 0.0;
      if (k < rl) {
        c[u] = __ldg(A.col + base + k * kSlice);
        av[u] = __ldg(A.aval + base + k * kSlice);
      }
    }
    double xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = (k0 + u < rl) ? __ldcg(v + c[u]) : 0.0;
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (k0 + u < rl) acc = fma(av[u], xv[u], acc);
  }
  return acc;
}

// Fused multiply-add in the accumulation type.
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

// Contiguous share [sa, sb) of nsl slices for warp w of nw (equal slice counts).
__device__ __forceinline__ void warp_slices(int nsl, int w, int nw, int& sa, int& sb) {
  sa = (int)((long long)nsl * w / nw);
  sb = (int)((long long)nsl * (w + 1) / nw);
}

// Gathered vectors are written by other blocks in an earlier phase of the same launch and read
// after a grid (or cluster) barrier: release increment, acquire wait, then bar.sync, which orders
// every later weak load of the block after the other blocks' writes.  They are read with
// ld.global.ca (__ldca: cached in L1 and L2), never through the read-only .nc path, whose
// contents may go stale within a launch; neighbouring rows of a warp's contiguous share gather
// mostly the same entries, so L1 serves most of them.

// No operands to fetch ahead for a row (see spmv_stream).
struct NoPre {};
struct NoBegin {
  __device__ NoPre operator()(int) const { return NoPre(); }
};

// Streamed product of the rows of slices [sa, sb) of a SELL-32 matrix with `lpr` lanes per row
// (SellHost) by one warp: for every row < nrows, emit(row, sum of val * g(col) over its stored
// entries, pre), in slice order, on the row's first lane.  The elements of consecutive slices
// are contiguous (slice s + 1 starts where slice s ends), so the warp walks them as one stream
// of 32-wide steps and fetches them in batches of U steps whatever the row lengths: the U
// column and value loads of a batch are issued together, then its U gathers, so every lane keeps
// U independent loads in flight even on rows of a few entries.  Padding slots (column 0,
// value 0) are read like the others and add nothing.  At a slice boundary (warp-uniform) the
// lanes of each row combine their partial sums by shuffles and the row is emitted; a slice
// without steps emits zeros.  `begin(row)` runs on the row's first lane when its slice starts
// and returns the row's own operands (`pre`), so that their loads overlap the slice's stream
// instead of stalling the emit.  TA is the accumulation type, TV the stored value type.
template <typename TA, int U, typename TV, class G, class Begin, class Emit>
__device__ __forceinline__ void spmv_stream(const int32_t* __restrict__ sl_ptr, const int32_t* __restrict__ sl_w,
                                            const int32_t* __restrict__ col, const TV* __restrict__ val, int nrows,
                                            int lpr, int sa, int sb, int lane, G g, Begin begin, Emit emit) {
  if (sa >= sb) return;
  const int lg = __ffs(lpr) - 1;        // log2(lanes per row)
  const int rsub = lane >> lg;          // row of the slice this lane works on
  const bool lead = (lane & (lpr - 1)) == 0;
  const int e0 = __ldg(sl_ptr + sa);
  const int nsteps = (__ldg(sl_ptr + sb) - e0) >> 5;
  const int32_t* __restrict__ cp = col + e0 + lane;
  const TV* __restrict__ vp = val + e0 + lane;
  // widths of 32 slices at a time: lane t holds the width of slice sbase + t
  int sbase = sa;
  int wreg = sa + lane < sb ? __ldg(sl_w + sa + lane) : 0;
  int s = sa;
  int rem = __shfl_sync(0xffffffffu, wreg, 0);
  decltype(begin(0)) pre{};
  auto enter = [&]() {
    const int row = (s << (5 - lg)) + rsub;
    if (lead && row < nrows) pre = begin(row);
  };
  auto finish = [&](TA v) {
    for (int o = lpr >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int row = (s << (5 - lg)) + rsub;
    if (lead && row < nrows) emit(row, v, pre);
  };
  auto next_slice = [&]() {
    ++s;
    if (s < sb) {
      if (s - sbase == 32) {
        sbase = s;
        wreg = s + lane < sb ? __ldg(sl_w + s + lane) : 0;
      }
      rem = __shfl_sync(0xffffffffu, wreg, s - sbase);
      enter();
    }
  };
  auto skip_empty = [&]() {
    while (rem == 0 && s < sb) {
      finish(TA(0));
      next_slice();
    }
  };
  enter();
  skip_empty();
  // software pipeline: the column and value loads of batch k + 1 are issued before the gathers
  // of batch k are consumed, so the stream's memory latency overlaps the gathers' latency.  The
  // operator's elements are read once per product: loaded with the evict-first policy (.cs) so
  // that they do not push the gathered vectors out of L2.
  int c[U], cn[U];
  TV v[U], vn[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    c[u] = 0;
    v[u] = TV(0);
    if (u < nsteps) {
      c[u] = __ldcs(cp + (size_t)u * kSlice);
      v[u] = __ldcs(vp + (size_t)u * kSlice);
    }
  }
  TA acc = TA(0);
  for (int j0 = 0; j0 < nsteps; j0 += U) {
    TA x[U];
#pragma unroll
    for (int u = 0; u < U; ++u) x[u] = j0 + u < nsteps ? (TA)g(c[u]) : TA(0);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + U + u;
      cn[u] = 0;
      vn[u] = TV(0);
      if (j < nsteps) {
        cn[u] = __ldcs(cp + (size_t)j * kSlice);
        vn[u] = __ldcs(vp + (size_t)j * kSlice);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (j0 + u < nsteps) {
        acc = fma_t((TA)v[u], x[u], acc);
        if (--rem == 0) {
          finish(acc);
          acc = TA(0);
          next_slice();
          skip_empty();
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      c[u] = cn[u];
      v[u] = vn[u];
    }
  }
}

template <typename TA, int U, typename T, class G, class Begin, class Emit>
__device__ __forceinline__ void spmv_stream(const SellMatT<T>& M, int sa, int sb, int lane, G g, Begin begin,
                                            Emit emit) {
  spmv_stream<TA, U>(M.sl_ptr, M.sl_w, M.col, M.val, M.n, M.lpr, sa, sb, lane, g, begin, emit);
}

}  // namespace avip
