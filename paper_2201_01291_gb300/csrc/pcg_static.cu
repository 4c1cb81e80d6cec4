// No-allocation entry point: Jacobi-preconditioned CG on a symmetric positive definite CSR
// matrix that the caller already holds in device memory, with every work vector in a
// fixed-size scratch array compiled into this library.
//
// Who needs it: callers that must not call cudaMalloc or any allocating routine at all, e.g.
// real-time loops with a fixed memory budget that forbid allocation after start-up (an
// allocation can block on the driver or fail under fragmentation at the worst moment), or
// hosts whose framework has reserved all device memory through its own pool, so that a
// cudaMalloc from a library would fail or steal from it.  Such callers cannot create a mesh
// handle (mesh_create allocates), but they can solve the same Poisson system from CSR arrays
// they placed in device memory themselves.
//
// The call is synchronous: it queues the solve on the caller's stream, copies the status back
// to the host and waits for that stream, so it blocks the calling host thread until the solve
// has finished.
//
// The scratch array lives in every GPU that loads the library until the process exits
// (kStaticMaxRows rows, about 10.5 MB).  All calls share it and it keeps the last call's
// contents: every call clears the barrier words it needs and overwrites the work vectors
// before reading them.  Calls that overlap on the GPU (different streams or host threads
// without ordering) race and corrupt each other.
//
// Its device address is looked up once per device, by the first call made with that device
// current (cudaGetSymbolAddress, which allocates nothing).  cudaDeviceReset destroys the
// context that address belongs to: a process that resets a device must not call this entry
// point on that device again.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <mutex>

#include "avip_internal.h"
#include "grid_sync.cuh"

namespace avip {

constexpr int kStaticMaxRows = 262144;
constexpr int kStaticTPB = 256;
constexpr int kStaticMaxBlocks = 1024;
// layout (doubles): [control: 32 doubles = 256 B][parts: 2 * kStaticMaxBlocks * 4][dinv][r][z][p][q]
// control: GridSync (abort word) at 0, barrier counter at double 12, status at 16, relres at 20
constexpr size_t kFlagDoubles = 32;
constexpr size_t kPartDoubles = 2 * (size_t)kStaticMaxBlocks * 4;
constexpr size_t kStaticDoubles = kFlagDoubles + kPartDoubles + 5 * (size_t)kStaticMaxRows;

static_assert(sizeof(GridSync) <= 12 * sizeof(double), "control area layout");
static __device__ __align__(256) double g_pcg_scratch[kStaticDoubles];

struct StaticPcgArgs {
  int32_t n;
  const int32_t* row_ptr;
  const int32_t* col;
  const double* val;
  const double* b;
  double* x;
  double* scratch;  // device address of g_pcg_scratch
  double rtol;
  int32_t max_iter;
  int32_t* status_out;  // in scratch: [0] status, [1] iterations
  double* relres_out;   // in scratch
};

// row i of A v (CSR)
__device__ __forceinline__ double csr_row(const StaticPcgArgs& a, int i, const double* v) {
  double acc = 0.0;
  const int e1 = __ldg(a.row_ptr + i + 1);
  for (int e = __ldg(a.row_ptr + i); e < e1; ++e) acc = fma(__ldg(a.val + e), __ldcg(v + __ldg(a.col + e)), acc);
  return acc;
}

__global__ void __launch_bounds__(kStaticTPB) pcg_csr_static_kernel(StaticPcgArgs a) {
  __shared__ double smem[2 * 32 * 4];
  double* base = a.scratch;
  GridSync* gs = reinterpret_cast<GridSync*>(base);  // abort word
  unsigned* flags = reinterpret_cast<unsigned*>(base + 12);
  double* parts = base + kFlagDoubles;
  double* dinv = parts + kPartDoubles;
  double* r = dinv + kStaticMaxRows;
  double* z = r + kStaticMaxRows;
  double* p = z + kStaticMaxRows;
  double* q = p + kStaticMaxRows;
  FlagSync fs{flags, parts, gs, 0u, kSpinLimitNs, (int)gridDim.x, (int)blockIdx.x};
  const int n = a.n;
  const int stride = gridDim.x * blockDim.x;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  double one[1];

  // diagonal (read back only by the same thread), r = b - A x, z = D^-1 r, p = q = 0
  double red[3] = {0.0, 0.0, 0.0};  // r.z, r.r, b.b
  for (int i = t0; i < n; i += stride) {
    double d = 0.0;
    const int e1 = __ldg(a.row_ptr + i + 1);
    for (int e = __ldg(a.row_ptr + i); e < e1; ++e)
      if (__ldg(a.col + e) == i) d += __ldg(a.val + e);
    dinv[i] = d > 0.0 ? 1.0 / d : 1.0;
  }
  for (int i = t0; i < n; i += stride) {
    const double bi = a.b[i];
    const double ri = bi - csr_row(a, i, a.x);
    const double zi = dinv[i] * ri;
    r[i] = ri;
    z[i] = zi;
    p[i] = 0.0;
    q[i] = 0.0;
    red[0] = fma(ri, zi, red[0]);
    red[1] = fma(ri, ri, red[1]);
    red[2] = fma(bi, bi, red[2]);
  }
  if (!grid_allsum<3>(red, fs, smem)) goto timeout;
  if (red[2] == 0.0) {  // b = 0: the solution is x = 0, whatever the initial guess
    for (int i = t0; i < n; i += stride) a.x[i] = 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.status_out[0] = AVIP_OK;
      a.status_out[1] = 0;
      a.relres_out[0] = 0.0;  // b - A 0 = 0 exactly
    }
    return;
  }
  {
    double rz = red[0], rr = red[1];
    const double bb = red[2];
    const double thresh = a.rtol * a.rtol * bb;
    double beta = 0.0, rr_true = rr;
    int it = 0, restarts = 0, status = AVIP_OK;
    while (true) {
      if (rr <= thresh || it >= a.max_iter) {
        // true residual of x; restart from it when the recursion drifted (bounded restarts)
        double tr[2] = {0.0, 0.0};
        for (int i = t0; i < n; i += stride) {
          // x is complete: the last reduction separates its writes from these reads
          const double ri = a.b[i] - csr_row(a, i, a.x);
          const double zi = dinv[i] * ri;
          r[i] = ri;
          z[i] = zi;
          p[i] = 0.0;
          q[i] = 0.0;
          tr[0] = fma(ri, zi, tr[0]);
          tr[1] = fma(ri, ri, tr[1]);
        }
        if (!grid_allsum<2>(tr, fs, smem)) goto timeout;
        rr_true = tr[1];
        if (rr_true <= thresh) break;
        if (it >= a.max_iter || restarts >= 8) {
          status = AVIP_ENOTCONV;
          break;
        }
        ++restarts;
        rz = tr[0];
        rr = tr[1];
        beta = 0.0;
      }
      double pq[1] = {0.0};
      for (int i = t0; i < n; i += stride) {
        const double w = csr_row(a, i, z);
        const double qn = fma(beta, q[i], w);
        const double pn = fma(beta, p[i], z[i]);
        q[i] = qn;
        p[i] = pn;
        pq[0] = fma(pn, qn, pq[0]);
      }
      const double rz_now = rz;
      if (!grid_allsum<1, 1>(pq, one, fs, smem, [rz_now](const double* t, double* e) { e[0] = rz_now / t[0]; }))
        goto timeout;
      const double alpha = one[0];
      double rn[2] = {0.0, 0.0};
      for (int i = t0; i < n; i += stride) {
        a.x[i] = fma(alpha, p[i], a.x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        const double zi = dinv[i] * ri;
        r[i] = ri;
        z[i] = zi;
        rn[0] = fma(ri, zi, rn[0]);
        rn[1] = fma(ri, ri, rn[1]);
      }
      double bs[1];
      if (!grid_allsum<2, 1>(rn, bs, fs, smem, [rz_now](const double* t, double* e) { e[0] = t[0] / rz_now; }))
        goto timeout;
      beta = bs[0];
      rz = rn[0];
      rr = rn[1];
      ++it;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.status_out[0] = status;
      a.status_out[1] = it;
      a.relres_out[0] = sqrt(rr_true / bb);  // true residual of the x returned
    }
    return;
  }
timeout:
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.status_out[0] = AVIP_ETIMEOUT;
    a.status_out[1] = -1;
  }
}

namespace {
std::mutex g_static_mu;
void* g_static_ptr[128];  // per device: device address of g_pcg_scratch (set-up once)
}  // namespace

}  // namespace avip

using namespace avip;

extern "C" int pcg_csr_static(int32_t n, const int32_t* row_ptr, const int32_t* col, const double* val,
                              const double* b, double* x, double rtol, int32_t max_iter, void* stream,
                              int32_t* iters_out, double* relres_out) {
  if (n < 1 || !row_ptr || !col || !val || !b || !x || !(rtol > 0) || max_iter < 1) return AVIP_EINVAL;
  if (n > kStaticMaxRows) {
    std::fprintf(stderr, "pcg_csr_static: %d rows exceed the compiled-in maximum of %d\n", n, kStaticMaxRows);
    return AVIP_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
    cudaGetLastError();
    return AVIP_ECUDA;
  }
  void* scratch = nullptr;
  {
    // one-time set-up per device, with that device current: the host-side name of a
    // __device__ array is not a device address, so ask the runtime for the address
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_pcg_scratch);
      if (e != cudaSuccess || !ptr) {
        cudaGetLastError();
        return AVIP_ECUDA;
      }
      g_static_ptr[dev] = ptr;
    }
    scratch = g_static_ptr[dev];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* base = static_cast<double*>(scratch);
  // the barrier flags and the abort word must start at zero; everything else is overwritten
  cudaError_t e = cudaMemsetAsync(base, 0, kFlagDoubles * sizeof(double), st);
  int sms = 0, occ = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pcg_csr_static_kernel, kStaticTPB, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return AVIP_ECUDA;
  }
  int blocks = (n + kStaticTPB - 1) / kStaticTPB;
  blocks = std::min(blocks, std::min(occ * sms, kStaticMaxBlocks));
  if (blocks < 1) blocks = 1;
  // status words live in the flag area (after the barrier counter and the abort word)
  int32_t* status_dev = reinterpret_cast<int32_t*>(base + 16);
  double* relres_dev = base + 20;
  StaticPcgArgs args{n, row_ptr, col, val, b, x, base, rtol, max_iter, status_dev, relres_dev};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kStaticTPB);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, pcg_csr_static_kernel, args);
  int32_t hst[2] = {AVIP_ECUDA, 0};
  double hrr = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(hst, status_dev, sizeof(hst), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hrr, relres_dev, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return AVIP_ECUDA;
  }
  if (iters_out) *iters_out = hst[1];
  if (relres_out) *relres_out = hrr;
  return hst[0];
}
