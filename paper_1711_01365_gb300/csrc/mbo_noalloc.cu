// mbo_diffuse_noalloc: the diffusion step for callers that cannot allocate
// device memory.  Its workspace and tables live in one file-scope device
// array (g_noalloc_scratch, MBO_NOALLOC_SCRATCH_BYTES) instead of memory from
// cudaMalloc.  The kernels are the library's own transform passes; only the
// place their scratch lives differs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "../../include/mbo.h"
#include "mbo_dev.cuh"
#include "mbo_internal.h"

namespace mbo {
namespace {

// The scratch array.  Every device that loads this module holds it until the
// process exits.  In host code the name is only a stand-in: kernels receive
// the device address obtained from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[MBO_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 256;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (with that device current).
cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// Fill one axis's tables in place: per-stage twiddles [j-1][n1] and the
// multiplier g and 1 - g at the digit-reversed positions of the forward
// network.  Same definitions as the tables the handle-based calls build on
// the host, computed here with the device math library.
template <typename R>
__global__ void k_noalloc_tables(Plan pl, int N, int ntw, double tau, typename VT<R>::V* tw,
                                 R* g, R* om) {
  using V = typename VT<R>::V;
  const int total = max(ntw, N);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    if (i < ntw) {
      for (int st = 0; st < pl.nst; ++st) {
        const Stage& s = pl.st[st];
        const int cnt = s.m > 1 ? s.m * (s.rad - 1) : 0;
        if (i >= s.tw && i < s.tw + cnt) {
          const int loc = i - s.tw;
          const int j = loc / s.m + 1;
          const int n1 = loc - (j - 1) * s.m;
          const long long e = ((long long)n1 * j) % s.lb;
          double sn, cs;
          sincospi(2.0 * (double)e / (double)s.lb, &sn, &cs);
          tw[i] = V{(R)cs, (R)(-sn)};
        }
      }
    }
    if (i < N) {
      int kk = i, len = N, pos = 0;
      for (int st = 0; st < pl.nst; ++st) {
        const int r = pl.st[st].rad;
        const int Ms = len / r;
        pos += Ms * (kk % r);
        kk /= r;
        len = Ms;
      }
      const double kf = (2 * i <= N) ? (double)i : (double)(i - N);
      const double ex = -4.0 * 3.14159265358979323846 * 3.14159265358979323846 * tau * kf * kf;
      g[pos] = (R)exp(ex);
      om[pos] = (R)(-expm1(ex));
    }
  }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

template <typename R>
mbo_status diffuse_noalloc(const Geom& g, const void* A, void* At, cudaStream_t s) {
  using V = typename VT<R>::V;
  const int lens[3] = {g.nx, g.ny, g.nz};
  Tables<R> t{};
  size_t off = align256((size_t)g.Q * (size_t)g.P * sizeof(V));  // workspace first
  size_t off_tw[3], off_g[3], off_om[3];
  int ntw[3];
  for (int ax = 0; ax < 3; ++ax) {
    t.plan[ax] = make_plan(lens[ax]);
    ntw[ax] = plan_twiddles(t.plan[ax]);
    off_tw[ax] = off;
    off = align256(off + (size_t)std::max(ntw[ax], 1) * sizeof(V));
    off_g[ax] = off;
    off = align256(off + (size_t)lens[ax] * sizeof(R));
    off_om[ax] = off;
    off = align256(off + (size_t)lens[ax] * sizeof(R));
  }
  if (off > (size_t)MBO_NOALLOC_SCRATCH_BYTES) return MBO_ERR_UNSUPPORTED_SIZE;
  const int tx = pick_tx(g.nx, sizeof(R) == 4 ? 8 : 4);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MBO_ERR_CUDA;
  // The row and strided passes keep whole rows / column tiles in shared
  // memory: refuse, before any launch, a problem whose tiles exceed the
  // device's per-block limit (as mbo_create does), so that no kernel
  // attribute call can fail and leave an error behind.
  int maxsm = 0;
  if (cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return MBO_ERR_CUDA;
  if (row_smem_bytes(g, sizeof(R), false) > (size_t)maxsm ||
      axis_smem_bytes(std::max(g.ny, g.nz), tx, sizeof(R)) > (size_t)maxsm)
    return MBO_ERR_UNSUPPORTED_SIZE;
  // Both fields must live on the current device: the kernels and the scratch
  // array used are those of the current device.
  const void* fields[2] = {A, At};
  for (const void* p : fields) {
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
      (void)cudaGetLastError();  // the failed query's error is ours, not the caller's
      return MBO_ERR_INVALID_ARG;
    }
    if (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) return MBO_ERR_INVALID_ARG;
    if (pa.device != dev) return MBO_ERR_INVALID_ARG;
  }
  void* base = nullptr;
  if (scratch_address(dev, &base) != cudaSuccess) return MBO_ERR_CUDA;
  char* b = static_cast<char*>(base);
  for (int ax = 0; ax < 3; ++ax) {
    t.tw[ax] = b + off_tw[ax];
    t.g[ax] = reinterpret_cast<const R*>(b + off_g[ax]);
    t.om[ax] = reinterpret_cast<const R*>(b + off_om[ax]);
    const int n = std::max(ntw[ax], lens[ax]);
    k_noalloc_tables<R><<<(n + 255) / 256, 256, 0, s>>>(
        t.plan[ax], lens[ax], ntw[ax], g.tau, reinterpret_cast<V*>(b + off_tw[ax]),
        reinterpret_cast<R*>(b + off_g[ax]), reinterpret_cast<R*>(b + off_om[ax]));
    if (cudaGetLastError() != cudaSuccess) return MBO_ERR_CUDA;
  }
  t.inv_p = (R)(1.0 / (double)g.P);
  void* W = base;
  const int row_threads = g.nx >= 1024 ? 256 : (g.nx >= 256 ? 128 : (g.nx >= 64 ? 64 : 32));
  const int axis_threads = 256;
  StatsPtrs none{};
  none.respect_stop = 0;
  none.do_stats = 0;
  none.tol = -1.0;
  cudaError_t e = launch_row<R>(ROW_FWD, g, t, static_cast<const R*>(A), nullptr, W, none, 0.0,
                                row_threads, s);
  if (e == cudaSuccess) {
    if (g.ndim == 2) {
      e = launch_axis<R>(AXIS_FGI, 1, g, t, W, none, tx, axis_threads, s);
    } else {
      e = launch_axis<R>(AXIS_FWD, 1, g, t, W, none, tx, axis_threads, s);
      if (e == cudaSuccess) e = launch_axis<R>(AXIS_FGI, 2, g, t, W, none, tx, axis_threads, s);
      if (e == cudaSuccess) e = launch_axis<R>(AXIS_INV, 1, g, t, W, none, tx, axis_threads, s);
    }
  }
  if (e == cudaSuccess)
    e = launch_row<R>(ROW_INV_OUT, g, t, nullptr, static_cast<R*>(At), W, none, 0.0, row_threads, s);
  return e == cudaSuccess ? MBO_OK : MBO_ERR_CUDA;
}

}  // namespace
}  // namespace mbo

using namespace mbo;

extern "C" mbo_status mbo_diffuse_noalloc(int ndim, const int64_t* dims, int n, double tau,
                                          mbo_dtype dtype, const void* A, void* A_tilde,
                                          void* stream) {
  if ((ndim != 2 && ndim != 3) || !dims || n < 1 || n > 4 || !(tau > 0) || !std::isfinite(tau) ||
      (dtype != MBO_F32 && dtype != MBO_F64))
    return MBO_ERR_INVALID_ARG;
  if (!A || !A_tilde || reinterpret_cast<uintptr_t>(A) % 16 || reinterpret_cast<uintptr_t>(A_tilde) % 16)
    return MBO_ERR_INVALID_ARG;
  for (int i = 0; i < ndim; ++i) {
    int a, b;
    if (dims[i] < 2 || dims[i] > 2048 || !factor23(dims[i], a, b)) return MBO_ERR_UNSUPPORTED_SIZE;
  }
  Geom g{};
  g.ndim = ndim;
  g.nx = (int)dims[ndim - 1];
  g.ny = (int)dims[ndim - 2];
  g.nz = ndim == 3 ? (int)dims[0] : 1;
  g.P = (long long)g.nx * g.ny * g.nz;
  g.n = n;
  g.C = n * n;
  g.Q = (g.C + 1) / 2;
  g.tau = tau;
  g.xh = g.nx;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dtype == MBO_F32) return diffuse_noalloc<float>(g, A, A_tilde, s);
  return diffuse_noalloc<double>(g, A, A_tilde, s);
}
