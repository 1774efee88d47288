// Host side of the C ABI declared in include/mbo.h: validation, radix plans,
// twiddle and heat-multiplier tables, workspace ownership, the launch
// sequences of the diffusion / projection / step / energy calls, and the run
// loop (CUDA-graph replay of one step, host polling of the device step
// records every few steps).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/mbo.h"
#include "mbo_dev.cuh"
#include "mbo_internal.h"
#include "mbo_tma.cuh"

namespace mbo {

size_t row_smem_bytes(const Geom& g, size_t elem_bytes, bool fallback) {
  size_t b = (size_t)g.Q * (size_t)row_pad(g.nx) * 2 * elem_bytes;
  if (fallback) b += (size_t)kFallbackCap * ((size_t)g.C * sizeof(float) + sizeof(int));
  return (b + 15) & ~(size_t)15;
}
size_t axis_smem_bytes(int len, int tx, size_t elem_bytes) {
  return (size_t)row_pad(len) * tx * 2 * elem_bytes;
}

bool factor23(int64_t N, int& a, int& b) {
  a = b = 0;
  while (N % 2 == 0) { N /= 2; ++a; }
  while (N % 3 == 0) { N /= 3; ++b; }
  return N == 1;
}

FastDiv make_div(unsigned d) {
  FastDiv f{};
  if ((d & (d - 1)) == 0) {
    f.shift = 0;
    while ((1u << f.shift) < d) ++f.shift;
    f.mul = 0;
  } else {
    f.shift = -1;
    f.mul = (unsigned)((((unsigned long long)1 << 32) + d - 1) / d);
  }
  return f;
}

// Radix plan: the power of two in ceil(a/4) stages of 16 / 8 / 4 / 2 (bits
// spread evenly, larger radices first), then one radix-3 stage per factor 3.
// Stage twiddle offsets are assigned in stage order.
Plan make_plan(int N) {
  Plan p{};
  p.len = N;
  int a, b;
  factor23(N, a, b);
  int rad[kMaxStages];
  int ns = 0;
  if (a > 0) {
    const int n2 = (a + 3) / 4;
    for (int i = 0; i < n2; ++i) rad[ns++] = 1 << (a / n2 + (i < a % n2 ? 1 : 0));
  }
  for (int i = 0; i < b; ++i) rad[ns++] = 3;
  p.nst = ns;
  int lb = N, tw = 0;
  for (int i = 0; i < ns; ++i) {
    Stage& s = p.st[i];
    s.rad = rad[i];
    s.lb = lb;
    s.m = lb / rad[i];
    s.dm = make_div((unsigned)s.m);
    s.dnr = make_div((unsigned)(N / rad[i]));
    s.tw = tw;
    if (s.m > 1) tw += s.m * (s.rad - 1);
    // affine padded addressing: m a multiple of 8 (p/8 advances by m/8 per j), or
    // the whole butterfly inside one 8-aligned block (lb divides 8)
    s.pstride = (s.m % 8 == 0) ? s.m + s.m / 8 : ((s.lb <= 8 && 8 % s.lb == 0) ? s.m : 0);
    lb /= rad[i];
  }
  return p;
}

Plan axis_plan(const Geom& g, int axis, bool f32) {
  const int N = axis == 0 ? g.nx : axis == 1 ? g.ny : g.nz;
  if (f32 && warp_plan_length(N) && (axis == 0 || warp_tile(N, g.nx, 8) != 0) &&
      (axis == 0 || axis < g.ndim)) {
    Plan p{};
    p.len = N;
    p.rad0 = warp_plan_radix(N);
    p.lq = N / p.rad0 == 1024 ? 32 : 16;
    return p;
  }
  return make_plan(N);
}

int plan_twiddles(const Plan& p) {
  if (p.lq) return p.len;
  int n = 0;
  for (int i = 0; i < p.nst; ++i)
    if (p.st[i].m > 1) n += p.st[i].m * (p.st[i].rad - 1);
  return n;
}

// pos[k]: digit-reversed position where the forward network leaves frequency k.
void digit_positions(const Plan& p, int N, std::vector<int>& pos) {
  pos.assign(N, 0);
  if (p.lq) {  // warp-cooperative plans leave the spectrum in natural order
    for (int k = 0; k < N; ++k) pos[k] = k;
    return;
  }
  for (int k = 0; k < N; ++k) {
    int kk = k, len = N, off = 0;
    for (int st = 0; st < p.nst; ++st) {
      const int r = p.st[st].rad;
      const int M = len / r;
      off += M * (kk % r);
      kk /= r;
      len = M;
    }
    pos[k] = off;
  }
}

// Blocks along x per axis tile: largest power of two dividing nx, capped.
int pick_tx(int nx, int cap) {
  int t = 1;
  while (t < cap && nx % (2 * t) == 0) t *= 2;
  return t;
}

}  // namespace mbo

using namespace mbo;

struct mbo_ctx {
  int dev = 0;
  Geom g{};
  int64_t dims_user[3] = {0, 0, 0};
  mbo_dtype dtype = MBO_F32;
  mbo_config cfg{};
  size_t elem = 4;
  // device memory
  void* W = nullptr;
  void* tabs = nullptr;  // twiddles, multipliers (one allocation)
  size_t tabs_bytes = 0;
  double* part = nullptr;     // per-block partials, then per-group totals
  double* epart = nullptr;    // per-block energy partials of the fused step's multiplier pass
  unsigned int* cnt = nullptr;  // per-group arrival counters + the group counter
  size_t ngroups = 0;
  RunState* st = nullptr;
  Hist hist{};
  void* hist_mem = nullptr;
  void* field = nullptr;  // staging field for host-pointer runs
  // volume-preserving step buffers (allocated on first use)
  void* vp_at = nullptr;                 // the diffused field
  unsigned long long* vp_keys = nullptr; // one selection key per point
  SelectState* vp_ss = nullptr;
  // host mirrors
  RunState* h_st = nullptr;  // pinned
  void* h_hist = nullptr;    // pinned ring copy
  // launch configuration
  Tables<float> tf{};
  Tables<double> td{};
  int row_threads = 256, axis_threads = 256, tx = 8;
  int axis_stages = 1;  // tile buffers per block of the FP32 warp-plan strided passes
  bool pdl = false;     // programmatic dependent launch of the FP32 warp-plan passes
  bool xpers = false;   // FP32 warp-plan x pass as one wave of blocks over the row groups
  // TMA descriptors of W for the FP32 warp-plan strided passes (index = axis)
  CUtensorMap wmap[3];
  bool wmap_ok[3] = {false, false, false};
  size_t bytes_total = 0;
  // workspace validity for MBO_STEP_CONTINUE
  const void* w_valid_for = nullptr;
  // captured step graph
  cudaStream_t cap = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const void* g_ptr = nullptr;
  double g_tol = 0;
  // per-pass device timing (mbo_profile_*)
  bool prof = false;
  std::vector<cudaEvent_t> ev_free;
  struct Pending { int pass; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  double prof_ms[MBO_PROFILE_PASSES] = {0};
  long long prof_n[MBO_PROFILE_PASSES] = {0};
  char err[512] = {0};
};

namespace {

mbo_status fail(mbo_ctx* h, mbo_status s, const char* fmt, ...) {
  if (h) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(h->err, sizeof(h->err), fmt, ap);
    va_end(ap);
  }
  return s;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(h, e_ == cudaErrorMemoryAllocation ? MBO_ERR_OOM : MBO_ERR_CUDA,        \
                  "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);   \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

template <typename R> struct TabBuild {
  std::vector<unsigned char> bytes;
  size_t off_tw[3], off_g[3], off_om[3];
};

template <typename R>
void build_tables(mbo_ctx* h, TabBuild<R>& tb, Tables<R>& t) {
  const int lens[3] = {h->g.nx, h->g.ny, h->g.nz};
  size_t off = 0;
  auto reserve = [&](size_t n) {
    size_t o = (off + 255) & ~(size_t)255;
    off = o + n;
    return o;
  };
  for (int ax = 0; ax < 3; ++ax) {
    const int N = lens[ax];
    t.plan[ax] = axis_plan(h->g, ax, sizeof(R) == 4);
    tb.off_tw[ax] = reserve((size_t)std::max(plan_twiddles(t.plan[ax]), 1) * 2 * sizeof(R));
    tb.off_g[ax] = reserve((size_t)N * sizeof(R));
    tb.off_om[ax] = reserve((size_t)N * sizeof(R));
  }
  tb.bytes.assign(off, 0);
  const double pi = 3.14159265358979323846;
  for (int ax = 0; ax < 3; ++ax) {
    const int N = lens[ax];
    const Plan& pl = t.plan[ax];
    R* tw = reinterpret_cast<R*>(&tb.bytes[tb.off_tw[ax]]);
    if (pl.lq) {
      // N = rad0 * Mw: the length-Mw table [k2][l] = exp(-2 pi i l k2 / Mw), then
      // the pre-stage twiddles exp(-2 pi i r k' / N) at Mw + (r - 1) Mw + k'
      const int Mw = N / pl.rad0, E = Mw / pl.lq;
      for (int k2 = 0; k2 < E; ++k2)
        for (int l = 0; l < pl.lq; ++l) {
          const long long e = ((long long)l * k2) % Mw;
          const double ang = 2.0 * pi * (double)e / (double)Mw;
          const size_t i = (size_t)k2 * pl.lq + l;
          tw[2 * i] = (R)std::cos(ang);
          tw[2 * i + 1] = (R)(-std::sin(ang));
        }
      for (int r = 1; r < pl.rad0; ++r)
        for (int k = 0; k < Mw; ++k) {
          const long long e = ((long long)r * k) % N;
          const double ang = 2.0 * pi * (double)e / (double)N;
          const size_t i = (size_t)Mw + (size_t)(r - 1) * Mw + k;
          tw[2 * i] = (R)std::cos(ang);
          tw[2 * i + 1] = (R)(-std::sin(ang));
        }
    }
    for (int st = 0; st < pl.nst; ++st) {
      const Stage& s = pl.st[st];
      if (s.m <= 1) continue;
      for (int n1 = 0; n1 < s.m; ++n1)
        for (int j = 1; j < s.rad; ++j) {
          const long long e = ((long long)n1 * j) % s.lb;
          const double ang = 2.0 * pi * (double)e / (double)s.lb;
          const size_t i = (size_t)s.tw + (size_t)(j - 1) * s.m + n1;
          tw[2 * i] = (R)std::cos(ang);
          tw[2 * i + 1] = (R)(-std::sin(ang));
        }
    }
    std::vector<int> pos;
    digit_positions(pl, N, pos);
    R* gt = reinterpret_cast<R*>(&tb.bytes[tb.off_g[ax]]);
    R* om = reinterpret_cast<R*>(&tb.bytes[tb.off_om[ax]]);
    for (int k = 0; k < N; ++k) {
      const double kf = (2 * k <= N) ? (double)k : (double)(k - N);
      const double e = -4.0 * pi * pi * h->g.tau * kf * kf;
      gt[pos[k]] = (R)std::exp(e);
      om[pos[k]] = (R)(-std::expm1(e));
    }
  }
  t.inv_p = (R)(1.0 / (double)h->g.P);
}

template <typename R> void bind_tables(mbo_ctx* h, const TabBuild<R>& tb, Tables<R>& t) {
  const char* base = static_cast<const char*>(h->tabs);
  for (int ax = 0; ax < 3; ++ax) {
    t.tw[ax] = base + tb.off_tw[ax];
    t.g[ax] = reinterpret_cast<const R*>(base + tb.off_g[ax]);
    t.om[ax] = reinterpret_cast<const R*>(base + tb.off_om[ax]);
  }
}

StatsPtrs stats_ptrs(mbo_ctx* h, bool stats, bool respect_stop, double tol) {
  StatsPtrs sp{};
  sp.st = h->st;
  sp.hist = h->hist;
  sp.rb.part = h->part;
  sp.rb.gpart = h->part + h->ngroups * kReduceGroup;
  sp.rb.gcount = h->cnt;
  sp.rb.done = h->cnt + h->ngroups;
  sp.respect_stop = respect_stop ? 1 : 0;
  sp.do_stats = stats ? 1 : 0;
  sp.tol = tol;
  sp.epart = nullptr;
  return sp;
}

cudaError_t row_launch(mbo_ctx* h, RowMode mode, const void* Ain, void* Aout,
                       const StatsPtrs& sp, cudaStream_t s);
cudaError_t axis_launch(mbo_ctx* h, AxisMode mode, int axis, const StatsPtrs& sp, cudaStream_t s,
                        const void* l2_hint);

cudaEvent_t take_event(mbo_ctx* h) {
  if (!h->ev_free.empty()) {
    cudaEvent_t e = h->ev_free.back();
    h->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Launch f on stream s; when profiling, bracket it with events (pass id).
template <class F> cudaError_t timed(mbo_ctx* h, int pass, cudaStream_t s, F&& f) {
  if (!h->prof) return f();
  cudaEvent_t a = take_event(h), b = take_event(h);
  cudaEventRecord(a, s);
  cudaError_t e = f();
  cudaEventRecord(b, s);
  h->pending.push_back({pass, a, b});
  return e;
}

cudaError_t row_pass(mbo_ctx* h, RowMode mode, const void* Ain, void* Aout, const StatsPtrs& sp,
                     cudaStream_t s) {
  const int pass = mode == ROW_FWD ? MBO_PASS_ROW_FWD
                   : mode == ROW_INV_OUT ? MBO_PASS_ROW_INV : MBO_PASS_ROW_PROJECT;
  return timed(h, pass, s, [&]() { return row_launch(h, mode, Ain, Aout, sp, s); });
}

cudaError_t axis_pass(mbo_ctx* h, AxisMode mode, int axis, const StatsPtrs& sp, cudaStream_t s,
                      const void* l2_hint = nullptr) {
  const int pass = mode == AXIS_FWD ? MBO_PASS_AXIS_FWD
                   : mode == AXIS_INV ? MBO_PASS_AXIS_INV
                   : mode == AXIS_FGI ? MBO_PASS_AXIS_FGI : MBO_PASS_AXIS_ENERGY;
  return timed(h, pass, s, [&]() { return axis_launch(h, mode, axis, sp, s, l2_hint); });
}

cudaError_t row_launch(mbo_ctx* h, RowMode mode, const void* Ain, void* Aout, const StatsPtrs& sp,
                       cudaStream_t s) {
  pdl_flag() = h->pdl;
  wrow_persistent_flag() = h->xpers;
  if (h->dtype == MBO_F32)
    return launch_row<float>(mode, h->g, h->tf, static_cast<const float*>(Ain),
                             static_cast<float*>(Aout), h->W, sp, h->cfg.fallback_sigma,
                             h->row_threads, s);
  return launch_row<double>(mode, h->g, h->td, static_cast<const double*>(Ain),
                            static_cast<double*>(Aout), h->W, sp, 0.0, h->row_threads, s);
}

// The field and the workspace together fit in L2 comfortably: the last
// strided pass of a step may then pull the field (which the x pass reads for
// its step statistics) into L2 while it transforms.
constexpr size_t kL2HintBytes = 96u << 20;

cudaError_t axis_launch(mbo_ctx* h, AxisMode mode, int axis, const StatsPtrs& sp, cudaStream_t s,
                        const void* l2_hint) {
  const size_t abytes = (size_t)h->g.C * (size_t)h->g.P * h->elem;
  const size_t wbytes = (size_t)h->g.Q * (size_t)h->g.P * 2 * h->elem;
  if (abytes + wbytes > kL2HintBytes) l2_hint = nullptr;
  pdl_flag() = h->pdl;
  if (h->dtype == MBO_F32)
    return launch_axis<float>(mode, axis, h->g, h->tf, h->W, sp, h->tx, h->axis_threads, s,
                              h->wmap_ok[axis] ? &h->wmap[axis] : nullptr, h->axis_stages,
                              l2_hint, l2_hint ? (long long)abytes : 0);
  return launch_axis<double>(mode, axis, h->g, h->td, h->W, sp, h->tx, h->axis_threads, s);
}

// Transform passes between the forward and the inverse x pass.
// mode AXIS_FGI: diffuse; AXIS_ENERGY: energy only (workspace not restored in 3-D).
// A_next: the field the following x pass reads (L2 hint), or nullptr.
cudaError_t middle_passes(mbo_ctx* h, AxisMode mode, const StatsPtrs& sp, cudaStream_t s,
                          const void* A_next = nullptr) {
  const StatsPtrs none = [&] {
    StatsPtrs n = sp;
    n.do_stats = 0;
    return n;
  }();
  cudaError_t e;
  if (h->g.ndim == 2) return axis_pass(h, mode, 1, sp, s, A_next);
  if ((e = axis_pass(h, AXIS_FWD, 1, none, s)) != cudaSuccess) return e;
  if ((e = axis_pass(h, mode, 2, sp, s)) != cudaSuccess) return e;
  if (mode == AXIS_FGI) return axis_pass(h, AXIS_INV, 1, none, s, A_next);
  return cudaSuccess;
}

// The steady-state step: middle passes + inverse x / projection / forward x.
cudaError_t step_passes(mbo_ctx* h, void* A, bool respect_stop, double tol, cudaStream_t s) {
  StatsPtrs sp = stats_ptrs(h, true, respect_stop, tol);
  sp.epart = h->epart;  // the energy is reduced by the x pass's finaliser
  cudaError_t e = middle_passes(h, AXIS_FGI, sp, s);
  if (e != cudaSuccess) return e;
  return row_pass(h, ROW_INV_PROJECT_FWD, nullptr, A, sp, s);
}

mbo_status check_field_ptr(mbo_ctx* h, const void* p, const char* what) {
  if (!p) return fail(h, MBO_ERR_INVALID_ARG, "%s is NULL", what);
  if (reinterpret_cast<uintptr_t>(p) % 16 != 0)
    return fail(h, MBO_ERR_INVALID_ARG, "%s is not 16-byte aligned", what);
  return MBO_OK;
}

void invalidate_graph(mbo_ctx* h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  h->gexec = nullptr;
  h->g_ptr = nullptr;
}

// ---------------------------------------------------------------------------
// Launch-shape autotuner.  Candidates: the strided passes' tile width (and, for
// FP32 warp-plan axes, one or two tile buffers per block; for the in-place
// network, threads per block), then the row pass's threads per block where
// the x axis takes the network.  Each candidate runs a fresh step and one
// more on a scratch field, then three timed steps; the fastest is kept and
// cached per (dims, n, dtype) for the process.
// ---------------------------------------------------------------------------
struct LaunchShape {
  int tx, stages, axis_threads, row_threads;
  bool pdl, xpers;
};
using TuneKey = std::tuple<int, int, int, int, int, int>;
std::mutex g_tune_mu;
std::map<TuneKey, LaunchShape> g_tune_cache;

template <typename R> __global__ void k_tune_fill(R* A, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = (unsigned long long)i * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    A[i] = (R)((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);  // uniform in [-1, 1)
  }
}

bool shape_fits(mbo_ctx* h, const LaunchShape& c, int maxsm) {
  const Geom& g = h->g;
  if (c.tx < 1 || g.nx % c.tx) return false;
  for (int ax = 1; ax < g.ndim; ++ax) {
    const int L = ax == 1 ? g.ny : g.nz;
    if (h->dtype == MBO_F32 && h->tf.plan[ax].lq) {
      const int wt = warp_tile(L, g.nx, c.tx);
      if (!wt || wcol_smem_bytes(L, wt, c.stages) > (size_t)maxsm) return false;
    } else if (axis_smem_bytes(L, c.tx, h->elem) > (size_t)maxsm) {
      return false;
    }
  }
  return true;
}

cudaError_t apply_shape(mbo_ctx* h, const LaunchShape& c) {
  h->tx = c.tx;
  h->axis_stages = c.stages;
  h->axis_threads = c.axis_threads;
  h->row_threads = c.row_threads;
  h->pdl = c.pdl;
  h->xpers = c.xpers;
  invalidate_graph(h);
  const Geom& g = h->g;
  cudaError_t e = h->dtype == MBO_F32 ? prepare_kernels<float>(g, h->tf, h->tx, h->axis_stages)
                                      : prepare_kernels<double>(g, h->td, h->tx, 1);
  if (e != cudaSuccess) return e;
  if (h->dtype == MBO_F32) {
    for (int ax = 1; ax < g.ndim; ++ax) {
      if (!h->tf.plan[ax].lq) continue;
      const int L = ax == 1 ? g.ny : g.nz;
      if (!wcol_tensor_map(&h->wmap[ax], h->W, g, ax, warp_tile(L, g.nx, h->tx)))
        return cudaErrorInvalidValue;
      h->wmap_ok[ax] = true;
    }
  }
  return cudaSuccess;
}

// ms per step of the handle's current launch shapes on field A
cudaError_t time_shape(mbo_ctx* h, void* A, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1,
                       float& ms) {
  cudaError_t e = row_pass(h, ROW_FWD, A, nullptr, stats_ptrs(h, true, false, -1.0), s);
  if (e == cudaSuccess) e = step_passes(h, A, false, -1.0, s);
  if (e == cudaSuccess) e = step_passes(h, A, false, -1.0, s);
  if (e != cudaSuccess) return e;
  cudaEventRecord(e0, s);
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = step_passes(h, A, false, -1.0, s);
  cudaEventRecord(e1, s);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  ms = t / 3.f;
  return cudaGetLastError();
}

mbo_status autotune(mbo_ctx* h, int maxsm) {
  const Geom& g = h->g;
  const mbo_config& c = h->cfg;
  const TuneKey key{g.ndim, g.nz, g.ny, g.nx, g.n, (int)h->dtype};
  LaunchShape best{h->tx, h->axis_stages, h->axis_threads, h->row_threads, h->pdl, h->xpers};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      LaunchShape sh = it->second;
      if (c.axis_tx) sh.tx = h->tx;
      if (c.axis_stages) sh.stages = h->axis_stages;
      if (c.axis_threads) sh.axis_threads = h->axis_threads;
      if (c.row_threads) sh.row_threads = h->row_threads;
      if (c.pdl) sh.pdl = h->pdl;
      return apply_shape(h, sh) == cudaSuccess ? MBO_OK : MBO_ERR_CUDA;
    }
  }
  const bool f32 = h->dtype == MBO_F32;
  bool warp_axis = false, net_axis = false;
  for (int ax = 1; ax < g.ndim; ++ax) {
    if (f32 && h->tf.plan[ax].lq) warp_axis = true;
    else net_axis = true;
  }
  const bool net_row = !(f32 && h->tf.plan[0].lq);
  std::vector<int> txs, stages, athreads, rthreads;
  for (int t : {h->tx, 2 * h->tx, h->tx / 2, 4})
    if (t >= 1 && t <= 16 && std::find(txs.begin(), txs.end(), t) == txs.end()) txs.push_back(t);
  if (c.axis_tx) txs = {h->tx};
  stages = (warp_axis && !c.axis_stages) ? std::vector<int>{1, 2, 3} : std::vector<int>{h->axis_stages};
  athreads = (net_axis && !c.axis_threads) ? std::vector<int>{128, 256, 384}
                                           : std::vector<int>{h->axis_threads};
  rthreads = (net_row && !c.row_threads) ? std::vector<int>{64, 128, 192, 256, 384}
                                         : std::vector<int>{h->row_threads};
  const size_t fbytes = (size_t)g.C * (size_t)g.P * h->elem;
  void* A = nullptr;
  if (cudaMalloc(&A, fbytes) != cudaSuccess) return MBO_ERR_OOM;
  cudaStream_t s = h->cap;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaError_t e = cudaSuccess;
  const long long nv = (long long)g.C * g.P;
  if (f32) {
    k_tune_fill<float><<<256, 256, 0, s>>>(static_cast<float*>(A), nv);
    e = launch_project<float>(g, static_cast<float*>(A), static_cast<float*>(A), nullptr, 0.0, s);
  } else {
    k_tune_fill<double><<<256, 256, 0, s>>>(static_cast<double*>(A), nv);
    e = launch_project<double>(g, static_cast<double*>(A), static_cast<double*>(A), nullptr, 0.0, s);
  }
  float best_ms = 1e30f;
  auto consider = [&](const LaunchShape& sh) {
    if (e != cudaSuccess || !shape_fits(h, sh, maxsm)) return;
    if ((e = apply_shape(h, sh)) != cudaSuccess) return;
    float ms = 0.f;
    if ((e = time_shape(h, A, s, e0, e1, ms)) != cudaSuccess) return;
    if (ms < best_ms) {
      best_ms = ms;
      best = sh;
    }
  };
  // strided passes first (row threads at their default), then the row pass
  const LaunchShape start = best;
  for (int t : txs)
    for (int st : stages)
      for (int at : athreads) consider(LaunchShape{t, st, at, start.row_threads, start.pdl, start.xpers});
  const LaunchShape mid = best;
  for (int rt : rthreads)
    if (rt != mid.row_threads)
      consider(LaunchShape{mid.tx, mid.stages, mid.axis_threads, rt, mid.pdl, mid.xpers});
  if (f32 && !net_row) {
    if (!c.pdl) {  // programmatic dependent launch on or off
      LaunchShape alt = best;
      alt.pdl = !alt.pdl;
      consider(alt);
    }
    LaunchShape alt = best;  // the x pass as one wave of blocks, or one block per row group
    alt.xpers = !alt.xpers;
    consider(alt);
  }
  if (e == cudaSuccess) e = apply_shape(h, best);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(A);
  if (e == cudaSuccess)
    e = cudaMemset(h->st, 0, sizeof(RunState)) == cudaSuccess &&
                cudaMemset(h->hist_mem, 0, (size_t)kRing * 5 * sizeof(double)) == cudaSuccess
            ? cudaSuccess
            : cudaErrorUnknown;
  h->w_valid_for = nullptr;
  if (e != cudaSuccess) {
    (void)cudaGetLastError();  // no stale error for the caller's next launch
    return MBO_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = best;
  return MBO_OK;
}

}  // namespace

extern "C" {

const char* mbo_status_string(mbo_status s) {
  switch (s) {
    case MBO_OK: return "ok";
    case MBO_ERR_INVALID_ARG: return "invalid argument";
    case MBO_ERR_UNSUPPORTED_SIZE: return "unsupported size (axis length must be 2^a 3^b in [2, 2048])";
    case MBO_ERR_OOM: return "device out of memory";
    case MBO_ERR_CUDA: return "CUDA error";
    case MBO_ERR_NUMERIC: return "non-finite values in the field";
    case MBO_ERR_DEVICE_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

const char* mbo_last_error(mbo_handle h) { return h ? h->err : ""; }

void mbo_default_config(mbo_config* cfg) {
  if (!cfg) return;
  cfg->fallback_sigma = 0.0;
  cfg->check_interval = 16;
  cfg->use_graph = 1;
  cfg->row_threads = 0;
  cfg->axis_threads = 0;
  cfg->axis_tx = 0;
  cfg->axis_stages = 0;
  cfg->autotune = 0;
  cfg->pdl = 0;
}

int64_t mbo_workspace_bytes(mbo_handle h) { return h ? (int64_t)h->bytes_total : 0; }

mbo_status mbo_destroy(mbo_handle h) {
  if (!h) return MBO_ERR_INVALID_ARG;
  DeviceGuard dg(h->dev);
  cudaDeviceSynchronize();
  invalidate_graph(h);
  for (auto& p : h->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : h->ev_free) cudaEventDestroy(e);
  if (h->cap) cudaStreamDestroy(h->cap);
  cudaFree(h->W);
  cudaFree(h->tabs);
  cudaFree(h->part);
  cudaFree(h->cnt);
  cudaFree(h->st);
  cudaFree(h->epart);
  cudaFree(h->hist_mem);
  cudaFree(h->field);
  cudaFree(h->vp_at);
  cudaFree(h->vp_keys);
  cudaFree(h->vp_ss);
  cudaFreeHost(h->h_st);
  cudaFreeHost(h->h_hist);
  delete h;
  return MBO_OK;
}

mbo_status mbo_create(mbo_handle* out, int ndim, const int64_t* dims, int n, double tau,
                      mbo_dtype dtype, const mbo_config* cfg) {
  if (!out) return MBO_ERR_INVALID_ARG;
  *out = nullptr;
  if ((ndim != 2 && ndim != 3) || !dims || n < 1 || n > 4 || !(tau > 0) || !std::isfinite(tau) ||
      (dtype != MBO_F32 && dtype != MBO_F64))
    return MBO_ERR_INVALID_ARG;
  for (int i = 0; i < ndim; ++i) {
    int a, b;
    if (dims[i] < 2 || dims[i] > 2048 || !factor23(dims[i], a, b)) return MBO_ERR_UNSUPPORTED_SIZE;
  }
  mbo_ctx* h = new mbo_ctx();
  if (cfg) h->cfg = *cfg;
  else mbo_default_config(&h->cfg);
  if (h->cfg.check_interval < 1) h->cfg.check_interval = 1;
  if (h->cfg.check_interval > kRing / 2) h->cfg.check_interval = kRing / 2;
  h->dtype = dtype;
  h->elem = dtype == MBO_F32 ? 4 : 8;
  Geom& g = h->g;
  g.ndim = ndim;
  g.nx = (int)dims[ndim - 1];
  g.ny = (int)dims[ndim - 2];
  g.nz = ndim == 3 ? (int)dims[0] : 1;
  for (int i = 0; i < ndim; ++i) h->dims_user[i] = dims[i];
  g.P = (long long)g.nx * g.ny * g.nz;
  g.n = n;
  g.C = n * n;
  g.Q = (g.C + 1) / 2;
  g.tau = tau;
  g.xh = g.nx;
  if ((g.C & 1) && dtype == MBO_F32 && axis_plan(g, 0, true).lq)
    g.xh = std::min(g.nx, ((g.nx / 2 + 1 + 15) / 16) * 16);
  cudaGetDevice(&h->dev);
  // launch shapes
  h->tx = pick_tx(g.nx, dtype == MBO_F32 ? 8 : 4);
  // measured on GB300 (1024^2, n = 3): 192 threads best for FP32 rows, 128 for FP64
  h->row_threads = g.nx >= 2048 ? 256
                   : g.nx >= 1024 ? (dtype == MBO_F32 ? 192 : 128)
                   : (g.nx >= 256 ? 128 : (g.nx >= 64 ? 64 : 32));
  h->axis_threads = 256;
  if (dtype == MBO_F32) {
    // FP32 warp-plan strided passes, measured on GB300: 16-column tiles (one
    // 128-byte line per tile row) where an axis of 512 is strided (512^3:
    // 13.7 -> 10.4 ms per step; 512^2, n = 2: 32 -> 26 us), and split staging
    // with them and in 3-D (512^3: 10.4 -> 9.9 ms; 256^3: 1.36 -> 1.28 ms)
    bool l512 = false;
    for (int ax = 1; ax < ndim; ++ax)
      l512 = l512 || ((ax == 1 ? g.ny : g.nz) == 512 && axis_plan(g, ax, true).lq);
    if (l512 && g.nx % 16 == 0) h->tx = 16;
    if (h->tx == 16 || ndim == 3) h->axis_stages = 3;
  }
  const mbo_config& c = h->cfg;
  if (c.row_threads) {
    if (c.row_threads < 32 || c.row_threads > kMaxThreads || c.row_threads % 32) {
      delete h;
      return MBO_ERR_INVALID_ARG;
    }
    h->row_threads = c.row_threads;
  }
  if (c.axis_tx) {
    if (c.axis_tx < 1 || c.axis_tx > 16 || (c.axis_tx & (c.axis_tx - 1)) || g.nx % c.axis_tx) {
      delete h;
      return MBO_ERR_INVALID_ARG;
    }
    h->tx = c.axis_tx;
  }
  if (c.axis_stages) {
    if (c.axis_stages < 1 || c.axis_stages > 3) {
      delete h;
      return MBO_ERR_INVALID_ARG;
    }
    h->axis_stages = c.axis_stages;
  }
  if (c.axis_threads) {
    if (c.axis_threads < 64 || c.axis_threads > kMaxThreads || c.axis_threads % 32) {
      delete h;
      return MBO_ERR_INVALID_ARG;
    }
    h->axis_threads = c.axis_threads;
  }
  if (c.pdl < 0 || c.pdl > 2) {
    delete h;
    return MBO_ERR_INVALID_ARG;
  }
  // programmatic dependent launch: measured to help where the projecting x
  // pass runs in at most two waves of blocks, and to cost a little beyond
  if (dtype == MBO_F32 && axis_plan(g, 0, true).lq) {
    const double waves = wrow_waves(g);
    h->pdl = c.pdl == 1 || (c.pdl == 0 && waves <= 2.0);
    // beyond two waves a grid of one wave walking the row groups with a stride
    // of the grid was measured faster (768^2 n=3: 84.6 -> 78.7 us per step,
    // 2048^2: 367.8 -> 359.5); at 1024^2 dependent launch gains more
    h->xpers = waves > 2.0;
  }
  size_t rs = row_smem_bytes(g, h->elem, true);
  size_t as = 0;       // shared memory of the strided passes, each by its own plan
  int min_tx = h->tx;  // narrowest column tile of any strided pass
  if (dtype == MBO_F32 && axis_plan(g, 0, true).lq) rs = std::max(rs, wrow_smem_bytes(g, g.nx, true));
  for (int ax = 1; ax < ndim; ++ax) {
    const int L = ax == 1 ? g.ny : g.nz;
    if (dtype == MBO_F32 && axis_plan(g, ax, true).lq) {
      const int wt = warp_tile(L, g.nx, h->tx);
      as = std::max(as, wcol_smem_bytes(L, wt, h->axis_stages));
      min_tx = std::min(min_tx, wt);
    } else {
      as = std::max(as, axis_smem_bytes(L, h->tx, h->elem));
    }
  }
  int maxsm = 0;
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->dev);
  if (rs > (size_t)maxsm || as > (size_t)maxsm) {
    delete h;
    return MBO_ERR_UNSUPPORTED_SIZE;
  }
  mbo_status rc = MBO_OK;
  auto alloc = [&](void** p, size_t bytes) -> bool {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      rc = MBO_ERR_OOM;
      return false;
    }
    h->bytes_total += bytes;
    return true;
  };
  const size_t wbytes = (size_t)g.Q * (size_t)g.P * 2 * h->elem;
  const int rows = g.nz * g.ny;
  // the autotuner may narrow the column tiles (down to half, or 4 columns)
  if (c.autotune && !c.axis_tx) min_tx = std::max(1, std::min(min_tx, std::min(h->tx / 2, 4)));
  const int tiles = g.Q * std::max(g.nz, g.ny) * (g.nx / min_tx);
  const size_t nparts = (size_t)std::max(rows, tiles);
  h->ngroups = (nparts + kReduceGroup - 1) / kReduceGroup;
  if (!alloc(&h->W, wbytes) ||
      !alloc((void**)&h->part, (h->ngroups * kReduceGroup + h->ngroups) * sizeof(double)) ||
      !alloc((void**)&h->epart, h->ngroups * kReduceGroup * sizeof(double)) ||
      !alloc((void**)&h->cnt, (h->ngroups + 1) * sizeof(unsigned int)) ||
      !alloc((void**)&h->st, sizeof(RunState)) ||
      !alloc(&h->hist_mem, (size_t)kRing * 5 * sizeof(double))) {
    mbo_destroy(h);
    return rc;
  }
  char* hm = static_cast<char*>(h->hist_mem);
  h->hist.energy = reinterpret_cast<double*>(hm);
  h->hist.maxdelta = reinterpret_cast<double*>(hm + kRing * 8);
  h->hist.flips = reinterpret_cast<long long*>(hm + 2 * kRing * 8);
  h->hist.fallback = reinterpret_cast<long long*>(hm + 3 * kRing * 8);
  h->hist.nonfinite = reinterpret_cast<long long*>(hm + 4 * kRing * 8);
  if (dtype == MBO_F32) {
    TabBuild<float> tb;
    build_tables(h, tb, h->tf);
    if (!alloc(&h->tabs, tb.bytes.size())) { mbo_destroy(h); return rc; }
    cudaMemcpy(h->tabs, tb.bytes.data(), tb.bytes.size(), cudaMemcpyHostToDevice);
    bind_tables(h, tb, h->tf);
  } else {
    TabBuild<double> tb;
    build_tables(h, tb, h->td);
    if (!alloc(&h->tabs, tb.bytes.size())) { mbo_destroy(h); return rc; }
    cudaMemcpy(h->tabs, tb.bytes.data(), tb.bytes.size(), cudaMemcpyHostToDevice);
    bind_tables(h, tb, h->td);
  }
  const cudaError_t pe = dtype == MBO_F32 ? prepare_kernels<float>(g, h->tf, h->tx, h->axis_stages)
                                          : prepare_kernels<double>(g, h->td, h->tx, 1);
  if (pe != cudaSuccess) {
    (void)cudaGetLastError();  // the failed attribute call must not surface at a later launch
    mbo_destroy(h);
    return MBO_ERR_CUDA;
  }
  if (dtype == MBO_F32) {
    for (int ax = 1; ax < ndim; ++ax) {
      if (!h->tf.plan[ax].lq) continue;
      const int L = ax == 1 ? g.ny : g.nz;
      if (!wcol_tensor_map(&h->wmap[ax], h->W, g, ax, warp_tile(L, g.nx, h->tx))) {
        mbo_destroy(h);
        return MBO_ERR_CUDA;
      }
      h->wmap_ok[ax] = true;
    }
  }
  if (cudaMemset(h->st, 0, sizeof(RunState)) != cudaSuccess ||
      cudaMemset(h->cnt, 0, (h->ngroups + 1) * sizeof(unsigned int)) != cudaSuccess ||
      cudaMemset(h->hist_mem, 0, (size_t)kRing * 5 * sizeof(double)) != cudaSuccess ||
      cudaMallocHost((void**)&h->h_st, sizeof(RunState)) != cudaSuccess ||
      cudaMallocHost(&h->h_hist, (size_t)kRing * 5 * sizeof(double)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) {
    mbo_destroy(h);
    return MBO_ERR_CUDA;
  }
  if (c.autotune) {
    const mbo_status ts = autotune(h, maxsm);
    if (ts != MBO_OK) {
      mbo_destroy(h);
      return ts;
    }
  }
  *out = h;
  return MBO_OK;
}

mbo_status mbo_launch_config(mbo_handle h, mbo_config* out) {
  if (!h || !out) return MBO_ERR_INVALID_ARG;
  *out = h->cfg;
  out->row_threads = h->row_threads;
  out->axis_threads = h->axis_threads;
  out->axis_tx = h->tx;
  out->axis_stages = h->axis_stages;
  out->pdl = h->pdl ? 1 : 2;
  return MBO_OK;
}

mbo_status mbo_diffuse(mbo_handle h, const void* A, void* A_tilde, void* stream) {
  if (!h) return MBO_ERR_INVALID_ARG;
  mbo_status rc;
  if ((rc = check_field_ptr(h, A, "A")) != MBO_OK) return rc;
  if ((rc = check_field_ptr(h, A_tilde, "A_tilde")) != MBO_OK) return rc;
  DeviceGuard dg(h->dev);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const StatsPtrs none = stats_ptrs(h, false, false, -1.0);
  h->w_valid_for = nullptr;
  CK(row_pass(h, ROW_FWD, A, nullptr, none, s));
  CK(middle_passes(h, AXIS_FGI, none, s));
  CK(row_pass(h, ROW_INV_OUT, nullptr, A_tilde, none, s));
  return MBO_OK;
}

mbo_status mbo_project(mbo_handle h, const void* A_tilde, void* B, int8_t* det_sign,
                       void* stream) {
  if (!h) return MBO_ERR_INVALID_ARG;
  mbo_status rc;
  if ((rc = check_field_ptr(h, A_tilde, "A_tilde")) != MBO_OK) return rc;
  if ((rc = check_field_ptr(h, B, "B")) != MBO_OK) return rc;
  DeviceGuard dg(h->dev);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (B == h->w_valid_for) h->w_valid_for = nullptr;
  CK(timed(h, MBO_PASS_PROJECT, s, [&]() {
    if (h->dtype == MBO_F32)
      return launch_project<float>(h->g, static_cast<const float*>(A_tilde),
                                   static_cast<float*>(B), det_sign, h->cfg.fallback_sigma, s);
    return launch_project<double>(h->g, static_cast<const double*>(A_tilde),
                                  static_cast<double*>(B), det_sign, 0.0, s);
  }));
  return MBO_OK;
}

static mbo_status read_record(mbo_handle h, long long slot, mbo_stats* out) {
  double v[5];
  CK(cudaMemcpy(&v[0], h->hist.energy + slot, 8, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&v[1], h->hist.maxdelta + slot, 8, cudaMemcpyDeviceToHost));
  long long f[3];
  CK(cudaMemcpy(&f[0], h->hist.flips + slot, 8, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&f[1], h->hist.fallback + slot, 8, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&f[2], h->hist.nonfinite + slot, 8, cudaMemcpyDeviceToHost));
  out->energy = v[0];
  out->max_delta = v[1];
  out->det_flips = f[0];
  out->fallback_points = f[1];
  out->nonfinite = f[2];
  return MBO_OK;
}

// Self-test of the bounded-wait error path: one block waits on an mbarrier
// phase that nothing completes (no arrival, no copy), with the same bounded
// wait the TMA passes use, and records the timeout in the run state's error
// word as they do.
__global__ void k_wait_timeout_selftest(RunState* st, long long limit) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  const bool ok = __syncthreads_and(mbar_wait_bounded(&bar, 0, limit)) != 0;
  if (!ok && threadIdx.x == 0) atomicOr(&st->err, kErrWaitTimeout);
}

// Device error bits of the last synchronised read of the run state: a
// kernel whose bounded wait gave up left them set.  The bits are cleared so
// that later calls start clean.
static mbo_status device_errors(mbo_handle h) {
  const unsigned bits = h->h_st->err;
  if (!bits) return MBO_OK;
  h->h_st->err = 0;
  cudaMemset(&h->st->err, 0, sizeof(unsigned int));
  return fail(h, MBO_ERR_DEVICE_TIMEOUT, "a bounded device wait gave up (error bits 0x%x)", bits);
}

mbo_status mbo_step(mbo_handle h, void* A, int flags, mbo_stats* stats, void* stream) {
  if (!h) return MBO_ERR_INVALID_ARG;
  mbo_status rc;
  if ((rc = check_field_ptr(h, A, "A")) != MBO_OK) return rc;
  DeviceGuard dg(h->dev);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool cont = (flags & MBO_STEP_CONTINUE) && h->w_valid_for == A;
  if (!cont) CK(row_pass(h, ROW_FWD, A, nullptr, stats_ptrs(h, true, false, -1.0), s));
  CK(step_passes(h, A, false, -1.0, s));
  h->w_valid_for = A;
  if (stats) {
    CK(cudaStreamSynchronize(s));
    CK(cudaMemcpy(h->h_st, h->st, sizeof(RunState), cudaMemcpyDeviceToHost));
    if ((rc = device_errors(h)) != MBO_OK) return rc;
    const long long slot = (h->h_st->step - 1) & (kRing - 1);
    if ((rc = read_record(h, slot, stats)) != MBO_OK) return rc;
    if (stats->nonfinite) return fail(h, MBO_ERR_NUMERIC, "%lld non-finite points", (long long)stats->nonfinite);
  }
  return MBO_OK;
}

mbo_status mbo_selftest_wait_timeout(mbo_handle h, int64_t limit_cycles, void* stream) {
  if (!h || limit_cycles < 1 || limit_cycles > kWaitCycles) return MBO_ERR_INVALID_ARG;
  DeviceGuard dg(h->dev);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_wait_timeout_selftest<<<1, 64, 0, s>>>(h->st, (long long)limit_cycles);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  CK(cudaMemcpy(h->h_st, h->st, sizeof(RunState), cudaMemcpyDeviceToHost));
  return device_errors(h);
}

mbo_status mbo_lyapunov(mbo_handle h, const void* A, double* E, void* stream) {
  if (!h || !E) return MBO_ERR_INVALID_ARG;
  mbo_status rc;
  if ((rc = check_field_ptr(h, A, "A")) != MBO_OK) return rc;
  DeviceGuard dg(h->dev);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const StatsPtrs sp = stats_ptrs(h, true, false, -1.0);
  CK(row_pass(h, ROW_FWD, A, nullptr, sp, s));
  CK(middle_passes(h, AXIS_ENERGY, sp, s));
  h->w_valid_for = (h->g.ndim == 2) ? A : nullptr;
  CK(cudaStreamSynchronize(s));
  CK(cudaMemcpy(h->h_st, h->st, sizeof(RunState), cudaMemcpyDeviceToHost));
  if ((rc = device_errors(h)) != MBO_OK) return rc;
  *E = h->h_st->energy_last;
  return MBO_OK;
}

mbo_status mbo_run_until_stationary(mbo_handle h, void* A, int max_steps, double tol,
                                    int* steps_taken, int* stationary, double* energies,
                                    double* max_deltas, int64_t* det_flips, mbo_stats* last,
                                    void* stream) {
  if (!h || max_steps < 0) return MBO_ERR_INVALID_ARG;
  if (!A) return fail(h, MBO_ERR_INVALID_ARG, "A is NULL");
  DeviceGuard dg(h->dev);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t fbytes = (size_t)h->g.C * (size_t)h->g.P * h->elem;
  cudaPointerAttributes pa{};
  CK(cudaPointerGetAttributes(&pa, A));
  const bool host = pa.type == cudaMemoryTypeUnregistered || pa.type == cudaMemoryTypeHost;
  void* dA = A;
  if (host) {
    if (!h->field) {
      CK(cudaMalloc(&h->field, fbytes));
      h->bytes_total += fbytes;
    }
    dA = h->field;
    CK(cudaMemcpyAsync(dA, A, fbytes, cudaMemcpyHostToDevice, s));
  } else {
    mbo_status rc = check_field_ptr(h, A, "A");
    if (rc != MBO_OK) return rc;
  }
  CK(cudaMemsetAsync(h->st, 0, sizeof(RunState), s));
  CK(row_pass(h, ROW_FWD, dA, nullptr, stats_ptrs(h, true, false, -1.0), s));

  const bool use_graph = h->cfg.use_graph != 0 && !h->prof;
  // the first step is launched directly (kernel attributes get set outside
  // capture); later steps replay a graph captured for this field and tol
  if (use_graph && (h->g_ptr != dA || h->g_tol != tol)) invalidate_graph(h);
  const int K = h->cfg.check_interval;
  double* hh = static_cast<double*>(h->h_hist);
  long long copied = 0;  // energies[0..copied) / deltas[0..copied) already copied out
  long long nonfinite = 0;
  int done = 0;
  bool stopped = false;
  auto harvest = [&](long long upto_step, bool final_energy) -> mbo_status {
    CK(cudaMemcpy(h->h_hist, h->hist_mem, (size_t)kRing * 5 * sizeof(double),
                  cudaMemcpyDeviceToHost));
    const long long* fl = reinterpret_cast<const long long*>(hh + 2 * kRing);
    const long long* nf = reinterpret_cast<const long long*>(hh + 4 * kRing);
    for (long long i = copied; i < upto_step; ++i) {
      const long long sl = i & (kRing - 1);
      nonfinite += nf[sl];
      if (energies) energies[i] = hh[sl];
      if (max_deltas) max_deltas[i] = hh[kRing + sl];
      if (det_flips) det_flips[i] = fl[sl];
    }
    if (final_energy && energies) energies[upto_step] = hh[upto_step & (kRing - 1)];
    copied = upto_step;
    return MBO_OK;
  };
  while (done < max_steps && !stopped) {
    const int chunk = std::min(K, max_steps - done);
    for (int i = 0; i < chunk; ++i) {
      if (use_graph && done + i > 0) {
        if (!h->gexec) {
          cudaGraph_t graph = nullptr;
          CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
          cudaError_t e = step_passes(h, dA, true, tol, h->cap);
          cudaError_t e2 = cudaStreamEndCapture(h->cap, &graph);
          if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail(h, MBO_ERR_CUDA, "graph capture failed: %s / %s", cudaGetErrorString(e),
                        cudaGetErrorString(e2));
          }
          cudaError_t e3 = cudaGraphInstantiate(&h->gexec, graph, 0);
          cudaGraphDestroy(graph);
          if (e3 != cudaSuccess) return fail(h, MBO_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e3));
          h->g_ptr = dA;
          h->g_tol = tol;
        }
        CK(cudaGraphLaunch(h->gexec, s));
      } else {
        CK(step_passes(h, dA, true, tol, s));
      }
    }
    done += chunk;
    CK(cudaMemcpyAsync(h->h_st, h->st, sizeof(RunState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (mbo_status de = device_errors(h)) return de;
    stopped = h->h_st->stop != 0;
    mbo_status rc = harvest(h->h_st->step, false);
    if (rc != MBO_OK) return rc;
    if (stopped) break;
  }
  const long long steps = h->h_st->step;
  // energy of the final field: its forward x transform is in the workspace
  CK(middle_passes(h, AXIS_ENERGY, stats_ptrs(h, true, false, -1.0), s));
  CK(cudaStreamSynchronize(s));
  mbo_status rc = harvest(steps, true);
  if (rc != MBO_OK) return rc;
  h->w_valid_for = (h->g.ndim == 2 && !host) ? dA : nullptr;
  if (host) {
    CK(cudaMemcpyAsync(A, dA, fbytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  if (steps_taken) *steps_taken = (int)steps;
  if (stationary) *stationary = stopped ? 1 : 0;
  const long long* nf = reinterpret_cast<const long long*>(hh + 4 * kRing);
  if (last) {
    if (steps > 0) {
      const long long sl = (steps - 1) & (kRing - 1);
      const long long* fl = reinterpret_cast<const long long*>(hh + 2 * kRing);
      const long long* fb = reinterpret_cast<const long long*>(hh + 3 * kRing);
      last->energy = hh[sl];
      last->max_delta = hh[kRing + sl];
      last->det_flips = fl[sl];
      last->fallback_points = fb[sl];
      last->nonfinite = nf[sl];
    } else {
      memset(last, 0, sizeof(*last));
      last->energy = hh[0];
    }
  }
  if (nonfinite) return fail(h, MBO_ERR_NUMERIC, "%lld non-finite points during the run", nonfinite);
  return MBO_OK;
}

mbo_status mbo_profile_enable(mbo_handle h, int enable) {
  if (!h) return MBO_ERR_INVALID_ARG;
  DeviceGuard dg(h->dev);
  for (auto& p : h->pending) {
    cudaEventSynchronize(p.b);
    h->ev_free.push_back(p.a);
    h->ev_free.push_back(p.b);
  }
  h->pending.clear();
  for (int i = 0; i < MBO_PROFILE_PASSES; ++i) {
    h->prof_ms[i] = 0;
    h->prof_n[i] = 0;
  }
  h->prof = enable != 0;
  return MBO_OK;
}

mbo_status mbo_profile_read(mbo_handle h, double* ms, int64_t* launches, int npass) {
  if (!h || npass < 0) return MBO_ERR_INVALID_ARG;
  DeviceGuard dg(h->dev);
  for (auto& p : h->pending) {
    CK(cudaEventSynchronize(p.b));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, p.a, p.b));
    h->prof_ms[p.pass] += t;
    h->prof_n[p.pass] += 1;
    h->ev_free.push_back(p.a);
    h->ev_free.push_back(p.b);
  }
  h->pending.clear();
  for (int i = 0; i < npass && i < MBO_PROFILE_PASSES; ++i) {
    if (ms) ms[i] = h->prof_ms[i];
    if (launches) launches[i] = h->prof_n[i];
  }
  return MBO_OK;
}

// ---------------------------------------------------------------------------
// Volume-preserving MBO (Sec. 7)
// ---------------------------------------------------------------------------

static mbo_status vp_buffers(mbo_handle h) {
  if (h->vp_at) return MBO_OK;
  const size_t fbytes = (size_t)h->g.C * (size_t)h->g.P * h->elem;
  CK(cudaMalloc(&h->vp_at, fbytes));
  CK(cudaMalloc((void**)&h->vp_keys, (size_t)h->g.P * sizeof(unsigned long long)));
  CK(cudaMalloc((void**)&h->vp_ss, sizeof(SelectState)));
  h->bytes_total += fbytes + (size_t)h->g.P * 8 + sizeof(SelectState);
  return MBO_OK;
}

static cudaError_t vp_launch(mbo_handle h, int which, const void* At, void* A, const StatsPtrs& sp,
                             cudaStream_t s) {
  long long blocks = (h->g.P + 255) / 256;
  const long long cap = std::min<long long>((long long)h->ngroups * kReduceGroup, 152 * 16);
  if (blocks > cap) blocks = cap;
  if (h->dtype == MBO_F32)
    return launch_volume<float>(which, h->g, static_cast<const float*>(At), static_cast<float*>(A),
                                h->vp_keys, h->vp_ss, sp, h->cfg.fallback_sigma, (int)blocks, s);
  return launch_volume<double>(which, h->g, static_cast<const double*>(At), static_cast<double*>(A),
                               h->vp_keys, h->vp_ss, sp, 0.0, (int)blocks, s);
}

// One volume-preserving step: diffuse (energy of A recorded), dE keys,
// selection of n_plus (< 0: the count of det > 0 points of A), assignment.
static mbo_status vp_step(mbo_handle h, void* A, long long n_plus, bool respect_stop, double tol,
                          cudaStream_t s) {
  const StatsPtrs sp = stats_ptrs(h, true, respect_stop, tol);
  StatsPtrs none = sp;
  none.do_stats = 0;
  CK(row_pass(h, ROW_FWD, A, nullptr, sp, s));
  CK(middle_passes(h, AXIS_FGI, sp, s));
  CK(row_pass(h, ROW_INV_OUT, nullptr, h->vp_at, none, s));
  CK(vp_launch(h, 0, h->vp_at, A, none, s));
  if (n_plus < 0) {
    CK(cudaMemsetAsync(&h->vp_ss->n_plus, 0, sizeof(unsigned long long), s));
    CK(vp_launch(h, 1, h->vp_at, A, none, s));
  }
  CK(launch_select_init(h->vp_ss, n_plus, s));
  long long blocks = std::min<long long>((h->g.P + 255) / 256, 152 * 16);
  CK(launch_select(h->vp_keys, h->g.P, h->vp_ss, (int)blocks, s));
  CK(vp_launch(h, 2, h->vp_at, A, sp, s));
  h->w_valid_for = nullptr;
  return MBO_OK;
}

mbo_status mbo_step_volume(mbo_handle h, void* A, int64_t n_plus, mbo_stats* stats, void* stream) {
  if (!h) return MBO_ERR_INVALID_ARG;
  if (h->g.n > 3) return fail(h, MBO_ERR_UNSUPPORTED_SIZE, "the volume-preserving step supports n <= 3");
  mbo_status rc;
  if ((rc = check_field_ptr(h, A, "A")) != MBO_OK) return rc;
  if (n_plus > h->g.P) return fail(h, MBO_ERR_INVALID_ARG, "n_plus exceeds the number of points");
  DeviceGuard dg(h->dev);
  if ((rc = vp_buffers(h)) != MBO_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((rc = vp_step(h, A, n_plus, false, -1.0, s)) != MBO_OK) return rc;
  if (stats) {
    CK(cudaStreamSynchronize(s));
    CK(cudaMemcpy(h->h_st, h->st, sizeof(RunState), cudaMemcpyDeviceToHost));
    const long long slot = (h->h_st->step - 1) & (kRing - 1);
    if ((rc = read_record(h, slot, stats)) != MBO_OK) return rc;
    if (stats->nonfinite) return fail(h, MBO_ERR_NUMERIC, "%lld non-finite points", (long long)stats->nonfinite);
  }
  return MBO_OK;
}

mbo_status mbo_run_volume(mbo_handle h, void* A, int64_t n_plus, int max_steps, double tol,
                          int* steps_taken, int* stationary, double* energies, void* stream) {
  if (!h || max_steps < 0) return MBO_ERR_INVALID_ARG;
  if (h->g.n > 3) return fail(h, MBO_ERR_UNSUPPORTED_SIZE, "the volume-preserving step supports n <= 3");
  mbo_status rc;
  if ((rc = check_field_ptr(h, A, "A")) != MBO_OK) return rc;
  if (n_plus > h->g.P) return fail(h, MBO_ERR_INVALID_ARG, "n_plus exceeds the number of points");
  DeviceGuard dg(h->dev);
  if ((rc = vp_buffers(h)) != MBO_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaMemsetAsync(h->st, 0, sizeof(RunState), s));
  if (n_plus < 0) {  // fix the volume of the initial field once
    const StatsPtrs none = stats_ptrs(h, false, false, -1.0);
    CK(cudaMemsetAsync(&h->vp_ss->n_plus, 0, sizeof(unsigned long long), s));
    CK(vp_launch(h, 1, nullptr, A, none, s));
    unsigned long long cnt = 0;
    CK(cudaMemcpyAsync(&cnt, &h->vp_ss->n_plus, sizeof(cnt), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    n_plus = (long long)cnt;
  }
  const int K = h->cfg.check_interval;
  int done = 0;
  bool stopped = false;
  while (done < max_steps && !stopped) {
    const int chunk = std::min(K, max_steps - done);
    for (int i = 0; i < chunk; ++i)
      if ((rc = vp_step(h, A, n_plus, true, tol, s)) != MBO_OK) return rc;
    done += chunk;
    CK(cudaMemcpyAsync(h->h_st, h->st, sizeof(RunState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    stopped = h->h_st->stop != 0;
  }
  const long long steps = h->h_st->step;
  CK(row_pass(h, ROW_FWD, A, nullptr, stats_ptrs(h, true, false, -1.0), s));
  CK(middle_passes(h, AXIS_ENERGY, stats_ptrs(h, true, false, -1.0), s));
  CK(cudaStreamSynchronize(s));
  CK(cudaMemcpy(h->h_hist, h->hist_mem, (size_t)kRing * 5 * sizeof(double), cudaMemcpyDeviceToHost));
  const double* hh = static_cast<const double*>(h->h_hist);
  if (energies) {
    const long long first = std::max(0LL, steps + 1 - kRing);
    for (long long i = first; i <= steps; ++i) energies[i] = hh[i & (kRing - 1)];
  }
  h->w_valid_for = (h->g.ndim == 2) ? A : nullptr;
  if (steps_taken) *steps_taken = (int)steps;
  if (stationary) *stationary = stopped ? 1 : 0;
  return MBO_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches of independent fields (uneven sizes and orders).  Each field keeps
// its own single-field context; one step of the whole batch is one CUDA graph
// whose per-field branches (spread over worker streams) are independent, so
// fields of different sizes run concurrently and the host launches once per
// step.
// ---------------------------------------------------------------------------

struct mbo_batch_ctx {
  int dev = 0;
  int count = 0;
  mbo_config cfg{};
  std::vector<mbo_ctx*> f;
  std::vector<cudaStream_t> ws;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<const void*> g_ptrs;
  double g_tol = 0;
  int g_run = -1;
  char err[512] = {0};
};

namespace mbo {

bool set_axis_multipliers(mbo_ctx* h, const double* const* mult) {
  if (!h || !mult) return false;
  DeviceGuard dg(h->dev);
  const int lens[3] = {h->g.nx, h->g.ny, h->g.nz};
  const bool f32 = h->dtype == MBO_F32;
  for (int ax = 0; ax < h->g.ndim; ++ax) {
    if (!mult[ax]) return false;
    const int N = lens[ax];
    const Plan& pl = f32 ? h->tf.plan[ax] : h->td.plan[ax];
    std::vector<int> pos;
    digit_positions(pl, N, pos);
    std::vector<double> g(N), om(N);
    for (int k = 0; k < N; ++k) {
      g[pos[k]] = mult[ax][k];
      om[pos[k]] = 1.0 - mult[ax][k];
    }
    cudaError_t e;
    if (f32) {
      std::vector<float> gf(g.begin(), g.end()), of(om.begin(), om.end());
      e = cudaMemcpy(const_cast<float*>(h->tf.g[ax]), gf.data(), N * sizeof(float), cudaMemcpyHostToDevice);
      if (e == cudaSuccess)
        e = cudaMemcpy(const_cast<float*>(h->tf.om[ax]), of.data(), N * sizeof(float), cudaMemcpyHostToDevice);
    } else {
      e = cudaMemcpy(const_cast<double*>(h->td.g[ax]), g.data(), N * sizeof(double), cudaMemcpyHostToDevice);
      if (e == cudaSuccess)
        e = cudaMemcpy(const_cast<double*>(h->td.om[ax]), om.data(), N * sizeof(double), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) return false;
  }
  return true;
}

}  // namespace mbo

namespace {

constexpr int kBatchStreams = 8;

mbo_status bfail(mbo_batch_ctx* b, mbo_status s, const char* what, cudaError_t e) {
  if (b) snprintf(b->err, sizeof(b->err), "%s: %s", what, cudaGetErrorString(e));
  return s;
}

#define BCK(call)                                                                            \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return bfail(b, e_ == cudaErrorMemoryAllocation ? MBO_ERR_OOM : MBO_ERR_CUDA, #call, e_); \
  } while (0)

// Capture one step of every field (run: stop flags respected, tol) into b->gexec.
mbo_status batch_capture(mbo_batch_ctx* b, void* const* A, bool run, double tol) {
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  cudaGraph_t graph = nullptr;
  BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaEventRecord(b->fork, b->cap);
  for (size_t k = 0; k < b->ws.size() && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->ws[k], b->fork, 0);
  for (int i = 0; i < b->count && e == cudaSuccess; ++i)
    e = step_passes(b->f[i], A[i], run, run ? tol : -1.0, b->ws[i % b->ws.size()]);
  for (size_t k = 0; k < b->ws.size() && e == cudaSuccess; ++k) {
    e = cudaEventRecord(b->join[k], b->ws[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->join[k], 0);
  }
  cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return bfail(b, MBO_ERR_CUDA, "batch graph capture", e != cudaSuccess ? e : e2);
  }
  e = cudaGraphInstantiate(&b->gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return bfail(b, MBO_ERR_CUDA, "batch graph instantiate", e);
  b->g_ptrs.assign(A, A + b->count);
  b->g_tol = tol;
  b->g_run = run ? 1 : 0;
  return MBO_OK;
}

bool batch_graph_matches(const mbo_batch_ctx* b, void* const* A, bool run, double tol) {
  if (!b->gexec || b->g_run != (run ? 1 : 0) || (run && b->g_tol != tol)) return false;
  for (int i = 0; i < b->count; ++i)
    if (b->g_ptrs[i] != A[i]) return false;
  return true;
}

}  // namespace

extern "C" {

mbo_status mbo_batch_destroy(mbo_batch h) {
  if (!h) return MBO_ERR_INVALID_ARG;
  DeviceGuard dg(h->dev);
  cudaDeviceSynchronize();
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  for (auto s : h->ws) cudaStreamDestroy(s);
  for (auto e : h->join) cudaEventDestroy(e);
  if (h->fork) cudaEventDestroy(h->fork);
  if (h->cap) cudaStreamDestroy(h->cap);
  for (auto f : h->f)
    if (f) mbo_destroy(f);
  delete h;
  return MBO_OK;
}

mbo_status mbo_batch_create(mbo_batch* out, int count, const int* ndim, const int64_t* dims,
                            const int* n, const double* tau, mbo_dtype dtype,
                            const mbo_config* cfg) {
  if (!out || count < 1 || !ndim || !dims || !n || !tau) return MBO_ERR_INVALID_ARG;
  *out = nullptr;
  mbo_batch_ctx* b = new mbo_batch_ctx();
  b->count = count;
  if (cfg) b->cfg = *cfg;
  else mbo_default_config(&b->cfg);
  cudaGetDevice(&b->dev);
  b->f.assign(count, nullptr);
  for (int i = 0; i < count; ++i) {
    mbo_status rc = mbo_create(&b->f[i], ndim[i], dims + 3 * (size_t)i, n[i], tau[i], dtype, &b->cfg);
    if (rc != MBO_OK) {
      snprintf(b->err, sizeof(b->err), "field %d: %s", i, mbo_status_string(rc));
      mbo_batch_destroy(b);
      return rc;
    }
  }
  const int nws = std::min(count, kBatchStreams);
  b->ws.assign(nws, nullptr);
  b->join.assign(nws, nullptr);
  bool ok = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; k < nws && ok; ++k)
    ok = cudaStreamCreateWithFlags(&b->ws[k], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    mbo_batch_destroy(b);
    return MBO_ERR_CUDA;
  }
  *out = b;
  return MBO_OK;
}

int64_t mbo_batch_workspace_bytes(mbo_batch h) {
  if (!h) return 0;
  int64_t t = 0;
  for (auto f : h->f) t += mbo_workspace_bytes(f);
  return t;
}

const char* mbo_batch_last_error(mbo_batch h) { return h ? h->err : ""; }

mbo_status mbo_batch_step(mbo_batch b, void* const* A, int flags, mbo_stats* stats, void* stream) {
  if (!b || !A) return MBO_ERR_INVALID_ARG;
  DeviceGuard dg(b->dev);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < b->count; ++i) {
    mbo_ctx* h = b->f[i];
    mbo_status rc = check_field_ptr(h, A[i], "A[i]");
    if (rc != MBO_OK) {
      snprintf(b->err, sizeof(b->err), "field %d: %s", i, h->err);
      return rc;
    }
    if (!((flags & MBO_STEP_CONTINUE) && h->w_valid_for == A[i]))
      BCK(row_pass(h, ROW_FWD, A[i], nullptr, stats_ptrs(h, true, false, -1.0), s));
  }
  if (!batch_graph_matches(b, A, false, -1.0)) {
    mbo_status rc = batch_capture(b, A, false, -1.0);
    if (rc != MBO_OK) return rc;
  }
  BCK(cudaGraphLaunch(b->gexec, s));
  for (int i = 0; i < b->count; ++i) b->f[i]->w_valid_for = A[i];
  if (stats) {
    BCK(cudaStreamSynchronize(s));
    for (int i = 0; i < b->count; ++i) {
      mbo_ctx* h = b->f[i];
      BCK(cudaMemcpy(h->h_st, h->st, sizeof(RunState), cudaMemcpyDeviceToHost));
      const long long slot = (h->h_st->step - 1) & (kRing - 1);
      mbo_status rc = read_record(h, slot, &stats[i]);
      if (rc != MBO_OK) return rc;
      if (stats[i].nonfinite) {
        snprintf(b->err, sizeof(b->err), "field %d: non-finite values", i);
        return MBO_ERR_NUMERIC;
      }
    }
  }
  return MBO_OK;
}

mbo_status mbo_batch_run(mbo_batch b, void* const* A, int max_steps, double tol, int* steps_taken,
                         int* stationary, double* energies, mbo_stats* last, void* stream) {
  if (!b || !A || max_steps < 0) return MBO_ERR_INVALID_ARG;
  DeviceGuard dg(b->dev);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int C = b->count;
  for (int i = 0; i < C; ++i) {
    mbo_ctx* h = b->f[i];
    mbo_status rc = check_field_ptr(h, A[i], "A[i]");
    if (rc != MBO_OK) {
      snprintf(b->err, sizeof(b->err), "field %d: %s", i, h->err);
      return rc;
    }
    BCK(cudaMemsetAsync(h->st, 0, sizeof(RunState), s));
    BCK(row_pass(h, ROW_FWD, A[i], nullptr, stats_ptrs(h, true, false, -1.0), s));
  }
  if (max_steps > 0 && !batch_graph_matches(b, A, true, tol)) {
    mbo_status rc = batch_capture(b, A, true, tol);
    if (rc != MBO_OK) return rc;
  }
  const int K = b->cfg.check_interval < 1 ? 1 : std::min(b->cfg.check_interval, kRing / 2);
  const size_t stride = (size_t)max_steps + 1;
  std::vector<long long> copied(C, 0), nonfinite(C, 0);
  std::vector<int> stopped(C, 0);
  auto harvest = [&](int i, long long upto, bool final_energy) -> mbo_status {
    mbo_ctx* h = b->f[i];
    BCK(cudaMemcpy(h->h_hist, h->hist_mem, (size_t)kRing * 5 * sizeof(double), cudaMemcpyDeviceToHost));
    const double* hh = static_cast<const double*>(h->h_hist);
    const long long* nf = reinterpret_cast<const long long*>(hh + 4 * kRing);
    for (long long t = copied[i]; t < upto; ++t) {
      nonfinite[i] += nf[t & (kRing - 1)];
      if (energies) energies[i * stride + t] = hh[t & (kRing - 1)];
    }
    if (final_energy && energies) energies[i * stride + upto] = hh[upto & (kRing - 1)];
    copied[i] = upto;
    return MBO_OK;
  };
  int done = 0;
  while (done < max_steps) {
    const int chunk = std::min(K, max_steps - done);
    for (int k = 0; k < chunk; ++k) BCK(cudaGraphLaunch(b->gexec, s));
    done += chunk;
    for (int i = 0; i < C; ++i)
      BCK(cudaMemcpyAsync(b->f[i]->h_st, b->f[i]->st, sizeof(RunState), cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));
    int all = 1;
    for (int i = 0; i < C; ++i) {
      stopped[i] = b->f[i]->h_st->stop != 0;
      all &= stopped[i];
      mbo_status rc = harvest(i, b->f[i]->h_st->step, false);
      if (rc != MBO_OK) return rc;
    }
    if (all) break;
  }
  for (int i = 0; i < C; ++i)
    BCK(middle_passes(b->f[i], AXIS_ENERGY, stats_ptrs(b->f[i], true, false, -1.0), s));
  BCK(cudaStreamSynchronize(s));
  for (int i = 0; i < C; ++i) {
    mbo_ctx* h = b->f[i];
    BCK(cudaMemcpy(h->h_st, h->st, sizeof(RunState), cudaMemcpyDeviceToHost));
    const long long st = h->h_st->step;
    mbo_status rc = harvest(i, st, true);
    if (rc != MBO_OK) return rc;
    h->w_valid_for = (h->g.ndim == 2) ? A[i] : nullptr;
    if (steps_taken) steps_taken[i] = (int)st;
    if (stationary) stationary[i] = stopped[i];
    if (last) {
      const double* hh = static_cast<const double*>(h->h_hist);
      const long long* fl = reinterpret_cast<const long long*>(hh + 2 * kRing);
      const long long* fb = reinterpret_cast<const long long*>(hh + 3 * kRing);
      const long long* nf = reinterpret_cast<const long long*>(hh + 4 * kRing);
      const long long sl = (st > 0 ? st - 1 : 0) & (kRing - 1);
      last[i].energy = hh[sl];
      last[i].max_delta = st > 0 ? hh[kRing + sl] : 0.0;
      last[i].det_flips = st > 0 ? fl[sl] : 0;
      last[i].fallback_points = st > 0 ? fb[sl] : 0;
      last[i].nonfinite = st > 0 ? nf[sl] : 0;
    }
  }
  for (int i = 0; i < C; ++i)
    if (nonfinite[i]) {
      snprintf(b->err, sizeof(b->err), "field %d: non-finite values during the run", i);
      return MBO_ERR_NUMERIC;
    }
  return MBO_OK;
}

}  // extern "C"
