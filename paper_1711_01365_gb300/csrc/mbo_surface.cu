// Closed-surface path of the MBO step (Sec. 5.2 and Algorithm 2 of Osting &
// Wang, arXiv:1711.01365), declared in include/mbo_surface.h.
//
// The diffusion of Algorithm 2 is the double sum
//   A~(x_t) = (h/2pi)^3 Re sum_m e^{-h^2 tau |m|^2} e^{i h m.x_t} sum_q w_q A(x_q^c) e^{-i h m.x_q}
// over m in {-M..M-1}^3.  With theta = h (x - centre) every point lies in
// [-pi/2, pi/2]^3, and the two non-uniform sums are computed on a periodic grid
// of nf points per axis (spacing 2 pi / nf, nf >= 4M):
//   k_spread   type-1 spreading: every source adds w_q A(x_q^c) phi(2 (j - u_q) / W)
//              to the W^3 grid points j around its grid coordinate u_q, with the
//              "exponential of semicircle" kernel phi(z) = exp(beta (sqrt(1 - z^2) - 1))
//              (Barnett, Magland, af Klinteberg, SIAM J. Sci. Comput. 41, 2019).
//              Sources are sorted into bins of kBin^3 grid cells; one block per
//              (bin, channel group) accumulates into a shared-memory tile of
//              (kBin + W)^3 points and adds the tile to the grid at the end.
//   (the library's 3-D FFT diffusion with the per-axis multiplier
//              nf (h / 2 pi) win(k) e^{-k^2 h^2 tau} / psi(k)^2, psi the kernel's
//              Fourier transform: forward FFT, multiplier, inverse FFT, in one
//              call of the torus path)
//   k_interp   type-2 interpolation: each target sums phi-weighted grid values
//              around its coordinate (one warp per target, lanes over the W^3
//              points), then, in the step, a lane per target projects the
//              matrix (Lemma 1.1) and writes it back with the step statistics.
// win(k) = 1 for |k| < M, 1/2 at |k| = M (the real part of the sum over
// -M..M-1), 0 beyond.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/mbo_surface.h"
#include "mbo_internal.h"
#include "mbo_kernels.cuh"

namespace mbo {
namespace {

constexpr int kBin = 8;          // spreading / interpolation bin: kBin^3 grid cells
constexpr int kMaxWidth = 12;    // kernel width limit (FP64)
constexpr int kMaxWidthF32 = 8;  // FP32: single precision holds no more digits
constexpr int kSpreadThreads = 256;
constexpr int kInterpThreads = 256;
constexpr size_t kTileBudget = 76 * 1024;  // shared bytes of one spreading tile

template <typename T> struct V4 { T x, y, z, w; };

struct SurfStats {
  unsigned long long maxd_bits;  // max |delta| as double bits (non-negative)
  unsigned long long flips, fallback, nonfinite;
};

template <typename T> __device__ __forceinline__ T es_kernel(T z, T beta) {
  const T a = T(1) - z * z;
  return a > T(0) ? exp(beta * (sqrt(a) - T(1))) : T(0);
}

// First footprint index of a coordinate o (offset from the bin origin, grid
// units) relative to the tile origin (bin origin - W/2), clamped so that the
// W points stay inside the tile whatever the rounding of o.
template <typename T> __device__ __forceinline__ int foot0(T o, int W) {
  int t = (int)ceil(o - T(0.5) * T(W)) + W / 2;
  return min(max(t, 0), kBin);
}

template <typename T> struct SpreadArgs {
  const T* A;            // surface field, C x nq
  const V4<T>* su;       // sources sorted by bin: offsets from the bin origin, weight
  const int* sidx;       // source -> field point
  const int* bstart;     // per non-empty bin: first source (nbins + 1 entries)
  const int* bid;        // per non-empty bin: bin id (bz nb + by) nb + bx
  T* F;                  // grid, C x nf^3
  long long nq;
  int C, nf, nb, W;
  T beta;
};

// One block per (non-empty bin, group of CG channels).
template <typename T, int CG>
__global__ void __launch_bounds__(kSpreadThreads) k_spread(SpreadArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);
  const int W = a.W, TS = kBin + W, TV = TS * TS * TS;
  const int c0 = blockIdx.y * CG;
  const int cg = min(CG, a.C - c0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < CG * TV; i += kSpreadThreads) tile[i] = T(0);
  __syncthreads();

  const int s0 = a.bstart[blockIdx.x], s1 = a.bstart[blockIdx.x + 1];
  const int W2 = W * W, W3 = W2 * W, iters = (W3 + 31) >> 5;
  for (int s = s0 + warp; s < s1; s += kSpreadThreads / 32) {
    const V4<T> u = a.su[s];
    const long long src = a.sidx[s];
    const int tx = foot0(u.x, W), ty = foot0(u.y, W), tz = foot0(u.z, W);
    // lane l < 3W: the 1-D weight of point l % W along axis l / W
    T wt = T(0);
    if (lane < 3 * W) {
      const int ax = lane / W, i = lane - ax * W;
      const T o = ax == 0 ? u.x : (ax == 1 ? u.y : u.z);
      const int t0 = ax == 0 ? tx : (ax == 1 ? ty : tz);
      const T z = (T(t0 + i - W / 2) - o) * (T(2) / T(W));
      wt = es_kernel(z, a.beta);
    }
    T str[CG];
#pragma unroll
    for (int c = 0; c < CG; ++c) str[c] = (c < cg) ? a.A[(long long)(c0 + c) * a.nq + src] * u.w : T(0);
    for (int it = 0; it < iters; ++it) {
      const int p = lane + 32 * it;
      const bool ok = p < W3;
      const int pp = ok ? p : 0;
      const int k = pp / W2, r = pp - k * W2, j = r / W, i = r - j * W;
      const T wx = __shfl_sync(0xffffffffu, wt, i);
      const T wy = __shfl_sync(0xffffffffu, wt, W + j);
      const T wz = __shfl_sync(0xffffffffu, wt, 2 * W + k);
      if (ok) {
        const T wgt = wx * wy * wz;
        const int addr = ((tz + k) * TS + ty + j) * TS + tx + i;
#pragma unroll
        for (int c = 0; c < CG; ++c)
          if (c < cg) atomicAdd(&tile[c * TV + addr], wgt * str[c]);
      }
    }
  }
  __syncthreads();

  // add the tile to the periodic grid
  const int b = a.bid[blockIdx.x];
  const int bx = b % a.nb, by = (b / a.nb) % a.nb, bz = b / (a.nb * a.nb);
  const int nf = a.nf;
  const long long P = (long long)nf * nf * nf;
  const int lx = bx * kBin - W / 2 + nf, ly = by * kBin - W / 2 + nf, lz = bz * kBin - W / 2 + nf;
  for (int c = 0; c < cg; ++c) {
    T* Fc = a.F + (long long)(c0 + c) * P;
    for (int i = tid; i < TV; i += kSpreadThreads) {
      const T v = tile[c * TV + i];
      if (v == T(0)) continue;
      const int x = i % TS, y = (i / TS) % TS, z = i / (TS * TS);
      const int gx = (lx + x) % nf, gy = (ly + y) % nf, gz = (lz + z) % nf;
      atomicAdd(&Fc[((long long)gz * nf + gy) * nf + gx], v);
    }
  }
}

template <typename T> struct InterpArgs {
  const T* F;          // grid, C x nf^3
  const V4<T>* tu;     // targets sorted by bin: offsets from the bin origin
  const int* tbin;     // target bin id
  const int* tidx;     // target -> field point
  T* out;              // C x nq: diffused field (diffuse) or the field itself (step)
  SurfStats* st;       // step statistics (step only)
  long long nq;
  int nf, nb, W;
  T beta, fb;
};

// One warp per group of 32 sorted targets: for each target the lanes sum the
// W^3 grid points (lane-parallel) and reduce; then lane l finishes target l.
template <typename T, int NM, bool STEP>
__global__ void __launch_bounds__(kInterpThreads) k_interp(InterpArgs<T> a) {
  constexpr int C = NM * NM;
  __shared__ T res[kInterpThreads / 32][32][C];
  __shared__ double redd[32];
  __shared__ int redi[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long base = ((long long)blockIdx.x * (kInterpThreads / 32) + warp) * 32;
  const int W = a.W, W2 = W * W, W3 = W2 * W, iters = (W3 + 31) >> 5;
  const int nf = a.nf;
  const long long P = (long long)nf * nf * nf;
  for (int e = 0; e < 32; ++e) {
    const long long t = base + e;
    if (t >= a.nq) break;  // warp-uniform
    const V4<T> u = a.tu[t];
    const int b = a.tbin[t];
    const int bx = b % a.nb, by = (b / a.nb) % a.nb, bz = b / (a.nb * a.nb);
    const int tx = foot0(u.x, W), ty = foot0(u.y, W), tz = foot0(u.z, W);
    T wt = T(0);
    if (lane < 3 * W) {
      const int ax = lane / W, i = lane - ax * W;
      const T o = ax == 0 ? u.x : (ax == 1 ? u.y : u.z);
      const int t0 = ax == 0 ? tx : (ax == 1 ? ty : tz);
      const T z = (T(t0 + i - W / 2) - o) * (T(2) / T(W));
      wt = es_kernel(z, a.beta);
    }
    const int lx = bx * kBin - W / 2 + tx + nf, ly = by * kBin - W / 2 + ty + nf,
              lz = bz * kBin - W / 2 + tz + nf;
    T acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = T(0);
    for (int it = 0; it < iters; ++it) {
      const int p = lane + 32 * it;
      const bool ok = p < W3;
      const int pp = ok ? p : 0;
      const int k = pp / W2, r = pp - k * W2, j = r / W, i = r - j * W;
      const T wx = __shfl_sync(0xffffffffu, wt, i);
      const T wy = __shfl_sync(0xffffffffu, wt, W + j);
      const T wz = __shfl_sync(0xffffffffu, wt, 2 * W + k);
      if (ok) {
        const T wgt = wx * wy * wz;
        const long long o = ((long long)((lz + k) % nf) * nf + (ly + j) % nf) * nf + (lx + i) % nf;
#pragma unroll
        for (int c = 0; c < C; ++c) acc[c] += wgt * __ldg(&a.F[c * P + o]);
      }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
      T v = acc[c];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (lane == 0) res[warp][e][c] = v;
    }
  }
  __syncwarp();

  const long long t = base + lane;
  PointStats<T> ps;
  if (t < a.nq) {
    const long long q = a.tidx[t];
    T m[C];
#pragma unroll
    for (int c = 0; c < C; ++c) m[c] = res[warp][lane][c];
    if constexpr (!STEP) {
#pragma unroll
      for (int c = 0; c < C; ++c) a.out[c * a.nq + q] = m[c];
    } else {
      T old[C], bb[C], sg;
#pragma unroll
      for (int c = 0; c < C; ++c) old[c] = a.out[c * a.nq + q];
      bool fin = true;
#pragma unroll
      for (int c = 0; c < C; ++c) fin = fin && isfinite(m[c]);
      ps.nonfinite += fin ? 0 : 1;
      if (!project_point<NM>(m, bb, sg, a.fb)) {
        sg = project_point_f64<NM>(m, bb);
        ps.fallback += 1;
      }
      T d = T(0);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        d = fmax(d, fabs(bb[c] - old[c]));
        a.out[c * a.nq + q] = bb[c];
      }
      ps.maxd = fmax(ps.maxd, d);
      ps.flips += (det_sign<NM>(old) != sg) ? 1 : 0;
    }
  }
  if constexpr (STEP) {
    const double mx = block_max((double)ps.maxd, redd);
    const int fl = block_sum(ps.flips, redi);
    const int nfin = block_sum(ps.nonfinite, redi);
    const int nfb = block_sum(ps.fallback, redi);
    if (tid == 0) {
      atomicMax(&a.st->maxd_bits, (unsigned long long)__double_as_longlong(mx));
      if (fl) atomicAdd(&a.st->flips, (unsigned long long)fl);
      if (nfin) atomicAdd(&a.st->nonfinite, (unsigned long long)nfin);
      if (nfb) atomicAdd(&a.st->fallback, (unsigned long long)nfb);
    }
  }
}

// ----------------------------------------------------------------------------
// host-side geometry (Algorithm 2, step 1) and plan parameters
// ----------------------------------------------------------------------------

double tail_T(double x) { return 2.0 * x / std::sqrt(M_PI) * std::exp(-x * x) + std::erfc(x); }

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on the
// three-term recurrence of P_n, starting from the Chebyshev-like guesses
// cos(pi (i - 1/4) / (n + 1/2))).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

bool smooth23(int N) {
  while (N % 2 == 0) N /= 2;
  while (N % 3 == 0) N /= 3;
  return N == 1;
}

}  // namespace
}  // namespace mbo

using namespace mbo;

struct mbo_surface_ctx {
  int dev = 0;
  mbo_dtype dtype = MBO_F32;
  int n = 0, C = 0;
  long long nq = 0;
  double tau = 0, eps = 0;
  mbo_surface_params prm{};
  int nb = 0;  // bins per axis
  int nbins = 0;  // non-empty source bins
  int cg = 1, ngroups = 1;
  size_t tile_bytes = 0;
  mbo_handle fine = nullptr;  // 3-D FFT diffusion on the nf^3 grid
  void* F = nullptr;          // grid, C x nf^3
  void* su = nullptr;         // V4<T> sources
  int* sidx = nullptr;
  int* bstart = nullptr;
  int* bid = nullptr;
  void* tu = nullptr;         // V4<T> targets
  int* tbin = nullptr;
  int* tidx = nullptr;
  SurfStats* st = nullptr;
  SurfStats* h_st = nullptr;  // pinned
  size_t bytes = 0;
  char err[512] = {0};
};

namespace {

mbo_status sfail(mbo_surface_ctx* s, mbo_status rc, const char* fmt, const char* what = "") {
  if (s) snprintf(s->err, sizeof(s->err), fmt, what);
  return rc;
}

#define SCK(call)                                                                           \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return sfail(s, e_ == cudaErrorMemoryAllocation ? MBO_ERR_OOM : MBO_ERR_CUDA,         \
                   "%s", cudaGetErrorString(e_));                                           \
  } while (0)

template <typename T, int CG> cudaError_t spread_cg(const SpreadArgs<T>& a, dim3 grid, size_t smem,
                                                    cudaStream_t st) {
  auto k = k_spread<T, CG>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k<<<grid, kSpreadThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_spread(mbo_surface_ctx* s, const void* A, cudaStream_t st) {
  SpreadArgs<T> a;
  a.A = static_cast<const T*>(A);
  a.su = static_cast<const V4<T>*>(s->su);
  a.sidx = s->sidx;
  a.bstart = s->bstart;
  a.bid = s->bid;
  a.F = static_cast<T*>(s->F);
  a.nq = s->nq;
  a.C = s->C;
  a.nf = s->prm.nf;
  a.nb = s->nb;
  a.W = s->prm.width;
  a.beta = (T)s->prm.beta;
  const dim3 grid(s->nbins, s->ngroups);
  switch (s->cg) {
    case 1: return spread_cg<T, 1>(a, grid, s->tile_bytes, st);
    case 2: return spread_cg<T, 2>(a, grid, s->tile_bytes, st);
    case 3: return spread_cg<T, 3>(a, grid, s->tile_bytes, st);
    case 4: return spread_cg<T, 4>(a, grid, s->tile_bytes, st);
    case 5: return spread_cg<T, 5>(a, grid, s->tile_bytes, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, bool STEP>
cudaError_t launch_interp(mbo_surface_ctx* s, void* out, cudaStream_t st) {
  InterpArgs<T> a;
  a.F = static_cast<const T*>(s->F);
  a.tu = static_cast<const V4<T>*>(s->tu);
  a.tbin = s->tbin;
  a.tidx = s->tidx;
  a.out = static_cast<T*>(out);
  a.st = s->st;
  a.nq = s->nq;
  a.nf = s->prm.nf;
  a.nb = s->nb;
  a.W = s->prm.width;
  a.beta = (T)s->prm.beta;
  a.fb = T(0);
  const long long per = (kInterpThreads / 32) * 32;
  const unsigned blocks = (unsigned)((s->nq + per - 1) / per);
  switch (s->n) {
    case 1: k_interp<T, 1, STEP><<<blocks, kInterpThreads, 0, st>>>(a); break;
    case 2: k_interp<T, 2, STEP><<<blocks, kInterpThreads, 0, st>>>(a); break;
    case 3: k_interp<T, 3, STEP><<<blocks, kInterpThreads, 0, st>>>(a); break;
    default: k_interp<T, 4, STEP><<<blocks, kInterpThreads, 0, st>>>(a); break;
  }
  return cudaGetLastError();
}

mbo_status surface_diffusion(mbo_surface_ctx* s, const void* A, cudaStream_t st) {
  const long long P = (long long)s->prm.nf * s->prm.nf * s->prm.nf;
  const size_t elem = s->dtype == MBO_F32 ? 4 : 8;
  SCK(cudaMemsetAsync(s->F, 0, (size_t)s->C * P * elem, st));
  SCK(s->dtype == MBO_F32 ? launch_spread<float>(s, A, st) : launch_spread<double>(s, A, st));
  const mbo_status rc = mbo_diffuse(s->fine, s->F, s->F, st);
  if (rc != MBO_OK) return sfail(s, rc, "grid diffusion: %s", mbo_last_error(s->fine));
  return MBO_OK;
}

template <typename T> void pack_points(const std::vector<V4<double>>& in, void* dst) {
  std::vector<V4<T>> v(in.size());
  for (size_t i = 0; i < in.size(); ++i) v[i] = V4<T>{(T)in[i].x, (T)in[i].y, (T)in[i].z, (T)in[i].w};
  cudaMemcpy(dst, v.data(), v.size() * sizeof(V4<T>), cudaMemcpyHostToDevice);
}

}  // namespace

extern "C" {

double mbo_surface_band_width(double eps, double tau) {
  if (!(eps > 0 && eps < 1) || !(tau > 0) || !std::isfinite(tau)) return -1.0;
  double lo = 0.0, hi = 1.0;
  while (tail_T(hi) > eps) hi *= 2.0;
  for (int i = 0; i < 200 && hi - lo > 0; ++i) {
    const double mid = 0.5 * (lo + hi);
    (tail_T(mid) > eps ? lo : hi) = mid;
  }
  return 2.0 * std::sqrt(tau) * hi;
}

mbo_status mbo_surface_heat_modes(double eps, double tau, double R, double* h, int* M) {
  if (!(eps > 0 && eps < 0.5) || !(tau > 0) || !(R > 0) || !std::isfinite(tau) || !std::isfinite(R))
    return MBO_ERR_INVALID_ARG;
  const double hh = std::min(M_PI / R, M_PI / (2.0 * std::sqrt(tau * std::fabs(std::log(eps)))));
  const double lg = std::log(2.0 * hh * std::sqrt(tau) / (std::sqrt(M_PI) * eps));
  const double mm = std::ceil(std::sqrt(std::max(lg, 0.0) / tau) / hh);
  if (h) *h = hh;
  if (M) *M = (int)std::max(1.0, std::min(mm, 1e9));
  return MBO_OK;
}

mbo_status mbo_surface_sphere_band(double radius, double dx, double wb, int p, double* xq,
                                   double* wq, double* xc, int64_t capacity, int64_t* count) {
  if (!(radius > 0) || !(dx > 0) || !(wb > 0) || p < 1 || p > 16 || !count) return MBO_ERR_INVALID_ARG;
  // nodes cos((2k - 1) pi / (2p)) and Fejer's first-rule weights on [-1, 1]
  std::vector<double> t(p), w(p);
  for (int k = 0; k < p; ++k) {
    const double th = (2.0 * (k + 1) - 1.0) * M_PI / (2.0 * p);
    t[k] = std::cos(th);
    double s = 0.0;
    for (int j = 1; j <= p / 2; ++j) s += std::cos(2.0 * j * th) / (4.0 * j * j - 1.0);
    w[k] = (2.0 / p) * (1.0 - 2.0 * s);
  }
  std::vector<double> off(p), wc(p);
  for (int k = 0; k < p; ++k) {
    off[k] = dx * (1.0 + t[k]) / 2.0;
    wc[k] = w[k] * dx / 2.0;
  }
  const long long lim = (long long)std::ceil((radius + wb) / dx) + 1;
  const long long per = (long long)p * p * p;
  int64_t n = 0;
  const bool fill = xq && wq && xc;
  for (long long i = -lim; i <= lim; ++i)
    for (long long j = -lim; j <= lim; ++j)
      for (long long k = -lim; k <= lim; ++k) {
        const double gx = dx * i, gy = dx * j, gz = dx * k;
        if (!(std::fabs(std::sqrt(gx * gx + gy * gy + gz * gz) - radius) < wb)) continue;
        if (fill && n + per <= capacity) {
          for (int a = 0; a < p; ++a)
            for (int b = 0; b < p; ++b)
              for (int c = 0; c < p; ++c) {
                const int64_t q = n + ((int64_t)a * p + b) * p + c;
                const double x = gx + off[a], y = gy + off[b], z = gz + off[c];
                xq[3 * q] = x;
                xq[3 * q + 1] = y;
                xq[3 * q + 2] = z;
                wq[q] = wc[a] * wc[b] * wc[c];
                const double r = std::sqrt(x * x + y * y + z * z);
                if (r > 0) {
                  xc[3 * q] = radius * x / r;
                  xc[3 * q + 1] = radius * y / r;
                  xc[3 * q + 2] = radius * z / r;
                } else {
                  xc[3 * q] = 0.0;
                  xc[3 * q + 1] = 0.0;
                  xc[3 * q + 2] = radius;
                }
              }
        }
        n += per;
      }
  *count = n;
  if (fill && n > capacity) return MBO_ERR_INVALID_ARG;
  return MBO_OK;
}

mbo_status mbo_surface_destroy(mbo_surface s) {
  if (!s) return MBO_ERR_INVALID_ARG;
  int prev = -1;
  if (cudaGetDevice(&prev) == cudaSuccess && prev != s->dev) cudaSetDevice(s->dev);
  else prev = -1;
  cudaDeviceSynchronize();
  if (s->fine) mbo_destroy(s->fine);
  void* bufs[] = {s->F, s->su, s->sidx, s->bstart, s->bid, s->tu, s->tbin, s->tidx, s->st};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (s->h_st) cudaFreeHost(s->h_st);
  if (prev >= 0) cudaSetDevice(prev);
  delete s;
  return MBO_OK;
}

mbo_status mbo_surface_create(mbo_surface* out, int64_t nq, const double* xq, const double* wq,
                              const double* xc, int n, double tau, double eps, mbo_dtype dtype) {
  if (!out) return MBO_ERR_INVALID_ARG;
  *out = nullptr;
  if (nq < 1 || nq >= (1LL << 31) || !xq || !wq || !xc || n < 1 || n > 4 || !(tau > 0) ||
      !std::isfinite(tau) || !(eps > 1e-12 && eps < 0.5) || (dtype != MBO_F32 && dtype != MBO_F64))
    return MBO_ERR_INVALID_ARG;
  for (int64_t i = 0; i < 3 * nq; ++i)
    if (!std::isfinite(xq[i]) || !std::isfinite(xc[i])) return MBO_ERR_INVALID_ARG;
  for (int64_t i = 0; i < nq; ++i)
    if (!std::isfinite(wq[i])) return MBO_ERR_INVALID_ARG;

  mbo_surface_ctx* s = new mbo_surface_ctx();
  cudaGetDevice(&s->dev);
  s->dtype = dtype;
  s->n = n;
  s->C = n * n;
  s->nq = nq;
  s->tau = tau;
  s->eps = eps;
  mbo_surface_params& prm = s->prm;

  // extent and centre of all points
  double lo[3], hi[3];
  for (int a = 0; a < 3; ++a) lo[a] = hi[a] = xq[a];
  for (int64_t i = 0; i < nq; ++i)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], std::min(xq[3 * i + a], xc[3 * i + a]));
      hi[a] = std::max(hi[a], std::max(xq[3 * i + a], xc[3 * i + a]));
    }
  prm.R = 0;
  for (int a = 0; a < 3; ++a) {
    prm.center[a] = 0.5 * (lo[a] + hi[a]);
    prm.R = std::max(prm.R, hi[a] - lo[a]);
  }
  if (!(prm.R > 0)) prm.R = 1.0;  // a single point: any radius
  mbo_surface_heat_modes(eps, tau, prm.R, &prm.h, &prm.M);
  int W = (int)std::ceil(std::log10(1.0 / eps)) + 1;
  W = std::max(2, std::min(W, dtype == MBO_F32 ? kMaxWidthF32 : kMaxWidth));
  prm.width = W;
  prm.beta = 2.30 * W;
  int nf = std::max(std::max(4 * prm.M, 2 * W), 8);
  while (!smooth23(nf)) ++nf;
  prm.nf = nf;
  if (nf > 2048) {
    mbo_surface_destroy(s);
    return MBO_ERR_UNSUPPORTED_SIZE;
  }
  const int nb = (nf + kBin - 1) / kBin;
  s->nb = nb;

  // grid coordinates u = (h (x - centre) + pi) nf / (2 pi), binned
  const double sc = (double)nf / (2.0 * M_PI);
  auto grid_coord = [&](const double* x, double* u) {
    for (int a = 0; a < 3; ++a) {
      double v = (prm.h * (x[a] - prm.center[a]) + M_PI) * sc;
      u[a] = std::min(std::max(v, 0.0), std::nextafter((double)nf, 0.0));
    }
  };
  auto bin_of = [&](const double* u, double* o) {
    int b[3];
    for (int a = 0; a < 3; ++a) {
      b[a] = std::min((int)(u[a] / kBin), nb - 1);
      o[a] = u[a] - (double)b[a] * kBin;
    }
    return (b[2] * nb + b[1]) * nb + b[0];
  };
  const int nbin_all = nb * nb * nb;
  std::vector<int> sb(nq), tb(nq);
  std::vector<V4<double>> so(nq), to(nq);
  for (int64_t i = 0; i < nq; ++i) {
    double u[3], o[3];
    grid_coord(xq + 3 * i, u);
    sb[i] = bin_of(u, o);
    so[i] = V4<double>{o[0], o[1], o[2], wq[i]};
    grid_coord(xc + 3 * i, u);
    tb[i] = bin_of(u, o);
    to[i] = V4<double>{o[0], o[1], o[2], 0.0};
  }
  // counting sorts by bin (stable: original order within a bin)
  auto sort_by = [&](const std::vector<int>& key, std::vector<int>& perm, std::vector<int>& cnt) {
    cnt.assign(nbin_all + 1, 0);
    for (int64_t i = 0; i < nq; ++i) ++cnt[key[i] + 1];
    for (int b = 0; b < nbin_all; ++b) cnt[b + 1] += cnt[b];
    std::vector<int> pos(cnt.begin(), cnt.end() - 1);
    perm.assign(nq, 0);
    for (int64_t i = 0; i < nq; ++i) perm[pos[key[i]]++] = (int)i;
  };
  std::vector<int> sperm, scnt, tperm, tcnt;
  sort_by(sb, sperm, scnt);
  sort_by(tb, tperm, tcnt);
  std::vector<int> bstart, bid;
  for (int b = 0; b < nbin_all; ++b)
    if (scnt[b + 1] > scnt[b]) {
      bid.push_back(b);
      bstart.push_back(scnt[b]);
    }
  bstart.push_back((int)nq);
  s->nbins = (int)bid.size();
  prm.bins = s->nbins;
  std::vector<V4<double>> sos(nq), tos(nq);
  std::vector<int> tbs(nq);
  for (int64_t i = 0; i < nq; ++i) {
    sos[i] = so[sperm[i]];
    tos[i] = to[tperm[i]];
    tbs[i] = tb[tperm[i]];
  }

  // channel groups of the spreading tile
  const size_t elem = dtype == MBO_F32 ? 4 : 8;
  const size_t tv = (size_t)(kBin + W) * (kBin + W) * (kBin + W);
  const size_t per_ch = tv * elem;
  int fit = (int)std::max<size_t>(1, kTileBudget / per_ch);
  fit = std::min(fit, 5);
  s->ngroups = (s->C + fit - 1) / fit;
  s->cg = (s->C + s->ngroups - 1) / s->ngroups;
  s->tile_bytes = (size_t)s->cg * per_ch;
  int maxsm = 0;
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->dev);
  if (s->tile_bytes > (size_t)maxsm) {
    mbo_surface_destroy(s);
    return MBO_ERR_UNSUPPORTED_SIZE;
  }

  // the grid's FFT diffusion with the deconvolved heat factor
  const int64_t dims[3] = {nf, nf, nf};
  mbo_status rc = mbo_create(&s->fine, 3, dims, n, 1.0, dtype, nullptr);
  if (rc != MBO_OK) {
    snprintf(s->err, sizeof(s->err), "grid plan: %s", mbo_status_string(rc));
    mbo_surface_destroy(s);
    return rc;
  }
  std::vector<double> gx, gwt, mult(nf);
  gauss_legendre(128, gx, gwt);
  for (int k = 0; k < nf; ++k) {
    const int kf = (2 * k <= nf) ? k : k - nf;
    const int ak = std::abs(kf);
    const double win = ak < prm.M ? 1.0 : (ak == prm.M ? 0.5 : 0.0);
    if (win == 0.0) {
      mult[k] = 0.0;
      continue;
    }
    // psi(k) = (W/2) int_{-1}^{1} phi(z) cos(pi k W z / nf) dz
    double psi = 0.0;
    for (size_t i = 0; i < gx.size(); ++i) {
      const double z = gx[i];
      psi += gwt[i] * std::exp(prm.beta * (std::sqrt(1.0 - z * z) - 1.0)) * std::cos(M_PI * kf * W * z / nf);
    }
    psi *= 0.5 * W;
    mult[k] = nf * (prm.h / (2.0 * M_PI)) * win * std::exp(-(double)kf * kf * prm.h * prm.h * tau) / (psi * psi);
  }
  const double* mm[3] = {mult.data(), mult.data(), mult.data()};
  if (!set_axis_multipliers(s->fine, mm)) {
    snprintf(s->err, sizeof(s->err), "grid multipliers: %s", cudaGetErrorString(cudaGetLastError()));
    mbo_surface_destroy(s);
    return MBO_ERR_CUDA;
  }

  // device tables
  const long long P = (long long)nf * nf * nf;
  auto alloc = [&](void** p, size_t b) {
    if (cudaMalloc(p, b) != cudaSuccess) return false;
    s->bytes += b;
    return true;
  };
  const size_t v4 = dtype == MBO_F32 ? sizeof(V4<float>) : sizeof(V4<double>);
  if (!alloc(&s->F, (size_t)s->C * P * elem) || !alloc(&s->su, nq * v4) ||
      !alloc((void**)&s->sidx, nq * sizeof(int)) || !alloc((void**)&s->bstart, bstart.size() * sizeof(int)) ||
      !alloc((void**)&s->bid, std::max<size_t>(bid.size(), 1) * sizeof(int)) || !alloc(&s->tu, nq * v4) ||
      !alloc((void**)&s->tbin, nq * sizeof(int)) || !alloc((void**)&s->tidx, nq * sizeof(int)) ||
      !alloc((void**)&s->st, sizeof(SurfStats)) ||
      cudaMallocHost((void**)&s->h_st, sizeof(SurfStats)) != cudaSuccess) {
    mbo_surface_destroy(s);
    return MBO_ERR_OOM;
  }
  if (dtype == MBO_F32) {
    pack_points<float>(sos, s->su);
    pack_points<float>(tos, s->tu);
  } else {
    pack_points<double>(sos, s->su);
    pack_points<double>(tos, s->tu);
  }
  cudaMemcpy(s->sidx, sperm.data(), nq * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(s->bstart, bstart.data(), bstart.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (!bid.empty()) cudaMemcpy(s->bid, bid.data(), bid.size() * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(s->tbin, tbs.data(), nq * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(s->tidx, tperm.data(), nq * sizeof(int), cudaMemcpyHostToDevice);
  const cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    snprintf(s->err, sizeof(s->err), "table upload: %s", cudaGetErrorString(e));
    mbo_surface_destroy(s);
    return MBO_ERR_CUDA;
  }
  *out = s;
  return MBO_OK;
}

mbo_status mbo_surface_get_params(mbo_surface s, mbo_surface_params* p) {
  if (!s || !p) return MBO_ERR_INVALID_ARG;
  *p = s->prm;
  return MBO_OK;
}

mbo_status mbo_surface_diffuse(mbo_surface s, const void* A, void* A_tilde, void* stream) {
  if (!s || !A || !A_tilde || ((uintptr_t)A & 15) || ((uintptr_t)A_tilde & 15)) return MBO_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  mbo_status rc = surface_diffusion(s, A, st);
  if (rc != MBO_OK) return rc;
  SCK((s->dtype == MBO_F32 ? launch_interp<float, false>(s, A_tilde, st)
                           : launch_interp<double, false>(s, A_tilde, st)));
  return MBO_OK;
}

mbo_status mbo_surface_step(mbo_surface s, void* A, mbo_stats* stats, void* stream) {
  if (!s || !A || ((uintptr_t)A & 15)) return MBO_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  mbo_status rc = surface_diffusion(s, A, st);
  if (rc != MBO_OK) return rc;
  SCK(cudaMemsetAsync(s->st, 0, sizeof(SurfStats), st));
  SCK((s->dtype == MBO_F32 ? launch_interp<float, true>(s, A, st)
                           : launch_interp<double, true>(s, A, st)));
  if (stats) {
    SCK(cudaMemcpyAsync(s->h_st, s->st, sizeof(SurfStats), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    stats->energy = NAN;
    double md;
    std::memcpy(&md, &s->h_st->maxd_bits, sizeof(md));
    stats->max_delta = md;
    stats->det_flips = (int64_t)s->h_st->flips;
    stats->fallback_points = (int64_t)s->h_st->fallback;
    stats->nonfinite = (int64_t)s->h_st->nonfinite;
    if (stats->nonfinite) {
      snprintf(s->err, sizeof(s->err), "non-finite values in the projected field");
      return MBO_ERR_NUMERIC;
    }
  }
  return MBO_OK;
}

int64_t mbo_surface_workspace_bytes(mbo_surface s) {
  if (!s) return -1;
  return (int64_t)s->bytes + (s->fine ? mbo_workspace_bytes(s->fine) : 0);
}

const char* mbo_surface_last_error(mbo_surface s) { return s ? s->err : "null plan"; }

}  // extern "C"
