// Closed-surface path of the MBO step (Sec. 5.2 and Algorithm 2 of Osting &
// Wang, arXiv:1711.01365), declared in include/mbo_surface.h.
//
// The diffusion of Algorithm 2 is the double sum
//   A~(x_t) = (h/2pi)^3 Re sum_m e^{-h^2 tau |m|^2} e^{i h m.x_t} sum_q w_q A(x_q^c) e^{-i h m.x_q}
// over m in {-M..M-1}^3.  With theta = h (x - centre) every point lies in
// [-pi/2, pi/2]^3, and the two non-uniform sums are computed on a periodic grid
// of nf points per axis (spacing 2 pi / nf, nf >= 4M) with the "exponential
// of semicircle" kernel phi(z) = exp(beta (sqrt(1 - z^2) - 1)) of width W grid
// points (Barnett, Magland, af Klinteberg, SIAM J. Sci. Comput. 41, 2019):
//   k_spread   type-1 spreading: source q adds w_q A(x_q^c) phi(2 (j - u_q) / W) to
//              the W^3 grid points j around its grid coordinate u_q (phi of a
//              vector: the product of its three coordinates' factors).
//   (the library's 3-D FFT diffusion with the per-axis multiplier
//              nf (h / 2 pi) win(k) e^{-k^2 h^2 tau} / psi(k)^2, psi the kernel's
//              Fourier transform: forward FFT, multiplier, inverse FFT, in one
//              call of the torus path)
//   k_interp   type-2 interpolation: target t sums the phi-weighted grid values
//              around its coordinate.
//   k_sproject projection of every target (Lemma 1.1) with the step statistics.
// win(k) = 1 for |k| < M, 1/2 at |k| = M (the real part of the sum over
// -M..M-1), 0 beyond.  The volume-preserving step (Sec. 7, Algorithm 3) runs
// the diffusion into the caller's point order, the flat-torus dE keys and
// class assignment (k_vp_delta / k_vp_assign) on the points, and between them
// a weighted radix selection (k_wselect_*).
//
// Points whose footprints (the W^3 grid points spread to or read from) start
// at the same grid point share their footprint, and the plan sorts them into
// such groups once (the geometry is fixed).  Spreading: one warp per group of
// sources, a lane per footprint column (x, y) holding the W points along z for
// CG channels in registers; the group's sources are summed there and added once
// to a shared-memory tile of the group's bin of kBin^3 cells, which goes to the
// grid at the end.  Interpolation: one block per group of targets stages the
// footprint values in shared memory once and evaluates every target of the
// group from them, a thread per target.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <type_traits>
#include <vector>

#include "../../include/mbo_surface.h"
#include "mbo_internal.h"
#include "mbo_kernels.cuh"

namespace mbo {
namespace {

constexpr int kBin = 8;         // spreading bin: kBin^3 grid cells
constexpr int kMaxW = 8;        // kernel width limit (register arrays)
constexpr int kMinW = 4;
constexpr int kSpreadThreads = 512;
constexpr int kProjThreads = 256;

template <typename T> struct V4 { T x, y, z, w; };

struct SurfStats {
  unsigned long long maxd_bits;  // max |delta| as double bits (non-negative)
  unsigned long long flips, fallback, nonfinite;
};

template <typename T> __device__ __forceinline__ T es_kernel(T z, T beta) {
  const T a = T(1) - z * z;
  return a > T(0) ? exp(beta * (sqrt(a) - T(1))) : T(0);
}

template <typename T> struct SpreadArgs {
  const T* A;            // surface field, C x nq
  const V4<T>* su;       // sources sorted by (bin, group): d per axis, weight w_q
  const int* sidx;       // source -> field point
  const int* gsrc;       // group -> first source (ngroups + 1)
  const int* gt0;        // group -> footprint start in the bin tile, t0x | t0y << 4 | t0z << 8
  const int* bgrp;       // bin -> first group (nbins + 1)
  const int* bid;        // bin -> bin id (bz nb + by) nb + bx
  T* F;                  // grid, C x nf^3
  long long nq;
  int C, nf, nb, W;
  T beta;
};

// One block per (non-empty bin, group of CG channels); one warp per point
// group.  A group holds the sources of a bin whose footprints start at the
// same z and within a 2 x 2 block in (x, y), so its footprint is
// (W + 1) x (W + 1) x W points (a source's weights vanish outside its own W^3).
// The warp stages chunk_of<T>() sources at a time in shared memory, lane l the
// l-th source (its one-dimensional weights, z first, and strengths w_q A, in
// 16-byte vectors; the per-source stride makes the vector stores of a quarter
// warp hit distinct banks); then lane p of round rd owns footprint column
// (x, y) = (p % (W+1), p / (W+1)), p = lane + 32 rd, sums it over the chunk, W
// points along z for CG channels in registers, and adds it to the bin tile.
// WT: the kernel width as a compile-time constant (the width of eps = 1e-6,
// the paper's choice, has its own instantiation), or 0 for the runtime width.
template <typename T> __host__ __device__ constexpr int chunk_of() { return sizeof(T) == 4 ? 32 : 16; }
// Tile column of x in tile row y.  At width 7 the rows are 16 wide and a flush
// writes 4 rows x 8 columns from an even (x, y) start: x ^ 8 on rows with bit 1
// of y set puts those 32 lanes on 32 distinct banks.
template <int WT> __device__ __forceinline__ int swz(int x, int y) {
  if constexpr (WT == 7) return x ^ (((y >> 1) & 1) << 3);
  return x;
}
constexpr int kWS = 9;     // weight slots of x and of y per source (>= W + 1)
constexpr int kWSrc = 28;  // per source: z[8] | x[kWS] | y[kWS] | 2 pad, then strengths
template <typename T> __host__ __device__ constexpr int src_stride() { return sizeof(T) == 4 ? 44 : 34; }
template <typename T, int CG, int WT>
__global__ void __launch_bounds__(kSpreadThreads) k_spread(SpreadArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int CH = chunk_of<T>(), SRC = src_stride<T>();
  constexpr int VW = 16 / sizeof(T);  // elements per 16-byte vector
  constexpr int CGP = (CG + VW - 1) / VW * VW;
  static_assert(kWSrc + CGP <= SRC, "strengths must fit the source stride");
  using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  const int W = WT ? WT : a.W, FW = W + 1, TX = kBin + FW, TZ = kBin + W, TV = TX * TX * TZ;
  T* tile = reinterpret_cast<T*>(smem_raw);  // [c][z][y][x], TX x TX x TZ
  const int c0 = blockIdx.y * CG;
  const int cg = min(CG, a.C - c0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  T* stg = tile + ((CG * TV + VW - 1) / VW) * VW + warp * CH * SRC;  // 16-byte aligned
  for (int i = tid; i < CG * TV; i += kSpreadThreads) tile[i] = T(0);
  __syncthreads();

  const int F2 = FW * FW;
  const T sc2 = T(2) / T(W);
  const int g0 = a.bgrp[blockIdx.x], g1 = a.bgrp[blockIdx.x + 1];
  for (int g = g0 + warp; g < g1; g += kSpreadThreads / 32) {
    const int pk = a.gt0[g];
    const int tx = pk & 15, ty = (pk >> 4) & 15, tz = (pk >> 8) & 15;
    const int s0 = a.gsrc[g], s1 = a.gsrc[g + 1];
    for (int cs = s0; cs < s1; cs += CH) {
      const int ns = min(CH, s1 - cs);
      __syncwarp();
      if (lane < ns) {
        const V4<T> u = a.su[cs + lane];  // distance past the group footprint start
        const long long src = a.sidx[cs + lane];
        T r[SRC];
#pragma unroll
        for (int k = 0; k < 8; ++k) r[k] = (k < W) ? es_kernel((T(k) - u.z) * sc2, a.beta) : T(0);
#pragma unroll
        for (int i = 0; i < kWS; ++i) {
          r[8 + i] = (i < FW) ? es_kernel((T(i) - u.x) * sc2, a.beta) : T(0);
          r[8 + kWS + i] = (i < FW) ? es_kernel((T(i) - u.y) * sc2, a.beta) : T(0);
        }
#pragma unroll
        for (int e = 8 + 2 * kWS; e < kWSrc; ++e) r[e] = T(0);
#pragma unroll
        for (int c = 0; c < SRC - kWSrc; ++c)
          r[kWSrc + c] = (c < cg) ? a.A[(long long)(c0 + c) * a.nq + src] * u.w : T(0);
        V* dst = reinterpret_cast<V*>(stg + lane * SRC);
#pragma unroll
        for (int v = 0; v < SRC / VW; ++v) {
          if constexpr (VW == 4) dst[v] = make_float4(r[4 * v], r[4 * v + 1], r[4 * v + 2], r[4 * v + 3]);
          else dst[v] = make_double2(r[2 * v], r[2 * v + 1]);
        }
      }
      __syncwarp();
      for (int rd = 0; rd * 32 < F2; ++rd) {
        const int p = lane + 32 * rd;
        const bool ok = p < F2;
        const int j = ok ? p / FW : 0, i = ok ? p - j * FW : 0;
        T acc[kMaxW][CG];
#pragma unroll
        for (int k = 0; k < kMaxW; ++k)
#pragma unroll
          for (int c = 0; c < CG; ++c) acc[k][c] = T(0);
        for (int q = 0; q < ns; ++q) {
          const T* wq = stg + q * SRC;
          const T wxy = wq[8 + i] * wq[8 + kWS + j];
          T wz[8], str[CGP];
#pragma unroll
          for (int v = 0; v < 8 / VW; ++v) {
            const V x = reinterpret_cast<const V*>(wq)[v];
            if constexpr (VW == 4) { wz[4 * v] = x.x; wz[4 * v + 1] = x.y; wz[4 * v + 2] = x.z; wz[4 * v + 3] = x.w; }
            else { wz[2 * v] = x.x; wz[2 * v + 1] = x.y; }
          }
#pragma unroll
          for (int v = 0; v < CGP / VW; ++v) {
            const V x = reinterpret_cast<const V*>(wq + kWSrc)[v];
            if constexpr (VW == 4) { str[4 * v] = x.x; str[4 * v + 1] = x.y; str[4 * v + 2] = x.z; str[4 * v + 3] = x.w; }
            else { str[2 * v] = x.x; str[2 * v + 1] = x.y; }
          }
#pragma unroll
          for (int k = 0; k < kMaxW; ++k) {
            if (k < W) {
              const T w = wz[k] * wxy;
#pragma unroll
              for (int c = 0; c < CG; ++c) acc[k][c] += w * str[c];
            }
          }
        }
        if (ok) {
          int addr = (tz * TX + ty + j) * TX + swz<WT>(tx + i, ty + j);
#pragma unroll
          for (int k = 0; k < kMaxW; ++k) {
            if (k < W) {
#pragma unroll
              for (int c = 0; c < CG; ++c)  // channels past cg add their zeros
                atomicAdd(&tile[c * TV + addr], acc[k][c]);
            }
            addr += TX * TX;
          }
        }
      }
    }
  }
  __syncthreads();

  // add the tile to the periodic grid: one warp per tile row
  const int b = a.bid[blockIdx.x];
  const int bx = b % a.nb, by = (b / a.nb) % a.nb, bz = b / (a.nb * a.nb);
  const int nf = a.nf;
  const long long P = (long long)nf * nf * nf;
  const int lx = (bx * kBin - W / 2 + nf) % nf, ly = (by * kBin - W / 2 + nf) % nf,
            lz = (bz * kBin - W / 2 + nf) % nf;
  for (int row = warp; row < cg * TZ * TX; row += kSpreadThreads / 32) {
    const int c = row / (TZ * TX), zy = row - c * TZ * TX, z = zy / TX, y = zy - z * TX;
    int gy = ly + y, gz = lz + z;
    gy -= gy >= nf ? nf : 0;
    gz -= gz >= nf ? nf : 0;
    T* Frow = a.F + (long long)(c0 + c) * P + ((long long)gz * nf + gy) * nf;
    const T* trow = tile + c * TV + zy * TX;
    for (int x = lane; x < TX; x += 32) {
      const T v = trow[swz<WT>(x, y)];
      if (v == T(0)) continue;
      int gx = lx + x;
      gx -= gx >= nf ? nf : 0;
      atomicAdd(&Frow[gx], v);
    }
  }
}

template <typename T> struct InterpArgs {
  const T* F;          // grid, C x nf^3
  const V4<T>* tu;     // targets sorted by group: d per axis
  const int* tidx;     // target -> field point
  const int* tgrp;     // group -> first target (ngroups + 1)
  const int4* tg0;     // group -> first footprint point on the grid (gx, gy, gz)
  T* dst;              // C x nq: out[c][tidx[t]] (diffuse) or scratch[c][t] (step)
  long long nq;
  int nf, W;
  bool scatter;        // write at tidx[t] (true) or at t (false)
  T beta;
};

// One block per target group: the group's W^3 footprint values (C channels
// padded to CP, point-major) are staged in shared memory once; each thread
// evaluates one target from them (all lanes of a warp read the same values:
// broadcast), with its 3W one-dimensional weights in registers.
constexpr int kInterpBlock = 128;
template <typename T, int C> __host__ __device__ constexpr int padded_channels() {
  return C == 1 ? 1 : (sizeof(T) == 4 ? (C + 3) / 4 * 4 : (C + 1) / 2 * 2);
}
template <typename T, int NM, int WT>
__global__ void __launch_bounds__(kInterpBlock) k_interp(InterpArgs<T> a) {
  constexpr int C = NM * NM, CP = padded_channels<T, C>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* fp = reinterpret_cast<T*>(smem_raw);  // [W^3][CP]
  const int W = WT ? WT : a.W, W2 = W * W, W3 = W2 * W, nf = a.nf;
  const long long P = (long long)nf * nf * nf;
  const int g = blockIdx.x;
  const int4 g0 = a.tg0[g];
  for (int e = threadIdx.x; e < CP * W3; e += kInterpBlock) {
    const int c = e / W3, p = e - c * W3;
    T v = T(0);
    if (c < C) {
      const int k = p / W2, r = p - k * W2, j = r / W, i = r - j * W;
      int gx = g0.x + i, gy = g0.y + j, gz = g0.z + k;
      gx -= gx >= nf ? nf : 0;
      gy -= gy >= nf ? nf : 0;
      gz -= gz >= nf ? nf : 0;
      v = __ldg(&a.F[c * P + ((long long)gz * nf + gy) * nf + gx]);
    }
    fp[p * CP + c] = v;
  }
  __syncthreads();
  const int t1 = a.tgrp[g + 1];
  const T sc2 = T(2) / T(W);
  for (int t = a.tgrp[g] + threadIdx.x; t < t1; t += kInterpBlock) {
    const V4<T> u = a.tu[t];
    T wx[kMaxW], wy[kMaxW];
#pragma unroll
    for (int i = 0; i < kMaxW; ++i) {
      wx[i] = (i < W) ? es_kernel((T(i) - u.x) * sc2, a.beta) : T(0);
      wy[i] = (i < W) ? es_kernel((T(i) - u.y) * sc2, a.beta) : T(0);
    }
    T acc[CP];
#pragma unroll
    for (int c = 0; c < CP; ++c) acc[c] = T(0);
    for (int k = 0; k < W; ++k) {
      const T wz = es_kernel((T(k) - u.z) * sc2, a.beta);
      const T* plane = fp + k * W2 * CP;
#pragma unroll
      for (int j = 0; j < kMaxW; ++j) {
        if (j < W) {
          const T wyz = wz * wy[j];
#pragma unroll
          for (int i = 0; i < kMaxW; ++i) {
            if (i < W) {
              const T w = wyz * wx[i];
              const T* pt = plane + (j * W + i) * CP;
              if constexpr (CP % 4 == 0 && sizeof(T) == 4) {
#pragma unroll
                for (int v = 0; v < CP / 4; ++v) {
                  const float4 x = reinterpret_cast<const float4*>(pt)[v];
                  acc[4 * v] += w * x.x;
                  acc[4 * v + 1] += w * x.y;
                  acc[4 * v + 2] += w * x.z;
                  acc[4 * v + 3] += w * x.w;
                }
              } else if constexpr (CP % 2 == 0 && sizeof(T) == 8) {
#pragma unroll
                for (int v = 0; v < CP / 2; ++v) {
                  const double2 x = reinterpret_cast<const double2*>(pt)[v];
                  acc[2 * v] += w * x.x;
                  acc[2 * v + 1] += w * x.y;
                }
              } else {
#pragma unroll
                for (int c = 0; c < CP; ++c) acc[c] += w * pt[c];
              }
            }
          }
        }
      }
    }
    const long long q = a.scatter ? (long long)a.tidx[t] : (long long)t;
#pragma unroll
    for (int c = 0; c < C; ++c) a.dst[c * a.nq + q] = acc[c];
  }
}

template <typename T> struct ProjArgs {
  const T* At;        // C x nq diffused values, sorted target order
  const int* tidx;    // target -> field point
  T* A;               // field, C x nq (read: previous; written: projected)
  SurfStats* st;
  long long nq;
  T fb;
};

// Projection of every target (Lemma 1.1) and the step statistics.
template <typename T, int NM>
__global__ void __launch_bounds__(kProjThreads) k_sproject(ProjArgs<T> a) {
  constexpr int C = NM * NM;
  __shared__ double redd[32];
  __shared__ int redi[32];
  const long long t = (long long)blockIdx.x * kProjThreads + threadIdx.x;
  PointStats<T> ps;
  if (t < a.nq) {
    const long long q = a.tidx[t];
    T m[C], old[C], bb[C], sg;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      m[c] = a.At[c * a.nq + t];
      old[c] = a.A[c * a.nq + q];
    }
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
      a.A[c * a.nq + q] = bb[c];
    }
    ps.maxd = d;
    ps.flips = (det_sign<NM>(old) != sg) ? 1 : 0;
  }
  const double mx = block_max((double)ps.maxd, redd);
  const int fl = block_sum(ps.flips, redi);
  const int nfin = block_sum(ps.nonfinite, redi);
  const int nfb = block_sum(ps.fallback, redi);
  if (threadIdx.x == 0) {
    atomicMax(&a.st->maxd_bits, (unsigned long long)__double_as_longlong(mx));
    if (fl) atomicAdd(&a.st->flips, (unsigned long long)fl);
    if (nfin) atomicAdd(&a.st->nonfinite, (unsigned long long)nfin);
    if (nfb) atomicAdd(&a.st->fallback, (unsigned long long)nfb);
  }
}

// Step statistics of the volume-preserving step: compare the previous field
// with the assigned one, point by point (both in the caller's order).
template <typename T, int NM>
__global__ void __launch_bounds__(kProjThreads) k_sdelta(const T* old, const T* A, long long nq, SurfStats* st) {
  constexpr int C = NM * NM;
  __shared__ double redd[32];
  __shared__ int redi[32];
  const long long q = (long long)blockIdx.x * kProjThreads + threadIdx.x;
  PointStats<T> ps;
  if (q < nq) {
    T o[C], b[C];
    bool fin = true;
    T d = T(0);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      o[c] = old[c * nq + q];
      b[c] = A[c * nq + q];
      fin = fin && isfinite(b[c]);
      d = fmax(d, fabs(b[c] - o[c]));
    }
    ps.maxd = d;
    ps.nonfinite = fin ? 0 : 1;
    ps.flips = (det_sign<NM>(o) != det_sign<NM>(b)) ? 1 : 0;
  }
  const double mx = block_max((double)ps.maxd, redd);
  const int fl = block_sum(ps.flips, redi);
  const int nfin = block_sum(ps.nonfinite, redi);
  if (threadIdx.x == 0) {
    atomicMax(&st->maxd_bits, (unsigned long long)__double_as_longlong(mx));
    if (fl) atomicAdd(&st->flips, (unsigned long long)fl);
    if (nfin) atomicAdd(&st->nonfinite, (unsigned long long)nfin);
  }
}

// Weighted selection of Algorithm 3 (Sec. 7 on surfaces): with points ordered
// by decreasing dE (ascending key, lower index first on equal keys), the
// smallest prefix whose weight reaches the target volume V.  Weights are
// fixed-point integers (the plan scales every w_q so that all of them sum to
// 2^62), so the sums are exact and independent of the summation order.  Twelve
// MSB-first passes over 8-bit digits of the 96-bit (key, index) composite, as
// in the count-based selection, with weight sums per digit instead of counts;
// the result goes into a SelectState for the class assignment (a point takes
// SO(n) iff its (key, index) <= (hi, lo) and the target is positive).
struct WSelect {
  unsigned long long hi;      // key part of the prefix / result
  unsigned int lo;            // index part
  int all;                    // the target exceeds the total weight: select every point
  unsigned long long vrem;    // weight still to reach inside the current prefix
  unsigned long long target;  // V
  unsigned long long hist[256];
};

__device__ __forceinline__ unsigned wdigit(unsigned long long key, unsigned idx, int d) {
  return d < 8 ? (unsigned)((key >> (56 - 8 * d)) & 0xffu) : ((idx >> (24 - 8 * (d - 8))) & 0xffu);
}

__device__ __forceinline__ bool wprefix(unsigned long long key, unsigned idx, unsigned long long hi,
                                        unsigned lo, int d) {
  if (d == 0) return true;
  if (d <= 8) {
    const int sh = 64 - 8 * d;
    return (key >> sh) == (hi >> sh);
  }
  if (key != hi) return false;
  const int sh = 32 - 8 * (d - 8);
  return (idx >> sh) == (lo >> sh);
}

// V = the weight of the points with det A > 0 (the input's own volume).
template <typename T, int NM>
__global__ void __launch_bounds__(256) k_wvolume(const T* A, const unsigned long long* w, long long nq,
                                                 WSelect* ws) {
  constexpr int C = NM * NM;
  __shared__ unsigned long long part[8];
  unsigned long long v = 0;
  for (long long q = blockIdx.x * 256LL + threadIdx.x; q < nq; q += (long long)gridDim.x * 256) {
    T m[C];
#pragma unroll
    for (int c = 0; c < C; ++c) m[c] = A[c * nq + q];
    if (det_sign<NM>(m) > T(0)) v += w[q];
  }
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int i = 0; i < 8; ++i) t += part[i];
    atomicAdd(&ws->target, t);
  }
}

__global__ void k_wselect_init(WSelect* ws, unsigned long long target, int use_given) {
  if (threadIdx.x == 0) {
    if (use_given) ws->target = target;
    ws->hi = 0;
    ws->lo = 0;
    ws->all = 0;
    ws->vrem = ws->target;
  }
  for (int i = threadIdx.x; i < 256; i += blockDim.x) ws->hist[i] = 0;
}

__global__ void __launch_bounds__(256) k_wselect_hist(const unsigned long long* __restrict__ keys,
                                                      const unsigned long long* __restrict__ w, long long nq,
                                                      WSelect* ws, int d) {
  __shared__ unsigned long long h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const unsigned long long hi = ws->hi;
  const unsigned lo = ws->lo;
  const bool active = ws->target > 0 && !ws->all;
  if (active) {
    for (long long x = blockIdx.x * 256LL + threadIdx.x; x < nq; x += (long long)gridDim.x * 256) {
      const unsigned long long key = keys[x];
      if (wprefix(key, (unsigned)x, hi, lo, d)) atomicAdd(&h[wdigit(key, (unsigned)x, d)], w[x]);
    }
  }
  __syncthreads();
  if (active)
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
      if (h[i]) atomicAdd(&ws->hist[i], h[i]);
}

__global__ void k_wselect_pick(WSelect* ws, SelectState* ss, int d) {
  if (threadIdx.x != 0) return;
  if (ws->target > 0 && !ws->all) {
    const unsigned long long v = ws->vrem;
    unsigned long long cum = 0;
    int b = 0;
    for (; b < 256; ++b) {
      if (cum + ws->hist[b] >= v) break;
      cum += ws->hist[b];
    }
    if (b == 256) {  // only on the first pass: V exceeds the total weight
      ws->all = 1;
      ws->hi = ~0ull;
      ws->lo = ~0u;
    } else {
      ws->vrem = v - cum;
      if (d < 8) ws->hi |= ((unsigned long long)b) << (56 - 8 * d);
      else ws->lo |= ((unsigned)b) << (24 - 8 * (d - 8));
    }
  }
  for (int i = 0; i < 256; ++i) ws->hist[i] = 0;
  if (d == 11) {
    ss->hi = ws->hi;
    ss->lo = ws->lo;
    ss->n_plus = ws->target > 0 ? 1 : 0;
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

// Band cells and quadrature points (Algorithm 2, step 1): the cells
// x_g + [0, dx]^3 of the grid dx Z^3 with |i| <= li, |j|, |k| <= lr whose corner
// x_g is in the band, each with p^3 points (the tensor product of the Chebyshev
// nodes cos((2k - 1) pi / (2p)) mapped to [0, dx], with Fejer's first-rule
// weights) and their closest points.  Order: cells (i, j, k) lexicographic, k
// fastest, then the nodes (a, b, c), c fastest.  With any output NULL only the
// count is produced.
template <typename InBand, typename Closest>
mbo_status emit_band(double dx, int p, long long li, long long lr, InBand in_band, Closest closest,
                     double* xq, double* wq, double* xc, int64_t capacity, int64_t* count) {
  std::vector<double> off(p), wc(p);
  for (int k = 0; k < p; ++k) {
    const double th = (2.0 * (k + 1) - 1.0) * M_PI / (2.0 * p);
    double s = 0.0;
    for (int j = 1; j <= p / 2; ++j) s += std::cos(2.0 * j * th) / (4.0 * j * j - 1.0);
    off[k] = dx * (1.0 + std::cos(th)) / 2.0;
    wc[k] = (2.0 / p) * (1.0 - 2.0 * s) * dx / 2.0;
  }
  const long long per = (long long)p * p * p;
  int64_t n = 0;
  const bool fill = xq && wq && xc;
  for (long long i = -li; i <= li; ++i)
    for (long long j = -lr; j <= lr; ++j)
      for (long long k = -lr; k <= lr; ++k) {
        const double gx = dx * i, gy = dx * j, gz = dx * k;
        if (!in_band(gx, gy, gz)) continue;
        if (fill && n + per <= capacity) {
          for (int a = 0; a < p; ++a)
            for (int b = 0; b < p; ++b)
              for (int c = 0; c < p; ++c) {
                const int64_t q = n + ((int64_t)a * p + b) * p + c;
                xq[3 * q] = gx + off[a];
                xq[3 * q + 1] = gy + off[b];
                xq[3 * q + 2] = gz + off[c];
                wq[q] = wc[a] * wc[b] * wc[c];
                closest(xq[3 * q], xq[3 * q + 1], xq[3 * q + 2], xc + 3 * q);
              }
        }
        n += per;
      }
  *count = n;
  if (fill && n > capacity) return MBO_ERR_INVALID_ARG;
  return MBO_OK;
}

// Generating curve of the peanut surface (Sec. 6.3), t in [-1, 1]: x = 3t - t^3
// and rho = sqrt((1 + x^2)(4 - x^2)) / 2, written as (1 - t^2) sqrt((1 + x^2)(4 - t^2)) / 2
// (4 - x^2 = (1 - t^2)^2 (4 - t^2)), which stays real to the ends.
void peanut_curve(double t, double& x, double& rho) {
  x = 3.0 * t - t * t * t;
  rho = 0.5 * (1.0 - t * t) * std::sqrt((1.0 + x * x) * (4.0 - t * t));
}

// Closest point c on the peanut surface to (x, y, z) and its distance.  The
// surface is one of revolution about the x axis, so the closest point is that of
// (x, |(y, z)|) on the generating curve, turned into the point's meridian (the
// +y meridian on the axis): a scan of 257 values of t, then a golden-section
// search between the neighbours of the nearest one.
double peanut_closest(double px, double py, double pz, double* c) {
  const double r = std::sqrt(py * py + pz * pz);
  auto D = [&](double t) {
    double x, rho;
    peanut_curve(t, x, rho);
    return (x - px) * (x - px) + (rho - r) * (rho - r);
  };
  constexpr int kScan = 257;
  int best = 0;
  double dbest = D(-1.0);
  for (int i = 1; i < kScan; ++i) {
    const double d = D(-1.0 + 2.0 * i / (kScan - 1));
    if (d < dbest) {
      dbest = d;
      best = i;
    }
  }
  const double step = 2.0 / (kScan - 1);
  double lo = std::max(-1.0, -1.0 + step * (best - 1)), hi = std::min(1.0, -1.0 + step * (best + 1));
  const double g = 0.5 * (std::sqrt(5.0) - 1.0);
  double a = hi - g * (hi - lo), b = lo + g * (hi - lo), fa = D(a), fb = D(b);
  for (int it = 0; it < 80; ++it) {
    if (fa < fb) {
      hi = b;
      b = a;
      fb = fa;
      a = hi - g * (hi - lo);
      fa = D(a);
    } else {
      lo = a;
      a = b;
      fa = fb;
      b = lo + g * (hi - lo);
      fb = D(b);
    }
  }
  const double t = 0.5 * (lo + hi);
  double x, rho;
  peanut_curve(t, x, rho);
  const double uy = r > 0 ? py / r : 1.0, uz = r > 0 ? pz / r : 0.0;
  c[0] = x;
  c[1] = rho * uy;
  c[2] = rho * uz;
  return std::sqrt(D(t));
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
  int nb = 0;        // bins per axis
  int nbins = 0;     // non-empty source bins
  int sgroups = 0;   // source groups
  int tgroups = 0;   // target groups
  int cg = 1, chgroups = 1;  // channels per spreading block, channel groups
  size_t tile_bytes = 0;
  mbo_handle fine = nullptr;  // 3-D FFT diffusion on the nf^3 grid
  void* F = nullptr;          // grid, C x nf^3
  void* At = nullptr;         // diffused values in sorted target order, C x nq
  // volume-preserving step (allocated on first use)
  void* Au = nullptr;                      // diffused values in the caller's order, C x nq
  unsigned long long* vkeys = nullptr;     // one selection key per point
  SelectState* vss = nullptr;
  WSelect* vws = nullptr;
  unsigned long long* vw = nullptr;        // fixed-point weights (caller's order), sum 2^62
  double wscale = 0;                       // fixed-point units per unit of w_q
  std::vector<double> hw;                  // the weights w_q (host copy)
  void* su = nullptr;         // V4<T> sources
  int* sidx = nullptr;
  int* gsrc = nullptr;
  int* gt0 = nullptr;
  int* bgrp = nullptr;
  int* bid = nullptr;
  void* tu = nullptr;         // V4<T> targets
  int* tidx = nullptr;
  int* tgrp = nullptr;
  int4* tg0 = nullptr;
  SurfStats* st = nullptr;
  SurfStats* h_st = nullptr;  // pinned
  size_t bytes = 0;
  // per-pass timing (mbo_surface_profile_*)
  bool prof = false;
  struct Pending { int pass; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> ev_free;
  double prof_ms[MBO_SURFACE_PROFILE_PASSES] = {0};
  long long prof_n[MBO_SURFACE_PROFILE_PASSES] = {0};
  char err[512] = {0};
};

namespace {

cudaEvent_t take_event(mbo_surface_ctx* s) {
  if (!s->ev_free.empty()) {
    cudaEvent_t e = s->ev_free.back();
    s->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Run f (a launch sequence on stream st); when profiling, bracket it with events.
template <typename Fn> cudaError_t timed(mbo_surface_ctx* s, int pass, cudaStream_t st, Fn&& f) {
  if (!s->prof) return f();
  cudaEvent_t a = take_event(s), b = take_event(s);
  cudaEventRecord(a, st);
  const cudaError_t e = f();
  cudaEventRecord(b, st);
  s->pending.push_back({pass, a, b});
  return e;
}

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

// Shared bytes of a spreading block: the tile and the per-warp staging.
size_t spread_smem(int cg, size_t elem, size_t tv) {
  const size_t vw = 16 / elem;
  const size_t chunk = elem == 4 ? chunk_of<float>() : chunk_of<double>();
  const size_t stride = elem == 4 ? src_stride<float>() : src_stride<double>();
  return (((size_t)cg * tv + vw - 1) / vw * vw + (size_t)(kSpreadThreads / 32) * chunk * stride) * elem;
}

// Channels per spreading block for n*n channels: the largest instantiated
// group that fits in `limit` shared bytes (0 if none fits).
int spread_cg(int C, size_t elem, size_t tv, size_t limit) {
  const int cand[] = {9, 8, 4, 3, 1};
  for (int cg : cand) {
    if (cg > C || (elem == 8 && cg > 4)) continue;  // FP64: at most 4 (registers)
    if (spread_smem(cg, elem, tv) <= limit) return cg;
  }
  return 0;
}

template <typename T, int CG> cudaError_t spread_run(const SpreadArgs<T>& a, dim3 grid, size_t smem,
                                                     cudaStream_t st) {
  auto k = a.W == 7 ? k_spread<T, CG, 7> : k_spread<T, CG, 0>;
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
  a.gsrc = s->gsrc;
  a.gt0 = s->gt0;
  a.bgrp = s->bgrp;
  a.bid = s->bid;
  a.F = static_cast<T*>(s->F);
  a.nq = s->nq;
  a.C = s->C;
  a.nf = s->prm.nf;
  a.nb = s->nb;
  a.W = s->prm.width;
  a.beta = (T)s->prm.beta;
  const dim3 grid(s->nbins, s->chgroups);
  switch (s->cg) {
    case 1: return spread_run<T, 1>(a, grid, s->tile_bytes, st);
    case 3: return spread_run<T, 3>(a, grid, s->tile_bytes, st);
    case 4: return spread_run<T, 4>(a, grid, s->tile_bytes, st);
    default: break;
  }
  if constexpr (sizeof(T) == 4) {  // FP64 groups stop at 4 channels (registers)
    if (s->cg == 8) return spread_run<T, 8>(a, grid, s->tile_bytes, st);
    if (s->cg == 9) return spread_run<T, 9>(a, grid, s->tile_bytes, st);
  }
  return cudaErrorInvalidValue;
}

template <typename T, int NM> cudaError_t interp_run(const InterpArgs<T>& a, int groups, size_t smem,
                                                      cudaStream_t st) {
  auto k = a.W == 7 ? k_interp<T, NM, 7> : k_interp<T, NM, 0>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k<<<groups, kInterpBlock, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T> cudaError_t launch_interp(mbo_surface_ctx* s, void* dst, bool scatter, cudaStream_t st) {
  InterpArgs<T> a;
  a.F = static_cast<const T*>(s->F);
  a.tu = static_cast<const V4<T>*>(s->tu);
  a.tidx = s->tidx;
  a.tgrp = s->tgrp;
  a.tg0 = s->tg0;
  a.dst = static_cast<T*>(dst);
  a.nq = s->nq;
  a.nf = s->prm.nf;
  a.W = s->prm.width;
  a.scatter = scatter;
  a.beta = (T)s->prm.beta;
  const int W3 = s->prm.width * s->prm.width * s->prm.width;
  const int CP = s->C == 1 ? 1 : (sizeof(T) == 4 ? (s->C + 3) / 4 * 4 : (s->C + 1) / 2 * 2);
  const size_t smem = (size_t)W3 * CP * sizeof(T);
  switch (s->n) {
    case 1: return interp_run<T, 1>(a, s->tgroups, smem, st);
    case 2: return interp_run<T, 2>(a, s->tgroups, smem, st);
    case 3: return interp_run<T, 3>(a, s->tgroups, smem, st);
    default: return interp_run<T, 4>(a, s->tgroups, smem, st);
  }
}

template <typename T> cudaError_t launch_project(mbo_surface_ctx* s, void* A, cudaStream_t st) {
  ProjArgs<T> a;
  a.At = static_cast<const T*>(s->At);
  a.tidx = s->tidx;
  a.A = static_cast<T*>(A);
  a.st = s->st;
  a.nq = s->nq;
  a.fb = T(0);
  const unsigned blocks = (unsigned)((s->nq + kProjThreads - 1) / kProjThreads);
  switch (s->n) {
    case 1: k_sproject<T, 1><<<blocks, kProjThreads, 0, st>>>(a); break;
    case 2: k_sproject<T, 2><<<blocks, kProjThreads, 0, st>>>(a); break;
    case 3: k_sproject<T, 3><<<blocks, kProjThreads, 0, st>>>(a); break;
    default: k_sproject<T, 4><<<blocks, kProjThreads, 0, st>>>(a); break;
  }
  return cudaGetLastError();
}

mbo_status surface_diffusion(mbo_surface_ctx* s, const void* A, void* dst, bool scatter, cudaStream_t st) {
  const long long P = (long long)s->prm.nf * s->prm.nf * s->prm.nf;
  const size_t elem = s->dtype == MBO_F32 ? 4 : 8;
  SCK(cudaMemsetAsync(s->F, 0, (size_t)s->C * P * elem, st));
  SCK(timed(s, 0, st, [&] {
    return s->dtype == MBO_F32 ? launch_spread<float>(s, A, st) : launch_spread<double>(s, A, st);
  }));
  mbo_status rc = MBO_OK;
  timed(s, 1, st, [&] {
    rc = mbo_diffuse(s->fine, s->F, s->F, st);
    return cudaSuccess;
  });
  if (rc != MBO_OK) return sfail(s, rc, "grid diffusion: %s", mbo_last_error(s->fine));
  SCK(timed(s, 2, st, [&] {
    return s->dtype == MBO_F32 ? launch_interp<float>(s, dst, scatter, st)
                               : launch_interp<double>(s, dst, scatter, st);
  }));
  return MBO_OK;
}

template <typename T> void upload_points(const std::vector<V4<double>>& in, void* dst) {
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
  const long long lim = (long long)std::ceil((radius + wb) / dx) + 1;
  auto in_band = [&](double x, double y, double z) {
    return std::fabs(std::sqrt(x * x + y * y + z * z) - radius) < wb;
  };
  auto closest = [&](double x, double y, double z, double* c) {
    const double r = std::sqrt(x * x + y * y + z * z);
    if (r > 0) {
      c[0] = radius * x / r;
      c[1] = radius * y / r;
      c[2] = radius * z / r;
    } else {
      c[0] = 0.0;
      c[1] = 0.0;
      c[2] = radius;
    }
  };
  return emit_band(dx, p, lim, lim, in_band, closest, xq, wq, xc, capacity, count);
}

mbo_status mbo_surface_peanut_band(double dx, double wb, int p, double* xq, double* wq, double* xc,
                                   int64_t capacity, int64_t* count) {
  if (!(dx > 0) || !(wb > 0) || p < 1 || p > 16 || !count) return MBO_ERR_INVALID_ARG;
  double rho_max = 0.0;
  for (int i = 0; i <= 4096; ++i) {
    double x, rho;
    peanut_curve(-1.0 + 2.0 * i / 4096, x, rho);
    rho_max = std::max(rho_max, rho);
  }
  const long long lx = (long long)std::ceil((2.0 + wb) / dx) + 1;
  const long long lr = (long long)std::ceil((rho_max + wb) / dx) + 1;
  auto in_band = [&](double x, double y, double z) {
    double c[3];
    return peanut_closest(x, y, z, c) < wb;
  };
  auto closest = [&](double x, double y, double z, double* c) { peanut_closest(x, y, z, c); };
  return emit_band(dx, p, lx, lr, in_band, closest, xq, wq, xc, capacity, count);
}

mbo_status mbo_surface_destroy(mbo_surface s) {
  if (!s) return MBO_ERR_INVALID_ARG;
  int prev = -1;
  if (cudaGetDevice(&prev) == cudaSuccess && prev != s->dev) cudaSetDevice(s->dev);
  else prev = -1;
  cudaDeviceSynchronize();
  if (s->fine) mbo_destroy(s->fine);
  void* bufs[] = {s->F, s->At, s->su, s->sidx, s->gsrc, s->gt0, s->bgrp, s->bid,
                  s->tu, s->tidx, s->tgrp, s->tg0, s->st, s->Au, s->vkeys, s->vss, s->vws, s->vw};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (s->h_st) cudaFreeHost(s->h_st);
  for (auto& p : s->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (cudaEvent_t e : s->ev_free) cudaEventDestroy(e);
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
  s->hw.assign(wq, wq + nq);
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
  W = std::max(kMinW, std::min(W, kMaxW));
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

  // grid coordinates u = (h (x - centre) + pi) nf / (2 pi); the footprint of a
  // point starts at g = ceil(u - W/2) on each axis (W points), and d = u - g
  const double sc = (double)nf / (2.0 * M_PI);
  auto grid_coord = [&](const double* x, double* u) {
    for (int a = 0; a < 3; ++a) {
      const double v = (prm.h * (x[a] - prm.center[a]) + M_PI) * sc;
      u[a] = std::min(std::max(v, 0.0), std::nextafter((double)nf, 0.0));
    }
  };
  // sources: key (bin, footprint start in the bin tile); targets: footprint start
  std::vector<long long> skey(nq), tkey(nq);
  std::vector<V4<double>> sd(nq), td(nq);
  std::vector<int> sgx(3 * nq);
  for (int64_t i = 0; i < nq; ++i) {
    double u[3];
    int b[3], t0[3], g[3];
    grid_coord(xq + 3 * i, u);
    for (int a = 0; a < 3; ++a) {
      b[a] = std::min((int)(u[a] / kBin), nb - 1);
      // footprint start relative to the tile origin b kBin - W/2, kept in [0, kBin];
      // the group start rounds it down to even in x and y
      t0[a] = (int)std::ceil(u[a] - 0.5 * W) - (b[a] * kBin - W / 2);
      t0[a] = std::min(std::max(t0[a], 0), kBin);
      if (a < 2) t0[a] &= ~1;
      g[a] = b[a] * kBin - W / 2 + t0[a];
    }
    const long long bin = ((long long)b[2] * nb + b[1]) * nb + b[0];
    skey[i] = bin * 4096 + (t0[2] << 8 | t0[1] << 4 | t0[0]);
    sd[i] = V4<double>{u[0] - g[0], u[1] - g[1], u[2] - g[2], wq[i]};
    grid_coord(xc + 3 * i, u);
    for (int a = 0; a < 3; ++a) g[a] = (int)std::ceil(u[a] - 0.5 * W);
    // wrapped start on the periodic grid (u >= 0, so g >= -W/2)
    const int gx = (g[0] + nf) % nf, gy = (g[1] + nf) % nf, gz = (g[2] + nf) % nf;
    tkey[i] = ((long long)gz * nf + gy) * nf + gx;
    td[i] = V4<double>{u[0] - g[0], u[1] - g[1], u[2] - g[2], 0.0};
  }
  std::vector<int> sperm(nq), tperm(nq);
  std::iota(sperm.begin(), sperm.end(), 0);
  std::iota(tperm.begin(), tperm.end(), 0);
  std::stable_sort(sperm.begin(), sperm.end(), [&](int x, int y) { return skey[x] < skey[y]; });
  std::stable_sort(tperm.begin(), tperm.end(), [&](int x, int y) { return tkey[x] < tkey[y]; });
  std::vector<int> gsrc, gt0, bgrp, bid, tgrp;
  std::vector<int4> tg0;
  std::vector<V4<double>> sds(nq), tds(nq);
  for (int64_t r = 0; r < nq; ++r) {
    const int i = sperm[r];
    sds[r] = sd[i];
    if (r == 0 || skey[i] != skey[sperm[r - 1]]) {
      const long long bin = skey[i] / 4096;
      if (r == 0 || bin != skey[sperm[r - 1]] / 4096) {
        bid.push_back((int)bin);
        bgrp.push_back((int)gsrc.size());
      }
      gsrc.push_back((int)r);
      gt0.push_back((int)(skey[i] % 4096));
    }
    const int j = tperm[r];
    tds[r] = td[j];
    if (r == 0 || tkey[j] != tkey[tperm[r - 1]]) {
      tgrp.push_back((int)r);
      const long long k = tkey[j];
      tg0.push_back(make_int4((int)(k % nf), (int)((k / nf) % nf), (int)(k / ((long long)nf * nf)), 0));
    }
  }
  gsrc.push_back((int)nq);
  tgrp.push_back((int)nq);
  bgrp.push_back((int)gt0.size());
  s->nbins = (int)bid.size();
  s->sgroups = (int)gt0.size();
  s->tgroups = (int)tg0.size();
  prm.bins = s->nbins;

  // channel groups of the spreading tile
  const size_t elem = dtype == MBO_F32 ? 4 : 8;
  const size_t tv = (size_t)(kBin + W + 1) * (kBin + W + 1) * (kBin + W);
  int maxsm = 0;
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->dev);
  s->cg = spread_cg(s->C, elem, tv, (size_t)maxsm);
  s->chgroups = s->cg ? (s->C + s->cg - 1) / s->cg : 0;
  s->tile_bytes = spread_smem(s->cg, elem, tv);
  if (s->cg == 0) {
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
    if (cudaMalloc(p, std::max<size_t>(b, 16)) != cudaSuccess) return false;
    s->bytes += b;
    return true;
  };
  const size_t v4 = dtype == MBO_F32 ? sizeof(V4<float>) : sizeof(V4<double>);
  if (!alloc(&s->F, (size_t)s->C * P * elem) || !alloc(&s->At, (size_t)s->C * nq * elem) ||
      !alloc(&s->su, nq * v4) || !alloc((void**)&s->sidx, nq * sizeof(int)) ||
      !alloc((void**)&s->gsrc, gsrc.size() * sizeof(int)) || !alloc((void**)&s->gt0, gt0.size() * sizeof(int)) ||
      !alloc((void**)&s->bgrp, bgrp.size() * sizeof(int)) || !alloc((void**)&s->bid, bid.size() * sizeof(int)) ||
      !alloc(&s->tu, nq * v4) || !alloc((void**)&s->tidx, nq * sizeof(int)) ||
      !alloc((void**)&s->tgrp, tgrp.size() * sizeof(int)) || !alloc((void**)&s->tg0, tg0.size() * sizeof(int4)) ||
      !alloc((void**)&s->st, sizeof(SurfStats)) ||
      cudaMallocHost((void**)&s->h_st, sizeof(SurfStats)) != cudaSuccess) {
    mbo_surface_destroy(s);
    return MBO_ERR_OOM;
  }
  if (dtype == MBO_F32) {
    upload_points<float>(sds, s->su);
    upload_points<float>(tds, s->tu);
  } else {
    upload_points<double>(sds, s->su);
    upload_points<double>(tds, s->tu);
  }
  cudaMemcpy(s->sidx, sperm.data(), nq * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(s->gsrc, gsrc.data(), gsrc.size() * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(s->gt0, gt0.data(), gt0.size() * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(s->bgrp, bgrp.data(), bgrp.size() * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(s->bid, bid.data(), bid.size() * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(s->tidx, tperm.data(), nq * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(s->tgrp, tgrp.data(), tgrp.size() * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(s->tg0, tg0.data(), tg0.size() * sizeof(int4), cudaMemcpyHostToDevice);
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
  return surface_diffusion(s, A, A_tilde, true, static_cast<cudaStream_t>(stream));
}

mbo_status mbo_surface_step(mbo_surface s, void* A, mbo_stats* stats, void* stream) {
  if (!s || !A || ((uintptr_t)A & 15)) return MBO_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  mbo_status rc = surface_diffusion(s, A, s->At, false, st);
  if (rc != MBO_OK) return rc;
  SCK(cudaMemsetAsync(s->st, 0, sizeof(SurfStats), st));
  SCK(timed(s, 3, st, [&] {
    return s->dtype == MBO_F32 ? launch_project<float>(s, A, st) : launch_project<double>(s, A, st);
  }));
  if (stats) {
    SCK(cudaMemcpyAsync(s->h_st, s->st, sizeof(SurfStats), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    double md;
    std::memcpy(&md, &s->h_st->maxd_bits, sizeof(md));
    stats->energy = NAN;
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

mbo_status mbo_surface_step_volume(mbo_surface s, void* A, double volume, mbo_stats* stats, void* stream) {
  if (!s || !A || ((uintptr_t)A & 15) || std::isnan(volume)) return MBO_ERR_INVALID_ARG;
  if (s->n > 3) return sfail(s, MBO_ERR_UNSUPPORTED_SIZE, "%s", "the volume-preserving step supports n <= 3");
  const size_t elem = s->dtype == MBO_F32 ? 4 : 8;
  const size_t fbytes = (size_t)s->C * (size_t)s->nq * elem;
  if (!s->Au) {
    // fixed-point weights: w_q scaled so that all of them sum to 2^62
    long double tot = 0;
    for (double w : s->hw) {
      if (!(w >= 0)) return sfail(s, MBO_ERR_INVALID_ARG, "%s", "the volume step needs weights w_q >= 0");
      tot += w;
    }
    if (!(tot > 0)) return sfail(s, MBO_ERR_INVALID_ARG, "%s", "the volume step needs a positive total weight");
    s->wscale = (double)(std::ldexp(1.0L, 62) / tot);
    std::vector<unsigned long long> wf(s->nq);
    for (long long q = 0; q < s->nq; ++q) wf[q] = (unsigned long long)((long double)s->hw[q] * s->wscale);
    // all buffers or none: a failed call leaves the plan as it was
    void* au = nullptr;
    void* keys = nullptr;
    void* ss = nullptr;
    void* ws = nullptr;
    void* w = nullptr;
    cudaError_t e = cudaMalloc(&au, fbytes);
    if (e == cudaSuccess) e = cudaMalloc(&keys, (size_t)s->nq * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&ss, sizeof(SelectState));
    if (e == cudaSuccess) e = cudaMalloc(&ws, sizeof(WSelect));
    if (e == cudaSuccess) e = cudaMalloc(&w, (size_t)s->nq * sizeof(unsigned long long));
    if (e == cudaSuccess)
      e = cudaMemcpy(w, wf.data(), (size_t)s->nq * sizeof(unsigned long long), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      void* bufs[] = {au, keys, ss, ws, w};
      for (void* b : bufs)
        if (b) cudaFree(b);
      return sfail(s, e == cudaErrorMemoryAllocation ? MBO_ERR_OOM : MBO_ERR_CUDA, "%s", cudaGetErrorString(e));
    }
    s->Au = au;
    s->vkeys = static_cast<unsigned long long*>(keys);
    s->vss = static_cast<SelectState*>(ss);
    s->vws = static_cast<WSelect*>(ws);
    s->vw = static_cast<unsigned long long*>(w);
    s->bytes += fbytes + (size_t)s->nq * 16 + sizeof(SelectState) + sizeof(WSelect);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the diffused field in the caller's order; the previous field kept for the statistics
  mbo_status rc = surface_diffusion(s, A, s->Au, true, st);
  if (rc != MBO_OK) return rc;
  SCK(cudaMemcpyAsync(s->At, A, fbytes, cudaMemcpyDeviceToDevice, st));
  // dE keys (the flat-torus volume step's kernels, on the nq points), the
  // weighted selection of Algorithm 3, class assignment
  Geom g{};
  g.P = s->nq;
  g.n = s->n;
  g.C = s->C;
  const StatsPtrs none{};
  const int blocks = (int)std::min<long long>((s->nq + 255) / 256, 152 * 16);
  auto vol = [&](int which) {
    return s->dtype == MBO_F32
               ? launch_volume<float>(which, g, static_cast<const float*>(s->Au), static_cast<float*>(A),
                                      s->vkeys, s->vss, none, 0.0, blocks, st)
               : launch_volume<double>(which, g, static_cast<const double*>(s->Au), static_cast<double*>(A),
                                       s->vkeys, s->vss, none, 0.0, blocks, st);
  };
  SCK(vol(0));
  if (volume < 0) {
    SCK(cudaMemsetAsync(&s->vws->target, 0, sizeof(unsigned long long), st));
#define MBO_WVOL(T, NM)                                                                              \
  k_wvolume<T, NM><<<blocks, 256, 0, st>>>(static_cast<const T*>(A), s->vw, s->nq, s->vws)
    if (s->dtype == MBO_F32) {
      if (s->n == 1) MBO_WVOL(float, 1); else if (s->n == 2) MBO_WVOL(float, 2); else MBO_WVOL(float, 3);
    } else {
      if (s->n == 1) MBO_WVOL(double, 1); else if (s->n == 2) MBO_WVOL(double, 2); else MBO_WVOL(double, 3);
    }
#undef MBO_WVOL
    k_wselect_init<<<1, 256, 0, st>>>(s->vws, 0, 0);
  } else {
    const long double t = std::min((long double)volume * s->wscale, std::ldexp(1.0L, 63));
    k_wselect_init<<<1, 256, 0, st>>>(s->vws, (unsigned long long)std::llround((double)t), 1);
  }
  for (int d = 0; d < 12; ++d) {
    k_wselect_hist<<<blocks, 256, 0, st>>>(s->vkeys, s->vw, s->nq, s->vws, d);
    k_wselect_pick<<<1, 32, 0, st>>>(s->vws, s->vss, d);
  }
  SCK(cudaGetLastError());
  SCK(vol(2));
  SCK(cudaMemsetAsync(s->st, 0, sizeof(SurfStats), st));
  const unsigned pb = (unsigned)((s->nq + kProjThreads - 1) / kProjThreads);
#define MBO_SDELTA(T, NM)                                                                   \
  k_sdelta<T, NM><<<pb, kProjThreads, 0, st>>>(static_cast<const T*>(s->At), static_cast<const T*>(A), s->nq, s->st)
  if (s->dtype == MBO_F32) {
    if (s->n == 1) MBO_SDELTA(float, 1); else if (s->n == 2) MBO_SDELTA(float, 2); else MBO_SDELTA(float, 3);
  } else {
    if (s->n == 1) MBO_SDELTA(double, 1); else if (s->n == 2) MBO_SDELTA(double, 2); else MBO_SDELTA(double, 3);
  }
#undef MBO_SDELTA
  SCK(cudaGetLastError());
  if (stats) {
    SCK(cudaMemcpyAsync(s->h_st, s->st, sizeof(SurfStats), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
    double md;
    std::memcpy(&md, &s->h_st->maxd_bits, sizeof(md));
    stats->energy = NAN;
    stats->max_delta = md;
    stats->det_flips = (int64_t)s->h_st->flips;
    stats->fallback_points = 0;
    stats->nonfinite = (int64_t)s->h_st->nonfinite;
    if (stats->nonfinite) {
      snprintf(s->err, sizeof(s->err), "non-finite values in the assigned field");
      return MBO_ERR_NUMERIC;
    }
  }
  return MBO_OK;
}

mbo_status mbo_surface_profile_enable(mbo_surface s, int enable) {
  if (!s) return MBO_ERR_INVALID_ARG;
  for (auto& p : s->pending) {
    cudaEventSynchronize(p.b);
    s->ev_free.push_back(p.a);
    s->ev_free.push_back(p.b);
  }
  s->pending.clear();
  for (int i = 0; i < MBO_SURFACE_PROFILE_PASSES; ++i) {
    s->prof_ms[i] = 0;
    s->prof_n[i] = 0;
  }
  s->prof = enable != 0;
  return MBO_OK;
}

mbo_status mbo_surface_profile_read(mbo_surface s, double* ms, int64_t* launches, int npass) {
  if (!s || npass < 0) return MBO_ERR_INVALID_ARG;
  for (auto& p : s->pending) {
    SCK(cudaEventSynchronize(p.b));
    float t = 0.f;
    SCK(cudaEventElapsedTime(&t, p.a, p.b));
    s->prof_ms[p.pass] += t;
    s->prof_n[p.pass] += 1;
    s->ev_free.push_back(p.a);
    s->ev_free.push_back(p.b);
  }
  s->pending.clear();
  for (int i = 0; i < npass && i < MBO_SURFACE_PROFILE_PASSES; ++i) {
    if (ms) ms[i] = s->prof_ms[i];
    if (launches) launches[i] = s->prof_n[i];
  }
  return MBO_OK;
}

int64_t mbo_surface_workspace_bytes(mbo_surface s) {
  if (!s) return -1;
  return (int64_t)s->bytes + (s->fine ? mbo_workspace_bytes(s->fine) : 0);
}

const char* mbo_surface_last_error(mbo_surface s) { return s ? s->err : "null plan"; }

}  // extern "C"
