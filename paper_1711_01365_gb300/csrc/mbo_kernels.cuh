// Kernels of the flat-torus MBO step (Algorithm 1 of Osting & Wang,
// arXiv:1711.01365) and their launchers.  Instantiated per element type in
// k_f32.cu and k_f64.cu.
//
// Data layout in HBM
//   field A      planar: channel c = i*n + j, P values each, row-major (z, y, x)
//   workspace W  Q = ceil(n*n/2) complex planes of P points; plane q packs
//                channels 2q (real part) and 2q+1 (imaginary part).  Because
//                the heat multiplier is real and even, the packed transform of
//                two real channels diffuses both at once (Sec. 5.1 applies the
//                same convolution "entry by entry").
//
// Transforms along each axis are in place in shared memory: forward DIF
// (spectrum left digit-reversed along that axis), inverse DIT.
// Passes of one step (steady state, 2-D):
//   k_axis<FGI>   along y: forward DFT, x g(k)/P (Sec. 5.1), energy partials
//                 (Sec. 4 functional, Parseval form), inverse DFT
//   k_row<INV_PROJECT_FWD> along x: inverse DFT, per-point polar factor
//                 (Lemma 1.1), step statistics, then the forward x-DFT of the
//                 new field for the next step
// 3-D adds k_axis<FWD> and k_axis<INV> along y around the z pass.
#pragma once
#include "mbo_dev.cuh"

namespace mbo {

// Statistics of the points a thread projected.
template <typename R> struct PointStats {
  R maxd = R(0);
  R defect = R(0);
  int flips = 0;
  int nonfinite = 0;
  int fallback = 0;
};

// Out-of-line forms of the rarely taken projections (quaternion form, FP64
// re-projection): their code stays out of the hot loop's instruction stream.
// Matrices pass by value so that the callers' arrays stay in registers.
template <int NM> struct MatV { float v[NM * NM]; };
template <int NM> struct ProjV {
  float b[NM * NM];
  float sg;
  float gap;
};

// Points the fixed FP32 n = 3 schedule did not settle: the convergence-tested
// iteration, continued from the current iterate.
static __device__ __noinline__ ProjV<3> newton_cold(MatV<3> x) {
  ProjV<3> r;
  float est = 0.f;
  r.sg = polar_newton<3, 10, 2>(x.v, r.b, est, 0.f, 0.f);
  r.gap = est;
  return r;
}

template <int NM> __device__ __noinline__ ProjV<NM> quat_cold(MatV<NM> m, float sg) {
  ProjV<NM> r;
  r.sg = sg;
  r.gap = polar3_quat(m.v, sg, r.b);
  return r;
}

template <int NM> __device__ __noinline__ ProjV<NM> f64_cold(MatV<NM> m) {
  constexpr int C = NM * NM;
  double md[C], bd[C], sd;
#pragma unroll
  for (int c = 0; c < C; ++c) md[c] = (double)m.v[c];
  ProjV<NM> r;
  r.sg = (float)polar_f64<NM>(md, bd, sd);
#pragma unroll
  for (int c = 0; c < C; ++c) r.b[c] = (float)bd[c];
  r.gap = 0.f;
  return r;
}

// The quaternion projection's accuracy bound (s2 + s3) / |m|_F >= kQuatGap
// keeps its error (about 4e-7 / ((s2 + s3) / s1) in FP32) well inside the
// FP32 step tolerance.
constexpr float kQuatGap = 0.05f;

// Project one point in the element type R.  Returns false when the point
// must be re-projected in FP64 instead.  FP32, n = 3: the scaled Newton
// iteration for points whose smallest singular value is at least fb (the
// configured threshold) and not small to single precision; below that the
// quaternion form, whose error grows with 1 / (s2 + s3) instead of 1 / s3;
// FP64 only where s2 + s3 is small too.  FP32, n = 4: the same Newton
// iteration, FP64 below the limit.  FP32, n = 2: points whose smallest
// singular value is below fb.  FP64 elements are always projected here.
template <int NM, typename R>
__device__ __forceinline__ bool project_point(const R* m, R* b, R& sg, R fb) {
  if constexpr (sizeof(R) == 8) {
    double sm;
    sg = polar_f64<NM>(m, b, sm);
    return true;
  } else if constexpr (NM >= 3) {
    float nx = 0.f;
#pragma unroll
    for (int k = 0; k < NM * NM; ++k) nx += m[k] * m[k];
    float est = 0.f;
    const float lim = fmaxf(fb, 1e-6f * sqrtf(nx));
    // |cof m|_F > 1e-5 |m|_F^(n-1): above the FP32 rounding error of cof
    const float cf = NM == 3 ? nx * nx : nx * nx * nx;
    if constexpr (NM == 3) {
      bool done;
      sg = polar3_fixed(m, b, est, lim, 1e-10f * cf, done);
      if (est > lim && !done) {
        MatV<3> xv;
#pragma unroll
        for (int k = 0; k < 9; ++k) xv.v[k] = b[k];
        const ProjV<3> r = newton_cold(xv);
#pragma unroll
        for (int k = 0; k < 9; ++k) b[k] = r.b[k];
        sg = r.sg;
        if (!(fabsf(b[0]) < 1e30f)) est = 0.f;
      }
    } else {
      sg = polar_newton<NM, 10, 2>(m, b, est, lim, 1e-10f * cf);
    }
    if (est > lim) return true;
    if constexpr (NM == 3) {
      MatV<3> mv;
#pragma unroll
      for (int k = 0; k < 9; ++k) mv.v[k] = m[k];
      const ProjV<3> r = quat_cold<3>(mv, sg);
#pragma unroll
      for (int k = 0; k < 9; ++k) b[k] = r.b[k];
      return r.gap >= kQuatGap;
    } else {
      return false;
    }
  } else {
    float sm;
    sg = polar<NM>(m, b, sm);
    return !(NM >= 2 && sm < fb);
  }
}

// FP64 projection of an element-type point (the re-projection path).
template <int NM, typename R>
__device__ __forceinline__ R project_point_f64(const R* m, R* b) {
  constexpr int C = NM * NM;
  if constexpr (sizeof(R) == 4) {
    MatV<NM> mv;
#pragma unroll
    for (int c = 0; c < C; ++c) mv.v[c] = m[c];
    const ProjV<NM> r = f64_cold<NM>(mv);
#pragma unroll
    for (int c = 0; c < C; ++c) b[c] = r.b[c];
    return r.sg;
  } else {
    double sd;
    return polar_f64<NM>(m, b, sd);
  }
}

// Record a projected point: compare with the old field, write the new value
// to global memory and, packed, to shared memory (plane q at dst[q * qstride]).
template <int NM, typename R, typename V>
__device__ __forceinline__ void finish_point(R* __restrict__ A, long long P, long long off, int x,
                                             const R* old, const R* b, R sg, V* dst, int qstride,
                                             PointStats<R>& ps) {
  constexpr int C = NM * NM, Q = (C + 1) / 2;
  R d = R(0), nb = R(0);
#pragma unroll
  for (int c = 0; c < C; ++c) {
    d = fmax(d, fabs(b[c] - old[c]));
    nb += b[c] * b[c];
  }
  ps.maxd = fmax(ps.maxd, d);
  ps.flips += (det_sign<NM>(old) != sg) ? 1 : 0;
  ps.defect += R(NM) - nb;
#pragma unroll
  for (int c = 0; c < C; ++c) A[c * P + off + x] = b[c];
#pragma unroll
  for (int q = 0; q < Q; ++q) dst[q * qstride] = V{b[2 * q], (2 * q + 1 < C) ? b[2 * q + 1] : R(0)};
}

// Reduce a block's point statistics and, in the last block of the grid,
// record the step (energy slot filled earlier by the transform pass; max
// delta, flips, re-projections, non-finite count), decide stationarity
// (tol >= 0), reset the accumulators and advance the step counter.
template <typename R>
__device__ __forceinline__ void finalize_step_stats(long long P, double tau, const StatsPtrs& sp,
                                                    const PointStats<R>& ps, double* redd, int* redi,
                                                    int* s_flag) {
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  // one fused block reduction (blocks of at most 16 warps): the defect sum,
  // the largest change, and the three counts in 21-bit fields of one integer
  // (a block holds far fewer than 2^21 points)
  double dsum = (double)ps.defect, mx = (double)ps.maxd;
  unsigned long long cnt = (unsigned long long)ps.flips |
                           ((unsigned long long)ps.nonfinite << 21) |
                           ((unsigned long long)ps.fallback << 42);
  auto warp_fold = [&]() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
      mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
  };
  warp_fold();
  __syncthreads();  // the slots may still be read by an earlier reduction
  if (l == 0) {
    redd[w] = dsum;
    redd[16 + w] = mx;
    redi[w] = (int)(unsigned)cnt;
    redi[16 + w] = (int)(unsigned)(cnt >> 32);
  }
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    const bool in = l < nw;
    dsum = in ? redd[l] : 0.0;
    mx = in ? redd[16 + l] : 0.0;
    cnt = in ? ((unsigned long long)(unsigned)redi[l] | ((unsigned long long)(unsigned)redi[16 + l] << 32))
             : 0ull;
    warp_fold();
  }
  const int fl = (int)(cnt & 0x1FFFFFull);
  const int nfin = (int)((cnt >> 21) & 0x1FFFFFull);
  const int nfb = (int)(cnt >> 42);
  if (tid == 0) {
    atomicMax(&sp.st->maxdelta_bits, (unsigned long long)__double_as_longlong(mx));
    if (fl) atomicAdd(&sp.st->flips, (unsigned long long)fl);
    if (nfin) atomicAdd(&sp.st->nonfinite, (unsigned long long)nfin);
    if (nfb) atomicAdd(&sp.st->fallback, (unsigned long long)nfb);
  }
  double all, esum = 0.0;
  // deferred energy of this step's input: the multiplier pass's partials
  // (block order), summed by the last block with the defects; the defect of
  // A_s is still in st->defect
  if (grid_sum(dsum, sp.rb, redd, s_flag, &all, sp.epart, sp.epart ? &sp.st->nep : nullptr, &esum)) {
    if (tid == 0) {
      RunState* st = sp.st;
      const long long slot = st->step & (kRing - 1);
      if (sp.epart) {
        const double Pd = (double)P;
        const double E_tau = (esum / Pd + st->defect) / (Pd * tau);
        st->energy_last = E_tau;
        sp.hist.energy[slot] = E_tau;
      }
      st->defect = all;
      const double md = __longlong_as_double((long long)atomicAdd(&st->maxdelta_bits, 0ull));
      const unsigned long long f = atomicAdd(&st->flips, 0ull);
      const unsigned long long nb = atomicAdd(&st->fallback, 0ull);
      const unsigned long long nn = atomicAdd(&st->nonfinite, 0ull);
      sp.hist.maxdelta[slot] = md;
      sp.hist.flips[slot] = (long long)f;
      sp.hist.fallback[slot] = (long long)nb;
      sp.hist.nonfinite[slot] = (long long)nn;
      if (sp.tol >= 0.0 && f == 0 && md <= sp.tol) st->stop = 1;
      st->maxdelta_bits = 0;
      st->flips = 0;
      st->fallback = 0;
      st->nonfinite = 0;
      st->step += 1;
    }
  }
}

template <typename R, int NM, int MODE>
__global__ void __launch_bounds__(kMaxThreads, sizeof(R) == 4 ? 2 : 1)
k_row(Geom g, Tables<R> t, const R* __restrict__ Ain, R* A, typename VT<R>::V* W, StatsPtrs sp,
      R fb_sigma) {
  using V = typename VT<R>::V;
  constexpr int C = NM * NM, Q = (C + 1) / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double redd[32];
  __shared__ int redi[32];
  __shared__ int s_flag, s_nfb;
  if (sp.respect_stop && *(volatile int*)&sp.st->stop) return;

  V* s = reinterpret_cast<V*>(smem_raw);
  const int nx = g.nx;
  const int S = row_pad(nx);
  const RowLayout lay{S};
  const long long P = g.P;
  const long long off = (long long)blockIdx.x * nx;
  const int T = blockDim.x, tid = threadIdx.x;
  const V* tw = static_cast<const V*>(t.tw[0]);
  const bool is_f32 = sizeof(R) == 4;

  if (MODE == ROW_FWD) {
    R defect = R(0);
    for (int x = tid; x < nx; x += T) {
      R sq = R(0);
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const R re = Ain[(2 * q) * P + off + x];
        const R im = (2 * q + 1 < C) ? Ain[(2 * q + 1) * P + off + x] : R(0);
        s[lay.addr(q, x)] = V{re, im};
        sq += re * re + im * im;
      }
      defect += R(NM) - sq;
    }
    __syncthreads();
    fft_fwd(s, lay, nx, Q, t.plan[0], tw);
#pragma unroll
    for (int q = 0; q < Q; ++q)
      for (int x = tid; x < nx; x += T) W[q * P + off + x] = s[lay.addr(q, x)];
    if (sp.do_stats) {
      const double tot = block_sum((double)defect, redd);
      double all;
      if (grid_sum(tot, sp.rb, redd, &s_flag, &all) && tid == 0) sp.st->defect = all;
    }
    return;
  }

  // inverse modes: load the spectrum rows (asynchronous copies)
#pragma unroll
  for (int q = 0; q < Q; ++q)
    for (int x = tid; x < nx; x += T) cp_async_elem(&s[lay.addr(q, x)], &W[q * P + off + x]);
  cp_async_wait_all();
  __syncthreads();
  fft_inv(s, lay, nx, Q, t.plan[0], tw);

  if (MODE == ROW_INV_OUT) {
    for (int x = tid; x < nx; x += T) {
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const V z = s[lay.addr(q, x)];
        A[(2 * q) * P + off + x] = z.x;
        if (2 * q + 1 < C) A[(2 * q + 1) * P + off + x] = z.y;
      }
    }
    return;
  }

  // ROW_INV_PROJECT_FWD
  float* fbM = reinterpret_cast<float*>(s + Q * S);
  int* fbX = reinterpret_cast<int*>(fbM + kFallbackCap * C);
  if (tid == 0) s_nfb = 0;
  __syncthreads();
  PointStats<R> ps;
  for (int x = tid; x < nx; x += T) {
    R old[C];
#pragma unroll
    for (int c = 0; c < C; ++c) old[c] = A[c * P + off + x];
    R m[C];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const V z = s[lay.addr(q, x)];
      m[2 * q] = z.x;
      if (2 * q + 1 < C) m[2 * q + 1] = z.y;
    }
    bool fin = true;
#pragma unroll
    for (int c = 0; c < C; ++c) fin = fin && isfinite(m[c]);
    ps.nonfinite += fin ? 0 : 1;
    R b[C];
    R sg;
    if (!project_point<NM>(m, b, sg, fb_sigma) && fin) {
      const int slot = atomicAdd(&s_nfb, 1);
      if (slot < kFallbackCap) {
        fbX[slot] = x;
#pragma unroll
        for (int c = 0; c < C; ++c) fbM[slot * C + c] = (float)m[c];
        continue;
      }
      sg = project_point_f64<NM>(m, b);
      ps.fallback += 1;
    }
    finish_point<NM>(A, P, off, x, old, b, sg, s + lay.addr(0, x), lay.S, ps);
  }
  if (is_f32 && NM >= 2) {
    __syncthreads();
    const int nf = min(s_nfb, kFallbackCap);
    for (int k = tid; k < nf; k += T) {
      const int x = fbX[k];
      R m[C], b[C], old[C];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        m[c] = (R)fbM[k * C + c];
        old[c] = A[c * P + off + x];
      }
      const R sg = project_point_f64<NM>(m, b);
      ps.fallback += 1;
      finish_point<NM>(A, P, off, x, old, b, sg, s + lay.addr(0, x), lay.S, ps);
    }
  }
  __syncthreads();
  fft_fwd(s, lay, nx, Q, t.plan[0], tw);
#pragma unroll
  for (int q = 0; q < Q; ++q)
    for (int x = tid; x < nx; x += T) W[q * P + off + x] = s[lay.addr(q, x)];

  if (!sp.do_stats) return;
  finalize_step_stats(g.P, g.tau, sp, ps, redd, redi, &s_flag);
}

// Strided-axis pass (y in 2-D; y and z in 3-D).  One block owns a tile of tx
// adjacent x-columns of one complex plane along the whole axis.
template <typename R, int MODE>
__global__ void __launch_bounds__(kMaxThreads, sizeof(R) == 4 ? 2 : 1)
k_axis(Geom g, Tables<R> t, typename VT<R>::V* W, StatsPtrs sp, int axis, int ltx) {
  using V = typename VT<R>::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double redd[32];
  __shared__ int s_flag;
  if (sp.respect_stop && *(volatile int*)&sp.st->stop) return;

  V* s = reinterpret_cast<V*>(smem_raw);
  const int tx = 1 << ltx;
  const int L = (axis == 1) ? g.ny : g.nz;
  const long long es = (axis == 1) ? (long long)g.nx : (long long)g.nx * g.ny;
  const int nouter = (axis == 1) ? g.nz : g.ny;
  const long long ostride = (axis == 1) ? (long long)g.nx * g.ny : (long long)g.nx;
  int q, o, x0;
  col_tile(g, nouter, 1 << ltx, blockIdx.x, q, o, x0);
  V* base = W + (long long)q * g.P + (long long)o * ostride + x0;
  const ColLayout lay{ltx};
  const int T = blockDim.x, tid = threadIdx.x;
  const V* tw = static_cast<const V*>(t.tw[axis]);

  // Thread tid always owns column m = tid % tx of the tile (T is a multiple of
  // tx); it walks the axis with a fixed pointer stride.
  const int mcol = tid & (tx - 1);
  const int p0 = tid >> ltx, dp = T >> ltx;
  const long long gstep = (long long)dp * es;
  {
    const V* src = base + mcol + (long long)p0 * es;
    for (int p = p0; p < L; p += dp, src += gstep) cp_async_elem(&s[lay.addr(mcol, p)], src);
  }
  cp_async_wait_all();
  __syncthreads();
  if (MODE != AXIS_INV) fft_fwd(s, lay, L, tx, t.plan[axis], tw);
  R acc = R(0);
  if (MODE == AXIS_FGI || MODE == AXIS_ENERGY) {
    // the last axis applies g(k) = g_x g_y (g_z); in 3-D the y frequency is
    // the outer index o of this tile (the y pass ran before).
    R go = R(1), omo = R(0);
    if (g.ndim == 3) {
      go = t.g[1][o];
      omo = t.om[1][o];
    }
    const R* gL = t.g[axis];
    const R* omL = t.om[axis];
    const int x = x0 + mcol;
    const R gxx = t.g[0][x];
    const R omx = t.om[0][x];
    const R fo = gxx * go * t.inv_p;
    const R omo2 = gxx * go;
    const R wx = (R)col_weight(g, q, x);
    for (int p = p0; p < L; p += dp) {
      const int e = lay.addr(mcol, p);
      const R omv = omx + gxx * omo + omo2 * omL[p];  // 1 - g without cancellation
      V z = s[e];
      acc += wx * omv * (z.x * z.x + z.y * z.y);
      if (MODE == AXIS_FGI) {
        const R f = fo * gL[p];
        s[e] = V{z.x * f, z.y * f};
      }
    }
    __syncthreads();
  }
  if (MODE == AXIS_FGI || MODE == AXIS_INV) fft_inv(s, lay, L, tx, t.plan[axis], tw);
  if (MODE != AXIS_ENERGY) {
    V* dst = base + mcol + (long long)p0 * es;
    for (int p = p0; p < L; p += dp, dst += gstep) *dst = s[lay.addr(mcol, p)];
  }
  if ((MODE == AXIS_FGI || MODE == AXIS_ENERGY) && sp.do_stats) {
    const double tot = block_sum((double)acc, redd);
    if (MODE == AXIS_FGI && sp.epart) {  // the x pass's finaliser adds these up
      if (tid == 0) {
        sp.epart[blockIdx.x] = tot;
        if (blockIdx.x == 0) sp.st->nep = gridDim.x;
      }
      return;
    }
    double all;
    if (grid_sum(tot, sp.rb, redd, &s_flag, &all)) {
      if (tid == 0) {
        RunState* st = sp.st;
        const double Pd = (double)g.P;
        const double E_tau = (all / Pd + st->defect) / (Pd * g.tau);
        st->energy_last = E_tau;
        sp.hist.energy[st->step & (kRing - 1)] = E_tau;
      }
    }
  }
}

// Pointwise projection of a diffused field (the unfused projection step).
template <typename R, int NM>
__global__ void __launch_bounds__(256)
k_project(long long P, const R* At, R* B, int8_t* ds, R fb_sigma) {
  constexpr int C = NM * NM;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < P;
       x += (long long)gridDim.x * blockDim.x) {
    R m[C], b[C], sg;
#pragma unroll
    for (int c = 0; c < C; ++c) m[c] = At[c * P + x];
    if (!project_point<NM>(m, b, sg, fb_sigma)) sg = project_point_f64<NM>(m, b);
#pragma unroll
    for (int c = 0; c < C; ++c) B[c * P + x] = b[c];
    if (ds) ds[x] = (sg > R(0)) ? 1 : -1;
  }
}

// ---------------------------------------------------------------------------
// Volume-preserving step (Sec. 7)
// ---------------------------------------------------------------------------

// Order-preserving map of a double to an unsigned 64-bit key, complemented so
// that ascending keys are descending values.
__device__ __forceinline__ unsigned long long desc_key(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const unsigned long long asc = (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
  return ~asc;
}

// dE and both class candidates of a point in R, re-done in FP64 where the FP32
// smallest singular value is below fb.
template <int NM, typename R>
__device__ __forceinline__ R class_pair_checked(const R* m, R* tp, R* tm, R& dE, R fb, int& fbk) {
  const R smin = class_pair<NM>(m, tp, tm, dE);
  if (sizeof(R) == 4 && NM >= 2 && smin < fb) {
    constexpr int C = NM * NM;
    double md[C], pd[C], qd[C], ed;
#pragma unroll
    for (int c = 0; c < C; ++c) md[c] = (double)m[c];
    class_pair<NM>(md, pd, qd, ed);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      tp[c] = (R)pd[c];
      tm[c] = (R)qd[c];
    }
    dE = (R)ed;
    fbk = 1;
  }
  return smin;
}

// keys[x] = desc_key(dE(x)) for the diffused field At.
template <typename R, int NM>
__global__ void __launch_bounds__(256)
k_vp_delta(long long P, const R* __restrict__ At, unsigned long long* keys, R fb) {
  constexpr int C = NM * NM;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < P;
       x += (long long)gridDim.x * blockDim.x) {
    R m[C], tp[C], tm[C], dE;
    int fbk = 0;
#pragma unroll
    for (int c = 0; c < C; ++c) m[c] = At[c * P + x];
    class_pair_checked<NM>(m, tp, tm, dE, fb, fbk);
    keys[x] = desc_key((double)dE);
  }
}

// Points with det A(x) > 0 are counted into *count.
template <typename R, int NM>
__global__ void __launch_bounds__(256)
k_count_positive(long long P, const R* __restrict__ A, unsigned long long* count) {
  constexpr int C = NM * NM;
  __shared__ int redi[32];
  int cnt = 0;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < P;
       x += (long long)gridDim.x * blockDim.x) {
    R m[C];
#pragma unroll
    for (int c = 0; c < C; ++c) m[c] = A[c * P + x];
    R d;
    if constexpr (NM == 1) d = m[0];
    else if constexpr (NM == 2) d = m[0] * m[3] - m[1] * m[2];
    else
      d = m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) +
          m[2] * (m[3] * m[7] - m[4] * m[6]);
    cnt += (d > R(0)) ? 1 : 0;
  }
  cnt = block_sum(cnt, redi);
  if (threadIdx.x == 0 && cnt) atomicAdd(count, (unsigned long long)cnt);
}

// Assign T+ to the n_plus points of smallest (key, index) and T- to the rest,
// write the field, and record the step like the projection pass.
template <typename R, int NM>
__global__ void __launch_bounds__(256)
k_vp_assign(long long P, const R* __restrict__ At, R* A, const unsigned long long* __restrict__ keys,
            const SelectState* __restrict__ ss, StatsPtrs sp, R fb) {
  constexpr int C = NM * NM;
  __shared__ double redd[32];
  __shared__ int redi[32];
  __shared__ int s_flag;
  if (sp.respect_stop && *(volatile int*)&sp.st->stop) return;
  const unsigned long long n_plus = ss->n_plus;
  const unsigned long long kh = ss->hi;
  const unsigned int kl = ss->lo;
  PointStats<R> ps;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < P;
       x += (long long)gridDim.x * blockDim.x) {
    R m[C], tp[C], tm[C], old[C], dE;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      m[c] = At[c * P + x];
      old[c] = A[c * P + x];
    }
    int fbk = 0;
    class_pair_checked<NM>(m, tp, tm, dE, fb, fbk);
    ps.fallback += fbk;
    const unsigned long long k = keys[x];
    const bool sel = n_plus > 0 && (k < kh || (k == kh && (unsigned int)x <= kl));
    bool fin = true;
#pragma unroll
    for (int c = 0; c < C; ++c) fin = fin && isfinite(m[c]);
    ps.nonfinite += fin ? 0 : 1;
    R d = R(0), nb = R(0);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const R b = sel ? tp[c] : tm[c];
      d = fmax(d, fabs(b - old[c]));
      nb += b * b;
      A[c * P + x] = b;
    }
    ps.maxd = fmax(ps.maxd, d);
    ps.defect += R(NM) - nb;
    R od;
    if constexpr (NM == 1) od = old[0];
    else if constexpr (NM == 2) od = old[0] * old[3] - old[1] * old[2];
    else
      od = old[0] * (old[4] * old[8] - old[5] * old[7]) - old[1] * (old[3] * old[8] - old[5] * old[6]) +
           old[2] * (old[3] * old[7] - old[4] * old[6]);
    ps.flips += ((od > R(0)) != sel) ? 1 : 0;
  }
  if (!sp.do_stats) return;
  finalize_step_stats(P, 0.0, sp, ps, redd, redi, &s_flag);  // the energy is the FGI pass's (no epart)
}

template <typename R>
cudaError_t launch_volume(int which, const Geom& g, const R* At, R* A, unsigned long long* keys,
                          SelectState* ss, const StatsPtrs& sp, double fb, int blocks,
                          cudaStream_t s) {
  const R f = (R)fb;
#define MBO_VP_CASE(NM)                                                                         \
  if (g.n == NM) {                                                                              \
    if (which == 0) k_vp_delta<R, NM><<<blocks, 256, 0, s>>>(g.P, At, keys, f);                 \
    else if (which == 1) k_count_positive<R, NM><<<blocks, 256, 0, s>>>(g.P, A, &ss->n_plus);   \
    else k_vp_assign<R, NM><<<blocks, 256, 0, s>>>(g.P, At, A, keys, ss, sp, f);                \
    return cudaGetLastError();                                                                  \
  }
  MBO_VP_CASE(1)
  MBO_VP_CASE(2)
  MBO_VP_CASE(3)
#undef MBO_VP_CASE
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
// Raise a kernel's dynamic shared-memory limit once (per process) to the
// largest size it was launched with; launches inside graph capture then make
// no attribute call.
template <typename K> static cudaError_t set_smem(K kernel, size_t bytes, size_t& done) {
  if (bytes <= 48 * 1024 || bytes <= done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done = bytes;
  return e;
}

template <typename R, int NM, int MODE>
static cudaError_t launch_row_nm(const Geom& g, const Tables<R>& t, const R* Ain, R* A, void* W,
                                 const StatsPtrs& sp, R fb, int threads, cudaStream_t s,
                                 bool prepare_only = false) {
  auto k = k_row<R, NM, MODE>;
  static size_t done = 0;
  const size_t smem = row_smem_bytes(g, sizeof(R), MODE == ROW_INV_PROJECT_FWD);
  cudaError_t e = set_smem(k, smem, done);
  if (e != cudaSuccess || prepare_only) return e;
  const int rows = g.nz * g.ny;
  k<<<rows, threads, smem, s>>>(g, t, Ain, A, static_cast<typename VT<R>::V*>(W), sp, fb);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_row(RowMode mode, const Geom& g, const Tables<R>& t, const R* A_in, R* A_out,
                       void* W, const StatsPtrs& sp, double fallback_sigma, int threads,
                       cudaStream_t s) {
  if constexpr (sizeof(R) == 4) {
    if (t.plan[0].lq) return launch_wrow(mode, g, t, A_in, A_out, W, sp, fallback_sigma, s, false);
  }
  const R fb = (R)fallback_sigma;
#define MBO_ROW_CASE(NM)                                                                   \
  if (g.n == NM) {                                                                         \
    if (mode == ROW_FWD)                                                                   \
      return launch_row_nm<R, NM, ROW_FWD>(g, t, A_in, A_out, W, sp, fb, threads, s);      \
    if (mode == ROW_INV_OUT)                                                               \
      return launch_row_nm<R, NM, ROW_INV_OUT>(g, t, A_in, A_out, W, sp, fb, threads, s);  \
    return launch_row_nm<R, NM, ROW_INV_PROJECT_FWD>(g, t, A_in, A_out, W, sp, fb, threads, \
                                                     s);                                   \
  }
  MBO_ROW_CASE(1)
  MBO_ROW_CASE(2)
  MBO_ROW_CASE(3)
  MBO_ROW_CASE(4)
#undef MBO_ROW_CASE
  return cudaErrorInvalidValue;
}

template <typename R, int MODE>
static cudaError_t launch_axis_m(const Geom& g, const Tables<R>& t, void* W, const StatsPtrs& sp,
                                 int axis, int tx, int threads, cudaStream_t s,
                                 bool prepare_only = false) {
  auto k = k_axis<R, MODE>;
  static size_t done = 0;
  const int L = axis == 1 ? g.ny : g.nz;
  const size_t smem = axis_smem_bytes(L, tx, sizeof(R));
  cudaError_t e = set_smem(k, smem, done);
  if (e != cudaSuccess || prepare_only) return e;
  int ltx = 0;
  while ((1 << ltx) < tx) ++ltx;
  const int nouter = axis == 1 ? g.nz : g.ny;
  const int tiles = col_tiles(g, nouter, tx);
  k<<<tiles, threads, smem, s>>>(g, t, static_cast<typename VT<R>::V*>(W), sp, axis, ltx);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_axis(AxisMode mode, int axis, const Geom& g, const Tables<R>& t, void* W,
                        const StatsPtrs& sp, int tx, int threads, cudaStream_t s,
                        const CUtensorMap* tm, int stages, const void* l2_hint,
                        long long l2_hint_bytes) {
  if constexpr (sizeof(R) == 4) {
    if (t.plan[axis].lq)
      return launch_wcol(mode, axis, g, t, W, sp, tx, s, false, tm, stages, l2_hint, l2_hint_bytes);
  }
  switch (mode) {
    case AXIS_FWD: return launch_axis_m<R, AXIS_FWD>(g, t, W, sp, axis, tx, threads, s);
    case AXIS_INV: return launch_axis_m<R, AXIS_INV>(g, t, W, sp, axis, tx, threads, s);
    case AXIS_FGI: return launch_axis_m<R, AXIS_FGI>(g, t, W, sp, axis, tx, threads, s);
    default: return launch_axis_m<R, AXIS_ENERGY>(g, t, W, sp, axis, tx, threads, s);
  }
}

template <typename R>
cudaError_t launch_project(const Geom& g, const R* At, R* B, int8_t* det_sign,
                           double fallback_sigma, cudaStream_t s) {
  const int threads = 256;
  long long blocks = (g.P + threads - 1) / threads;
  if (blocks > 152 * 64) blocks = 152 * 64;
  const R fb = (R)fallback_sigma;
  if (g.n == 1) k_project<R, 1><<<(int)blocks, threads, 0, s>>>(g.P, At, B, det_sign, fb);
  else if (g.n == 2) k_project<R, 2><<<(int)blocks, threads, 0, s>>>(g.P, At, B, det_sign, fb);
  else if (g.n == 3) k_project<R, 3><<<(int)blocks, threads, 0, s>>>(g.P, At, B, det_sign, fb);
  else k_project<R, 4><<<(int)blocks, threads, 0, s>>>(g.P, At, B, det_sign, fb);
  return cudaGetLastError();
}

// Raise the shared-memory limit of every kernel a geometry uses, without
// launching (so that later launches inside stream capture make no attribute
// call).
template <typename R> cudaError_t prepare_kernels(const Geom& g, const Tables<R>& tabs, int tx,
                                                  int stages) {
  Tables<R> t{};
  StatsPtrs sp{};
  cudaError_t e = cudaSuccess;
  if constexpr (sizeof(R) == 4) {
    if (tabs.plan[0].lq) {
      for (int m = ROW_FWD; m <= ROW_INV_PROJECT_FWD && e == cudaSuccess; ++m)
        e = launch_wrow((RowMode)m, g, tabs, nullptr, nullptr, nullptr, sp, 0.0, 0, true);
    }
    for (int axis = 1; axis <= (g.ndim == 3 ? 2 : 1) && e == cudaSuccess; ++axis) {
      if (!tabs.plan[axis].lq) continue;
      for (int m = AXIS_FWD; m <= AXIS_ENERGY && e == cudaSuccess; ++m)
        e = launch_wcol((AxisMode)m, axis, g, tabs, nullptr, sp, tx, 0, true, nullptr, stages);
    }
  }
#define MBO_PREP_ROW(NM)                                                                       \
  if (g.n == NM) {                                                                             \
    if (e == cudaSuccess)                                                                      \
      e = launch_row_nm<R, NM, ROW_FWD>(g, t, nullptr, nullptr, nullptr, sp, R(0), 32, 0, true); \
    if (e == cudaSuccess)                                                                      \
      e = launch_row_nm<R, NM, ROW_INV_OUT>(g, t, nullptr, nullptr, nullptr, sp, R(0), 32, 0,  \
                                            true);                                             \
    if (e == cudaSuccess)                                                                      \
      e = launch_row_nm<R, NM, ROW_INV_PROJECT_FWD>(g, t, nullptr, nullptr, nullptr, sp, R(0), \
                                                    32, 0, true);                              \
  }
  MBO_PREP_ROW(1)
  MBO_PREP_ROW(2)
  MBO_PREP_ROW(3)
  MBO_PREP_ROW(4)
#undef MBO_PREP_ROW
  for (int axis = 1; axis <= (g.ndim == 3 ? 2 : 1) && e == cudaSuccess; ++axis) {
    if (sizeof(R) == 4 && tabs.plan[axis].lq) continue;  // the warp-plan pass above takes this axis
    e = launch_axis_m<R, AXIS_FWD>(g, t, nullptr, sp, axis, tx, 64, 0, true);
    if (e == cudaSuccess) e = launch_axis_m<R, AXIS_INV>(g, t, nullptr, sp, axis, tx, 64, 0, true);
    if (e == cudaSuccess) e = launch_axis_m<R, AXIS_FGI>(g, t, nullptr, sp, axis, tx, 64, 0, true);
    if (e == cudaSuccess)
      e = launch_axis_m<R, AXIS_ENERGY>(g, t, nullptr, sp, axis, tx, 64, 0, true);
  }
  return e;
}

#define MBO_INSTANTIATE(R)                                                                     \
  template cudaError_t prepare_kernels<R>(const Geom&, const Tables<R>&, int, int);            \
  template cudaError_t launch_row<R>(RowMode, const Geom&, const Tables<R>&, const R*, R*,     \
                                     void*, const StatsPtrs&, double, int, cudaStream_t);      \
  template cudaError_t launch_axis<R>(AxisMode, int, const Geom&, const Tables<R>&, void*,     \
                                      const StatsPtrs&, int, int, cudaStream_t,                \
                                      const CUtensorMap*, int, const void*, long long);        \
  template cudaError_t launch_project<R>(const Geom&, const R*, R*, int8_t*, double,          \
                                         cudaStream_t);                                        \
  template cudaError_t launch_volume<R>(int, const Geom&, const R*, R*, unsigned long long*,   \
                                        SelectState*, const StatsPtrs&, double, int,           \
                                        cudaStream_t);

}  // namespace mbo
