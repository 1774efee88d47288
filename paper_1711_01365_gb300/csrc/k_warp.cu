// FP32 passes of the MBO step (Algorithm 1 of Osting & Wang,
// arXiv:1711.01365) for axes whose plan is the warp-cooperative four-step
// transform (mbo_wfft.cuh): lengths 256, 512 and 1024.
//
//   k_wrow  x axis: one sequence (row, complex plane) per LQ lanes.  Inverse
//           transform in registers, exchange through shared memory so that one
//           thread sees all n*n channels of a point, projection (Lemma 1.1) and
//           step statistics, exchange back, forward transform of the new field.
//   k_wcol  y / z axis: a tile of TX adjacent columns of one plane is staged
//           through shared memory with coalesced copies; one sequence per
//           column; forward transform, multiplier g(k)/P and the energy
//           partials of the Sec. 4 functional (Parseval form), inverse
//           transform, all in registers.
// Data layout in HBM is that of the generic passes (mbo_kernels.cuh); spectra
// along these axes are in natural order.
#include "mbo_kernels.cuh"
#include "mbo_wfft.cuh"

namespace mbo {
namespace {

__host__ __device__ constexpr int wrow_lq(int N) { return N == 1024 ? 32 : 16; }
__host__ __device__ constexpr int wrow_rb(int N) { return N == 1024 ? 1 : 2; }  // rows per block: whole warps

// Blocks per SM the register budget is sized for (x pass, n <= 3: 160-thread
// blocks at 96 registers; n = 4: 256-thread blocks at 128; strided passes:
// 128 registers whatever the tile).
__host__ __device__ constexpr int wrow_minb(int N, int NM) { return N > 0 && NM <= 3 ? 4 : 2; }
__host__ __device__ constexpr int wcol_minb(int L, int TX) {
  return 512 / (TX * (L == 1024 ? 32 : 16)) > 0 ? 512 / (TX * (L == 1024 ? 32 : 16)) : 1;
}

template <int NM, int MODE, int N>
__global__ void __launch_bounds__(wrow_rb(N) * ((NM * NM + 1) / 2) * wrow_lq(N), wrow_minb(N, NM))
k_wrow(Geom g, Tables<float> t, const float* __restrict__ Ain, float* A, float2* W, StatsPtrs sp,
       float fb_sigma) {
  constexpr int LQ = wrow_lq(N), RB = wrow_rb(N);
  using F = WarpFFT<N, LQ>;
  constexpr int C = NM * NM, Q = (C + 1) / 2, E = F::E, RS = F::RS, NT = RB * Q * LQ;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double redd[32];
  __shared__ int redi[32];
  __shared__ int s_flag, s_nfb;
  if (sp.respect_stop && *(volatile int*)&sp.st->stop) return;

  float2* sm = reinterpret_cast<float2*>(smem_raw);
  const int tid = threadIdx.x;
  const int seq = tid / LQ, l = tid - seq * LQ;
  const int row = seq / Q, q = seq - row * Q;
  const long long P = g.P;
  const long long rows = P / N;
  const long long row0 = (long long)blockIdx.x * RB;
  const bool live = row0 + row < rows;  // a whole sequence is live or not
  const long long off = (row0 + row) * N;
  float2* buf = sm + seq * RS;
  const float2* tw = static_cast<const float2*>(t.tw[0]);
  float2 v[E];

  if (MODE == ROW_FWD) {
    // per point: load all channels, accumulate n - |A|^2, park the planes
    double defect = 0.0;
    for (int p = tid; p < RB * N; p += NT) {
      const int r = p / N, x = p - r * N;
      if (row0 + r >= rows) continue;
      const long long o = (row0 + r) * N + x;
      float sq = 0.f;
#pragma unroll
      for (int qq = 0; qq < Q; ++qq) {
        const float re = Ain[(2 * qq) * P + o];
        const float im = (2 * qq + 1 < C) ? Ain[(2 * qq + 1) * P + o] : 0.f;
        sm[(r * Q + qq) * RS + x] = float2{re, im};
        sq += re * re + im * im;
      }
      defect += (double)(float(NM) - sq);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < E; ++j) v[j] = buf[l + LQ * j];
    __syncwarp();
    F::fwd(v, buf, tw, l);
    if (live) {
#pragma unroll
      for (int j = 0; j < E; ++j)
        if (q < Q - 1 || l + LQ * j < g.xh) W[q * P + off + l + LQ * j] = v[j];
    }
    if (sp.do_stats) {
      const double tot = block_sum(defect, redd);
      double all;
      if (grid_sum(tot, sp.rb, redd, &s_flag, &all) && tid == 0) sp.st->defect = all;
    }
    return;
  }

  // inverse modes: the spectrum rows straight into registers (coalesced); a
  // Hermitian last plane supplies columns k > N/2 as conj(column N - k)
  const bool mirror = q == Q - 1 && g.xh < N;
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int k = l + LQ * j;
    float2 z = float2{0.f, 0.f};
    if (live) {
      if (mirror && 2 * k > N) {
        z = W[q * P + off + (N - k)];
        z.y = -z.y;
      } else {
        z = W[q * P + off + k];
      }
    }
    v[j] = z;
  }
  F::inv(v, buf, tw, l);

  if (MODE == ROW_INV_OUT) {
    if (live) {
#pragma unroll
      for (int j = 0; j < E; ++j) {
        A[(2 * q) * P + off + l + LQ * j] = v[j].x;
        if (2 * q + 1 < C) A[(2 * q + 1) * P + off + l + LQ * j] = v[j].y;
      }
    }
    return;
  }

  // ROW_INV_PROJECT_FWD
#pragma unroll
  for (int j = 0; j < E; ++j) buf[l + LQ * j] = v[j];
  float* fbM = reinterpret_cast<float*>(sm + RB * Q * RS);
  int* fbX = reinterpret_cast<int*>(fbM + kFallbackCap * C);
  if (tid == 0) s_nfb = 0;
  __syncthreads();
  PointStats<float> ps;
  for (int p = tid; p < RB * N; p += NT) {
    const int r = p / N, x = p - r * N;
    if (row0 + r >= rows) continue;
    const long long ro = (row0 + r) * N;
    float2* pt = sm + r * Q * RS + x;
    float old[C];
#pragma unroll
    for (int c = 0; c < C; ++c) old[c] = A[c * P + ro + x];
    float m[C];
#pragma unroll
    for (int qq = 0; qq < Q; ++qq) {
      const float2 z = pt[qq * RS];
      m[2 * qq] = z.x;
      if (2 * qq + 1 < C) m[2 * qq + 1] = z.y;
    }
    bool fin = true;
#pragma unroll
    for (int c = 0; c < C; ++c) fin = fin && isfinite(m[c]);
    ps.nonfinite += fin ? 0 : 1;
    float b[C];
    float sg;
    if (!project_point<NM>(m, b, sg, fb_sigma) && fin) {
      const int slot = atomicAdd(&s_nfb, 1);
      if (slot < kFallbackCap) {
        fbX[slot] = p;
#pragma unroll
        for (int c = 0; c < C; ++c) fbM[slot * C + c] = m[c];
        continue;
      }
      sg = project_point_f64<NM>(m, b);
      ps.fallback += 1;
    }
    finish_point<NM>(A, P, ro, x, old, b, sg, pt, RS, ps);
  }
  if (NM >= 2) {
    // the FP64 re-projections collected above, spread over the block
    __syncthreads();
    const int nf = min(s_nfb, kFallbackCap);
    for (int k = tid; k < nf; k += NT) {
      const int p = fbX[k];
      const int r = p / N, x = p - r * N;
      const long long ro = (row0 + r) * N;
      float m[C], b[C], old[C];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        m[c] = fbM[k * C + c];
        old[c] = A[c * P + ro + x];
      }
      const float sg = project_point_f64<NM>(m, b);
      ps.fallback += 1;
      finish_point<NM>(A, P, ro, x, old, b, sg, sm + r * Q * RS + x, RS, ps);
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < E; ++j) v[j] = buf[l + LQ * j];
  __syncwarp();
  F::fwd(v, buf, tw, l);
  if (live) {
#pragma unroll
    for (int j = 0; j < E; ++j)
      if (q < Q - 1 || l + LQ * j < g.xh) W[q * P + off + l + LQ * j] = v[j];
  }
  if (!sp.do_stats) return;
  finalize_step_stats(sp, ps, redd, redi, &s_flag);
}

__host__ __device__ constexpr int wcol_lq(int L) { return L == 1024 ? 32 : 16; }

// Strided-axis pass (y in 2-D; y and z in 3-D) on a tile of TX adjacent
// x-columns of one complex plane.
template <int MODE, int L, int TX>
__global__ void __launch_bounds__(TX * wcol_lq(L), wcol_minb(L, TX))
k_wcol(Geom g, Tables<float> t, float2* W, StatsPtrs sp, int axis) {
  constexpr int LQ = wcol_lq(L);
  using F = WarpFFT<L, LQ>;
  constexpr int E = F::E, NT = TX * LQ, TS = TX + 1;  // tile row stride (complex)
  static_assert(TX * F::RS <= L * TS, "transpose regions must fit in the tile");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double redd[32];
  __shared__ int s_flag;
  if (sp.respect_stop && *(volatile int*)&sp.st->stop) return;

  float2* tile = reinterpret_cast<float2*>(smem_raw);
  const long long es = (axis == 1) ? (long long)g.nx : (long long)g.nx * g.ny;
  const int nouter = (axis == 1) ? g.nz : g.ny;
  const long long ostride = (axis == 1) ? (long long)g.nx * g.ny : (long long)g.nx;
  int q, o, x0;
  col_tile(g, nouter, TX, blockIdx.x, q, o, x0);
  float2* base = W + (long long)q * g.P + (long long)o * ostride + x0;
  const int tid = threadIdx.x;
  const int c = tid / LQ, l = tid - c * LQ;
  const float2* tw = static_cast<const float2*>(t.tw[axis]);

  for (int i = tid; i < L * TX; i += NT) {
    const int p = i / TX, cc = i - p * TX;
    cp_async_elem(&tile[p * TS + cc], base + (long long)p * es + cc);
  }
  cp_async_wait_all();
  __syncthreads();
  float2 v[E];
#pragma unroll
  for (int j = 0; j < E; ++j) v[j] = tile[(l + LQ * j) * TS + c];
  __syncthreads();
  float2* buf = tile + c * F::RS;
  if (MODE != AXIS_INV) F::fwd(v, buf, tw, l);
  float acc = 0.f;
  if (MODE == AXIS_FGI || MODE == AXIS_ENERGY) {
    // the last axis applies g(k) = g_x g_y (g_z); in 3-D the y frequency is
    // the outer index o of this tile (the y pass ran before).
    float go = 1.f, omo = 0.f;
    if (g.ndim == 3) {
      go = t.g[1][o];
      omo = t.om[1][o];
    }
    const float* gL = t.g[axis];
    const float* omL = t.om[axis];
    const int x = x0 + c;
    const float gxx = t.g[0][x];
    const float omx = t.om[0][x];
    const float fo = gxx * go * t.inv_p;
    const float omo2 = gxx * go;
    const float wx = col_weight(g, q, x);
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const int p = l + LQ * j;
      const float omv = omx + gxx * omo + omo2 * __ldg(&omL[p]);  // 1 - g without cancellation
      const float2 z = v[j];
      acc += wx * omv * (z.x * z.x + z.y * z.y);
      if (MODE == AXIS_FGI) {
        const float f = fo * __ldg(&gL[p]);
        v[j] = float2{z.x * f, z.y * f};
      }
    }
  }
  if (MODE == AXIS_FGI || MODE == AXIS_INV) F::inv(v, buf, tw, l);
  if (MODE != AXIS_ENERGY) {
    __syncthreads();  // every column's transposes are done: the tile is free
#pragma unroll
    for (int j = 0; j < E; ++j) tile[(l + LQ * j) * TS + c] = v[j];
    __syncthreads();
    for (int i = tid; i < L * TX; i += NT) {
      const int p = i / TX, cc = i - p * TX;
      base[(long long)p * es + cc] = tile[p * TS + cc];
    }
  }
  if ((MODE == AXIS_FGI || MODE == AXIS_ENERGY) && sp.do_stats) {
    const double tot = block_sum((double)acc, redd);
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

template <typename K> cudaError_t set_smem_once(K kernel, size_t bytes, size_t& done) {
  if (bytes <= 48 * 1024 || bytes <= done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done = bytes;
  return e;
}

template <int NM, int MODE, int N>
cudaError_t wrow_nm(const Geom& g, const Tables<float>& t, const float* Ain, float* A, void* W,
                    const StatsPtrs& sp, float fb, cudaStream_t s, bool prepare_only) {
  auto k = k_wrow<NM, MODE, N>;
  static size_t done = 0;
  const size_t smem = wrow_smem_bytes(g, N, MODE == ROW_INV_PROJECT_FWD);
  cudaError_t e = set_smem_once(k, smem, done);
  if (e != cudaSuccess || prepare_only) return e;
  constexpr int RB = wrow_rb(N);
  const long long rows = g.P / N;
  const int blocks = (int)((rows + RB - 1) / RB);
  const int threads = RB * ((NM * NM + 1) / 2) * wrow_lq(N);
  k<<<blocks, threads, smem, s>>>(g, t, Ain, A, static_cast<float2*>(W), sp, fb);
  return cudaGetLastError();
}

template <int N>
cudaError_t wrow_n(RowMode mode, const Geom& g, const Tables<float>& t, const float* Ain, float* A,
                   void* W, const StatsPtrs& sp, float fb, cudaStream_t s, bool prep) {
#define MBO_WROW_CASE(NM)                                                                        \
  if (g.n == NM) {                                                                               \
    if (mode == ROW_FWD) return wrow_nm<NM, ROW_FWD, N>(g, t, Ain, A, W, sp, fb, s, prep);       \
    if (mode == ROW_INV_OUT) return wrow_nm<NM, ROW_INV_OUT, N>(g, t, Ain, A, W, sp, fb, s, prep); \
    return wrow_nm<NM, ROW_INV_PROJECT_FWD, N>(g, t, Ain, A, W, sp, fb, s, prep);                \
  }
  MBO_WROW_CASE(1)
  MBO_WROW_CASE(2)
  MBO_WROW_CASE(3)
  MBO_WROW_CASE(4)
#undef MBO_WROW_CASE
  return cudaErrorInvalidValue;
}

template <int MODE, int L, int TX>
cudaError_t wcol_m(const Geom& g, const Tables<float>& t, void* W, const StatsPtrs& sp, int axis,
                   cudaStream_t s, bool prepare_only) {
  auto k = k_wcol<MODE, L, TX>;
  static size_t done = 0;
  const size_t smem = wcol_smem_bytes(L, TX);
  cudaError_t e = set_smem_once(k, smem, done);
  if (e != cudaSuccess || prepare_only) return e;
  const int nouter = axis == 1 ? g.nz : g.ny;
  const int tiles = col_tiles(g, nouter, TX);
  k<<<tiles, TX * wcol_lq(L), smem, s>>>(g, t, static_cast<float2*>(W), sp, axis);
  return cudaGetLastError();
}

template <int L, int TX>
cudaError_t wcol_ltx(AxisMode mode, int axis, const Geom& g, const Tables<float>& t, void* W,
                     const StatsPtrs& sp, cudaStream_t s, bool prep) {
  switch (mode) {
    case AXIS_FWD: return wcol_m<AXIS_FWD, L, TX>(g, t, W, sp, axis, s, prep);
    case AXIS_INV: return wcol_m<AXIS_INV, L, TX>(g, t, W, sp, axis, s, prep);
    case AXIS_FGI: return wcol_m<AXIS_FGI, L, TX>(g, t, W, sp, axis, s, prep);
    default: return wcol_m<AXIS_ENERGY, L, TX>(g, t, W, sp, axis, s, prep);
  }
}

}  // namespace

bool warp_plan_length(int N) { return N == 256 || N == 512 || N == 1024; }

int warp_tile(int L, int nx, int tx) {
  (void)L;
  const int t = tx >= 8 ? 8 : 4;
  return (nx % t == 0) ? t : 0;
}

size_t wrow_smem_bytes(const Geom& g, int N, bool fallback) {
  const int LQ = wrow_lq(N), RB = wrow_rb(N);
  const size_t rs = (size_t)(LQ + 1) * (N / LQ);
  size_t b = (size_t)RB * g.Q * rs * sizeof(float2);
  if (fallback) b += (size_t)kFallbackCap * ((size_t)g.C * sizeof(float) + sizeof(int));
  return (b + 15) & ~(size_t)15;
}

size_t wcol_smem_bytes(int L, int tx) { return (size_t)L * (tx + 1) * sizeof(float2); }

cudaError_t launch_wrow(RowMode mode, const Geom& g, const Tables<float>& t, const float* Ain,
                        float* A, void* W, const StatsPtrs& sp, double fb, cudaStream_t s,
                        bool prepare_only) {
  const float f = (float)fb;
  switch (g.nx) {
    case 1024: return wrow_n<1024>(mode, g, t, Ain, A, W, sp, f, s, prepare_only);
    case 512: return wrow_n<512>(mode, g, t, Ain, A, W, sp, f, s, prepare_only);
    case 256: return wrow_n<256>(mode, g, t, Ain, A, W, sp, f, s, prepare_only);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_wcol(AxisMode mode, int axis, const Geom& g, const Tables<float>& t, void* W,
                        const StatsPtrs& sp, int tx, cudaStream_t s, bool prepare_only) {
  const int L = axis == 1 ? g.ny : g.nz;
  const int TX = warp_tile(L, g.nx, tx);
#define MBO_WCOL_CASE(LEN)                                                          \
  if (L == LEN) {                                                                   \
    if (TX == 8) return wcol_ltx<LEN, 8>(mode, axis, g, t, W, sp, s, prepare_only); \
    if (TX == 4) return wcol_ltx<LEN, 4>(mode, axis, g, t, W, sp, s, prepare_only); \
  }
  MBO_WCOL_CASE(1024)
  MBO_WCOL_CASE(512)
  MBO_WCOL_CASE(256)
#undef MBO_WCOL_CASE
  return cudaErrorInvalidValue;
}

}  // namespace mbo
