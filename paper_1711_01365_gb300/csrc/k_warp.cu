// FP32 x pass of the MBO step (Algorithm 1 of Osting & Wang,
// arXiv:1711.01365) for x axes whose plan is the warp-cooperative four-step
// transform (mbo_wfft.cuh): lengths 256, 512 and 1024, and 768 = 3 x 256,
// 1536 = 3 x 512, 2048 = 2 x 1024 through a radix-3 / radix-2 stage across
// groups of lanes.  The strided passes are in k_wcol.cu.
//
//   k_wrow  x axis: one sequence (row, complex plane) per LQ lanes.  Inverse
//           transform in registers, exchange through shared memory so that one
//           thread sees all n*n channels of a point, projection (Lemma 1.1) and
//           step statistics, exchange back, forward transform of the new field.
// Data layout in HBM is that of the generic passes (mbo_kernels.cuh); spectra
// along these axes are in natural order.
#include "mbo_kernels.cuh"
#include "mbo_tma.cuh"
#include "mbo_wfft.cuh"
#include "mbo_wshape.cuh"

namespace mbo {
namespace {

template <int NM, int MODE, int N, bool PERS>
__global__ void __launch_bounds__(wrow_threads(N, NM), wrow_minb(N, NM))
k_wrow(Geom g, Tables<float> t, const float* __restrict__ Ain, float* A, float2* W, StatsPtrs sp,
       float fb_sigma, int ahead) {
  constexpr int R = w_r(N), M = w_m(N), LQ = w_lq(N), RB = wrow_rb(N);
  using F = WarpFFTR<M, LQ, R>;
  constexpr int C = NM * NM, Q = (C + 1) / 2, E = F::E, RS = F::RS, NT = wrow_threads(N, NM);
  constexpr int PS = R * RS;  // slots of one (row, plane): R group regions, >= N
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double redd[32];
  __shared__ int redi[32];
  __shared__ int s_flag, s_nfb;
  pdl_wait();  // the previous pass's spectrum and run state are complete
  if (sp.respect_stop && *(volatile int*)&sp.st->stop) return;
  pdl_release();

  float2* sm = reinterpret_cast<float2*>(smem_raw);
  const int tid = threadIdx.x;
  const int grp = tid / LQ, l = tid - grp * LQ;  // group = (row, plane, r)
  const int seq = grp / R, r = grp - seq * R;
  const int row = seq / Q, q = seq - row * Q;
  const long long P = g.P;
  const long long rows = P / N;
  const long long ngroups = (rows + RB - 1) / RB;  // row groups: RB rows each
  float2* base = sm + seq * PS;  // this (row, plane)'s regions
  const float2* tw = static_cast<const float2*>(t.tw[0]);
  const float2* twr = tw + M;
  float* fbM = reinterpret_cast<float*>(sm + wrow_nseq(N, NM) * PS);
  int* fbX = reinterpret_cast<int*>(fbM + kFallbackCap * C);
  const bool mirror = q == Q - 1 && g.xh < N;
  float2 v[E];
  PointStats<float> ps;  // projection mode: over all of the block's rows
  double defect = 0.0;   // forward mode

  // Row groups of this block: its own index, or with PERS the groups
  // blockIdx.x, blockIdx.x + gridDim.x, ... (a grid of one wave).
  const long long gstep = PERS ? (long long)gridDim.x : ngroups;
  auto do_group = [&](long long gi) {
    const long long row0 = gi * RB;
    const bool live = seq < RB * Q && row0 + row < rows;  // a whole sequence is live or not
    const long long off = (row0 + row) * N;
    // the forward spectrum of this sequence to W; the last plane of an odd
    // channel count is Hermitian: columns k < xh only
    auto store_spectrum = [&](const float2(&u)[E]) {
      if (!live) return;
      float2* wdst = W + q * P + off;
      if (q < Q - 1 || g.xh == N) {
#pragma unroll
        for (int j = 0; j < E; ++j) wdst[l + M * r + LQ * j] = u[j];
      } else {
#pragma unroll
        for (int j = 0; j < E; ++j) {
          const int k = l + LQ * j + M * r;
          if (k < g.xh) wdst[k] = u[j];
        }
      }
    };

    if (MODE == ROW_FWD) {
      // per point: load all channels, accumulate n - |A|^2, park the planes
      for (int p = tid; p < RB * N; p += NT) {
        const int rw = p / N, x = p - rw * N;
        if (row0 + rw >= rows) continue;
        const long long o = (row0 + rw) * N + x;
        float sq = 0.f;
#pragma unroll
        for (int qq = 0; qq < Q; ++qq) {
          const float re = Ain[(2 * qq) * P + o];
          const float im = (2 * qq + 1 < C) ? Ain[(2 * qq + 1) * P + o] : 0.f;
          sm[(rw * Q + qq) * PS + x] = float2{re, im};
          sq += re * re + im * im;
        }
        defect += (double)(float(NM) - sq);
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < E; ++j) v[j] = base[R * (l + LQ * j) + r];
      if constexpr (R > 1) __syncthreads();  // regions are shared across groups
      else __syncwarp();
      F::fwd(v, base, r, tw, twr, l);
      store_spectrum(v);
      return;
    }

    if (MODE == ROW_INV_PROJECT_FWD && tid < C) {
      // the old field of this group's rows, wanted after the inverse transform
      const long long nr = rows - row0 < RB ? rows - row0 : RB;
      bulk_prefetch_l2(A + tid * P + row0 * N, (unsigned)(nr * N * sizeof(float)));
    } else if (tid >= 32 && tid < 32 + RB * Q && (PERS || ahead > 0)) {
      // the spectrum rows of the group this block (or a block of a later
      // wave) takes next
      const long long rn = (PERS ? row0 + gstep * RB : row0 + (long long)ahead * RB) + (tid - 32) / Q;
      const int qq = (tid - 32) % Q;
      if (rn < rows) {
        const int cols = qq == Q - 1 ? g.xh : N;
        bulk_prefetch_l2(W + qq * P + rn * N, (unsigned)((cols * sizeof(float2) + 15) & ~15u));
      }
    }

    // inverse modes: the spectrum rows straight into registers (coalesced); a
    // Hermitian last plane supplies columns k > N/2 as conj(column N - k)
    const float2* wrow = W + q * P + off;  // this sequence's spectrum row
    if (!live) {
#pragma unroll
      for (int j = 0; j < E; ++j) v[j] = float2{0.f, 0.f};
    } else if (!mirror) {  // warp-uniform: one address per element, constant offsets
#pragma unroll
      for (int j = 0; j < E; ++j) v[j] = wrow[l + M * r + LQ * j];
    } else {
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const int k = l + LQ * j + M * r;
        const bool up = 2 * k > N;
        float2 z = wrow[up ? N - k : k];
        z.y = up ? -z.y : z.y;
        v[j] = z;
      }
    }
    F::inv(v, base, r, tw, twr, l);

    if (MODE == ROW_INV_OUT) {
      if (live) {
#pragma unroll
        for (int j = 0; j < E; ++j) {
          const int x = R * (l + LQ * j) + r;
          A[(2 * q) * P + off + x] = v[j].x;
          if (2 * q + 1 < C) A[(2 * q + 1) * P + off + x] = v[j].y;
        }
      }
      return;
    }

    // ROW_INV_PROJECT_FWD
    if constexpr (R > 1) __syncthreads();  // every group's transposes are done: the regions hold points now
#pragma unroll
    for (int j = 0; j < E; ++j) base[R * (l + LQ * j) + r] = v[j];
    if (tid == 0) s_nfb = 0;
    __syncthreads();
    for (int p = tid; p < RB * N; p += NT) {
      const int rw = p / N, x = p - rw * N;
      if (row0 + rw >= rows) continue;
      // issued first, used last: the loads overlap the projection (the rows
      // were prefetched to L2 at the start of the group)
      float old[C];
      {
        const float* src = A + (row0 + rw) * N + x;
#pragma unroll
        for (int c = 0; c < C; ++c, src += P) old[c] = *src;
      }
      const long long ro = (row0 + rw) * N;
      float2* pt = sm + rw * Q * PS + x;
      float m[C];
#pragma unroll
      for (int qq = 0; qq < Q; ++qq) {
        const float2 z = pt[qq * PS];
        m[2 * qq] = z.x;
        if (2 * qq + 1 < C) m[2 * qq + 1] = z.y;
      }
      // finite entries have a finite sum of squares (up to overflow, which
      // the entry-wise test below settles)
      float nx = 0.f;
#pragma unroll
      for (int c = 0; c < C; ++c) nx += m[c] * m[c];
      bool fin = isfinite(nx);
      if (!fin) {
        fin = true;
#pragma unroll
        for (int c = 0; c < C; ++c) fin = fin && isfinite(m[c]);
      }
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
      finish_point<NM>(A, P, ro, x, old, b, sg, pt, PS, ps);
    }
    if (NM >= 2) {
      // the FP64 re-projections collected above, spread over the block
      __syncthreads();
      const int nf = min(s_nfb, kFallbackCap);
      for (int k = tid; k < nf; k += NT) {
        const int p = fbX[k];
        const int rw = p / N, x = p - rw * N;
        const long long ro = (row0 + rw) * N;
        float m[C], b[C], old[C];
#pragma unroll
        for (int c = 0; c < C; ++c) {
          m[c] = fbM[k * C + c];
          old[c] = A[c * P + ro + x];
        }
        const float sg = project_point_f64<NM>(m, b);
        ps.fallback += 1;
        finish_point<NM>(A, P, ro, x, old, b, sg, sm + rw * Q * PS + x, PS, ps);
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < E; ++j) v[j] = base[R * (l + LQ * j) + r];
    if constexpr (R > 1) __syncthreads();
    else __syncwarp();
    F::fwd(v, base, r, tw, twr, l);
    store_spectrum(v);
  };
  if constexpr (PERS) {
    for (long long gi = blockIdx.x; gi < ngroups; gi += gstep) {
      if (gi != blockIdx.x) __syncthreads();  // the previous group's regions are free
      do_group(gi);
    }
  } else {
    do_group(blockIdx.x);
  }

  if (!sp.do_stats || MODE == ROW_INV_OUT) return;
  if (MODE == ROW_FWD) {
    const double tot = block_sum(defect, redd);
    double all;
    if (grid_sum(tot, sp.rb, redd, &s_flag, &all) && tid == 0) sp.st->defect = all;
    return;
  }
  finalize_step_stats(g.P, g.tau, sp, ps, redd, redi, &s_flag);
}

template <int NM, int MODE, int N>
cudaError_t wrow_nm(const Geom& g, const Tables<float>& t, const float* Ain, float* A, void* W,
                    const StatsPtrs& sp, float fb, cudaStream_t s, bool prepare_only) {
  // the one-wave form is instantiated for the projecting pass only
  constexpr bool CAN_PERS = MODE == ROW_INV_PROJECT_FWD;
  auto k = k_wrow<NM, MODE, N, false>;
  auto kp = k_wrow<NM, MODE, N, CAN_PERS>;
  static size_t done = 0, done_p = 0;
  static int resident = 0;  // blocks of this kernel that fit on the device at once
  const size_t smem = wrow_smem_bytes(g, N, MODE == ROW_INV_PROJECT_FWD);
  cudaError_t e = set_smem_once(k, smem, done);
  if (e == cudaSuccess && CAN_PERS) e = set_smem_once(kp, smem, done_p);
  if (e != cudaSuccess) return e;
  if (!resident) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, wrow_threads(N, NM), smem);
    resident = sms * (per_sm > 0 ? per_sm : 1);
  }
  if (prepare_only) return cudaSuccess;
  constexpr int RB = wrow_rb(N);
  const long long rows = g.P / N;
  const int blocks = (int)((rows + RB - 1) / RB);
  // a block prefetches the spectrum rows of the block one wave later
  const int ahead = blocks > resident ? resident : 0;
  // persistent: one wave of blocks walks the row groups with a stride of the grid
  if (CAN_PERS && wrow_persistent_flag() && blocks > resident)
    return launch_pdl(kp, resident, wrow_threads(N, NM), smem, s, g, t, Ain, A, static_cast<float2*>(W),
                      sp, fb, 0);
  return launch_pdl(k, blocks, wrow_threads(N, NM), smem, s, g, t, Ain, A, static_cast<float2*>(W), sp,
                    fb, ahead);
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

}  // namespace

bool warp_plan_length(int N) {
  return N == 256 || N == 512 || N == 768 || N == 1024 || N == 1536 || N == 2048;
}
int warp_plan_radix(int N) { return w_r(N); }

size_t wrow_smem_bytes(const Geom& g, int N, bool fallback) {
  const int LQ = w_lq(N), RB = wrow_rb(N), R = w_r(N);
  const size_t rs = (size_t)(LQ + 1) * (w_m(N) / LQ);
  const int threads = (RB * g.Q * R * LQ + 31) / 32 * 32;
  const int nseq = (threads + R * LQ - 1) / (R * LQ);  // wrow_nseq(N, g.n)
  size_t b = (size_t)nseq * R * rs * sizeof(float2);
  if (fallback) b += (size_t)kFallbackCap * ((size_t)g.C * sizeof(float) + sizeof(int));
  return (b + 15) & ~(size_t)15;
}

namespace {
template <int NM, int N> double wrow_waves_nm(const Geom& g) {
  auto k = k_wrow<NM, ROW_INV_PROJECT_FWD, N, false>;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = wrow_smem_bytes(g, N, true);
  // a shape that does not fit is rejected by the caller; leave no error behind
  if ((smem > 48 * 1024 &&
       cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, wrow_threads(N, NM), smem) != cudaSuccess) {
    (void)cudaGetLastError();
    return 1e9;
  }
  const double blocks = (double)((g.P / N + wrow_rb(N) - 1) / wrow_rb(N));
  return blocks / ((double)sms * (per_sm > 0 ? per_sm : 1));
}
template <int N> double wrow_waves_n(const Geom& g) {
  switch (g.n) {
    case 1: return wrow_waves_nm<1, N>(g);
    case 2: return wrow_waves_nm<2, N>(g);
    case 3: return wrow_waves_nm<3, N>(g);
    default: return wrow_waves_nm<4, N>(g);
  }
}
}  // namespace

double wrow_waves(const Geom& g) {
  switch (g.nx) {
    case 2048: return wrow_waves_n<2048>(g);
    case 1536: return wrow_waves_n<1536>(g);
    case 1024: return wrow_waves_n<1024>(g);
    case 768: return wrow_waves_n<768>(g);
    case 512: return wrow_waves_n<512>(g);
    case 256: return wrow_waves_n<256>(g);
    default: return 0.0;
  }
}

bool& wrow_persistent_flag() {
  thread_local bool on = false;
  return on;
}

bool& pdl_flag() {
  thread_local bool on = true;
  return on;
}

cudaError_t launch_wrow(RowMode mode, const Geom& g, const Tables<float>& t, const float* Ain,
                        float* A, void* W, const StatsPtrs& sp, double fb, cudaStream_t s,
                        bool prepare_only) {
  const float f = (float)fb;
  switch (g.nx) {
    case 2048: return wrow_n<2048>(mode, g, t, Ain, A, W, sp, f, s, prepare_only);
    case 1536: return wrow_n<1536>(mode, g, t, Ain, A, W, sp, f, s, prepare_only);
    case 1024: return wrow_n<1024>(mode, g, t, Ain, A, W, sp, f, s, prepare_only);
    case 768: return wrow_n<768>(mode, g, t, Ain, A, W, sp, f, s, prepare_only);
    case 512: return wrow_n<512>(mode, g, t, Ain, A, W, sp, f, s, prepare_only);
    case 256: return wrow_n<256>(mode, g, t, Ain, A, W, sp, f, s, prepare_only);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mbo
