// FP32 strided passes (y in 2-D; y and z in 3-D) of the MBO step (Algorithm 1
// of Osting & Wang, arXiv:1711.01365) for axes whose plan is the
// warp-cooperative four-step transform (mbo_wfft.cuh).
//
//   k_wcol  a tile of TX adjacent columns of one plane is staged through
//           shared memory with coalesced copies; one sequence (R groups of
//           lanes) per column; forward transform, multiplier g(k)/P and the
//           energy partials of the Sec. 4 functional (Parseval form), inverse
//           transform, all in registers.
#include "mbo_kernels.cuh"
#include "mbo_wfft.cuh"
#include "mbo_wshape.cuh"

namespace mbo {
namespace {

// Strided-axis pass (y in 2-D; y and z in 3-D) on a tile of TX adjacent
// x-columns of one complex plane; each column is one sequence of R groups.
template <int MODE, int L, int TX>
__global__ void __launch_bounds__(TX * w_r(L) * w_lq(L), wcol_minb(L, TX))
k_wcol(Geom g, Tables<float> t, float2* W, StatsPtrs sp, int axis) {
  constexpr int R = w_r(L), M = w_m(L), LQ = w_lq(L);
  using F = WarpFFTR<M, LQ, R>;
  constexpr int E = F::E, NT = TX * R * LQ, TS = TX + 1;  // tile row stride (complex)
  constexpr int PS = R * F::RS;                          // transpose slots of one column
  static_assert(TX * PS <= L * TS, "transpose regions must fit in the tile");
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
  const int grp = tid / LQ, l = tid - grp * LQ;
  const int c = grp / R, r = grp - c * R;
  const float2* tw = static_cast<const float2*>(t.tw[axis]);
  const float2* twr = tw + M;

  for (int i = tid; i < L * TX; i += NT) {
    const int p = i / TX, cc = i - p * TX;
    cp_async_elem(&tile[p * TS + cc], base + (long long)p * es + cc);
  }
  cp_async_wait_all();
  __syncthreads();
  float2 v[E];
#pragma unroll
  for (int j = 0; j < E; ++j) v[j] = tile[(R * (l + LQ * j) + r) * TS + c];
  __syncthreads();
  float2* cbase = tile + c * PS;
  if (MODE != AXIS_INV) F::fwd(v, cbase, r, tw, twr, l);
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
      const int p = l + LQ * j + M * r;  // group r holds frequencies k' + M r
      const float omv = omx + gxx * omo + omo2 * __ldg(&omL[p]);  // 1 - g without cancellation
      const float2 z = v[j];
      acc += wx * omv * (z.x * z.x + z.y * z.y);
      if (MODE == AXIS_FGI) {
        const float f = fo * __ldg(&gL[p]);
        v[j] = float2{z.x * f, z.y * f};
      }
    }
  }
  if (MODE == AXIS_FGI || MODE == AXIS_INV) F::inv(v, cbase, r, tw, twr, l);
  if (MODE != AXIS_ENERGY) {
    __syncthreads();  // every column's transposes are done: the tile is free
#pragma unroll
    for (int j = 0; j < E; ++j) tile[(R * (l + LQ * j) + r) * TS + c] = v[j];
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
  k<<<tiles, TX * w_r(L) * w_lq(L), smem, s>>>(g, t, static_cast<float2*>(W), sp, axis);
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

int warp_tile(int L, int nx, int tx) {
  const int t = (tx >= 8 && L <= 1024) ? 8 : 4;  // 1536 and 2048: 4 columns (tile size)
  return (nx % t == 0) ? t : 0;
}

size_t wcol_smem_bytes(int L, int tx) { return (size_t)L * (tx + 1) * sizeof(float2); }

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
  MBO_WCOL_CASE(768)
  if (L == 1536 && TX == 4) return wcol_ltx<1536, 4>(mode, axis, g, t, W, sp, s, prepare_only);
  if (L == 2048 && TX == 4) return wcol_ltx<2048, 4>(mode, axis, g, t, W, sp, s, prepare_only);
#undef MBO_WCOL_CASE
  return cudaErrorInvalidValue;
}

}  // namespace mbo
