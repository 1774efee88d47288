// Internal types shared by the host API (mbo_api.cu) and the kernels
// (mbo_kernels.cuh).  Not part of the public ABI.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mbo {

constexpr int kMaxStages = 8;
constexpr int kRing = 1024;      // step-record ring (power of two)
// Row and axis kernels are launched with at most this many threads and are
// compiled so that 768 (FP32) or 384 (FP64) threads fit on an SM.
constexpr int kMaxThreads = 384;
constexpr int kFallbackCap = 64; // per-row FP64 re-projection slots (FP32 path)

// Division of x < 65536 by a fixed d < 65536: a shift when d is a power of
// two (shift >= 0), else the high word of x * ceil(2^32 / d), which is exact
// in that range.
struct FastDiv {
  unsigned mul;
  int shift;
};

// One forward stage: radix rad on blocks of length lb = N / (rad_0 ... rad_{st-1});
// a butterfly (block b, offset n1 < m = lb / rad) owns positions b*lb + n1 + m*j.
// tw is the offset of the stage's twiddles exp(-2 pi i n1 j / lb), stored
// [j - 1][n1] (n1 fastest, so lanes with consecutive n1 read consecutive
// entries), in the axis twiddle table (unused when m == 1).
struct Stage {
  int rad, lb, m, tw;
  int pstride;  // p -> p + p/8 maps base + j*m to phi(base) + j*pstride (0: not affine)
  FastDiv dm;   // division by m
  FastDiv dnr;  // division by N / rad
};

// Transform plan of one axis.
//   lq == 0: the in-place network of nst stages (forward stages applied in
//            order, product = N); the spectrum is left digit-reversed.
//   lq >  0: the warp-cooperative four-step transform of M = lq * (M / lq)
//            points held in registers by lq lanes per sequence, N = rad0 * M
//            (rad0 > 1: rad0 such sequences combined by a length-rad0 DFT);
//            the spectrum is in natural order and the twiddle table holds
//            exp(-2 pi i l k2 / M) at [k2][l] (k2 < M / lq, l < lq), then
//            exp(-2 pi i r k / N) at M + (r - 1) M + k (0 < r < rad0, k < M).
struct Plan {
  int nst;
  int lq;
  int len;   // N
  int rad0;  // warp plans: N = rad0 * M with a length-M warp transform (rad0 in 1..3)
  Stage st[kMaxStages];
};

// Device-resident state of a run.  Accumulators are reset by the finaliser
// of the projection pass at the end of every step.
struct RunState {
  unsigned long long maxdelta_bits;  // bit pattern of a non-negative double (atomicMax)
  unsigned long long flips;
  unsigned long long fallback;
  unsigned long long nonfinite;
  double defect;       // sum_x (n - |A(x)|_F^2) of the field whose spectrum is in the workspace
  double energy_last;  // last energy written by a transform pass
  long long step;      // steps completed in this run
  int stop;            // 1 once a stationary step was seen (run loop only)
  unsigned int err;    // device error bits (kErr*), surfaced by the host at sync points
  unsigned int nep;    // blocks of the last transform pass that left energy partials in epart
  unsigned int pad_;
};

// Device error bits of RunState::err.
constexpr unsigned int kErrWaitTimeout = 1u;  // a bounded wait (copy or barrier) gave up

// Step-record ring, indexed by step & (kRing - 1).
struct Hist {
  double* energy;
  double* maxdelta;
  long long* flips;
  long long* fallback;
  long long* nonfinite;
};

// Geometry of a field.  dims are (nz, ny, nx); nz = 1 in 2-D.
struct Geom {
  int ndim;
  int nx, ny, nz;
  long long P;
  int n, C, Q;
  double tau;
  // x-columns of the last complex plane that the workspace keeps and the
  // strided passes transform.  nx, unless that plane carries one real
  // channel (n*n odd) and the x spectrum is in natural order: its spectrum is
  // then Hermitian along x, columns kx > nx/2 are the conjugates of columns
  // nx - kx, and only the first xh = min(nx, roundup(nx/2 + 1, 16)) are kept.
  int xh;
};

// Tile count of a strided pass (tiles of tx x-columns, nouter outer rows per plane).
__host__ __device__ inline int col_tiles(const Geom& g, int nouter, int tx) {
  return (g.Q - 1) * nouter * (g.nx / tx) + nouter * (g.xh / tx);
}
// Plane q, outer index o and first column x0 of strided-pass tile b.
__host__ __device__ inline void col_tile(const Geom& g, int nouter, int tx, int b, int& q, int& o,
                                         int& x0) {
  const int xt = g.nx / tx;
  const int full = (g.Q - 1) * nouter * xt;
  if (b < full) {
    q = b / (nouter * xt);
    const int rem = b - q * nouter * xt;
    o = rem / xt;
    x0 = (rem - o * xt) * tx;
  } else {
    const int xtl = g.xh / tx;
    const int rem = b - full;
    q = g.Q - 1;
    o = rem / xtl;
    x0 = (rem - o * xtl) * tx;
  }
}
// Weight of spectrum column kx of plane q in the Parseval sums: 2 for the
// kept half of a Hermitian plane (each column stands for itself and its
// conjugate), 1 for its self-conjugate columns 0 and nx/2 and for full
// planes, 0 for the padding columns past nx/2.
__host__ __device__ inline float col_weight(const Geom& g, int q, int kx) {
  if (q != g.Q - 1 || g.xh == g.nx) return 1.f;
  if (kx == 0 || 2 * kx == g.nx) return 1.f;
  return 2 * kx < g.nx ? 2.f : 0.f;
}

// Per-axis tables in the element type R (0 = x, 1 = y, 2 = z).
template <typename R> struct Tables {
  const void* tw[3];   // per-stage twiddles of each axis (see Stage::tw)
  const R* g[3];       // exp(-4 pi^2 tau k^2), k the signed frequency held at each
                       // spectrum position of the forward transform (digit-reversed
                       // or natural, per the axis plan)
  const R* om[3];      // 1 - g at the same positions (computed as -expm1)
  Plan plan[3];
  R inv_p;             // 1 / P, folded into the multiplier
};

// Pass modes of the strided-axis kernel.
enum AxisMode { AXIS_FWD = 0, AXIS_INV = 1, AXIS_FGI = 2, AXIS_ENERGY = 3 };
// Modes of the row (x-axis) kernel.
enum RowMode { ROW_FWD = 0, ROW_INV_OUT = 1, ROW_INV_PROJECT_FWD = 2 };

// Buffers of the deterministic two-level grid sum (see grid_sum).
constexpr int kReduceGroup = 256;
constexpr unsigned kReduceOneLevel = 2048;  // grids up to this size reduce in one level
struct ReduceBufs {
  double* part;          // one partial per block
  double* gpart;         // one total per group of kReduceGroup blocks
  unsigned int* gcount;  // arrivals per group (zero between launches)
  unsigned int* done;    // groups finished (zero between launches)
};

struct StatsPtrs {
  RunState* st;
  Hist hist;
  ReduceBufs rb;       // per-block partial sums
  int respect_stop;    // 1: return at once if st->stop is set
  int do_stats;        // 1: accumulate and finalise statistics
  double tol;          // stationarity tolerance (< 0: never stop)
  // Deferred energy (fused step only; nullptr otherwise): the multiplier pass
  // leaves one Parseval partial per block here (and the block count in
  // RunState::nep) instead of reducing them itself, and the x pass's
  // finaliser, which runs next and reduces anyway, adds them up in block
  // order and records E^tau.  This takes one grid-wide reduction off the
  // critical path of each step.
  double* epart;
};

// Radix selection of the n_plus smallest (key, index) pairs (volume-preserving
// step).  After the passes, (hi, lo) is the n_plus-th smallest pair; a point is
// selected iff (key, index) <= (hi, lo) and n_plus > 0.
struct SelectState {
  unsigned long long hi;     // key part of the prefix / result
  unsigned int lo;           // index part
  unsigned int pad_;
  unsigned long long k;      // remaining rank (1-based) inside the current prefix
  unsigned long long n_plus; // points to select
  unsigned int hist[256];
};

cudaError_t launch_select(unsigned long long* keys, long long P, SelectState* ss, int blocks,
                          cudaStream_t s);
cudaError_t launch_select_init(SelectState* ss, long long n, cudaStream_t s);

// Launchers (defined per element type in k_f32.cu / k_f64.cu).
template <typename R>
cudaError_t launch_row(RowMode mode, const Geom& g, const Tables<R>& t, const R* A_in, R* A_out,
                       void* W, const StatsPtrs& sp, double fallback_sigma, int threads,
                       cudaStream_t s);
template <typename R>
cudaError_t launch_axis(AxisMode mode, int axis, const Geom& g, const Tables<R>& t, void* W,
                        const StatsPtrs& sp, int tx, int threads, cudaStream_t s,
                        const CUtensorMap* tm = nullptr, int stages = 1,
                        const void* l2_hint = nullptr, long long l2_hint_bytes = 0);
template <typename R>
cudaError_t launch_project(const Geom& g, const R* At, R* B, int8_t* det_sign,
                           double fallback_sigma, cudaStream_t s);

// Plan helpers (mbo_api.cu).
bool factor23(int64_t N, int& a, int& b);
FastDiv make_div(unsigned d);
Plan make_plan(int N);
// Plan of one axis of a geometry: the warp-cooperative plan (FP32, lengths
// 256, 512, 768, 1024, 1536, 2048; strided axes need nx % 4 == 0) where one
// exists, else make_plan.
Plan axis_plan(const Geom& g, int axis, bool f32);
int plan_twiddles(const Plan& p);
int pick_tx(int nx, int cap);

// FP32 passes over warp-plan axes (k_warp.cu).
bool& pdl_flag();  // programmatic dependent launch of these passes (per host thread)
bool& wrow_persistent_flag();  // x pass as one wave of blocks over the row groups (per host thread)
double wrow_waves(const Geom& g);  // waves of blocks of the projecting x pass
bool warp_plan_length(int N);
int warp_plan_radix(int N);
int warp_tile(int L, int nx, int tx);  // columns per tile of the strided pass (4, 8 or 16; 0: none)
size_t wrow_smem_bytes(const Geom& g, int N, bool fallback);
size_t wcol_smem_bytes(int L, int tx, int stages);
cudaError_t launch_wrow(RowMode mode, const Geom& g, const Tables<float>& t, const float* A_in,
                        float* A_out, void* W, const StatsPtrs& sp, double fallback_sigma,
                        cudaStream_t s, bool prepare_only);
cudaError_t launch_wcol(AxisMode mode, int axis, const Geom& g, const Tables<float>& t, void* W,
                        const StatsPtrs& sp, int tx, cudaStream_t s, bool prepare_only,
                        const CUtensorMap* tm, int stages, const void* l2_hint = nullptr,
                        long long l2_hint_bytes = 0);
// TMA descriptor of the workspace W (4-D: x, y, z, plane; float2 elements)
// with the box of the strided pass along `axis` (tile width tx).  Host.
bool wcol_tensor_map(CUtensorMap* map, void* W, const Geom& g, int axis, int tx);

template <typename R> cudaError_t prepare_kernels(const Geom& g, const Tables<R>& t, int tx,
                                                  int stages);
template <typename R>
cudaError_t launch_volume(int which, const Geom& g, const R* At, R* A, unsigned long long* keys,
                          SelectState* ss, const StatsPtrs& sp, double fb, int blocks,
                          cudaStream_t s);

// Replace the per-axis multipliers of a handle's diffusion (mbo_api.cu).
// mult[ax] (ax = 0: x, 1: y, 2: z; z ignored in 2-D) holds N_ax values in
// natural frequency order: index k is the signed frequency k (2k <= N) or
// k - N.  The diffusion then multiplies spectrum entry (kz, ky, kx) by
// mult[2][kz] mult[1][ky] mult[0][kx] / P.  Host; synchronous.
bool set_axis_multipliers(struct mbo_ctx* h, const double* const* mult);

// Shared memory bytes of the row kernel for a geometry.
size_t row_smem_bytes(const Geom& g, size_t elem_bytes, bool fallback);
size_t axis_smem_bytes(int len, int tx, size_t elem_bytes);

}  // namespace mbo
