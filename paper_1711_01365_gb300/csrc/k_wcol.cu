// FP32 strided passes (y in 2-D; y and z in 3-D) of the MBO step (Algorithm 1
// of Osting & Wang, arXiv:1711.01365) for axes whose plan is the
// warp-cooperative four-step transform (mbo_wfft.cuh).
//
//   k_wcol  persistent: each block walks the tiles b = blockIdx.x,
//           blockIdx.x + gridDim.x, ...; a tile is TX adjacent x-columns of
//           one complex plane along the whole axis.  The tile arrives in
//           shared memory by TMA (4-D tensor map over (x, y, z, plane), boxes
//           of TX x 256 elements, swizzled), each column becomes one sequence
//           (R groups of lanes): forward transform, multiplier g(k)/P and the
//           energy partials of the Sec. 4 functional (Parseval form), inverse
//           transform, all in registers; the result goes back by TMA store.
//           With NBUF = 2 the next tile's load is in flight while a tile is
//           transformed.
#include <type_traits>

#include "mbo_kernels.cuh"
#include "mbo_tma.cuh"
#include "mbo_wfft.cuh"
#include "mbo_wshape.cuh"

namespace mbo {
namespace {

constexpr int kBoxRows = 256;  // TMA box extent along the transformed axis (the hardware limit)

// Swizzle span of a tile (bytes): one tile row (TX * 8 bytes).
constexpr int wcol_swizzle(int L, int TX) { return (void)L, TX * 8; }

template <int L, int TX> struct WcolShape {
  static constexpr int R = w_r(L), M = w_m(L), LQ = w_lq(L);
  // 2048 = 2 x 1024: the cross-group stage first, so that a warp reads
  // consecutive tile rows (8 of 16 bank pairs per access instead of 4)
  static constexpr bool DIF = R == 2;
  using F = typename std::conditional<DIF, WarpFFTRdif<M, LQ, R, TwShared>,
                                      WarpFFTR<M, LQ, R, TwShared>>::type;
  static constexpr int E = F::E;
  static constexpr int NT = TX * R * LQ;
  static constexpr int PS = R * F::RS;  // transpose slots of one column (padded rows)
  static constexpr int TILE = L * TX;   // tile slots (float2), dense, swizzled by TMA
  static constexpr int BUF = (TILE > TX * PS ? TILE : TX * PS);
  static constexpr int BUF_BYTES = ((BUF * 8 + 1023) / 1024) * 1024;
  // split staging (NBUF = 3): a tile buffer the copies use and a separate
  // transpose / store buffer
  static constexpr int TILE_BYTES = ((TILE * 8 + 1023) / 1024) * 1024;
  static constexpr int SCR_BYTES = ((TX * PS * 8 + 1023) / 1024) * 1024;
  static constexpr int BOX = L < kBoxRows ? L : kBoxRows;
  static constexpr int NBOX = L / BOX;
  // 16-byte chunk swizzle of the TMA tile, span SWB bytes (wcol_swizzle)
  static constexpr int SWB = wcol_swizzle(L, TX);
  static constexpr int SWM = SWB / 16 - 1;
  static_assert(TX == 4 || TX == 8 || TX == 16, "tile widths 4, 8, 16");
  static_assert(((DIF ? 1 : R) * LQ * TX) % SWB == 0 && (M * TX) % SWB == 0,
                "the lane's swizzle term must not depend on j or r");
};

// Shared-memory bytes: NBUF tile buffers (NBUF = 3: one tile buffer and one
// transpose buffer), the axis twiddles (L complex) and the axis multiplier and
// 1 - g (L reals each), plus 1 KB of alignment slack.
template <int L, int TX> constexpr size_t wcol_smem(int nbuf) {
  using S = WcolShape<L, TX>;
  const size_t bufs = nbuf == 3 ? (size_t)S::TILE_BYTES + S::SCR_BYTES : (size_t)nbuf * S::BUF_BYTES;
  return 1024 + bufs + (size_t)L * 8 + (size_t)L * 8;
}

template <int MODE, int L, int TX, int NBUF>
__global__ void __launch_bounds__(WcolShape<L, TX>::NT, wcol_minb(L, TX))
k_wcol(Geom g, Tables<float> t, const __grid_constant__ CUtensorMap tm, StatsPtrs sp, int axis,
       int ntiles, const char* __restrict__ pf, long long pf_bytes) {
  using S = WcolShape<L, TX>;
  using F = typename S::F;
  constexpr int R = S::R, M = S::M, LQ = S::LQ, E = S::E, NT = S::NT, PS = S::PS;
  // NBUF = 3: the next tile's copy goes out as soon as a tile is in registers,
  // into the one tile buffer; transposes and the store use a buffer of their own
  constexpr bool SPLIT = NBUF == 3;
  constexpr int NBAR = SPLIT ? 1 : NBUF;  // tile buffers the copies land in
  extern __shared__ unsigned char smem_raw[];
  __shared__ double redd[32];
  __shared__ int s_flag;
  __shared__ __align__(8) unsigned long long bar[NBAR];

  // 1024-byte aligned tile buffers (the TMA swizzle works on address bits
  // 4..9); offsetting the shared array itself keeps every access below a
  // shared-memory instruction
  unsigned char* al = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  float2* s_tw = reinterpret_cast<float2*>(al + (SPLIT ? S::TILE_BYTES + S::SCR_BYTES : NBUF * S::BUF_BYTES));
  float2* scr = reinterpret_cast<float2*>(al + S::TILE_BYTES);  // SPLIT: transposes, store
  float* s_g = reinterpret_cast<float*>(s_tw + L);
  float* s_om = s_g + L;

  const int tid = threadIdx.x;
  const int grp = tid / LQ, l = tid - grp * LQ;
  const int c = grp / R, r = grp - c * R;
  const int nouter = (axis == 1) ? g.nz : g.ny;

  // tile b of this pass: plane q, outer index o, first column x0
  auto coords = [&](int b, int& q, int& o, int& x0) { col_tile(g, nouter, TX, b, q, o, x0); };
  auto issue_load = [&](int b, int buf) {  // thread 0 only
    int q, o, x0;
    coords(b, q, o, x0);
    float2* dst = reinterpret_cast<float2*>(al + buf * S::BUF_BYTES);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&bar[buf], (unsigned)(S::TILE * 8));
#pragma unroll
    for (int bx = 0; bx < S::NBOX; ++bx) {
      if (axis == 1) tma_load_4d(dst + bx * S::BOX * TX, &tm, x0, bx * S::BOX, o, q, &bar[buf]);
      else tma_load_4d(dst + bx * S::BOX * TX, &tm, x0, o, bx * S::BOX, q, &bar[buf]);
    }
  };
  auto prefetch_tile = [&](int b) {  // thread 0 only: DRAM -> L2 ahead of the load
    int q, o, x0;
    coords(b, q, o, x0);
#pragma unroll
    for (int bx = 0; bx < S::NBOX; ++bx) {
      if (axis == 1) tma_prefetch_4d(&tm, x0, bx * S::BOX, o, q);
      else tma_prefetch_4d(&tm, x0, o, bx * S::BOX, q);
    }
  };

  if (tid == 0) {
#pragma unroll
    for (int b = 0; b < NBAR; ++b) mbar_init(&bar[b], 1);
    fence_barrier_init();
  }
  {  // the tables are the handle's own: staged while the previous pass finishes
    const float2* tw = static_cast<const float2*>(t.tw[axis]);
    for (int i = tid; i < L; i += NT) {
      s_tw[i] = tw[i];
      if (MODE == AXIS_FGI || MODE == AXIS_ENERGY) {
        s_g[i] = t.g[axis][i];
        s_om[i] = t.om[axis][i];
      }
    }
  }
  pdl_wait();  // the previous pass's spectrum and run state are complete
  if (sp.respect_stop && *(volatile int*)&sp.st->stop) return;
  pdl_release();
  if (tid == 0) {
    for (int k = 0; k < NBAR && blockIdx.x + k * gridDim.x < ntiles; ++k)
      issue_load(blockIdx.x + k * gridDim.x, k);
    if (blockIdx.x + NBAR * gridDim.x < ntiles) prefetch_tile(blockIdx.x + NBAR * gridDim.x);
    // the caller's L2 hint: this block's share of a buffer the next pass reads
    if (pf_bytes > 0) {
      const long long chunk = ((pf_bytes / gridDim.x + 4095) / 4096) * 4096;
      const long long beg = chunk * blockIdx.x;
      const long long end = beg + chunk < pf_bytes ? beg + chunk : pf_bytes;
      for (long long o = beg; o < end; o += 65536) {
        const long long n = end - o < 65536 ? end - o : 65536;
        bulk_prefetch_l2(pf + o, (unsigned)(n & ~15LL));
      }
    }
  }
  __syncthreads();

  // the lane's rows are R (l + LQ j) + r; their swizzle term depends on l and r only
  // (TMA swizzle: the 16-byte chunk bits 4..6 of an offset XOR its bits 7..9)
  // rows: R (l + LQ j) + r, or with the cross-group stage first l + LQ j + M r
  const int row0 = S::DIF ? l + M * r : R * l + r;
  const int xr = (((row0 * TX * 8) >> 7) & S::SWM);
  const int lane_slot = (row0 * TX + c) ^ (xr << 1);
  constexpr int JSTRIDE = (S::DIF ? 1 : R) * LQ * TX;

  float acc = 0.f;
  bool ok = true;
  int it = 0;
  for (int b = blockIdx.x; b < ntiles; b += gridDim.x, ++it) {
    const int buf = NBAR == 1 ? 0 : (it & 1);
    const unsigned parity = NBAR == 1 ? (it & 1) : ((it >> 1) & 1);
    float2* tile = reinterpret_cast<float2*>(al + buf * S::BUF_BYTES);
    // this tile's per-column factors, loaded before the wait so that their
    // latency overlaps it: g_x, 1 - g_x and the Parseval weight of column x
    // (and g_y, 1 - g_y of the outer index in 3-D)
    int q, o, x0;
    coords(b, q, o, x0);
    float gxx = 0.f, omx = 0.f, wx = 0.f, go = 1.f, omo = 0.f;
    if (MODE == AXIS_FGI || MODE == AXIS_ENERGY) {
      const int x = x0 + c;
      gxx = t.g[0][x];
      omx = t.om[0][x];
      wx = col_weight(g, q, x);
      if (g.ndim == 3) {
        go = t.g[1][o];
        omo = t.om[1][o];
      }
    }
    ok = __syncthreads_and(mbar_wait_bounded(&bar[buf], parity)) != 0;
    if (!ok) break;
    // L2 prefetch of the tile loaded one copy later (SPLIT: the prologue
    // covered b + gridDim.x, loaded below)
    if (SPLIT) {
      if (tid == 0 && b + 2 * gridDim.x < ntiles) prefetch_tile(b + 2 * gridDim.x);
    } else if (tid == 0 && it > 0 && b + NBAR * gridDim.x < ntiles) {
      prefetch_tile(b + NBAR * gridDim.x);
    }
    float2 v[E];
#pragma unroll
    for (int j = 0; j < E; ++j) v[j] = tile[lane_slot + j * JSTRIDE];
    // SPLIT: the previous tile's store has read the transpose buffer
    if (SPLIT && tid == 0) bulk_wait_read_all();
    __syncthreads();  // the tile is in registers: its buffer is free (holds the transposes)
    if (SPLIT && tid == 0 && b + gridDim.x < ntiles) issue_load(b + gridDim.x, 0);
    float2* work = SPLIT ? scr : tile;  // transposes and the store
    float2* cbase = work + c * PS;
    const float2* tw = s_tw;
    const float2* twr = s_tw + M;
    if (MODE != AXIS_INV) F::fwd(v, cbase, r, tw, twr, l);
    if (MODE == AXIS_FGI || MODE == AXIS_ENERGY) {
      // the last axis applies g(k) = g_x g_y (g_z); in 3-D the y frequency is
      // the outer index o of this tile (the y pass ran before).
      const float fo = gxx * go * t.inv_p;
      const float omo2 = gxx * go;
      const float omb = omx + gxx * omo;
#pragma unroll
      for (int j = 0; j < E; ++j) {
        // group r holds frequencies k' + M r, or R k' + r (k' = l + LQ j)
        const int p = S::DIF ? R * (l + LQ * j) + r : l + LQ * j + M * r;
        const float omv = omb + omo2 * s_om[p];  // 1 - g without cancellation
        const float2 z = v[j];
        acc += wx * omv * (z.x * z.x + z.y * z.y);
        if (MODE == AXIS_FGI) {
          const float f = fo * s_g[p];
          v[j] = float2{z.x * f, z.y * f};
        }
      }
    }
    if (MODE == AXIS_FGI || MODE == AXIS_INV) F::inv(v, cbase, r, tw, twr, l);
    __syncthreads();  // every column's transposes are done
    const int nb = b + NBAR * gridDim.x;  // the tile that reuses this buffer (not SPLIT)
    if (MODE != AXIS_ENERGY) {
#pragma unroll
      for (int j = 0; j < E; ++j) work[lane_slot + j * JSTRIDE] = v[j];
      fence_proxy_async_smem();
      __syncthreads();
      if (tid == 0) {
#pragma unroll
        for (int bx = 0; bx < S::NBOX; ++bx) {
          if (axis == 1) tma_store_4d(&tm, x0, bx * S::BOX, o, q, work + bx * S::BOX * TX);
          else tma_store_4d(&tm, x0, o, bx * S::BOX, q, work + bx * S::BOX * TX);
        }
        bulk_commit();
        if (!SPLIT && nb < ntiles) {
          bulk_wait_read_all();  // the store has read the buffer: the next load may overwrite it
          issue_load(nb, buf);
        }
      }
    } else if (!SPLIT && tid == 0 && nb < ntiles) {
      issue_load(nb, buf);
    }
  }
  if (tid == 0) bulk_wait_all();
  if (!ok) {
    // a tile load did not land in time: record it, give the copies still in
    // flight a bounded wait, and leave (statistics of this launch are void)
    if (tid == 0) {
      atomicOr(&sp.st->err, kErrWaitTimeout);
      for (int k = 0; k < NBAR; ++k) (void)mbar_wait_bounded(&bar[k], 0), (void)mbar_wait_bounded(&bar[k], 1);
    }
    return;
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

// Blocks of a kernel that fit on one SM, and the SM count (cached per kernel).
template <typename K> int persistent_blocks(K kernel, int threads, size_t smem, int& per_sm) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  if (per_sm < 1) per_sm = 1;
  return sms * per_sm;
}

template <int MODE, int L, int TX, int NBUF>
cudaError_t wcol_m(const Geom& g, const Tables<float>& t, const CUtensorMap* tm, const StatsPtrs& sp,
                   int axis, cudaStream_t s, bool prepare_only, const void* pf, long long pf_bytes) {
  auto k = k_wcol<MODE, L, TX, NBUF>;
  static size_t done = 0;
  static int slots = 0, per_sm = 0;
  const size_t smem = wcol_smem<L, TX>(NBUF);
  cudaError_t e = set_smem_once(k, smem, done);
  if (e != cudaSuccess) return e;
  if (!slots) slots = persistent_blocks(k, WcolShape<L, TX>::NT, smem, per_sm);
  if (prepare_only) return cudaSuccess;
  if (!tm) return cudaErrorInvalidValue;
  const int nouter = axis == 1 ? g.nz : g.ny;
  const int tiles = col_tiles(g, nouter, TX);
  const int blocks = tiles < slots ? tiles : slots;
  return launch_pdl(k, blocks, WcolShape<L, TX>::NT, smem, s, g, t, *tm, sp, axis, tiles,
                    static_cast<const char*>(pf), pf ? pf_bytes : 0LL);
}

struct L2Hint {
  const void* p;
  long long bytes;
};

template <int L, int TX, int NB>
cudaError_t wcol_ltxb(AxisMode mode, int axis, const Geom& g, const Tables<float>& t,
                      const CUtensorMap* tm, const StatsPtrs& sp, cudaStream_t s, bool prep,
                      L2Hint pf) {
  switch (mode) {
    case AXIS_FWD: return wcol_m<AXIS_FWD, L, TX, NB>(g, t, tm, sp, axis, s, prep, pf.p, pf.bytes);
    case AXIS_INV: return wcol_m<AXIS_INV, L, TX, NB>(g, t, tm, sp, axis, s, prep, pf.p, pf.bytes);
    case AXIS_FGI: return wcol_m<AXIS_FGI, L, TX, NB>(g, t, tm, sp, axis, s, prep, pf.p, pf.bytes);
    default: return wcol_m<AXIS_ENERGY, L, TX, NB>(g, t, tm, sp, axis, s, prep, pf.p, pf.bytes);
  }
}

template <int L, int TX>
cudaError_t wcol_ltx(AxisMode mode, int axis, const Geom& g, const Tables<float>& t,
                     const CUtensorMap* tm, const StatsPtrs& sp, cudaStream_t s, bool prep,
                     int stages, L2Hint pf) {
  if (stages == 3) return wcol_ltxb<L, TX, 3>(mode, axis, g, t, tm, sp, s, prep, pf);
  if (stages == 2) return wcol_ltxb<L, TX, 2>(mode, axis, g, t, tm, sp, s, prep, pf);
  return wcol_ltxb<L, TX, 1>(mode, axis, g, t, tm, sp, s, prep, pf);
}

}  // namespace

int warp_tile(int L, int nx, int tx) {
  // 16 columns (one 128-byte line per tile row) up to 512 rows; 1536 and 2048:
  // 4 columns (tile size)
  if (tx >= 16 && L <= 512 && nx % 16 == 0) return 16;
  const int t = (tx >= 8 && L <= 1024) ? 8 : 4;
  return (nx % t == 0) ? t : 0;
}

size_t wcol_smem_bytes(int L, int tx, int stages) {
#define MBO_WSM(LEN)                                        \
  if (L == LEN) return tx == 8 ? wcol_smem<LEN, 8>(stages) : wcol_smem<LEN, 4>(stages);
  if (L == 256 && tx == 16) return wcol_smem<256, 16>(stages);
  if (L == 512 && tx == 16) return wcol_smem<512, 16>(stages);
  MBO_WSM(256)
  MBO_WSM(512)
  MBO_WSM(768)
  MBO_WSM(1024)
  MBO_WSM(1536)
  MBO_WSM(2048)
#undef MBO_WSM
  return 0;
}

bool wcol_tensor_map(CUtensorMap* map, void* W, const Geom& g, int axis, int tx) {
  using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                CUtensorMapFloatOOBfill);
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
      return false;
    fn = reinterpret_cast<EncodeFn>(p);
  }
  const int L = axis == 1 ? g.ny : g.nz;
  const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)g.Q};
  const cuuint64_t strides[3] = {(cuuint64_t)g.nx * 8, (cuuint64_t)g.nx * g.ny * 8,
                                 (cuuint64_t)g.P * 8};
  const cuuint32_t bx = (cuuint32_t)(L < kBoxRows ? L : kBoxRows);
  const cuuint32_t box[4] = {(cuuint32_t)tx, axis == 1 ? bx : 1u, axis == 1 ? 1u : bx, 1u};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  const int swb = wcol_swizzle(L, tx);
  const CUtensorMapSwizzle sw = swb == 128  ? CU_TENSOR_MAP_SWIZZLE_128B
                                : swb == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                            : CU_TENSOR_MAP_SWIZZLE_32B;
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, W, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_wcol(AxisMode mode, int axis, const Geom& g, const Tables<float>& t, void* W,
                        const StatsPtrs& sp, int tx, cudaStream_t s, bool prepare_only,
                        const CUtensorMap* tm, int stages, const void* l2_hint,
                        long long l2_hint_bytes) {
  (void)W;  // addressed through the tensor map
  const L2Hint pf{l2_hint, l2_hint_bytes};
  const int L = axis == 1 ? g.ny : g.nz;
  const int TX = warp_tile(L, g.nx, tx);
#define MBO_WCOL_CASE(LEN)                                                              \
  if (L == LEN) {                                                                       \
    if (TX == 8) return wcol_ltx<LEN, 8>(mode, axis, g, t, tm, sp, s, prepare_only, stages, pf); \
    if (TX == 4) return wcol_ltx<LEN, 4>(mode, axis, g, t, tm, sp, s, prepare_only, stages, pf); \
  }
  if (L == 512 && TX == 16)
    return wcol_ltx<512, 16>(mode, axis, g, t, tm, sp, s, prepare_only, stages, pf);
  if (L == 256 && TX == 16)
    return wcol_ltx<256, 16>(mode, axis, g, t, tm, sp, s, prepare_only, stages, pf);
  MBO_WCOL_CASE(1024)
  MBO_WCOL_CASE(512)
  MBO_WCOL_CASE(256)
  MBO_WCOL_CASE(768)
  if (L == 1536 && TX == 4)
    return wcol_ltx<1536, 4>(mode, axis, g, t, tm, sp, s, prepare_only, stages, pf);
  if (L == 2048 && TX == 4)
    return wcol_ltx<2048, 4>(mode, axis, g, t, tm, sp, s, prepare_only, stages, pf);
#undef MBO_WCOL_CASE
  return cudaErrorInvalidValue;
}

}  // namespace mbo
