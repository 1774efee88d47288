// Shapes and launch helpers shared by the FP32 warp-plan passes (k_warp.cu,
// k_wcol.cu).
#pragma once
#include <cuda_runtime.h>

namespace mbo {

// Length N = R * M with M in {256, 512, 1024} and R in {1, 2, 3} (see WarpFFTR).
inline __host__ __device__ constexpr int w_r(int N) { return N % 3 == 0 ? 3 : (N > 1024 ? 2 : 1); }
inline __host__ __device__ constexpr int w_m(int N) { return N / w_r(N); }
inline __host__ __device__ constexpr int w_lq(int N) { return w_m(N) == 1024 ? 32 : 16; }
// Rows per block of the x pass: one row where a sequence takes 32 lanes or
// three 16-lane groups, else two rows (whole warps for any channel count).
inline __host__ __device__ constexpr int wrow_rb(int N) {
  return (w_lq(N) == 32 || w_r(N) == 3) ? 1 : 2;
}
// Lanes of the block's sequences (rows x complex planes x groups x lanes),
// and threads: the lanes rounded up to whole warps.  The extra lanes (three
// 16-lane groups, odd plane counts) form a partial sequence that runs the
// warps' transposes on a shared-memory region of its own and stores nothing.
inline __host__ __device__ constexpr int wrow_lanes(int N, int NM) {
  return wrow_rb(N) * ((NM * NM + 1) / 2) * w_r(N) * w_lq(N);
}
inline __host__ __device__ constexpr int wrow_threads(int N, int NM) {
  return (wrow_lanes(N, NM) + 31) / 32 * 32;
}
// Sequences with a shared-memory region, the partial one included.
inline __host__ __device__ constexpr int wrow_nseq(int N, int NM) {
  return (wrow_threads(N, NM) + w_r(N) * w_lq(N) - 1) / (w_r(N) * w_lq(N));
}

// Blocks per SM the register budget is sized for: the x pass at 96 registers
// (n <= 3) or 128 (n = 4), the strided passes at 128.  Registers are
// allocated per SM sub-partition (16384 each, warps spread over four), so at
// B registers a thread an SM holds 4 * floor(16384 / (32 B)) warps.
inline __host__ __device__ constexpr int wrow_minb(int N, int NM) {
  return (4 * (16384 / (32 * (NM <= 3 ? 96 : 128)))) / (wrow_threads(N, NM) / 32) > 0
             ? (4 * (16384 / (32 * (NM <= 3 ? 96 : 128)))) / (wrow_threads(N, NM) / 32)
             : 1;
}
inline __host__ __device__ constexpr int wcol_minb(int L, int TX) {
  return 512 / (TX * w_r(L) * w_lq(L)) > 0 ? 512 / (TX * w_r(L) * w_lq(L)) : 1;
}

// Whether the warp-plan launchers ask for programmatic dependent launch; the
// host API sets it for each handle's launches (per host thread).
bool& pdl_flag();

// Launch with programmatic stream serialization (when pdl_flag()): the kernel
// may be scheduled while the previous kernel of the stream finishes, and must
// call pdl_wait() (mbo_tma.cuh) before it touches anything that kernel writes.
template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*kernel)(P...), int blocks, int threads, size_t smem,
                              cudaStream_t s, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_flag() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<A&&>(args)...);
}

template <typename K> inline cudaError_t set_smem_once(K kernel, size_t bytes, size_t& done) {
  if (bytes <= 48 * 1024 || bytes <= done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done = bytes;
  return e;
}

}  // namespace mbo
