// Radix selection of the n_plus smallest (key, index) pairs, for the
// volume-preserving step (Sec. 7: the n_plus points of largest dE take the
// SO(n) class; the key is dE complemented so that smaller keys are larger dE,
// and the grid index breaks ties, lower index first).  Twelve MSB-first passes
// over 8-bit digits of the 96-bit composite (64-bit key, 32-bit index); each
// pass histograms the digit among the points that match the prefix found so
// far, and one thread picks the bucket that holds the remaining rank.
#include "mbo_dev.cuh"

namespace mbo {

__device__ __forceinline__ unsigned digit_of(unsigned long long key, unsigned idx, int d) {
  return d < 8 ? (unsigned)((key >> (56 - 8 * d)) & 0xffu) : ((idx >> (24 - 8 * (d - 8))) & 0xffu);
}

// The top 8*d bits of (key, idx) equal those of the prefix found so far.
__device__ __forceinline__ bool prefix_match(unsigned long long key, unsigned idx,
                                             unsigned long long hi, unsigned lo, int d) {
  if (d == 0) return true;
  if (d <= 8) {
    const int sh = 64 - 8 * d;
    return (key >> sh) == (hi >> sh);
  }
  if (key != hi) return false;
  const int sh = 32 - 8 * (d - 8);
  return (idx >> sh) == (lo >> sh);
}

// n >= 0: select n points; n < 0: select the count already in ss->n_plus.
__global__ void k_select_init(SelectState* ss, long long n) {
  if (threadIdx.x == 0) {
    if (n >= 0) ss->n_plus = (unsigned long long)n;
    ss->hi = 0;
    ss->lo = 0;
    ss->k = ss->n_plus;
  }
  for (int i = threadIdx.x; i < 256; i += blockDim.x) ss->hist[i] = 0;
}

__global__ void __launch_bounds__(256)
k_select_hist(const unsigned long long* __restrict__ keys, long long P, SelectState* ss, int d) {
  __shared__ unsigned int h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const unsigned long long hi = ss->hi;
  const unsigned lo = ss->lo;
  if (ss->n_plus == 0) return;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < P;
       x += (long long)gridDim.x * blockDim.x) {
    const unsigned long long key = keys[x];
    if (prefix_match(key, (unsigned)x, hi, lo, d)) atomicAdd(&h[digit_of(key, (unsigned)x, d)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (h[i]) atomicAdd(&ss->hist[i], h[i]);
}

__global__ void k_select_pick(SelectState* ss, int d) {
  if (threadIdx.x != 0 || ss->n_plus == 0) return;
  const unsigned long long k = ss->k;
  unsigned long long cum = 0;
  int b = 0;
  for (; b < 255; ++b) {
    const unsigned long long c = ss->hist[b];
    if (cum + c >= k) break;
    cum += c;
  }
  ss->k = k - cum;
  if (d < 8) ss->hi |= ((unsigned long long)b) << (56 - 8 * d);
  else ss->lo |= ((unsigned)b) << (24 - 8 * (d - 8));
  for (int i = 0; i < 256; ++i) ss->hist[i] = 0;
}

cudaError_t launch_select(unsigned long long* keys, long long P, SelectState* ss, int blocks,
                          cudaStream_t s) {
  for (int d = 0; d < 12; ++d) {
    k_select_hist<<<blocks, 256, 0, s>>>(keys, P, ss, d);
    k_select_pick<<<1, 32, 0, s>>>(ss, d);
  }
  return cudaGetLastError();
}

cudaError_t launch_select_init(SelectState* ss, long long n, cudaStream_t s) {
  k_select_init<<<1, 256, 0, s>>>(ss, n);
  return cudaGetLastError();
}

}  // namespace mbo
