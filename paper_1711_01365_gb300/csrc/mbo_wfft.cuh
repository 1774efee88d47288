// Warp-cooperative four-step transforms for FP32 axes of length 256, 512 and
// 1024 (the diffusion of Sec. 5.1 of Osting & Wang, arXiv:1711.01365, along
// one axis).
//
// A sequence of N = LQ * E points is held by LQ lanes, E points each: lane l
// holds a[l + LQ j] in register j.  The forward transform
//   X[k] = sum_x a[x] exp(-2 pi i x k / N)
// factors with x = x1 + LQ x2 and k = k2 + E k1 as
//   X[k2 + E k1] = sum_x1 W_LQ^(x1 k1) W_N^(x1 k2) sum_x2 a[x1 + LQ x2] W_E^(x2 k2)
// (W_M = exp(-2 pi i / M)): a length-E DFT in each lane's registers, one
// twiddle per register, a transpose through the warp's own shared-memory
// region, and length-LQ DFTs in registers again.  The spectrum comes out in
// natural order with lane l holding X[l + LQ j] in register j -- the layout the
// inverse transform takes as input -- so a forward transform, a multiplier
// and an inverse transform run on registers with no block barrier.  The
// transposes need only __syncwarp.
#pragma once
#include "mbo_dev.cuh"

namespace mbo {

// cos(pi j / 16) for any integer j.
__host__ __device__ constexpr double cos_pi16(int j) {
  j = ((j % 32) + 32) % 32;
  const int a = j <= 16 ? j : 32 - j;  // cos(pi a / 16), 0 <= a <= 16
  const int b = a <= 8 ? a : 16 - a;   // |cos| = cos(pi b / 16), 0 <= b <= 8
  const double c = b == 0   ? 1.0
                   : b == 1 ? 0.98078528040323044913
                   : b == 2 ? 0.92387953251128675613
                   : b == 3 ? 0.83146961230254523708
                   : b == 4 ? 0.70710678118654752440
                   : b == 5 ? 0.55557023301960222474
                   : b == 6 ? 0.38268343236508977173
                   : b == 7 ? 0.19509032201612826785
                            : 0.0;
  return a <= 8 ? c : -c;
}

// a * W^j with W = exp(DIR 2 pi i / 32); j is a constant after unrolling.
template <int DIR, typename V> __device__ __forceinline__ V twiddle32(V a, int j) {
  using R = decltype(a.x);
  j &= 31;
  if (j == 0) return a;
  if (j == 8) return DIR < 0 ? V{a.y, -a.x} : V{-a.y, a.x};
  if (j == 16) return V{-a.x, -a.y};
  if (j == 24) return DIR < 0 ? V{-a.y, a.x} : V{a.y, -a.x};
  const R c = (R)cos_pi16(j), s = (R)(DIR * cos_pi16(j - 8));
  return V{a.x * c - a.y * s, a.x * s + a.y * c};
}

// Length-32 DFT in registers, natural order in and out: 32 = 4 x 8 with
// n = n1 + 8 n2, k = k2 + 4 k1 (length-4 DFTs over n2, twiddles W32^(n1 k2),
// length-8 DFTs over n1).
template <int DIR, typename V> __device__ __forceinline__ void dft32(V* v) {
  V u[8][4];
#pragma unroll
  for (int n1 = 0; n1 < 8; ++n1) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) u[n1][n2] = v[n1 + 8 * n2];
    dft4<DIR>(u[n1]);
#pragma unroll
    for (int k2 = 1; k2 < 4; ++k2) u[n1][k2] = twiddle32<DIR>(u[n1][k2], n1 * k2);
  }
#pragma unroll
  for (int k2 = 0; k2 < 4; ++k2) {
    V w[8];
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) w[n1] = u[n1][k2];
    dft8<DIR>(w);
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) v[k2 + 4 * k1] = w[k1];
  }
}

template <int DIR, int LEN, typename V> __device__ __forceinline__ void rdft(V* v) {
  if constexpr (LEN == 32) dft32<DIR>(v);
  else dft<DIR, LEN>(v);
}

// Twiddle-table loads: TwGlobal reads a global table through the read-only
// data path, TwShared a copy staged in shared memory.
struct TwGlobal {
  template <typename V> __device__ __forceinline__ static V ld(const V* p) { return __ldg(p); }
};
struct TwShared {
  template <typename V> __device__ __forceinline__ static V ld(const V* p) { return *p; }
};

template <int N, int LQ, class TW = TwGlobal> struct WarpFFT {
  static constexpr int E = N / LQ;         // points per lane
  static constexpr int G = E / LQ;         // length-LQ DFTs per lane in the second step
  static constexpr int RS = (LQ + 1) * E;  // transpose region of one sequence (complex)
  static_assert(E % LQ == 0 && (E == 16 || E == 32) && (LQ == 16 || LQ == 32),
                "supported shapes: 16x16, 16x32, 32x32");

  // v[j] = a[l + LQ j]  ->  v[j] = X[l + LQ j].  buf: the sequence's RS slots;
  // tw[k2 * LQ + l] = W_N^(l k2).
  template <typename V>
  __device__ __forceinline__ static void fwd(V (&v)[E], V* buf, const V* __restrict__ tw, int l) {
    rdft<-1, E>(v);
#pragma unroll
    for (int k2 = 1; k2 < E; ++k2) v[k2] = cmul(v[k2], TW::ld(&tw[k2 * LQ + l]));
#pragma unroll
    for (int k2 = 0; k2 < E; ++k2) buf[k2 * (LQ + 1) + l] = v[k2];
    __syncwarp();
#pragma unroll
    for (int r = 0; r < G; ++r) {
      V u[LQ];
#pragma unroll
      for (int x1 = 0; x1 < LQ; ++x1) u[x1] = buf[(l + LQ * r) * (LQ + 1) + x1];
      rdft<-1, LQ>(u);
#pragma unroll
      for (int k1 = 0; k1 < LQ; ++k1) v[r + G * k1] = u[k1];
    }
    __syncwarp();
  }

  // v[j] = X[l + LQ j]  ->  v[j] = sum_k X[k] exp(+2 pi i (l + LQ j) k / N)
  // (unnormalised): the forward steps transposed and conjugated, in reverse.
  template <typename V>
  __device__ __forceinline__ static void inv(V (&v)[E], V* buf, const V* __restrict__ tw, int l) {
#pragma unroll
    for (int r = 0; r < G; ++r) {
      V u[LQ];
#pragma unroll
      for (int k1 = 0; k1 < LQ; ++k1) u[k1] = v[r + G * k1];
      rdft<+1, LQ>(u);
#pragma unroll
      for (int x1 = 0; x1 < LQ; ++x1) buf[(l + LQ * r) * (LQ + 1) + x1] = u[x1];
    }
    __syncwarp();
#pragma unroll
    for (int k2 = 0; k2 < E; ++k2) v[k2] = buf[k2 * (LQ + 1) + l];
    __syncwarp();
#pragma unroll
    for (int k2 = 1; k2 < E; ++k2) {
      V c = TW::ld(&tw[k2 * LQ + l]);
      c.y = -c.y;
      v[k2] = cmul(v[k2], c);
    }
    rdft<+1, E>(v);
  }
};

}  // namespace mbo

namespace mbo {

// Lengths N = R * M (R = 2 or 3, M one of the lengths above): R groups of LQ
// lanes, group r holding the sub-sequence a[R x' + r] (x' = l + LQ j), run the
// length-M transform; a twiddle W_N^(r k') and a length-R DFT across the groups,
// through shared memory, complete it:
//   X[k' + M s] = sum_r W_R^(r s) W_N^(r k') Y_r[k'],   Y_r = DFT_M(a[R x' + r]),
// so group s ends up holding X[k' + M s] (k' = l + LQ j): natural order again.
// The inverse runs the steps transposed and conjugated.  Group r works in the
// r-th of R consecutive regions of RS slots; for R > 1 the cross-group steps
// end with a block barrier, so every thread of the block must call them.  For
// R = 1 the calls are those of WarpFFT.
template <int M, int LQ, int R, class TW = TwGlobal> struct WarpFFTR {
  using F = WarpFFT<M, LQ, TW>;
  static constexpr int E = F::E;
  static constexpr int RS = F::RS;

  // W_R^(e) for a constant e
  template <typename V> __device__ __forceinline__ static V rot(V a, int e) {
    e %= R;
    if (R == 2) return e ? V{-a.x, -a.y} : a;
    constexpr float h = 0.86602540378443864676f;  // sqrt(3)/2, W_3 = -1/2 - i h
    if (e == 0) return a;
    const float s = (e == 1) ? -h : h;  // Im W_3^e
    return V{-0.5f * a.x - s * a.y, -0.5f * a.y + s * a.x};
  }

  // tw: the length-M table [k2][l]; twr: W_N^(r k') at [(r - 1) * M + k'].
  template <typename V>
  __device__ __forceinline__ static void fwd(V (&v)[E], V* base, int r, const V* __restrict__ tw,
                                             const V* __restrict__ twr, int l) {
    if constexpr (R == 1) {
      F::fwd(v, base, tw, l);
      return;
    }
    F::fwd(v, base + r * RS, tw, l);
    if (r > 0) {
#pragma unroll
      for (int j = 0; j < E; ++j) v[j] = cmul(v[j], TW::ld(&twr[(r - 1) * M + l + LQ * j]));
    }
#pragma unroll
    for (int j = 0; j < E; ++j) base[r * RS + l + LQ * j] = v[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < E; ++j) {
      V acc = base[l + LQ * j];
#pragma unroll
      for (int rr = 1; rr < R; ++rr) acc = cadd(acc, rot(base[rr * RS + l + LQ * j], rr * r));
      v[j] = acc;
    }
    __syncthreads();
  }

  // group s holds X[k' + M s]  ->  group r holds sum_k X[k] exp(+2 pi i (R x' + r) k / N)
  template <typename V>
  __device__ __forceinline__ static void inv(V (&v)[E], V* base, int r, const V* __restrict__ tw,
                                             const V* __restrict__ twr, int l) {
    if constexpr (R == 1) {
      F::inv(v, base, tw, l);
      return;
    }
#pragma unroll
    for (int j = 0; j < E; ++j) base[r * RS + l + LQ * j] = v[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < E; ++j) {
      V acc = base[l + LQ * j];
#pragma unroll
      for (int s = 1; s < R; ++s) acc = cadd(acc, rot(base[s * RS + l + LQ * j], (R - 1) * s * r));
      if (r > 0) {
        V c = TW::ld(&twr[(r - 1) * M + l + LQ * j]);
        c.y = -c.y;
        acc = cmul(acc, c);
      }
      v[j] = acc;
    }
    __syncthreads();
    F::inv(v, base + r * RS, tw, l);
  }
};

// The same lengths with the cross-group stage first (decimation in frequency
// across the groups): group r holds the contiguous sub-sequence a[x' + M r]
// (x' = l + LQ j); a length-R DFT across the groups and the twiddle W_N^(x' s)
// precede the length-M transform, after which group s holds X[R k' + s] at
// k' = l + LQ j:
//   X[R k' + s] = sum_x' W_M^(x' k') W_N^(x' s) sum_r W_R^(r s) a[x' + M r].
// The spectrum is decimated across the groups, so this form serves passes that
// transform, multiply and transform back in registers (the strided passes):
// lanes of a group read consecutive rows of a tile.  The inverse runs the steps
// transposed and conjugated, in reverse (unnormalised).
template <int M, int LQ, int R, class TW = TwGlobal> struct WarpFFTRdif {
  using F = WarpFFT<M, LQ, TW>;
  using D = WarpFFTR<M, LQ, R, TW>;  // rot()
  static constexpr int E = F::E;
  static constexpr int RS = F::RS;

  // twr: W_N^(s x') at [(s - 1) * M + x']
  template <typename V>
  __device__ __forceinline__ static void fwd(V (&v)[E], V* base, int r, const V* __restrict__ tw,
                                             const V* __restrict__ twr, int l) {
    if constexpr (R == 1) {
      F::fwd(v, base, tw, l);
      return;
    }
#pragma unroll
    for (int j = 0; j < E; ++j) base[r * RS + l + LQ * j] = v[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < E; ++j) {  // this group now plays s = r
      V acc = base[l + LQ * j];
#pragma unroll
      for (int rr = 1; rr < R; ++rr) acc = cadd(acc, D::rot(base[rr * RS + l + LQ * j], rr * r));
      if (r > 0) acc = cmul(acc, TW::ld(&twr[(r - 1) * M + l + LQ * j]));
      v[j] = acc;
    }
    __syncthreads();
    F::fwd(v, base + r * RS, tw, l);
  }

  // group s holds X[R k' + s]  ->  group r holds sum_k X[k] exp(+2 pi i (x' + M r) k / N)
  template <typename V>
  __device__ __forceinline__ static void inv(V (&v)[E], V* base, int r, const V* __restrict__ tw,
                                             const V* __restrict__ twr, int l) {
    if constexpr (R == 1) {
      F::inv(v, base, tw, l);
      return;
    }
    F::inv(v, base + r * RS, tw, l);  // this group plays s = r
    if (r > 0) {
#pragma unroll
      for (int j = 0; j < E; ++j) {
        V c = TW::ld(&twr[(r - 1) * M + l + LQ * j]);
        c.y = -c.y;
        v[j] = cmul(v[j], c);
      }
    }
    // each group's region held only its own transposes: no barrier before
#pragma unroll
    for (int j = 0; j < E; ++j) base[r * RS + l + LQ * j] = v[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < E; ++j) {
      V acc = base[l + LQ * j];
#pragma unroll
      for (int ss = 1; ss < R; ++ss) acc = cadd(acc, D::rot(base[ss * RS + l + LQ * j], (R - 1) * ss * r));
      v[j] = acc;
    }
    __syncthreads();
  }
};

}  // namespace mbo
