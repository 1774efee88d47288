// Device building blocks of the GB300 MBO path: complex arithmetic, small
// register DFTs, in-place mixed-radix transforms over sequences held in shared
// memory, the per-point closest-orthogonal-matrix projections (Lemma 1.1 of
// Osting & Wang, arXiv:1711.01365) and block reductions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "mbo_internal.h"

namespace mbo {

// ---------------------------------------------------------------------------
// Complex helpers (interleaved re/im as float2 / double2)
// ---------------------------------------------------------------------------
template <typename R> struct VT;
template <> struct VT<float> { using V = float2; };
template <> struct VT<double> { using V = double2; };

template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return V{a.x + b.x, a.y + b.y}; }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return V{a.x - b.x, a.y - b.y}; }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return V{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a + DIR*i*t and a - DIR*i*t, lane by lane (the swap of t's parts costs
// nothing in scalar form).
template <int DIR, typename V> __device__ __forceinline__ V cadd_i(V a, V t) {
  return DIR < 0 ? V{a.x + t.y, a.y - t.x} : V{a.x - t.y, a.y + t.x};
}
template <int DIR, typename V> __device__ __forceinline__ V csub_i(V a, V t) {
  return DIR < 0 ? V{a.x - t.y, a.y + t.x} : V{a.x + t.y, a.y - t.x};
}
// FP32 complex add and subtract as one packed two-lane instruction each
// (sm_100 family); the same IEEE operations lane by lane as the scalar forms.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}

// ---------------------------------------------------------------------------
// Register DFTs: y_k = sum_l v_l exp(DIR 2 pi i l k / RAD), in place.
// ---------------------------------------------------------------------------
template <int DIR, typename V> __device__ __forceinline__ void dft2(V* v) {
  V a = v[0];
  v[0] = cadd(a, v[1]);
  v[1] = csub(a, v[1]);
}

template <int DIR, typename V> __device__ __forceinline__ void dft3(V* v) {
  using R = decltype(v[0].x);
  const R h = R(0.86602540378443864676);  // sqrt(3)/2
  V s = cadd(v[1], v[2]);
  V d = csub(v[1], v[2]);
  V t1 = V{v[0].x - R(0.5) * s.x, v[0].y - R(0.5) * s.y};
  const V hd = V{h * d.x, h * d.y};
  v[0] = cadd(v[0], s);
  v[1] = cadd_i<DIR>(t1, hd);
  v[2] = csub_i<DIR>(t1, hd);
}

template <int DIR, typename V> __device__ __forceinline__ void dft4(V* v) {
  V s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
  V s13 = cadd(v[1], v[3]), d13 = csub(v[1], v[3]);
  v[0] = cadd(s02, s13);
  v[2] = csub(s02, s13);
  v[1] = cadd_i<DIR>(d02, d13);
  v[3] = csub_i<DIR>(d02, d13);
}

template <int DIR, typename V> __device__ __forceinline__ void dft8(V* v) {
  using R = decltype(v[0].x);
  const R c = R(0.70710678118654752440);
  V e[4] = {v[0], v[2], v[4], v[6]};
  V o[4] = {v[1], v[3], v[5], v[7]};
  dft4<DIR>(e);
  dft4<DIR>(o);
  // W8^k = exp(DIR 2 pi i k / 8)
  o[1] = cmul(o[1], V{c, R(DIR) * c});
  o[3] = cmul(o[3], V{-c, R(DIR) * c});
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (k == 2) {  // W8^2 = DIR*i
      v[2] = cadd_i<DIR>(e[2], o[2]);
      v[6] = csub_i<DIR>(e[2], o[2]);
    } else {
      v[k] = cadd(e[k], o[k]);
      v[k + 4] = csub(e[k], o[k]);
    }
  }
}

template <int DIR, typename V> __device__ __forceinline__ void dft16(V* v) {
  using R = decltype(v[0].x);
  const R c1 = R(0.92387953251128675613), s1 = R(0.38268343236508977173);
  const R c2 = R(0.70710678118654752440);
  V e[8], o[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    e[k] = v[2 * k];
    o[k] = v[2 * k + 1];
  }
  dft8<DIR>(e);
  dft8<DIR>(o);
  // W16^k = (cos(2 pi k/16), DIR sin(2 pi k/16)), k = 1..7
  const R D = R(DIR);
  o[1] = cmul(o[1], V{c1, D * s1});
  o[2] = cmul(o[2], V{c2, D * c2});
  o[3] = cmul(o[3], V{s1, D * c1});
  o[5] = cmul(o[5], V{-s1, D * c1});
  o[6] = cmul(o[6], V{-c2, D * c2});
  o[7] = cmul(o[7], V{-c1, D * s1});
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k == 4) {  // W16^4 = DIR*i
      v[4] = cadd_i<DIR>(e[4], o[4]);
      v[12] = csub_i<DIR>(e[4], o[4]);
    } else {
      v[k] = cadd(e[k], o[k]);
      v[k + 8] = csub(e[k], o[k]);
    }
  }
}

template <int DIR, int RAD, typename V> __device__ __forceinline__ void dft(V* v) {
  if constexpr (RAD == 2) dft2<DIR>(v);
  else if constexpr (RAD == 3) dft3<DIR>(v);
  else if constexpr (RAD == 4) dft4<DIR>(v);
  else if constexpr (RAD == 8) dft8<DIR>(v);
  else dft16<DIR>(v);
}

// ---------------------------------------------------------------------------
// Fast division (see FastDiv) and asynchronous global -> shared copies.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned fdiv(const FastDiv& d, unsigned x) {
  return d.shift >= 0 ? (x >> d.shift) : __umulhi(x, d.mul);
}

// cp.async of one complex element (8 bytes for float2, 16 for double2); the
// copy proceeds while the thread issues more; cp_async_wait_all() then a
// barrier makes the data visible to the block.
template <typename V> __device__ __forceinline__ void cp_async_elem(V* dst, const V* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(V) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
  else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// ---------------------------------------------------------------------------
// Shared-memory layouts of M sequences of length N.  Both pad one slot per 8
// along the transformed axis: element p of a sequence sits at
// phi(p) = p + p/8.  That keeps the strided butterfly accesses free of bank
// conflicts and, for every stage whose span m is a multiple of 8 or whose
// block length divides 8, makes phi(base + j*m) = phi(base) + j*pstride (see
// Stage::pstride), so a butterfly addresses its RAD elements with one add
// each.
//   RowLayout: sequence m at m*S (S = row_pad(N)); butterflies map
//              sequence-major (consecutive threads, consecutive positions).
//   ColLayout: element (m, p) at row phi(p), column m of a tile of M = 2^ltx
//              adjacent columns; butterflies map column-fastest.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int pad8(int p) { return p + (p >> 3); }
__host__ __device__ __forceinline__ int row_pad(int N) { return N + (N >> 3) + 1; }

struct RowLayout {
  static constexpr bool kColumns = false;
  int S;
  __device__ __forceinline__ int at(int m, int q) const { return m * S + q; }  // q = phi(p)
  __device__ __forceinline__ int addr(int m, int p) const { return at(m, pad8(p)); }
};
struct ColLayout {
  static constexpr bool kColumns = true;
  int ltx;
  __device__ __forceinline__ int at(int m, int q) const { return (q << ltx) + m; }
  __device__ __forceinline__ int addr(int m, int p) const { return at(m, pad8(p)); }
};

// In-place mixed-radix transforms.  The forward transform is a decimation-in-
// frequency network: natural-order input, spectrum left in digit-reversed
// order.  The inverse is the matching decimation-in-time network (the
// conjugate transpose of the forward stages, applied in reverse order): it
// reads the digit-reversed spectrum and returns natural order.  Every
// butterfly reads and writes the same RAD slots, so threads never hold more
// than one butterfly and a stage needs only a barrier after it.  Multiplier
// tables are permuted on the host to the digit-reversed positions.
//
// Stage st works on blocks of length lb = N / (r_0 ... r_{st-1}); a butterfly
// (block b, offset n1 < m = lb / RAD) owns positions b*lb + n1 + m*j.  Its
// twiddles exp(-2 pi i n1 j / lb) come from the stage table [j - 1][n1].
template <int DIR, int RAD, typename V, class L>
__device__ __forceinline__ void radix_stage(V* s, const L& lay, int N, int M, const Stage& sd,
                                            const V* __restrict__ tw) {
  const int NR = N / RAD;
  const int m = sd.m, lb = sd.lb, ps = sd.pstride;
  const unsigned B = (unsigned)(NR * M);
  const V* __restrict__ tws = tw + sd.tw;
  const int da = lay.at(0, ps);  // the affine stride in layout units
  for (unsigned u = threadIdx.x; u < B; u += blockDim.x) {
    int seq, w;
    if constexpr (L::kColumns) {
      seq = (int)(u & ((1u << lay.ltx) - 1));
      w = (int)(u >> lay.ltx);
    } else {
      seq = (int)fdiv(sd.dnr, u);
      w = (int)u - seq * NR;
    }
    const int b = (int)fdiv(sd.dm, (unsigned)w);
    const int n1 = w - b * m;
    const int base = b * lb + n1;
    int a[RAD];
    if (ps) {
      const int a0 = lay.addr(seq, base);
#pragma unroll
      for (int j = 0; j < RAD; ++j) a[j] = a0 + j * da;
    } else {
#pragma unroll
      for (int j = 0; j < RAD; ++j) a[j] = lay.addr(seq, base + j * m);
    }
    V v[RAD];
#pragma unroll
    for (int j = 0; j < RAD; ++j) v[j] = s[a[j]];
    if (DIR < 0) {
      dft<-1, RAD>(v);
      if (m > 1) {
        const V* t = tws + n1;
#pragma unroll
        for (int j = 1; j < RAD; ++j) v[j] = cmul(v[j], __ldg(&t[(j - 1) * m]));
      }
    } else {
      if (m > 1) {
        const V* t = tws + n1;
#pragma unroll
        for (int j = 1; j < RAD; ++j) {
          V c = __ldg(&t[(j - 1) * m]);
          c.y = -c.y;
          v[j] = cmul(v[j], c);
        }
      }
      dft<+1, RAD>(v);
    }
#pragma unroll
    for (int j = 0; j < RAD; ++j) s[a[j]] = v[j];
  }
  __syncthreads();
}

template <int DIR, typename V, class L>
__device__ __forceinline__ void run_stage(V* s, const L& lay, int N, int M, const Stage& sd,
                                          const V* __restrict__ tw) {
  switch (sd.rad) {
    case 16: radix_stage<DIR, 16>(s, lay, N, M, sd, tw); break;
    case 8: radix_stage<DIR, 8>(s, lay, N, M, sd, tw); break;
    case 4: radix_stage<DIR, 4>(s, lay, N, M, sd, tw); break;
    case 3: radix_stage<DIR, 3>(s, lay, N, M, sd, tw); break;
    default: radix_stage<DIR, 2>(s, lay, N, M, sd, tw); break;
  }
}

// Forward transform (unnormalised, exp(-2 pi i k x / N)); caller synchronises before.
template <typename V, class L>
__device__ void fft_fwd(V* s, const L& lay, int N, int M, const Plan& pl, const V* __restrict__ tw) {
  for (int st = 0; st < pl.nst; ++st) run_stage<-1>(s, lay, N, M, pl.st[st], tw);
}

// Inverse transform (unnormalised, exp(+2 pi i k x / N)) of a digit-reversed spectrum.
template <typename V, class L>
__device__ void fft_inv(V* s, const L& lay, int N, int M, const Plan& pl, const V* __restrict__ tw) {
  for (int st = pl.nst - 1; st >= 0; --st) run_stage<+1>(s, lay, N, M, pl.st[st], tw);
}

// ---------------------------------------------------------------------------
// Closest orthogonal matrix (Lemma 1.1).  Input m and output b are row-major
// n x n.  Returns the class sign s = +1 if det m >= 0 else -1 (det b = s) and
// the smallest singular value of m in smin.
// ---------------------------------------------------------------------------
template <typename R> struct JacobiPrec;
template <> struct JacobiPrec<float> {
  static constexpr float tol = 1e-6f;
  static constexpr int sweeps = 6;
};
template <> struct JacobiPrec<double> {
  static constexpr double tol = 2e-15;
  static constexpr int sweeps = 12;
};

template <typename R> __device__ __forceinline__ R rsqrt_(R x);
template <> __device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }

// n = 1: nearest of {+1, -1}.
template <typename R> __device__ __forceinline__ R polar1(const R* m, R* b, R& smin) {
  const R s = (m[0] >= R(0)) ? R(1) : R(-1);
  b[0] = s;
  smin = fabs(m[0]);
  return s;
}

// n = 2, closed form.  With p = a+d, q = c-b, r = a-d, t = b+c for
// A = [[a,b],[c,d]]: sigma_{1,2} = (sqrt(p^2+q^2) +- sqrt(r^2+t^2)) / 2 and
// det A = ((p^2+q^2) - (r^2+t^2)) / 4.  The nearest rotation is the
// normalised [[p,-q],[q,p]], the nearest reflection the normalised
// [[r,t],[t,-r]]; the class follows the sign of det A.
template <typename R> __device__ __forceinline__ R polar2(const R* m, R* b, R& smin) {
  const R p = m[0] + m[3], q = m[2] - m[1], r = m[0] - m[3], t = m[1] + m[2];
  const R rho2 = p * p + q * q, sig2 = r * r + t * t;
  const R rho = sqrt(rho2), sig = sqrt(sig2);
  smin = R(0.5) * fabs(rho - sig);
  if (rho2 >= sig2) {
    if (rho2 > R(0)) {
      const R inv = R(1) / rho;
      b[0] = p * inv; b[1] = -q * inv; b[2] = q * inv; b[3] = p * inv;
    } else {
      b[0] = R(1); b[1] = R(0); b[2] = R(0); b[3] = R(1);
    }
    return R(1);
  }
  const R inv = R(1) / sig;
  b[0] = r * inv; b[1] = t * inv; b[2] = t * inv; b[3] = -r * inv;
  return R(-1);
}

template <typename R> __device__ __forceinline__ R dot3(const R* a, const R* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// One-sided Jacobi rotation of columns P and Q of A (and of V).
template <int P, int Q, typename R>
__device__ __forceinline__ void jacobi_pair(R (&a)[3][3], R (&v)[3][3], bool& rot) {
  const R al = dot3(a[P], a[P]);
  const R be = dot3(a[Q], a[Q]);
  const R ga = dot3(a[P], a[Q]);
  if (fabs(ga) > JacobiPrec<R>::tol * sqrt(al * be)) {
    const R ze = (be - al) / (R(2) * ga);
    const R t = copysign(R(1), ze) / (fabs(ze) + sqrt(R(1) + ze * ze));
    const R c = rsqrt_(R(1) + t * t);
    const R s = c * t;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const R ap = a[P][i], aq = a[Q][i];
      a[P][i] = c * ap - s * aq;
      a[Q][i] = s * ap + c * aq;
      const R vp = v[P][i], vq = v[Q][i];
      v[P][i] = c * vp - s * vq;
      v[Q][i] = s * vp + c * vq;
    }
    rot = true;
  }
}

template <typename R> __device__ __forceinline__ void cross3(const R* a, const R* b, R* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// Unit vector orthogonal to the unit vector u (Gram-Schmidt of the axis least
// aligned with u).
template <typename R> __device__ __forceinline__ void any_orthogonal(const R* u, R* w) {
  int k = 0;
  if (fabs(u[1]) < fabs(u[k])) k = 1;
  if (fabs(u[2]) < fabs(u[k])) k = 2;
  R e[3] = {R(0), R(0), R(0)};
  e[k] = R(1);
  const R d = u[k];
  R x[3] = {e[0] - d * u[0], e[1] - d * u[1], e[2] - d * u[2]};
  const R inv = rsqrt_(dot3(x, x));
  w[0] = x[0] * inv; w[1] = x[1] * inv; w[2] = x[2] * inv;
}

// n = 3: one-sided (Hestenes) Jacobi on the columns of m.  On return
// a[j] = m v_j (mutually orthogonal columns), V = [v_0 v_1 v_2] in SO(3)
// (re-orthonormalised), and U in SO(3) with columns u_big = a_big / |a_big|,
// u_mid from Gram-Schmidt and u_small = +-u_big x u_mid (orientation chosen
// so det U = +1); is = index of the smallest column, smin = |a_is|.  Then
// m = U diag(s_j) V^t with s_is = u_is . a_is carrying the sign of det m.
// Returns false (frame undefined) when m = 0 or is not finite.
template <typename R>
__device__ __forceinline__ bool jacobi3_frame(const R* m, R (&U)[3][3], R (&v)[3][3], R (&a)[3][3],
                                              int& is, R& smin) {
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      a[j][i] = m[i * 3 + j];
      v[j][i] = (i == j) ? R(1) : R(0);
    }
#pragma unroll 1
  for (int sw = 0; sw < JacobiPrec<R>::sweeps; ++sw) {
    bool rot = false;
    jacobi_pair<0, 1>(a, v, rot);
    jacobi_pair<0, 2>(a, v, rot);
    jacobi_pair<1, 2>(a, v, rot);
    if (!rot) break;
  }
  const R n0 = dot3(a[0], a[0]), n1 = dot3(a[1], a[1]), n2 = dot3(a[2], a[2]);
  // order the columns: ib (largest), im, is (smallest)
  int ib = 0;
  is = 0;
  if (n1 > n0) ib = 1;
  if (n2 > (ib == 0 ? n0 : n1)) ib = 2;
  if (n1 < n0) is = 1;
  if (n2 < (is == 0 ? n0 : n1)) is = 2;
  if (is == ib) is = (ib + 1) % 3;  // all equal
  const int im = 3 - ib - is;
  const R nn[3] = {n0, n1, n2};
  smin = sqrt(nn[is]);
  if (!(nn[ib] > R(0))) return false;
  {
    const R inv = rsqrt_(nn[ib]);
#pragma unroll
    for (int i = 0; i < 3; ++i) U[ib][i] = a[ib][i] * inv;
    const R dd = dot3(U[ib], a[im]);
    R w[3] = {a[im][0] - dd * U[ib][0], a[im][1] - dd * U[ib][1], a[im][2] - dd * U[ib][2]};
    const R ww = dot3(w, w);
    if (ww > R(0) && ww > nn[ib] * R(1e-30)) {
      const R iw = rsqrt_(ww);
      U[im][0] = w[0] * iw; U[im][1] = w[1] * iw; U[im][2] = w[2] * iw;
    } else {
      any_orthogonal(U[ib], U[im]);
    }
    // cyclic (ib, im, is) is an even permutation of (0, 1, 2)
    const R perm = (im == (ib + 1) % 3) ? R(1) : R(-1);
    R c[3];
    cross3(U[ib], U[im], c);
    U[is][0] = perm * c[0]; U[is][1] = perm * c[1]; U[is][2] = perm * c[2];
  }
  // re-orthonormalise V (a product of rotations: keep det V = +1)
  {
    const R i0 = rsqrt_(dot3(v[0], v[0]));
    v[0][0] *= i0; v[0][1] *= i0; v[0][2] *= i0;
    const R dd = dot3(v[0], v[1]);
    v[1][0] -= dd * v[0][0]; v[1][1] -= dd * v[0][1]; v[1][2] -= dd * v[0][2];
    const R i1 = rsqrt_(dot3(v[1], v[1]));
    v[1][0] *= i1; v[1][1] *= i1; v[1][2] *= i1;
    cross3(v[0], v[1], v[2]);
  }
  return true;
}

template <typename R>
__device__ __forceinline__ void frame_product(const R (&U)[3][3], const R (&v)[3][3], R* b) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) b[i * 3 + k] = U[0][i] * v[0][k] + U[1][i] * v[1][k] + U[2][i] * v[2][k];
}

// n = 3 polar factor from the Jacobi frame: U V^t with the smallest column of
// U oriented so that det(U V^t) = sign det m (Lemma 1.1; det m = 0 -> +1).
template <typename R> __device__ __forceinline__ R polar3(const R* m, R* b, R& smin) {
  const R det = m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) +
                m[2] * (m[3] * m[7] - m[4] * m[6]);
  const R sg = (det >= R(0)) ? R(1) : R(-1);
  R U[3][3], v[3][3], a[3][3];
  int is;
  if (!jacobi3_frame(m, U, v, a, is, smin)) {  // m = 0 (or not finite): identity
#pragma unroll
    for (int i = 0; i < 9; ++i) b[i] = (i % 4 == 0) ? R(1) : R(0);
    return (a[0][0] == R(0) && a[1][1] == R(0) && a[2][2] == R(0)) ? R(1) : sg;
  }
  U[is][0] *= sg; U[is][1] *= sg; U[is][2] *= sg;
  frame_product(U, v, b);
  return sg;
}

// Closest matrices of SO(n) (tp) and SO^-(n) (tm) and dE = <tp - tm, m>_F
// (Lemma 7.1, Sec. 7).  Returns the smallest singular value.
template <int NM, typename R>
__device__ __forceinline__ R class_pair(const R* m, R* tp, R* tm, R& dE) {
  if constexpr (NM == 1) {
    tp[0] = R(1);
    tm[0] = R(-1);
    dE = R(2) * m[0];
    return fabs(m[0]);
  } else if constexpr (NM == 2) {
    const R p = m[0] + m[3], q = m[2] - m[1], r = m[0] - m[3], t = m[1] + m[2];
    const R rho = sqrt(p * p + q * q), sig = sqrt(r * r + t * t);
    if (rho > R(0)) {
      const R i = R(1) / rho;
      tp[0] = p * i; tp[1] = -q * i; tp[2] = q * i; tp[3] = p * i;
    } else {
      tp[0] = R(1); tp[1] = R(0); tp[2] = R(0); tp[3] = R(1);
    }
    if (sig > R(0)) {
      const R i = R(1) / sig;
      tm[0] = r * i; tm[1] = t * i; tm[2] = t * i; tm[3] = -r * i;
    } else {
      tm[0] = R(1); tm[1] = R(0); tm[2] = R(0); tm[3] = R(-1);
    }
    dE = rho - sig;  // <rotation, m> = |(p, q)|, <reflection, m> = |(r, t)|
    return R(0.5) * fabs(rho - sig);
  } else {
    R U[3][3], v[3][3], a[3][3], smin;
    int is;
    if (!jacobi3_frame(m, U, v, a, is, smin)) {
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        tp[i] = (i % 4 == 0) ? R(1) : R(0);
        tm[i] = (i % 4 == 0) ? (i == 8 ? R(-1) : R(1)) : R(0);
      }
      dE = R(0);
      return smin;
    }
    frame_product(U, v, tp);  // U, V in SO(3): the closest rotation
    const R s = dot3(U[is], a[is]);  // signed smallest singular value
    dE = R(2) * s;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) tm[i * 3 + k] = tp[i * 3 + k] - R(2) * U[is][i] * v[is][k];
    return smin;
  }
}

// Reciprocal of a nonzero value: correctly rounded in FP32; in FP64 an FP32
// seed refined by two Newton steps (relative error at FP64 rounding level).
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) {
  double r = (double)__frcp_rn((float)x);
  r = r * (2.0 - x * r);
  r = r * (2.0 - x * r);
  return r;
}

// Cofactor matrix of a row-major 3x3 X (so X^{-t} = cof(X) / det X) and det X.
template <typename R> __device__ __forceinline__ R cofactor3(const R* X, R* C) {
  C[0] = X[4] * X[8] - X[5] * X[7];
  C[1] = X[5] * X[6] - X[3] * X[8];
  C[2] = X[3] * X[7] - X[4] * X[6];
  C[3] = X[2] * X[7] - X[1] * X[8];
  C[4] = X[0] * X[8] - X[2] * X[6];
  C[5] = X[1] * X[6] - X[0] * X[7];
  C[6] = X[1] * X[5] - X[2] * X[4];
  C[7] = X[2] * X[3] - X[0] * X[5];
  C[8] = X[0] * X[4] - X[1] * X[3];
  return X[0] * C[0] + X[1] * C[1] + X[2] * C[2];
}

// Determinant of a 4x4 matrix (row-major) by complementary 2x2 minors.
template <typename R> __device__ __forceinline__ R det4(const R* X) {
  const R t01 = X[0] * X[5] - X[1] * X[4], t02 = X[0] * X[6] - X[2] * X[4];
  const R t03 = X[0] * X[7] - X[3] * X[4], t12 = X[1] * X[6] - X[2] * X[5];
  const R t13 = X[1] * X[7] - X[3] * X[5], t23 = X[2] * X[7] - X[3] * X[6];
  const R b01 = X[8] * X[13] - X[9] * X[12], b02 = X[8] * X[14] - X[10] * X[12];
  const R b03 = X[8] * X[15] - X[11] * X[12], b12 = X[9] * X[14] - X[10] * X[13];
  const R b13 = X[9] * X[15] - X[11] * X[13], b23 = X[10] * X[15] - X[11] * X[14];
  return t01 * b23 - t02 * b13 + t03 * b12 + t12 * b03 - t13 * b02 + t23 * b01;
}

// n = 4: cofactor matrix C[i*4+j] = (-1)^(i+j) M_ij of X (row-major) from the
// 2x2 minors of rows (0, 1) and rows (2, 3): each 3x3 minor is expanded along
// the row that the deleted one leaves alone in its pair.  Returns det X.
template <typename R> __device__ __forceinline__ R cofactor4(const R* X, R* C) {
  const R t01 = X[0] * X[5] - X[1] * X[4], t02 = X[0] * X[6] - X[2] * X[4];
  const R t03 = X[0] * X[7] - X[3] * X[4], t12 = X[1] * X[6] - X[2] * X[5];
  const R t13 = X[1] * X[7] - X[3] * X[5], t23 = X[2] * X[7] - X[3] * X[6];
  const R b01 = X[8] * X[13] - X[9] * X[12], b02 = X[8] * X[14] - X[10] * X[12];
  const R b03 = X[8] * X[15] - X[11] * X[12], b12 = X[9] * X[14] - X[10] * X[13];
  const R b13 = X[9] * X[15] - X[11] * X[13], b23 = X[10] * X[15] - X[11] * X[14];
  C[0] = X[5] * b23 - X[6] * b13 + X[7] * b12;
  C[1] = -(X[4] * b23 - X[6] * b03 + X[7] * b02);
  C[2] = X[4] * b13 - X[5] * b03 + X[7] * b01;
  C[3] = -(X[4] * b12 - X[5] * b02 + X[6] * b01);
  C[4] = -(X[1] * b23 - X[2] * b13 + X[3] * b12);
  C[5] = X[0] * b23 - X[2] * b03 + X[3] * b02;
  C[6] = -(X[0] * b13 - X[1] * b03 + X[3] * b01);
  C[7] = X[0] * b12 - X[1] * b02 + X[2] * b01;
  C[8] = X[13] * t23 - X[14] * t13 + X[15] * t12;
  C[9] = -(X[12] * t23 - X[14] * t03 + X[15] * t02);
  C[10] = X[12] * t13 - X[13] * t03 + X[15] * t01;
  C[11] = -(X[12] * t12 - X[13] * t02 + X[14] * t01);
  C[12] = -(X[9] * t23 - X[10] * t13 + X[11] * t12);
  C[13] = X[8] * t23 - X[10] * t03 + X[11] * t02;
  C[14] = -(X[8] * t13 - X[9] * t03 + X[11] * t01);
  C[15] = X[8] * t12 - X[9] * t02 + X[10] * t01;
  return X[0] * C[0] + X[1] * C[1] + X[2] * C[2] + X[3] * C[3];
}

template <int NM, typename R> __device__ __forceinline__ R cofactor_n(const R* X, R* C) {
  if constexpr (NM == 3) return cofactor3(X, C);
  else return cofactor4(X, C);
}

// n = 3 and 4, scaled Newton iteration for the polar factor (Higham 1986):
//   X <- (zeta X + X^{-t} / zeta) / 2,  zeta = (|X^{-1}|_F / |X|_F)^{1/2},
// with X^{-t} = cof(X) / det(X).  With X = Q H, cof(X) = det(X) Q H^{-1}, so
// a X + c cof(X) = Q (a H + c det(X) H^{-1}) keeps the polar factor Q for any
// a > 0 and c det(X) > 0: the scaled phase only sets the speed, and its
// coefficients are computed in FP32 whatever R is (callers keep det m^2 in
// the FP32 range).  The scaled phase ends when
// |X|_F^2 = sum s_i^2 is within 1e-4 of n and zeta within 1e-5 of 1: then
// sum s_i^2 * sum s_i^-2 is within ~1e-4 of n^2, its minimum, which by the
// AM-HM inequality holds only when every s_i^2 is close to 1 (zeta = 1 alone
// does not suffice: s = (2, 1/2, 1) gives zeta = 1).  NUN unscaled iterations
// X <- (X + X^{-t}) / 2 follow; each squares the distance to orthogonality
// (d -> d^2 / 2) and their fixed point is exactly orthogonal.  det X keeps
// the sign of det m, and the returned class is the sign of det of the last
// iterate (the two differ only where det m is below its rounding error).
// est receives |det m| / |cof m|_F = 1 / |m^{-1}|_F, which lies in
// [sigma_min / sqrt(n), sigma_min], or 0 where |cof m|_F^2 <= cof2_floor
// (callers pass (c |m|_F^(n-1))^2 with c above the rounding error of cof:
// below it the matrix has rank <= n - 2 to working precision, est is noise
// over noise and the iteration would run on noise).  Points with
// est <= skip_below (exactly singular ones, where the iteration is undefined,
// included) are returned unprocessed, with the sign of det m, for the caller
// to route elsewhere, and est is set to 0 where the iteration overflowed.
template <int NM, int ITMAX, int NUN, typename R>
__device__ __forceinline__ R polar_newton(const R* m, R* b, R& est, R skip_below = R(0),
                                          R cof2_floor = R(0)) {
  constexpr int C2 = NM * NM;
  R X[C2], C[C2];
#pragma unroll
  for (int k = 0; k < C2; ++k) X[k] = m[k];
  R det = cofactor_n<NM>(X, C);
  const R sg = (det >= R(0)) ? R(1) : R(-1);
  {
    R nc = R(0);
#pragma unroll
    for (int k = 0; k < C2; ++k) nc += C[k] * C[k];
    est = fabs(det) * rsqrt_(nc);
    // at rank <= n - 2 (to working precision) cof m is rounding noise and est
    // noise over noise: callers pass a floor for |cof m|_F^2
    if (!(nc > cof2_floor)) est = R(0);
  }
  if (!(est > skip_below)) {  // singular, not finite or below the caller's limit: caller's fallback
#pragma unroll
    for (int k = 0; k < C2; ++k) b[k] = X[k];
    return sg;
  }
#pragma unroll 1
  for (int it = 0; it < ITMAX; ++it) {
    float nx = 0.f, nc = 0.f;
#pragma unroll
    for (int k = 0; k < C2; ++k) {
      nx += (float)X[k] * (float)X[k];
      nc += (float)C[k] * (float)C[k];
    }
    const float fd = (float)det;
    const float zf = rsqrtf(rsqrtf(__fdividef(nc, fd * fd * nx)));  // (nc / (det^2 nx))^{1/4}
    if (fabsf(zf - 1.0f) < 1e-5f && fabsf(nx - (float)NM) < 1e-4f) break;
    const R a = R(0.5f * zf);
    const R c = R(__fdividef(0.5f, zf * fd));
#pragma unroll
    for (int k = 0; k < C2; ++k) X[k] = a * X[k] + c * C[k];
    det = cofactor_n<NM>(X, C);
  }
  R c = R(0);
#pragma unroll
  for (int it = 0; it < NUN; ++it) {
    c = R(0.5) * recip(det);
#pragma unroll
    for (int k = 0; k < C2; ++k) X[k] = R(0.5) * X[k] + c * C[k];
    if (it + 1 < NUN) det = cofactor_n<NM>(X, C);
  }
#pragma unroll
  for (int k = 0; k < C2; ++k) b[k] = X[k];
  // At rank <= n - 2 (to working precision) the iteration runs on rounding
  // noise and can overflow: report it as singular (est = 0) for the caller's
  // fallback.
  if (!(fabs(c) < R(1e30)) || !(fabs(X[0]) < R(1e30))) est = R(0);
  // The class of the limit: det keeps its sign along the iteration, but where
  // det m is below its own rounding error its computed sign is noise and the
  // iterates settle the class; report the one b has.
  return det >= R(0) ? R(1) : R(-1);
}

// n = 3, FP32: a fixed schedule of the same iteration -- two Frobenius-
// scaled steps, then two unscaled ones -- with no convergence test inside.
// Newton's iteration for the polar factor converges quadratically, so when
// the last unscaled step moved no entry by more than kPolarAccept the
// remaining error is below about kPolarAccept^2 / 2 (5e-8, under the FP32
// rounding of the iterate itself) and b is accepted;
// else `done` is false and b holds the current iterate for the caller to
// finish.  est and the routing of small or singular points are as in
// polar_newton (points not iterated at all return done = true with est <=
// skip_below).  The returned class is the sign of det of the last iterate.
constexpr float kPolarAccept = 3e-4f;

__device__ __forceinline__ float polar3_fixed(const float* m, float* b, float& est, float skip_below,
                                              float cof2_floor, bool& done) {
  float X[9], C[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) X[k] = m[k];
  float det = cofactor3(X, C);
  const float sg = (det >= 0.f) ? 1.f : -1.f;
  float nx = 0.f, nc = 0.f;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    nx += X[k] * X[k];
    nc += C[k] * C[k];
  }
  est = fabsf(det) * rsqrtf(nc);
  if (!(nc > cof2_floor)) est = 0.f;
  done = true;
  if (!(est > skip_below)) {
#pragma unroll
    for (int k = 0; k < 9; ++k) b[k] = X[k];
    return sg;
  }
#pragma unroll
  for (int it = 0; it < 2; ++it) {  // scaled: zeta = (|X^-1|_F / |X|_F)^(1/2)
    if (it > 0) {
      det = cofactor3(X, C);
      nx = 0.f;
      nc = 0.f;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        nx += X[k] * X[k];
        nc += C[k] * C[k];
      }
    }
    const float zf = rsqrtf(rsqrtf(__fdividef(nc, det * det * nx)));
    const float a = 0.5f * zf;
    const float c = __fdividef(0.5f, zf * det);
#pragma unroll
    for (int k = 0; k < 9; ++k) X[k] = a * X[k] + c * C[k];
  }
  float delta = 0.f;
#pragma unroll
  for (int it = 0; it < 2; ++it) {  // unscaled
    det = cofactor3(X, C);
    const float c = 0.5f * __frcp_rn(det);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float xn = 0.5f * X[k] + c * C[k];
      if (it == 1) delta = fmaxf(delta, fabsf(xn - X[k]));
      X[k] = xn;
    }
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) b[k] = X[k];
  done = delta <= kPolarAccept;  // NaN: not done
  if (!(fabsf(X[0]) < 1e30f)) est = 0.f;
  return det >= 0.f ? 1.f : -1.f;
}

template <int ITMAX, int NUN, typename R>
__device__ __forceinline__ R polar3_newton(const R* m, R* b, R& est, R skip_below = R(0),
                                           R cof2_floor = R(0)) {
  return polar_newton<3, ITMAX, NUN>(m, b, est, skip_below, cof2_floor);
}

// n = 3, FP32: the nearest matrix of the class sg (det = sg) through the
// quaternion form of the problem (Horn 1987).  For a = sg m / |m|_F the
// nearest rotation R(q) maximises tr(R^t a) = q^t K q over unit quaternions q,
// K the symmetric traceless 4x4 matrix below, so q is the eigenvector of the
// largest eigenvalue l1 = s1 + s2 + s3 (the singular values of a, the
// smallest one signed by det a).  l1 is the largest root of
//   p(l) = det(K - l I) = l^4 - 2 |a|^2 l^2 - 8 det(a) l + det K,
// reached by Newton's method from the upper bound sqrt(3) |a|_F, and q is the
// column of adj(K - l1 I) = prod_{i>1} (l_i - l1) q q^t with the largest
// diagonal magnitude.  The other eigenvalues are s1 - s2 - s3, s2 - s1 - s3,
// s3 - s1 - s2, so p'(l1) = 8 (s2 + s3)(s1 + s3)(s1 + s2): the eigenvector's
// conditioning is that of the polar factor itself, 1 / (s2 + s3), and unlike
// the Newton iteration nothing here inverts a; the rounding of l1, however,
// enters q as eps / (s2 + s3)^2.  Returns p'(l1) / 32, a lower bound of
// (s2 + s3) / |m|_F, for the caller's accuracy test.
__device__ __forceinline__ float polar3_quat(const float* m, float sg, float* b) {
  float n2 = 0.f;
#pragma unroll
  for (int k = 0; k < 9; ++k) n2 += m[k] * m[k];
  const float sc = sg * rsqrtf(n2);
  float a[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) a[k] = m[k] * sc;
  float na = 0.f;
#pragma unroll
  for (int k = 0; k < 9; ++k) na += a[k] * a[k];
  const float adet = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                     a[2] * (a[3] * a[7] - a[4] * a[6]);
  // K (symmetric, upper triangle)
  const float k00 = a[0] + a[4] + a[8], k11 = a[0] - a[4] - a[8];
  const float k22 = -a[0] + a[4] - a[8], k33 = -a[0] - a[4] + a[8];
  const float k01 = a[7] - a[5], k02 = a[2] - a[6], k03 = a[3] - a[1];
  const float k12 = a[1] + a[3], k13 = a[2] + a[6], k23 = a[5] + a[7];
  // det K from the 2x2 minors of rows (0, 1) and rows (2, 3)
  float c0;
  {
    const float t01 = k00 * k11 - k01 * k01, t02 = k00 * k12 - k02 * k01;
    const float t03 = k00 * k13 - k03 * k01, t12 = k01 * k12 - k02 * k11;
    const float t13 = k01 * k13 - k03 * k11, t23 = k02 * k13 - k03 * k12;
    const float b01 = k02 * k13 - k12 * k03, b02 = k02 * k23 - k22 * k03;
    const float b03 = k02 * k33 - k23 * k03, b12 = k12 * k23 - k22 * k13;
    const float b13 = k12 * k33 - k23 * k13, b23 = k22 * k33 - k23 * k23;
    c0 = t01 * b23 - t02 * b13 + t03 * b12 + t12 * b03 - t13 * b02 + t23 * b01;
  }
  const float c2 = -2.f * na, c1 = -8.f * adet;
  float lam = sqrtf(3.f * na);
#pragma unroll 1
  for (int it = 0; it < 16; ++it) {
    const float l2 = lam * lam;
    const float p = fmaf(l2 + c2, l2, fmaf(c1, lam, c0));
    const float dp = fmaf(lam, fmaf(4.f, l2, 2.f * c2), c1);
    if (!(dp > 0.f)) break;
    const float step = p / dp;
    lam -= step;
    if (fabsf(step) <= 1e-7f * lam) break;
  }
  const float dp = fmaf(lam, fmaf(4.f, lam * lam, 2.f * c2), c1);
  // A = K - lam I; its 3x3 minors M(r, c) (symmetric), each expanded along
  // the row that deleting r leaves alone in its pair.
  const float a00 = k00 - lam, a11 = k11 - lam, a22 = k22 - lam, a33 = k33 - lam;
  const float a01 = k01, a02 = k02, a03 = k03, a12 = k12, a13 = k13, a23 = k23;
  const float t01 = a00 * a11 - a01 * a01, t02 = a00 * a12 - a02 * a01;
  const float t03 = a00 * a13 - a03 * a01, t12 = a01 * a12 - a02 * a11;
  const float t13 = a01 * a13 - a03 * a11;
  const float b01 = a02 * a13 - a12 * a03, b02 = a02 * a23 - a22 * a03;
  const float b03 = a02 * a33 - a23 * a03, b12 = a12 * a23 - a22 * a13;
  const float b13 = a12 * a33 - a23 * a13, b23 = a22 * a33 - a23 * a23;
  const float M00 = a11 * b23 - a12 * b13 + a13 * b12;
  const float M11 = a00 * b23 - a02 * b03 + a03 * b02;
  const float M22 = a03 * t13 - a13 * t03 + a33 * t01;
  const float M33 = a02 * t12 - a12 * t02 + a22 * t01;
  const float M01 = a01 * b23 - a12 * b03 + a13 * b02;
  const float M02 = a01 * b13 - a11 * b03 + a13 * b01;
  const float M03 = a01 * b12 - a11 * b02 + a12 * b01;
  const float M12 = a00 * b13 - a01 * b03 + a03 * b01;
  const float M13 = a00 * b12 - a01 * b02 + a02 * b01;
  const float M23 = a03 * t12 - a13 * t02 + a23 * t01;
  // adj = ((-1)^(i+j) M(i, j)); at l1 it is negative semidefinite: take the
  // column of the most negative diagonal entry.
  float w = M00, x = -M01, y = M02, z = -M03, best = M00;
  if (M11 < best) { best = M11; w = -M01; x = M11; y = -M12; z = M13; }
  if (M22 < best) { best = M22; w = M02; x = -M12; y = M22; z = -M23; }
  if (M33 < best) { best = M33; w = -M03; x = M13; y = -M23; z = M33; }
  const float ww = w * w, xx = x * x, yy = y * y, zz = z * z;
  const float f = sg / (ww + xx + yy + zz);
  b[0] = (ww + xx - yy - zz) * f;
  b[1] = 2.f * (x * y - w * z) * f;
  b[2] = 2.f * (x * z + w * y) * f;
  b[3] = 2.f * (x * y + w * z) * f;
  b[4] = (ww - xx + yy - zz) * f;
  b[5] = 2.f * (y * z - w * x) * f;
  b[6] = 2.f * (x * z - w * y) * f;
  b[7] = 2.f * (y * z + w * x) * f;
  b[8] = (ww - xx - yy + zz) * f;
  return dp * (1.f / 32.f);
}

template <int NM, typename R> __device__ __forceinline__ R polar(const R* m, R* b, R& smin) {
  if constexpr (NM == 1) return polar1(m, b, smin);
  else if constexpr (NM == 2) return polar2(m, b, smin);
  else return polar3(m, b, smin);
}

// n = 4, FP64, for matrices singular to working precision: one-sided
// (Hestenes) Jacobi on the columns of m gives m V = [a_0 .. a_3] with
// orthogonal columns; U = a_j / |a_j|, columns of negligible norm completed by
// Gram-Schmidt of the basis vector that leaves the largest remainder; the
// column of the smallest singular value is flipped when needed so that
// det(U V^t) = sign det m (Lemma 1.1, det m = 0 -> +1).  b = U V^t.
static __device__ __noinline__ double polar4_jacobi(const double* m, double* b, double& smin) {
  double a[4][4], v[4][4];  // a[j] = column j of m V, v[j] = column j of V
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      a[j][i] = m[i * 4 + j];
      v[j][i] = (i == j) ? 1.0 : 0.0;
    }
  auto dot4 = [](const double* x, const double* y) {
    return x[0] * y[0] + x[1] * y[1] + x[2] * y[2] + x[3] * y[3];
  };
#pragma unroll 1
  for (int sw = 0; sw < 16; ++sw) {
    bool rot = false;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = p + 1; q < 4; ++q) {
        const double al = dot4(a[p], a[p]), be = dot4(a[q], a[q]), ga = dot4(a[p], a[q]);
        if (fabs(ga) > 2e-15 * sqrt(al * be)) {
          const double ze = (be - al) / (2.0 * ga);
          const double t = copysign(1.0, ze) / (fabs(ze) + sqrt(1.0 + ze * ze));
          const double c = rsqrt(1.0 + t * t), s = c * t;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const double ap = a[p][i], aq = a[q][i];
            a[p][i] = c * ap - s * aq;
            a[q][i] = s * ap + c * aq;
            const double vp = v[p][i], vq = v[q][i];
            v[p][i] = c * vp - s * vq;
            v[q][i] = s * vp + c * vq;
          }
          rot = true;
        }
      }
    if (!rot) break;
  }
  double sgm[4], U[4][4];
  bool have[4];
  double nmax = 0.0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    sgm[j] = sqrt(dot4(a[j], a[j]));
    nmax = fmax(nmax, sgm[j]);
  }
  int is = 0;
#pragma unroll
  for (int j = 1; j < 4; ++j)
    if (sgm[j] < sgm[is]) is = j;
  smin = sgm[is];
  const double want = det4(m) >= 0.0 ? 1.0 : -1.0;
  if (!(nmax > 0.0)) {  // m = 0: the identity
#pragma unroll
    for (int k = 0; k < 16; ++k) b[k] = (k % 5 == 0) ? 1.0 : 0.0;
    return 1.0;
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    have[j] = sgm[j] > 1e-13 * nmax;
    const double inv = have[j] ? 1.0 / sgm[j] : 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i) U[j][i] = a[j][i] * inv;
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (have[j]) continue;
    double best[4] = {0.0, 0.0, 0.0, 0.0}, bn = -1.0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      double w[4] = {0.0, 0.0, 0.0, 0.0};
      w[e] = 1.0;
#pragma unroll
      for (int pass = 0; pass < 2; ++pass)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (!have[k]) continue;
          const double d = dot4(U[k], w);
#pragma unroll
          for (int i = 0; i < 4; ++i) w[i] -= d * U[k][i];
        }
      const double wn = dot4(w, w);
      if (wn > bn) {
        bn = wn;
#pragma unroll
        for (int i = 0; i < 4; ++i) best[i] = w[i];
      }
    }
    const double inv = rsqrt(bn);
#pragma unroll
    for (int i = 0; i < 4; ++i) U[j][i] = best[i] * inv;
    have[j] = true;
  }
  double um[16], vm[16];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      um[i * 4 + j] = U[j][i];
      vm[i * 4 + j] = v[j][i];
    }
  if ((det4(um) * det4(vm) >= 0.0 ? 1.0 : -1.0) != want) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (j == is)
#pragma unroll
        for (int i = 0; i < 4; ++i) U[j][i] = -U[j][i];
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k)
      b[i * 4 + k] = U[0][i] * v[0][k] + U[1][i] * v[1][k] + U[2][i] * v[2][k] + U[3][i] * v[3][k];
  return want;
}

// FP64 projection used by the FP64 path and by the FP32 path's
// re-projection: Newton, and the one-sided Jacobi construction for matrices
// that are singular to working precision (rank-deficient ties included).
template <int NM> __device__ __forceinline__ double polar_f64(const double* m, double* b, double& smin) {
  if constexpr (NM == 4) {
    double nx = 0.0;
#pragma unroll
    for (int k = 0; k < 16; ++k) nx += m[k] * m[k];
    // Newton only where det m stands clear of its rounding error and its
    // square of the FP32 range of the scaling coefficients; with two small
    // singular values est alone does not ensure either
    const double d = det4(m);
    if (nx > 1e-30 && nx < 1e30 && d * d > 1e-26 * nx * nx * nx * nx && fabs(d) > 1e-18) {
      double est = 0.0;
      const double sg = polar_newton<4, 16, 3>(m, b, est, 1e-12 * sqrt(nx), 1e-24 * nx * nx * nx);
      smin = est;
      if (est > 1e-12 * sqrt(nx)) return sg;
    }
    return polar4_jacobi(m, b, smin);
  } else if constexpr (NM == 3) {
    double nx = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k) nx += m[k] * m[k];
    double est = 0.0;
    const double sg = polar3_newton<16, 3>(m, b, est, 1e-12 * sqrt(nx), 1e-24 * nx * nx);
    smin = est;
    if (est > 1e-12 * sqrt(nx)) return sg;
    return polar3(m, b, smin);
  } else {
    return polar<NM>(m, b, smin);
  }
}

// Sign of det of an (orthogonal) matrix: +1 / -1.
template <int NM, typename R> __device__ __forceinline__ R det_sign(const R* m) {
  R d;
  if constexpr (NM == 1) d = m[0];
  else if constexpr (NM == 2) d = m[0] * m[3] - m[1] * m[2];
  else if constexpr (NM == 3)
    d = m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) +
        m[2] * (m[3] * m[7] - m[4] * m[6]);
  else
    d = det4(m);
  return d >= R(0) ? R(1) : R(-1);
}

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T> __device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum in a fixed order (deterministic).  red needs 32 slots.
template <typename T> __device__ T block_sum(T v, T* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  T r = T(0);
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    r = (l < nw) ? red[l] : T(0);
    r = warp_sum(r);
  }
  return r;  // valid in thread 0
}
template <typename T> __device__ T block_max(T v, T* red) {
  v = warp_max(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  T r = T(0);
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    r = (l < nw) ? red[l] : T(0);
    r = warp_max(r);
  }
  return r;
}

// Arrival counter: returns true in exactly one of `expected` arriving blocks
// (the last), after all of their earlier global writes are visible to it.
__device__ __forceinline__ bool last_to_arrive(unsigned int* counter, unsigned int expected,
                                               int* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int prev = atomicAdd(counter, 1u);
    *s_flag = (prev == expected - 1) ? 1 : 0;
  }
  __syncthreads();
  const bool last = *s_flag != 0;
  if (last) __threadfence();
  return last;
}

// Fixed-order sum of a partial array by one block (deterministic).
__device__ __forceinline__ double sum_partials(const double* p, int count, double* red) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) acc += __ldcg(&p[i]);
  return block_sum(acc, red);
}

// Two fixed-order partial sums by one block in one pass (their loads overlap):
// the same per-thread split and reduction tree as sum_partials, so each total
// is bit-identical to sum_partials of its array.  At most 16 warps; red needs
// 32 slots.
__device__ __forceinline__ void sum_partials2(const double* p1, int n1, const double* p2, int n2,
                                              double* red, double& s1, double& s2) {
  double a1 = 0.0, a2 = 0.0;
  const int n = n1 > n2 ? n1 : n2;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if (i < n1) a1 += __ldcg(&p1[i]);
    if (i < n2) a2 += __ldcg(&p2[i]);
  }
  a1 = warp_sum(a1);
  a2 = warp_sum(a2);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) {
    red[w] = a1;
    red[16 + w] = a2;
  }
  __syncthreads();
  s1 = s2 = 0.0;
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    s1 = warp_sum((l < nw) ? red[l] : 0.0);
    s2 = warp_sum((l < nw) ? red[16 + l] : 0.0);
  }
}

// Deterministic grid-wide sum of one double per block (thread 0's v).  Up to
// kReduceOneLevel blocks, the last block to arrive sums all partials in index
// order (one round of fence and counter); larger grids take two levels: blocks are grouped by kReduceGroup consecutive indices; the last
// block of a group to finish sums that group's partials in index order, and
// the last group to finish sums the group totals in index order.  Returns
// true in exactly one block, whose thread 0 receives the total.  The
// counters return to zero.
__device__ __forceinline__ bool grid_sum(double v, const ReduceBufs& rb, double* red, int* s_flag,
                                         double* total, const double* extra = nullptr,
                                         const unsigned* extra_n = nullptr, double* extra_total = nullptr) {
  const unsigned nb = gridDim.x, b = blockIdx.x;
  if (nb <= kReduceOneLevel) {
    // one level: the last block to arrive sums every partial in index order
    // (and, when asked, another partial array in the same pass)
    if (threadIdx.x == 0) rb.part[b] = v;
    if (!last_to_arrive(&rb.gcount[0], nb, s_flag)) return false;
    double t, te = 0.0;
    if (extra) sum_partials2(rb.part, (int)nb, extra, (int)*extra_n, red, t, te);
    else t = sum_partials(rb.part, (int)nb, red);
    if (threadIdx.x == 0) {
      *total = t;
      if (extra) *extra_total = te;
      rb.gcount[0] = 0;
    }
    return true;
  }
  const unsigned grp = b / kReduceGroup;
  const unsigned ngroups = (nb + kReduceGroup - 1) / kReduceGroup;
  const unsigned gsize = min((unsigned)kReduceGroup, nb - grp * kReduceGroup);
  if (threadIdx.x == 0) rb.part[b] = v;
  if (!last_to_arrive(&rb.gcount[grp], gsize, s_flag)) return false;
  const double gs = sum_partials(rb.part + grp * kReduceGroup, (int)gsize, red);
  if (threadIdx.x == 0) {
    rb.gpart[grp] = gs;
    rb.gcount[grp] = 0;
  }
  if (!last_to_arrive(rb.done, ngroups, s_flag)) return false;
  const double t = sum_partials(rb.gpart, (int)ngroups, red);
  const double te = extra ? sum_partials(extra, (int)*extra_n, red) : 0.0;
  if (threadIdx.x == 0) {
    *total = t;
    if (extra) *extra_total = te;
    *rb.done = 0;
  }
  return true;
}

}  // namespace mbo
