/*
 * FP64 CPU oracle for the generalized MBO scheme on a flat torus
 * (Osting & Wang, "A generalized MBO diffusion generated motion for
 * orthogonal matrix-valued fields", arXiv:1711.01365).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table
 * or helper with the CUDA library, and the CUDA library never calls it.
 *
 * What it computes, in the paper's order (Algorithm 1, "a:MBO"):
 *   1. Diffusion step (Sec. 5.1): every entry A_ij of the field is convolved
 *      with the periodic heat kernel G_{p,tau}; on the grid this is
 *      iFFT( g(k) * FFT(A_ij) ) with the exact torus multiplier
 *      g(k) = exp(-4 pi^2 tau |k|^2), k the signed integer frequency.
 *   2. Projection step (Lemma 1.1): at every grid point the diffused
 *      matrix is replaced by U V^t from its SVD, the closest orthogonal matrix,
 *      whose determinant sign equals that of the diffused matrix.
 *   3. Lyapunov functional (Sec. 4, the functional E^tau), discretised with the
 *      quadrature weight prod_j h_j:
 *        E^tau(A) = (prod h_j / tau) * sum_x ( n - <A(x), (e^{tau Delta} A)(x)>_F ).
 *   4. Stationarity: a step is stationary when no grid point changes the sign
 *      of its determinant (Prop. 4.6, "prop:MBOconverges2") and every entry
 *      moves by at most tol.
 *
 * Conventions.  Field layout is planar: channel c = i*n + j holds entry (i,j)
 * of every grid point, channels are contiguous blocks of P = prod(dims) values,
 * each block row-major over dims (last axis fastest).  The forward DFT uses
 * exp(-2 pi i k.x), the inverse exp(+2 pi i k.x) with a 1/P factor.
 *
 * Readings where the paper is silent (each restated in the design notes):
 *   - the multiplier is the exact exp(-4 pi^2 tau |k|^2), not the DFT of the
 *     sampled periodic kernel (they differ by aliasing terms ~exp(-pi^2 N^2 tau));
 *   - at det(A~) = 0 the positive class is chosen; A~ = 0 maps to the identity;
 *   - the energy constant is n (Sec. 4), with quadrature weight prod h_j.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORC_MAXN 8
#define ORC_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------- */
/* Threads                                                                    */
/* ------------------------------------------------------------------------- */

int orc_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
  return omp_get_max_threads();
#else
  (void)t;
  return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Compensated summation (Neumaier), so that energy sums do not depend on the  */
/* platform's long double.                                                    */
/* ------------------------------------------------------------------------- */

typedef struct { double s, c; } ksum;
static void ks_add(ksum* k, double v) {
  double t = k->s + v;
  if (fabs(k->s) >= fabs(v)) k->c += (k->s - t) + v;
  else k->c += (v - t) + k->s;
  k->s = t;
}
static double ks_val(const ksum* k) { return k->s + k->c; }

/* ------------------------------------------------------------------------- */
/* DFT / FFT                                                                  */
/* ------------------------------------------------------------------------- */

/* exp(sign * 2 pi i * e / N) with e reduced modulo N first. */
static cplx root_of_unity(int64_t e, int64_t N, int sign) {
  e %= N;
  if (e < 0) e += N;
  double ang = 2.0 * ORC_PI * (double)e / (double)N;
  return cos(ang) + (double)sign * I * sin(ang);
}

/* Textbook direct DFT: X[k] = sum_j x[j] exp(sign 2 pi i jk / N). */
static void dft_direct_strided(const cplx* in, int64_t stride, cplx* out, int64_t N, int sign) {
  for (int64_t k = 0; k < N; ++k) {
    cplx acc = 0;
    for (int64_t j = 0; j < N; ++j) acc += in[j * stride] * root_of_unity(j * k, N, sign);
    out[k] = acc;
  }
}

/* Recursive decimation-in-time Cooley-Tukey over the prime factors 2 and 3;
 * any other factor falls back to the direct DFT of that sub-length.
 * in is read with the given stride; out (length N) is contiguous. */
static void fft_rec(const cplx* in, int64_t stride, cplx* out, int64_t N, int sign) {
  if (N == 1) { out[0] = in[0]; return; }
  int p = (N % 2 == 0) ? 2 : (N % 3 == 0) ? 3 : 0;
  if (p == 0) { dft_direct_strided(in, stride, out, N, sign); return; }
  int64_t m = N / p;
  /* Sub-transforms of the decimated sequences x[r + p*j], r = 0..p-1. */
  for (int r = 0; r < p; ++r) fft_rec(in + r * stride, stride * p, out + r * m, m, sign);
  /* Butterfly: X[k + q m] = sum_r w_N^{r (k + q m)} Y_r[k]. */
  cplx* tmp = (cplx*)malloc(sizeof(cplx) * (size_t)N);
  for (int64_t k = 0; k < m; ++k) {
    for (int q = 0; q < p; ++q) {
      int64_t kk = k + q * m;
      cplx acc = 0;
      for (int r = 0; r < p; ++r) acc += root_of_unity((int64_t)r * kk, N, sign) * out[r * m + k];
      tmp[kk] = acc;
    }
  }
  memcpy(out, tmp, sizeof(cplx) * (size_t)N);
  free(tmp);
}

/* In-place unnormalised 1-D transform of interleaved complex data. */
int orc_fft(double* data, int64_t N, int sign) {
  if (N <= 0 || (sign != 1 && sign != -1)) return 1;
  cplx* x = (cplx*)data;
  cplx* out = (cplx*)malloc(sizeof(cplx) * (size_t)N);
  fft_rec(x, 1, out, N, sign);
  memcpy(x, out, sizeof(cplx) * (size_t)N);
  free(out);
  return 0;
}

/* Out-of-place direct DFT (self-check of orc_fft). */
int orc_dft_direct(const double* in, double* out, int64_t N, int sign) {
  if (N <= 0 || (sign != 1 && sign != -1)) return 1;
  dft_direct_strided((const cplx*)in, 1, (cplx*)out, N, sign);
  return 0;
}

/* Multi-dimensional transform: 1-D transforms along every axis in turn. */
int orc_fftn(double* data, int ndim, const int64_t* dims, int sign) {
  if (ndim < 1 || ndim > 3) return 1;
  cplx* x = (cplx*)data;
  int64_t P = 1;
  for (int a = 0; a < ndim; ++a) P *= dims[a];
  for (int a = 0; a < ndim; ++a) {
    int64_t N = dims[a];
    int64_t stride = 1;
    for (int b = a + 1; b < ndim; ++b) stride *= dims[b];
    int64_t lines = P / N;
#pragma omp parallel for schedule(static)
    for (int64_t l = 0; l < lines; ++l) {
      int64_t outer = l / stride, inner = l % stride;
      cplx* base = x + outer * N * stride + inner;
      cplx* line = (cplx*)malloc(sizeof(cplx) * (size_t)N);
      cplx* res = (cplx*)malloc(sizeof(cplx) * (size_t)N);
      for (int64_t j = 0; j < N; ++j) line[j] = base[j * stride];
      fft_rec(line, 1, res, N, sign);
      for (int64_t j = 0; j < N; ++j) base[j * stride] = res[j];
      free(line);
      free(res);
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Heat multiplier and diffusion (Sec. 5.1)                                   */
/* ------------------------------------------------------------------------- */

/* Signed integer frequency of DFT index i on an axis of N points. */
static double signed_freq(int64_t i, int64_t N) { return (double)((2 * i <= N) ? i : i - N); }

/* g(k) = exp(-4 pi^2 tau |k|^2) at flat index f of the spectrum. */
static double heat_multiplier(int64_t f, int ndim, const int64_t* dims, double tau) {
  double k2 = 0;
  for (int a = ndim - 1; a >= 0; --a) {
    int64_t i = f % dims[a];
    f /= dims[a];
    double k = signed_freq(i, dims[a]);
    k2 += k * k;
  }
  return exp(-4.0 * ORC_PI * ORC_PI * tau * k2);
}

/* 1 - g(k), without cancellation. */
static double one_minus_multiplier(int64_t f, int ndim, const int64_t* dims, double tau) {
  double k2 = 0;
  for (int a = ndim - 1; a >= 0; --a) {
    int64_t i = f % dims[a];
    f /= dims[a];
    double k = signed_freq(i, dims[a]);
    k2 += k * k;
  }
  return -expm1(-4.0 * ORC_PI * ORC_PI * tau * k2);
}

int orc_heat_multiplier(double* g, int ndim, const int64_t* dims, double tau) {
  int64_t P = 1;
  for (int a = 0; a < ndim; ++a) P *= dims[a];
  for (int64_t f = 0; f < P; ++f) g[f] = heat_multiplier(f, ndim, dims, tau);
  return 0;
}

/* At = e^{tau Delta} A, channel by channel ("entry by entry", Sec. 5.1 and 8).
 * max_imag (nullable) receives max |imag| of the inverse transforms, which is
 * rounding only because g is real and even. */
int orc_diffuse(const double* A, double* At, int ndim, const int64_t* dims, int C, double tau,
                double* max_imag) {
  if (ndim < 1 || ndim > 3 || C < 1 || !(tau >= 0)) return 1;
  int64_t P = 1;
  for (int a = 0; a < ndim; ++a) P *= dims[a];
  cplx* w = (cplx*)malloc(sizeof(cplx) * (size_t)P);
  double mi = 0;
  for (int c = 0; c < C; ++c) {
    for (int64_t f = 0; f < P; ++f) w[f] = A[c * P + f];
    orc_fftn((double*)w, ndim, dims, -1);
    for (int64_t f = 0; f < P; ++f) w[f] *= heat_multiplier(f, ndim, dims, tau);
    orc_fftn((double*)w, ndim, dims, +1);
    for (int64_t f = 0; f < P; ++f) {
      At[c * P + f] = creal(w[f]) / (double)P;
      double im = fabs(cimag(w[f]) / (double)P);
      if (im > mi) mi = im;
    }
  }
  free(w);
  if (max_imag) *max_imag = mi;
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Projection (Lemma 1.1): one-sided Jacobi SVD and the polar factor U V^t     */
/* ------------------------------------------------------------------------- */

/* Determinant by Gaussian elimination with partial pivoting (row-major n x n). */
double orc_det(const double* M, int n) {
  double a[ORC_MAXN * ORC_MAXN];
  memcpy(a, M, sizeof(double) * (size_t)(n * n));
  double det = 1.0;
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (fabs(a[i * n + k]) > fabs(a[piv * n + k])) piv = i;
    if (a[piv * n + k] == 0.0) return 0.0;
    if (piv != k) {
      for (int j = 0; j < n; ++j) { double t = a[k * n + j]; a[k * n + j] = a[piv * n + j]; a[piv * n + j] = t; }
      det = -det;
    }
    det *= a[k * n + k];
    for (int i = k + 1; i < n; ++i) {
      double l = a[i * n + k] / a[k * n + k];
      for (int j = k; j < n; ++j) a[i * n + j] -= l * a[k * n + j];
    }
  }
  return det;
}

/* Complete the column `col` of the column-major-by-index matrix U (U[i*n+j] =
 * entry (i,j)) to a unit vector orthogonal to the other columns listed in
 * `have` (Gram-Schmidt against the standard basis). */
static void complete_column(double* U, int n, int col, const int* have) {
  for (int e = 0; e < n; ++e) {
    double v[ORC_MAXN];
    for (int i = 0; i < n; ++i) v[i] = (i == e) ? 1.0 : 0.0;
    for (int pass = 0; pass < 2; ++pass)
      for (int j = 0; j < n; ++j) {
        if (!have[j]) continue;
        double d = 0;
        for (int i = 0; i < n; ++i) d += U[i * n + j] * v[i];
        for (int i = 0; i < n; ++i) v[i] -= d * U[i * n + j];
      }
    double nv = 0;
    for (int i = 0; i < n; ++i) nv += v[i] * v[i];
    nv = sqrt(nv);
    if (nv > 0.5) {
      for (int i = 0; i < n; ++i) U[i * n + col] = v[i] / nv;
      return;
    }
  }
}

/* Polar factor of one n x n matrix M (row-major) by a one-sided (Hestenes)
 * Jacobi SVD.  B = U D V^t where D = I except that the entry of the smallest
 * singular value is chosen so that sign det B = sign det M (Lemma 1.1; at
 * det M = 0 the positive class).  For nonsingular M this is exactly U V^t of
 * the SVD; the flip form is the opposite-class minimiser of Lemma 7.1.
 * sigma (nullable) receives the singular values in descending order.
 * Returns the number of Jacobi sweeps. */
static int polar_in_class(const double* M, double* B, double* sigma, int n, int cls);

int orc_polar(const double* M, double* B, double* sigma, int n) {
  return polar_in_class(M, B, sigma, n, 0);
}

/* Closest matrix of a prescribed class (cls = +1: SO(n), -1: SO^-(n)),
 * Lemma 7.1: U V^t when the class is that of det M, otherwise U D_n V^t with
 * D_n flipping the column of the smallest singular value. */
int orc_polar_class(const double* M, double* B, int n, int cls) {
  return polar_in_class(M, B, NULL, n, cls >= 0 ? 1 : -1);
}

static int polar_in_class(const double* M, double* B, double* sigma, int n, int cls) {
  if (n < 1 || n > ORC_MAXN) return -1;
  double a[ORC_MAXN * ORC_MAXN], v[ORC_MAXN * ORC_MAXN];
  memcpy(a, M, sizeof(double) * (size_t)(n * n));
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) v[i * n + j] = (i == j) ? 1.0 : 0.0;
  int sweeps = 0;
  for (; sweeps < 40; ++sweeps) {
    int rotated = 0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double alpha = 0, beta = 0, gamma = 0;
        for (int i = 0; i < n; ++i) {
          alpha += a[i * n + p] * a[i * n + p];
          beta += a[i * n + q] * a[i * n + q];
          gamma += a[i * n + p] * a[i * n + q];
        }
        if (gamma == 0.0 || fabs(gamma) <= 1e-15 * sqrt(alpha * beta)) continue;
        rotated = 1;
        double zeta = (beta - alpha) / (2.0 * gamma);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        for (int i = 0; i < n; ++i) {
          double ap = a[i * n + p], aq = a[i * n + q];
          a[i * n + p] = c * ap - s * aq;
          a[i * n + q] = s * ap + c * aq;
          double vp = v[i * n + p], vq = v[i * n + q];
          v[i * n + p] = c * vp - s * vq;
          v[i * n + q] = s * vp + c * vq;
        }
      }
    if (!rotated) break;
  }
  /* Singular values = column norms of A V; U = A V Sigma^{-1}. */
  double sg[ORC_MAXN], U[ORC_MAXN * ORC_MAXN];
  int have[ORC_MAXN];
  for (int j = 0; j < n; ++j) {
    double s2 = 0;
    for (int i = 0; i < n; ++i) s2 += a[i * n + j] * a[i * n + j];
    sg[j] = sqrt(s2);
    have[j] = sg[j] > 1e-300;
    for (int i = 0; i < n; ++i) U[i * n + j] = have[j] ? a[i * n + j] / sg[j] : 0.0;
  }
  int jmin = 0;
  for (int j = 1; j < n; ++j)
    if (sg[j] < sg[jmin]) jmin = j;
  int any = 0;
  for (int j = 0; j < n; ++j) any |= have[j];
  if (!any) { /* A~ = 0: the identity (diag(1, .., 1, -1) for the negative class). */
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) B[i * n + j] = (i == j) ? ((cls < 0 && i == n - 1) ? -1.0 : 1.0) : 0.0;
    if (sigma)
      for (int j = 0; j < n; ++j) sigma[j] = 0.0;
    return sweeps;
  }
  for (int j = 0; j < n; ++j)
    if (!have[j]) { complete_column(U, n, j, have); have[j] = 1; }
  /* Enforce sign det(U V^t) = sign det M (or the prescribed class) by the
   * smallest-singular-value column. */
  double want = cls != 0 ? (double)cls : ((orc_det(M, n) >= 0.0) ? 1.0 : -1.0);
  double du = orc_det(U, n), dv = orc_det(v, n);
  if ((du * dv >= 0.0 ? 1.0 : -1.0) != want)
    for (int i = 0; i < n; ++i) U[i * n + jmin] = -U[i * n + jmin];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double acc = 0;
      for (int k = 0; k < n; ++k) acc += U[i * n + k] * v[j * n + k];
      B[i * n + j] = acc;
    }
  if (sigma) {
    /* descending order */
    double s[ORC_MAXN];
    memcpy(s, sg, sizeof(double) * (size_t)n);
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j)
        if (s[j] > s[i]) { double t = s[i]; s[i] = s[j]; s[j] = t; }
    memcpy(sigma, s, sizeof(double) * (size_t)n);
  }
  return sweeps;
}

/* Project every grid point of a planar field (Algorithm 1, step 2).
 * det_sign (nullable) receives +1/-1 per point: the class chosen for B. */
int orc_project_field(const double* At, double* B, int8_t* det_sign, int64_t P, int n) {
  if (n < 1 || n > ORC_MAXN || P < 0) return 1;
  int C = n * n;
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < P; ++x) {
    double M[ORC_MAXN * ORC_MAXN], Bx[ORC_MAXN * ORC_MAXN];
    for (int c = 0; c < C; ++c) M[c] = At[c * P + x];
    orc_polar(M, Bx, NULL, n);
    for (int c = 0; c < C; ++c) B[c * P + x] = Bx[c];
    if (det_sign) det_sign[x] = (orc_det(M, n) >= 0.0) ? 1 : -1;
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* One step at sampled grid points, straight from the definition (Sec. 5.1):  */
/* A~(x) = sum_y K(x - y) A(y), K the discrete periodic heat kernel, i.e. the  */
/* inverse DFT of g; K is separable, K = K_z (x) K_y (x) K_x with             */
/* K_a(d) = (1/N_a) sum_k exp(-4 pi^2 tau k^2) cos(2 pi k d / N_a).           */
/* Each 1-D kernel is truncated to |d| <= r_a beyond which the Gaussian decay */
/* of K_a puts every dropped term below 1e-22 of K_a(0).  With project_input   */
/* the input is first projected point by point (Lemma 1.1), so the result is   */
/* one step of Algorithm 1 from the projected field.                          */
/* ------------------------------------------------------------------------- */

static void kernel_1d(int64_t N, double tau, double* K, int64_t* radius) {
  for (int64_t d = 0; d < N; ++d) {
    ksum s = {0, 0};
    for (int64_t k = 0; k < N; ++k) {
      double kf = signed_freq(k, N);
      ks_add(&s, exp(-4.0 * ORC_PI * ORC_PI * tau * kf * kf) * creal(root_of_unity(k * d, N, 1)));
    }
    K[d] = ks_val(&s) / (double)N;
  }
  /* The kernel is the periodised Gaussian of variance 2 tau (grid units:
   * 2 tau N^2), so K(d) / K(0) ~ exp(-d^2 / (4 tau N^2)).  Values computed
   * by the sum above bottom out at rounding (~1e-17 absolute), so the radius
   * comes from that decay: dropped terms are below 1e-22 of K(0). */
  double rr = sqrt(4.0 * tau * (double)N * (double)N * log(1e22));
  int64_t r = (int64_t)ceil(rr) + 1;
  if (r > N / 2) r = N / 2;
  *radius = r;
}

static int step_points_impl(const double* A, const float* Af, int ndim, const int64_t* dims,
                            int n, double tau, int project_input, const int64_t* pts,
                            int64_t npts, double* At_out, double* B_out) {
  if (ndim < 1 || ndim > 3 || n < 1 || n > ORC_MAXN) return 1;
  int64_t d3[3] = {1, 1, 1};
  for (int a = 0; a < ndim; ++a) d3[3 - ndim + a] = dims[a];
  int64_t P = d3[0] * d3[1] * d3[2];
  int C = n * n;
  double* K[3];
  int64_t lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    int64_t r;
    K[a] = (double*)malloc(sizeof(double) * (size_t)d3[a]);
    kernel_1d(d3[a], tau, K[a], &r);
    if (d3[a] == 1) { K[a][0] = 1.0; r = 0; }
    /* offsets -lo..hi visit every residue at most once */
    lo[a] = r < (d3[a] - 1) / 2 ? r : (d3[a] - 1) / 2;
    hi[a] = r < d3[a] / 2 ? r : d3[a] / 2;
  }
  const int64_t bz = lo[0] + hi[0] + 1, by = lo[1] + hi[1] + 1, bx = lo[2] + hi[2] + 1;
#pragma omp parallel for schedule(dynamic)
  for (int64_t s = 0; s < npts; ++s) {
    int64_t c3[3] = {0, 0, 0};
    for (int a = 0; a < ndim; ++a) c3[3 - ndim + a] = pts[s * ndim + a];
    /* gather the neighbourhood x - d, d in [-lo, hi]^3 (periodic), projected if asked */
    double* box = (double*)malloc(sizeof(double) * (size_t)(bz * by * bx * C));
    for (int64_t iz = 0; iz < bz; ++iz) {
      int64_t z = ((c3[0] - (iz - lo[0])) % d3[0] + d3[0]) % d3[0];
      for (int64_t iy = 0; iy < by; ++iy) {
        int64_t y = ((c3[1] - (iy - lo[1])) % d3[1] + d3[1]) % d3[1];
        for (int64_t ix = 0; ix < bx; ++ix) {
          int64_t x = ((c3[2] - (ix - lo[2])) % d3[2] + d3[2]) % d3[2];
          int64_t f = (z * d3[1] + y) * d3[2] + x;
          double* M = box + ((iz * by + iy) * bx + ix) * C;
          for (int c = 0; c < C; ++c) M[c] = A ? A[c * P + f] : (double)Af[c * P + f];
          if (project_input) {
            double Bq[ORC_MAXN * ORC_MAXN];
            orc_polar(M, Bq, NULL, n);
            for (int c = 0; c < C; ++c) M[c] = Bq[c];
          }
        }
      }
    }
    /* weighted sum K_z(dz) K_y(dy) K_x(dx) A(x - d), compensated */
    double acc[ORC_MAXN * ORC_MAXN];
    ksum ks[ORC_MAXN * ORC_MAXN];
    for (int c = 0; c < C; ++c) ks[c].s = ks[c].c = 0;
    for (int64_t iz = 0; iz < bz; ++iz) {
      int64_t dz = iz - lo[0];
      double kz = K[0][(dz % d3[0] + d3[0]) % d3[0]];
      for (int64_t iy = 0; iy < by; ++iy) {
        int64_t dy = iy - lo[1];
        double kzy = kz * K[1][(dy % d3[1] + d3[1]) % d3[1]];
        for (int64_t ix = 0; ix < bx; ++ix) {
          int64_t dx = ix - lo[2];
          double w = kzy * K[2][(dx % d3[2] + d3[2]) % d3[2]];
          const double* M = box + ((iz * by + iy) * bx + ix) * C;
          for (int c = 0; c < C; ++c) ks_add(&ks[c], w * M[c]);
        }
      }
    }
    free(box);
    for (int c = 0; c < C; ++c) acc[c] = ks_val(&ks[c]);
    if (At_out)
      for (int c = 0; c < C; ++c) At_out[s * C + c] = acc[c];
    if (B_out) {
      double Bp[ORC_MAXN * ORC_MAXN];
      orc_polar(acc, Bp, NULL, n);
      for (int c = 0; c < C; ++c) B_out[s * C + c] = Bp[c];
    }
  }
  for (int a = 0; a < 3; ++a) free(K[a]);
  return 0;
}

int orc_step_points(const double* A, int ndim, const int64_t* dims, int n, double tau,
                    int project_input, const int64_t* pts, int64_t npts, double* At_out,
                    double* B_out) {
  return step_points_impl(A, NULL, ndim, dims, n, tau, project_input, pts, npts, At_out, B_out);
}

/* Same, reading a float32 field (each value converted exactly to double). */
int orc_step_points_f32(const float* A, int ndim, const int64_t* dims, int n, double tau,
                        int project_input, const int64_t* pts, int64_t npts, double* At_out,
                        double* B_out) {
  return step_points_impl(NULL, A, ndim, dims, n, tau, project_input, pts, npts, At_out, B_out);
}

/* ------------------------------------------------------------------------- */
/* Lyapunov functional (Sec. 4 and its grid sum in Sec. 4.1)                 */
/* ------------------------------------------------------------------------- */

static double quad_weight(int ndim, const int64_t* dims) {
  double w = 1.0;
  for (int a = 0; a < ndim; ++a) w /= (double)dims[a];
  return w;
}

/* Physical form from a field and its diffusion:
 * (prod h / tau) * sum_x ( n - <A(x), At(x)>_F ). */
double orc_energy_from(const double* A, const double* At, int ndim, const int64_t* dims, int n,
                       double tau) {
  int64_t P = 1;
  for (int a = 0; a < ndim; ++a) P *= dims[a];
  int C = n * n;
  ksum tot = {0, 0};
  for (int64_t x = 0; x < P; ++x) {
    double ip = 0;
    for (int c = 0; c < C; ++c) ip += A[c * P + x] * At[c * P + x];
    ks_add(&tot, (double)n - ip);
  }
  return quad_weight(ndim, dims) / tau * ks_val(&tot);
}

double orc_energy(const double* A, int ndim, const int64_t* dims, int n, double tau) {
  int64_t P = 1;
  for (int a = 0; a < ndim; ++a) P *= dims[a];
  double* At = (double*)malloc(sizeof(double) * (size_t)(P * n * n));
  orc_diffuse(A, At, ndim, dims, n * n, tau, NULL);
  double e = orc_energy_from(A, At, ndim, dims, n, tau);
  free(At);
  return e;
}

/* Spectral (Parseval) form, free of the n - <A, GA> cancellation:
 * (prod h / tau) * [ (1/P) sum_k (1 - g(k)) sum_c |A^_c(k)|^2
 *                    + sum_x ( n - ||A(x)||_F^2 ) ]. */
double orc_energy_spectral(const double* A, int ndim, const int64_t* dims, int n, double tau) {
  int64_t P = 1;
  for (int a = 0; a < ndim; ++a) P *= dims[a];
  int C = n * n;
  cplx* w = (cplx*)malloc(sizeof(cplx) * (size_t)P);
  ksum spec = {0, 0}, defect = {0, 0};
  for (int c = 0; c < C; ++c) {
    for (int64_t f = 0; f < P; ++f) w[f] = A[c * P + f];
    orc_fftn((double*)w, ndim, dims, -1);
    for (int64_t f = 0; f < P; ++f) {
      double m2 = creal(w[f]) * creal(w[f]) + cimag(w[f]) * cimag(w[f]);
      ks_add(&spec, one_minus_multiplier(f, ndim, dims, tau) * m2);
    }
  }
  for (int64_t x = 0; x < P; ++x) {
    double nn = 0;
    for (int c = 0; c < C; ++c) nn += A[c * P + x] * A[c * P + x];
    ks_add(&defect, (double)n - nn);
  }
  free(w);
  return quad_weight(ndim, dims) / tau * (ks_val(&spec) / (double)P + ks_val(&defect));
}

/* ------------------------------------------------------------------------- */
/* One iteration and the loop (Algorithm 1)                                   */
/* ------------------------------------------------------------------------- */

typedef struct {
  double energy;      /* E^tau of the field entering the step            */
  double max_delta;   /* max over points and channels |A_new - A_old|     */
  int64_t det_flips;  /* points whose determinant sign changed            */
  double max_imag;    /* max |imag| left by the inverse transforms        */
} orc_stats;

/* A <- polar(e^{tau Delta} A) in place; fills st (nullable). */
int orc_step(double* A, int ndim, const int64_t* dims, int n, double tau, orc_stats* st) {
  int64_t P = 1;
  for (int a = 0; a < ndim; ++a) P *= dims[a];
  int C = n * n;
  double* At = (double*)malloc(sizeof(double) * (size_t)(P * C));
  double* Bn = (double*)malloc(sizeof(double) * (size_t)(P * C));
  double mi = 0;
  int rc = orc_diffuse(A, At, ndim, dims, C, tau, &mi);
  if (rc) { free(At); free(Bn); return rc; }
  double energy = orc_energy_from(A, At, ndim, dims, n, tau);
  orc_project_field(At, Bn, NULL, P, n);
  double md = 0;
  int64_t flips = 0;
  for (int64_t x = 0; x < P; ++x) {
    double Mo[ORC_MAXN * ORC_MAXN], Mn[ORC_MAXN * ORC_MAXN];
    for (int c = 0; c < C; ++c) {
      Mo[c] = A[c * P + x];
      Mn[c] = Bn[c * P + x];
      double d = fabs(Mn[c] - Mo[c]);
      if (d > md) md = d;
    }
    if ((orc_det(Mo, n) >= 0.0) != (orc_det(Mn, n) >= 0.0)) ++flips;
  }
  memcpy(A, Bn, sizeof(double) * (size_t)(P * C));
  free(At);
  free(Bn);
  if (st) { st->energy = energy; st->max_delta = md; st->det_flips = flips; st->max_imag = mi; }
  return 0;
}

/* Iterate until a step is stationary (no determinant sign flips and every
 * entry moved by <= tol) or max_steps steps were taken.
 * energies (nullable, length max_steps+1): E^tau(A_0), ..., E^tau(A_steps).
 * max_deltas / flips (nullable, length max_steps): per-step statistics. */
int orc_run(double* A, int ndim, const int64_t* dims, int n, double tau, int max_steps, double tol,
            int* steps_taken, int* stationary, double* energies, double* max_deltas,
            int64_t* flips) {
  int s = 0, stat = 0;
  for (; s < max_steps; ++s) {
    orc_stats st;
    int rc = orc_step(A, ndim, dims, n, tau, &st);
    if (rc) return rc;
    if (energies) energies[s] = st.energy;
    if (max_deltas) max_deltas[s] = st.max_delta;
    if (flips) flips[s] = st.det_flips;
    if (st.det_flips == 0 && st.max_delta <= tol) { stat = 1; ++s; break; }
  }
  if (energies) energies[s] = orc_energy(A, ndim, dims, n, tau);
  if (steps_taken) *steps_taken = s;
  if (stationary) *stationary = stat;
  return 0;
}

/* ------------------------------------------------------------------------- */
/* Volume-preserving step (Sec. 7): T+ / T- are the closest matrices of     */
/* SO(n) / SO^-(n) (Lemma 7.1), dE(x) = <T+(A~) - T-(A~), A~>_F, and the      */
/* n_plus points of largest dE (the set {dE >= lambda} of Lemma 7.2 on a      */
/* uniform grid, Algorithm 3 with equal weights) take T+, the others T-.      */
/* Equal dE values are ordered by grid index (lower index first).             */
/* ------------------------------------------------------------------------- */

typedef struct { double de; int64_t idx; } de_item;
static int de_cmp(const void* a, const void* b) {
  const de_item* x = (const de_item*)a;
  const de_item* y = (const de_item*)b;
  if (x->de > y->de) return -1;
  if (x->de < y->de) return 1;
  return (x->idx < y->idx) ? -1 : (x->idx > y->idx);
}

double orc_delta_energy(const double* M, int n) {
  double Tp[ORC_MAXN * ORC_MAXN], Tm[ORC_MAXN * ORC_MAXN];
  orc_polar_class(M, Tp, n, 1);
  orc_polar_class(M, Tm, n, -1);
  double s = 0;
  for (int c = 0; c < n * n; ++c) s += (Tp[c] - Tm[c]) * M[c];
  return s;
}

/* Number of points whose (orthogonal) matrix has det > 0. */
int64_t orc_count_positive(const double* A, int64_t P, int n) {
  int64_t cnt = 0;
  for (int64_t x = 0; x < P; ++x) {
    double M[ORC_MAXN * ORC_MAXN];
    for (int c = 0; c < n * n; ++c) M[c] = A[c * P + x];
    if (orc_det(M, n) > 0.0) ++cnt;
  }
  return cnt;
}

/* One volume-preserving step in place; n_plus < 0 keeps the count of A. */
int orc_step_volume(double* A, int ndim, const int64_t* dims, int n, double tau, int64_t n_plus,
                    orc_stats* st, double* dE_out) {
  int64_t P = 1;
  for (int a = 0; a < ndim; ++a) P *= dims[a];
  int C = n * n;
  if (n_plus < 0) n_plus = orc_count_positive(A, P, n);
  if (n_plus > P) return 1;
  double* At = (double*)malloc(sizeof(double) * (size_t)(P * C));
  double mi = 0;
  int rc = orc_diffuse(A, At, ndim, dims, C, tau, &mi);
  if (rc) { free(At); return rc; }
  double energy = orc_energy_from(A, At, ndim, dims, n, tau);
  de_item* items = (de_item*)malloc(sizeof(de_item) * (size_t)P);
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < P; ++x) {
    double M[ORC_MAXN * ORC_MAXN];
    for (int c = 0; c < C; ++c) M[c] = At[c * P + x];
    items[x].de = orc_delta_energy(M, n);
    items[x].idx = x;
  }
  if (dE_out)
    for (int64_t x = 0; x < P; ++x) dE_out[x] = items[x].de;
  qsort(items, (size_t)P, sizeof(de_item), de_cmp);
  double md = 0;
  int64_t flips = 0;
  for (int64_t r = 0; r < P; ++r) {
    int64_t x = items[r].idx;
    double M[ORC_MAXN * ORC_MAXN], Bx[ORC_MAXN * ORC_MAXN], Mo[ORC_MAXN * ORC_MAXN];
    for (int c = 0; c < C; ++c) {
      M[c] = At[c * P + x];
      Mo[c] = A[c * P + x];
    }
    orc_polar_class(M, Bx, n, r < n_plus ? 1 : -1);
    for (int c = 0; c < C; ++c) {
      double d = fabs(Bx[c] - Mo[c]);
      if (d > md) md = d;
      A[c * P + x] = Bx[c];
    }
    if ((orc_det(Mo, n) > 0.0) != (r < n_plus)) ++flips;
  }
  free(items);
  free(At);
  if (st) { st->energy = energy; st->max_delta = md; st->det_flips = flips; st->max_imag = mi; }
  return 0;
}

