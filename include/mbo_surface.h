/*
 * mbo_surface.h - C ABI of the closed-surface path of the GB300 (sm_103a)
 * generalized MBO library: Algorithm 1 of Osting & Wang (arXiv:1711.01365)
 * on a smooth closed surface in R^3, with the diffusion step computed as in
 * Sec. 5.2 and Algorithm 2:
 *   closest-point extension: the value at a quadrature point x_q of the band
 *              around the surface is the value at its closest surface point
 *              x_q^c;
 *   diffusion: the free-space heat kernel G_tau^3, replaced by its truncated
 *              Fourier sum (the heat-kernel approximation theorem of Sec. 5.2:
 *              spacing h, modes m in {-M..M-1}^3), applied as a type-1
 *              non-uniform transform of the band values (weights w_q), the
 *              factor exp(-h^2 tau |m|^2), and a type-2 non-uniform transform
 *              evaluated at the closest points:
 *                A~(x_t) = (h/2pi)^3 Re sum_m e^{-h^2 tau |m|^2} e^{i h m.x_t}
 *                                        sum_q w_q A(x_q^c) e^{-i h m.x_q};
 *   projection (Lemma 1.1): every x_t becomes the closest orthogonal matrix.
 * The non-uniform transforms run on the GPU as spreading onto an oversampled
 * periodic grid with the "exponential of semicircle" kernel
 * exp(beta (sqrt(1 - z^2) - 1)) (Barnett, Magland and af Klinteberg, SIAM J.
 * Sci. Comput. 41 (2019)), the library's own 3-D FFT with the deconvolved heat
 * factor, and interpolation from that grid.
 *
 * Conventions (as in mbo.h unless stated here)
 *   - A surface field is a planar array of n*n channels of nq values each:
 *     channel c = i*n + j holds matrix entry (i,j) at every point x_t, in the
 *     order the points were given.  Element type float (MBO_F32) or double
 *     (MBO_F64); caller-owned device pointers, 16-byte aligned.
 *   - Point arrays (xq, xc) are HOST arrays of nq rows (x, y, z), row-major,
 *     double; weights wq are host doubles.  The library copies them.
 *   - Source q (a quadrature point x_q with weight w_q) takes the value of
 *     point q (its closest point x_q^c): the field lives at the nq closest
 *     points, one per quadrature point.
 *   - Status codes, stream semantics and thread safety as in mbo.h.
 */
#ifndef MBO_GB300_SURFACE_H
#define MBO_GB300_SURFACE_H

#include "mbo.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mbo_surface_ctx* mbo_surface;

/* Band width w_b of the band-truncation theorem of Sec. 5.2: the root of
 * T(w_b / (2 sqrt(tau))) = eps, T(x) = 2x/sqrt(pi) exp(-x^2) + erfc(x).
 * Host only.  Returns a negative value if eps is not in (0, 1) or tau <= 0. */
MBO_API double mbo_surface_band_width(double eps, double tau);

/* Spacing h and mode count M of the heat-kernel approximation theorem of
 * Sec. 5.2 for spatial radius R (every per-axis point difference at most R):
 *   h = min(pi / R, pi / (2 sqrt(tau |ln eps|))),
 *   M = ceil( sqrt( ln(2 h sqrt(tau) / (sqrt(pi) eps)) / tau ) / h )
 * (the printed logarithm's argument read inverted, so that it exceeds 1).
 * Host only.  MBO_ERR_INVALID_ARG for eps not in (0, 1/2), tau <= 0, R <= 0. */
MBO_API mbo_status mbo_surface_heat_modes(double eps, double tau, double R, double* h, int* M);

/* Band, quadrature points and closest points of the sphere |x| = radius
 * (Algorithm 2, step 1).  Grid points x_g = dx (i, j, k) with
 * | |x_g| - radius | < wb; each cell x_g + [0, dx]^3 carries p^3 points, the
 * tensor product of the p Gauss-Chebyshev nodes cos((2k-1) pi / (2p)) mapped
 * to [0, dx] with Fejer's (interpolatory) weights; x_q^c = radius x_q / |x_q|
 * ((0, 0, radius) at the centre).  Order: grid points (i, j, k) lexicographic,
 * k fastest, then the cell's nodes (a, b, c) lexicographic, c fastest.
 * xq, xc (nq x 3) and wq (nq) are host arrays of capacity `capacity` points;
 * with any of them NULL only *count is set.  MBO_ERR_INVALID_ARG for
 * radius, dx or wb <= 0, p outside 1..16, or capacity < count (with *count
 * set to the size needed).  Host only. */
MBO_API mbo_status mbo_surface_sphere_band(double radius, double dx, double wb, int p, double* xq,
                                           double* wq, double* xc, int64_t capacity,
                                           int64_t* count);

/* The same for the peanut surface of Sec. 6.3: the surface of revolution about
 * the x axis of the curve x = 3t - t^3, rho = sqrt((1 + x^2)(4 - x^2)) / 2,
 * t in [-1, 1].  The band holds the grid points whose distance to the surface
 * is below wb; closest points come from the closest point of (x, |(y, z)|) on
 * the curve (a scan of t and a golden-section search; the +y meridian on the
 * axis), so the band costs a few hundred curve evaluations per point.  Same
 * arguments, order and errors as mbo_surface_sphere_band.  Host only. */
MBO_API mbo_status mbo_surface_peanut_band(double dx, double wb, int p, double* xq, double* wq,
                                           double* xc, int64_t capacity, int64_t* count);

/* Plan one surface geometry.
 *   nq        number of quadrature points (= field points), 1 <= nq < 2^31.
 *   xq, wq    quadrature points (nq x 3) and weights (nq), host arrays.
 *   xc        closest points (nq x 3), host array.
 *   n         matrix order 1..4; tau > 0 the diffusion time of one step.
 *   eps       accuracy in (1e-12, 1/2): it sets h and M (mbo_surface_heat_modes
 *             with R the largest coordinate extent of all xq and xc) and the
 *             spreading width ceil(log10(1/eps)) + 1, clamped to 4..8 (the
 *             spreading error is then about 10^(1 - width): below 1e-7 the
 *             non-uniform transforms, not eps, set the accuracy).
 * The oversampled grid has nf = the smallest 2^a 3^b >= max(4M, 2 width, 8)
 * points per axis (MBO_ERR_UNSUPPORTED_SIZE above 2048).  Allocates that
 * grid (n*n channels), the library's FFT workspace for it and the sorted
 * point tables on the current device.  Synchronous. */
MBO_API mbo_status mbo_surface_create(mbo_surface* out, int64_t nq, const double* xq,
                                      const double* wq, const double* xc, int n, double tau,
                                      double eps, mbo_dtype dtype);
MBO_API mbo_status mbo_surface_destroy(mbo_surface s);

/* Parameters the plan chose (host copy). */
typedef struct {
  double h;          /* spectral spacing                                         */
  int M;             /* modes per axis: m in {-M..M-1}                           */
  int nf;            /* oversampled grid points per axis                         */
  int width;         /* spreading kernel width (grid points per axis)            */
  double beta;       /* kernel shape parameter                                   */
  double R;          /* largest coordinate extent of the points                  */
  double center[3];  /* the points' bounding-box centre (phase origin)           */
  int64_t bins;      /* non-empty spreading bins                                 */
} mbo_surface_params;
MBO_API mbo_status mbo_surface_get_params(mbo_surface s, mbo_surface_params* p);

/* Diffusion step alone (Algorithm 2, steps 2-5): A_tilde = the diffused field
 * at the nq closest points.  A and A_tilde are device surface fields; they
 * may be the same pointer. */
MBO_API mbo_status mbo_surface_diffuse(mbo_surface s, const void* A, void* A_tilde, void* stream);

/* One iteration of Algorithm 1 on the surface, in place: A <- polar(diffused
 * A) (Lemma 1.1).  stats (nullable): if given, the call synchronises the
 * stream and fills max_delta, det_flips, fallback_points and nonfinite;
 * energy is NaN (the surface path defines no Lyapunov value). */
MBO_API mbo_status mbo_surface_step(mbo_surface s, void* A, mbo_stats* stats, void* stream);

/* One volume-preserving step on the surface (Sec. 7, Algorithm 3), in place.
 * After the diffusion above, every point gets dE = <T+ - T-, A~> (T+, T- the
 * closest matrices of SO(n) and SO^-(n) to the diffused A~, Lemma 7.1).  Taking
 * points in decreasing dE (equal dE: lower point index first) and adding their
 * weights w_q (the plan's quadrature weights: each point's share of the band
 * volume), the smallest prefix whose weight reaches `volume` takes T+ and the
 * other points take T- (Algorithm 3; Lemma 7.2), so the selected weight lies in
 * [volume, volume + the last point's weight).  volume < 0: the weight of the
 * points with det A > 0 in the input; repeated calls in that mode may then
 * gain up to one point's weight per step, so a run that must keep its volume
 * passes the same volume to every step.  Weights
 * are summed exactly in fixed point (w_q scaled so that all sum to 2^62).
 * n <= 3 (MBO_ERR_UNSUPPORTED_SIZE otherwise); negative weights or a NaN volume
 * are MBO_ERR_INVALID_ARG.  stats as in mbo_surface_step (fallback_points 0).
 * Allocates 2 n*n nq elements and 2 nq 64-bit words on first use. */
MBO_API mbo_status mbo_surface_step_volume(mbo_surface s, void* A, double volume, mbo_stats* stats,
                                           void* stream);

/* Per-pass device timing of the surface calls (CUDA events around each
 * launch on the caller's stream; off by default).  Passes, in this order:
 * spreading (k_spread), the grid's FFT diffusion (all its passes together),
 * interpolation (k_interp), projection (k_sproject).  mbo_surface_profile_enable
 * (re)starts the accumulation; mbo_surface_profile_read synchronises on the
 * recorded events and returns, for the first npass passes, the accumulated
 * milliseconds and the number of timed calls. */
enum { MBO_SURFACE_PROFILE_PASSES = 4 };
MBO_API mbo_status mbo_surface_profile_enable(mbo_surface s, int enable);
MBO_API mbo_status mbo_surface_profile_read(mbo_surface s, double* ms, int64_t* launches, int npass);

/* Device bytes the plan holds. */
MBO_API int64_t mbo_surface_workspace_bytes(mbo_surface s);

/* Text of the last error recorded in the plan (empty string if none). */
MBO_API const char* mbo_surface_last_error(mbo_surface s);

#ifdef __cplusplus
}
#endif

#endif /* MBO_GB300_SURFACE_H */
