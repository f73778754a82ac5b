/*
 * gm_oracle.c -- plain, slow FP64 CPU reference for batched galaxy-profile
 * fitting (arxiv 2404.07780, "galmoss").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file.  It shares no code, no
 * header and no constant table with the CUDA library; it is written straight
 * from the paper's definitions, in double precision, one pixel at a time:
 *
 *   light profiles at pixel centres ........ Sec. 4.1-4.2, Eqs. (r), (rmaj),
 *        (rmin), (sersic-intensity), (expdisk_I), (ferrer_I), (BE_S),
 *        (gaussion_I), (moffat_I), (sky_I)
 *   sum of PSF-convolved components, direct zero-padded correlation with
 *        the PSF, then the unconvolved components (the flat sky) ......
 *        Sec. 2 (workflow) and the conv2d(..., padding="same") call of App. C
 *   masked sigma-weighted chi^2 ............ Sec. 5.1, Eq. (chinu)
 *   Jacobian by central finite differences . (no analytic derivative here)
 *   Levenberg-Marquardt damped Gauss-Newton  Sec. 5.1 names LM as the
 *        classical alternative; the damping/acceptance rules are spelled out
 *        at or_fit_one() below
 *   covariance uncertainty ................. Sec. 5.2,
 *        sigma_p = sqrt(diag[(J^T W J)^-1]), W = 1/sigma^2
 *
 * Readings of points the paper leaves open (all listed in the design notes):
 *   - pixel centres x_j = j + 0.5, y_i = H - 0.5 - i (row 0 at the top), as in
 *     the grid built by the App. C listing;
 *   - PSF application is a cross-correlation, M[i,j] = sum_ab P[a,b] *
 *     I[i+a-c, j+b-c], zero outside the stamp, K odd, c = (K-1)/2 (torch
 *     conv2d semantics);
 *   - the elliptical radius (B = 0) is r = sqrt(X^2 + (Y/q)^2) with
 *     X =  cos(pa) dx + sin(pa) dy, Y = -sin(pa) dx + cos(pa) dy;
 *   - r is floored at 1e-4 px (the Sersic cusp);
 *   - the King bracket is read as [A(r) - A(r_t)] so that I(0) = I0, and both
 *     King and Ferrer are zero beyond their truncation radius;
 *   - Gaussian FWHM = 2 sqrt(2 ln 2) sigma;
 *   - mask: nonzero = excluded pixel.
 *
 * Parameter order of each component (geometric subset p_G first, then the
 * radial subset p_L, following the split of Sec. 2):
 *   SERSIC   x0 y0 q pa Ie Re n
 *   EXPDISK  x0 y0 q pa I0 rs
 *   FERRER   x0 y0 q pa I0 rout a b
 *   KING     x0 y0 q pa I0 rc rt alpha
 *   GAUSSIAN x0 y0 q pa I0 fwhm
 *   MOFFAT   x0 y0 q pa I0 fwhm n
 *   SKY      Isky
 *   TSKY     Isky kx ky   (tilted sky, Eq. new_sky_I: Isky + kx (x - W/2) + ky (y - H/2))
 */
#include <math.h>
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#include <stdlib.h>
#include <string.h>

#define OR_SERSIC 1
#define OR_EXPDISK 2
#define OR_FERRER 3
#define OR_KING 4
#define OR_GAUSSIAN 5
#define OR_MOFFAT 6
#define OR_SKY 7
#define OR_TSKY 8

#define OR_MAX_COMP 8
#define OR_MAX_SLOTS 24
#define OR_RFLOOR 1e-4

/* per-galaxy fit status */
#define OR_RUNNING 0
#define OR_CONVERGED 1
#define OR_MAX_ITER 2
#define OR_STALLED 3
#define OR_SINGULAR 4
#define OR_NONFINITE 5
#define OR_BAD_INPUT 6
#define OR_NO_DOF 7

typedef struct {
  int n_comp;
  int kind[OR_MAX_COMP];
  int convolve[OR_MAX_COMP];
  int slot[OR_MAX_COMP][8];
  int n_slots;
  int is_free[OR_MAX_SLOTS];
  int is_log[OR_MAX_SLOTS];
  double lo[OR_MAX_SLOTS];
  double hi[OR_MAX_SLOTS];
  int amp_is_mag[OR_MAX_COMP];  /* amplitude slot holds a magnitude ... */
  double mag_zero[OR_MAX_COMP]; /* ... with this zero point */
  int has_box[OR_MAX_COMP];     /* boxiness B in slot[or_n_params(kind)] */
} or_desc;

typedef struct {
  double tol;        /* relative chi^2 decrease that ends the fit */
  double xtol;       /* relative step size that ends the fit */
  double gtol;       /* Gauss-Newton decrement (relative to chi^2) that ends the fit */
  int max_iter;      /* model+Jacobian evaluations allowed */
  double lambda0, lambda_up, lambda_down, lambda_min, lambda_max;
  int polish;        /* 1: one final Gauss-Newton step after CONVERGED (step 7 of or_fit_one) */
  int canonical;     /* 1: rewrite q > 1 and wrap position angles at exit; 0: the best point as held */
  double *lambda_inout; /* NULL, or [G]: each galaxy's starting damping (when > 0, finite) in, its final one out */
} or_opts;

int or_n_params(int kind) {
  switch (kind) {
    case OR_SERSIC: return 7;
    case OR_EXPDISK: return 6;
    case OR_FERRER: return 8;
    case OR_KING: return 8;
    case OR_GAUSSIAN: return 6;
    case OR_MOFFAT: return 7;
    case OR_SKY: return 1;
    case OR_TSKY: return 3;
    default: return -1;
  }
}

/* ------------------------------------------------------------------------ */
/* Regularised lower incomplete gamma P(a, x) = gamma(a, x) / Gamma(a).       */
/* Power series for x < a + 1, Legendre continued fraction for Gamma(a, x)    */
/* (evaluated with the modified Lentz method) otherwise.                      */
/* ------------------------------------------------------------------------ */
double or_gammp(double a, double x) {
  if (!(a > 0.0) || x < 0.0) return NAN;
  if (x == 0.0) return 0.0;
  if (x < a + 1.0) {
    /* P = x^a e^-x / Gamma(a+1) * sum_k x^k / ((a+1)...(a+k)) */
    double term = 1.0, sum = 1.0, ap = a;
    for (int k = 1; k < 100000; ++k) {
      ap += 1.0;
      term *= x / ap;
      sum += term;
      if (fabs(term) < fabs(sum) * 1e-17) break;
    }
    return sum * exp(-x + a * log(x) - lgamma(a + 1.0));
  }
  /* Q = x^a e^-x / Gamma(a) * 1/(x+1-a- 1(1-a)/(x+3-a- 2(2-a)/(x+5-a- ...))) */
  const double tiny = 1e-300;
  double b = x + 1.0 - a;
  double c = 1.0 / tiny;
  double d = 1.0 / b;
  double h = d;
  for (int i = 1; i < 100000; ++i) {
    double an = -i * (i - a);
    b += 2.0;
    d = an * d + b;
    if (fabs(d) < tiny) d = tiny;
    c = b + an / c;
    if (fabs(c) < tiny) c = tiny;
    d = 1.0 / d;
    double del = d * c;
    h *= del;
    if (fabs(del - 1.0) < 1e-17) break;
  }
  double q = exp(-x + a * log(x) - lgamma(a)) * h;
  return 1.0 - q;
}

/* nu_n of Eq. (sersic-intensity): the half-light condition P(2n, nu) = 1/2,
 * solved by plain bisection (P is increasing in x; the median of a
 * Gamma(2n) variable lies below its mean 2n). */
double or_sersic_b(double n) {
  double a = 2.0 * n;
  double lo = 0.0, hi = a;
  while (or_gammp(a, hi) < 0.5) hi *= 2.0; /* never taken for a > 0, kept as a guard */
  for (int it = 0; it < 400; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (or_gammp(a, mid) < 0.5) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* Radius of Eqs. (r)-(rmin), floored at OR_RFLOOR: with r_maj = |X|, r_min = |Y|
 * (the absolute values read around the rotated coordinates),
 * r = (r_maj^(B+2) + (r_min/q)^(B+2))^(1/(B+2)); B = 0 is the ellipse. */
static double or_radius(double x, double y, double x0, double y0, double q, double pa, double B) {
  double dx = x - x0, dy = y - y0;
  double X = cos(pa) * dx + sin(pa) * dy;
  double Y = -sin(pa) * dx + cos(pa) * dy;
  double r;
  if (B == 0.0) {
    r = sqrt(X * X + (Y / q) * (Y / q));
  } else {
    double p = B + 2.0;
    r = pow(pow(fabs(X), p) + pow(fabs(Y / q), p), 1.0 / p);
  }
  return r < OR_RFLOOR ? OR_RFLOOR : r;
}

/* Eq. (rbox): the flux correction of a boxy ellipse, pi / (area of the unit
 * superellipse |x|^(B+2) + |y|^(B+2) = 1). */
double or_rbox(double B) {
  double a = 1.0 / (2.0 + B);
  double lnbeta = 2.0 * lgamma(a) - lgamma(2.0 * a);
  return M_PI * (2.0 + B) / (2.0 * exp(lnbeta));
}

/* Intensity of one component at the point (x, y); par in the order above.
 * nu is nu_n of the Sersic index (or_sersic_b(par[6])) for a Sersic
 * component and ignored otherwise. */
double or_component_value(int kind, const double *par, double nu, double B, double x, double y) {
  if (kind == OR_SKY) return par[0]; /* Eq. (sky_I) */
  if (kind == OR_TSKY) return par[0] + par[1] * x + par[2] * y; /* Eq. (new_sky_I); x, y from the stamp centre */
  double r = or_radius(x, y, par[0], par[1], par[2], par[3], B);
  switch (kind) {
    case OR_SERSIC: { /* Eq. (sersic-intensity) */
      double Ie = par[4], Re = par[5], n = par[6];
      return Ie * exp(-nu * (pow(r / Re, 1.0 / n) - 1.0));
    }
    case OR_EXPDISK: { /* Eq. (expdisk_I) */
      double I0 = par[4], rs = par[5];
      return I0 * exp(-r / rs);
    }
    case OR_FERRER: { /* Eq. (ferrer_I), zero beyond r_out */
      double I0 = par[4], rout = par[5], a = par[6], b = par[7];
      if (r >= rout) return 0.0;
      return I0 * pow(1.0 - pow(r / rout, 2.0 - b), a);
    }
    case OR_KING: { /* Eq. (BE_S), bracket read so that I(0) = I0 */
      double I0 = par[4], rc = par[5], rt = par[6], al = par[7];
      if (r >= rt) return 0.0;
      double At = pow(1.0 + (rt / rc) * (rt / rc), -1.0 / al);
      double Ar = pow(1.0 + (r / rc) * (r / rc), -1.0 / al);
      return I0 * pow(1.0 - At, -al) * pow(Ar - At, al);
    }
    case OR_GAUSSIAN: { /* Eq. (gaussion_I), FWHM = 2 sqrt(2 ln 2) sigma */
      double I0 = par[4], fwhm = par[5];
      double sig = fwhm / (2.0 * sqrt(2.0 * log(2.0)));
      return I0 * exp(-r * r / (2.0 * sig * sig));
    }
    case OR_MOFFAT: { /* Eqs. (moffat_I), (moffat_rd) */
      double I0 = par[4], fwhm = par[5], n = par[6];
      double rd = fwhm / (2.0 * sqrt(pow(2.0, 1.0 / n) - 1.0));
      return I0 * pow(1.0 + (r / rd) * (r / rd), -n);
    }
    default: return NAN;
  }
}

/* Amplitude of a component whose amplitude slot par[4] holds a magnitude m with
 * zero point m0: the amplitude giving the total flux F = 10^(-0.4 (m - m0))
 * (Sec. 4.1 Eq. sersicLtot, Sec. 4.2 Eqs. expdiskI0, ferrerI0, moffatI0, with
 * r_box = 1 for B = 0; the Gaussian's flux 2 pi q sigma^2 I0).  NAN for the
 * kinds without such a relation. */
double or_mag_amplitude(int kind, const double *par, double m0) {
  const double lnF = -0.4 * log(10.0) * (par[4] - m0);
  const double q = par[2];
  switch (kind) {
    case OR_SERSIC: {
      const double re = par[5], n = par[6], nu = or_sersic_b(n);
      return exp(2.0 * n * log(nu) + lnF - log(2.0 * M_PI * q * re * re * n) - lgamma(2.0 * n) - nu);
    }
    case OR_EXPDISK: return exp(lnF) / (2.0 * M_PI * q * par[5] * par[5]);
    case OR_FERRER: {
      const double rout = par[5], a = par[6], b = par[7], c = 1.0 + 2.0 / (2.0 - b);
      const double lnbeta = lgamma(a) + lgamma(c) - lgamma(a + c);
      return exp(lnF - log(M_PI * q * rout * rout * a) - lnbeta);
    }
    case OR_GAUSSIAN: {
      const double sig = par[5] / (2.0 * sqrt(2.0 * log(2.0)));
      return exp(lnF) / (2.0 * M_PI * q * sig * sig);
    }
    case OR_MOFFAT: {
      const double fw = par[5], n = par[6], rd = fw / (2.0 * sqrt(pow(2.0, 1.0 / n) - 1.0));
      return (n - 1.0) * exp(lnF) / (M_PI * q * rd * rd);
    }
    default: return NAN;
  }
}

/* Parameter count of component c: the profile's, plus B when it is boxy. */
static int or_np(const or_desc *d, int c) { return or_n_params(d->kind[c]) + (d->has_box[c] ? 1 : 0); }

/* Parameters of component c from the slot vector p, in profile units (a
 * magnitude replaced by its amplitude). */
static double or_gather(const or_desc *d, int c, const double *p, double *par) {
  int np = or_np(d, c);
  for (int k = 0; k < np; ++k) par[k] = p[d->slot[c][k]];
  double B = d->has_box[c] ? par[or_n_params(d->kind[c])] : 0.0;
  if (d->amp_is_mag[c]) par[4] = or_mag_amplitude(d->kind[c], par, d->mag_zero[c]) * or_rbox(B);
  return B;
}

/* Image of one component on the H x W stamp (no PSF). */
void or_component_image_box(int kind, const double *par, double B, int H, int W, double *out) {
  double nu = (kind == OR_SERSIC) ? or_sersic_b(par[6]) : 0.0;
  /* the tilted sky is measured from the stamp centre (W/2, H/2) */
  double xc = kind == OR_TSKY ? 0.5 * W : 0.0, yc = kind == OR_TSKY ? 0.5 * H : 0.0;
  for (int i = 0; i < H; ++i)
    for (int j = 0; j < W; ++j)
      out[(size_t)i * W + j] = or_component_value(kind, par, nu, B, j + 0.5 - xc, H - 0.5 - i - yc);
}

void or_component_image(int kind, const double *par, int H, int W, double *out) {
  or_component_image_box(kind, par, 0.0, H, W, out);
}

/* Direct zero-padded cross-correlation with a K x K PSF, same-size output. */
void or_correlate(const double *img, int H, int W, const double *psf, int K, double *out) {
  int c = (K - 1) / 2;
  for (int i = 0; i < H; ++i)
    for (int j = 0; j < W; ++j) {
      double s = 0.0;
      for (int a = 0; a < K; ++a) {
        int ii = i + a - c;
        if (ii < 0 || ii >= H) continue;
        for (int b = 0; b < K; ++b) {
          int jj = j + b - c;
          if (jj < 0 || jj >= W) continue;
          s += psf[a * K + b] * img[(size_t)ii * W + jj];
        }
      }
      out[(size_t)i * W + j] = s;
    }
}

/* Full model of one galaxy: correlated sum of the convolved components plus
 * the unconvolved ones.  work must hold 2*H*W doubles. */
void or_model_one(const or_desc *d, const double *p, int H, int W, const double *psf, int K,
                  double *model, double *work) {
  size_t N = (size_t)H * W;
  double *conv = work, *comp = work + N;
  double par[9];
  int any_conv = 0;
  for (size_t t = 0; t < N; ++t) { conv[t] = 0.0; model[t] = 0.0; }
  for (int c = 0; c < d->n_comp; ++c) {
    double B = or_gather(d, c, p, par);
    or_component_image_box(d->kind[c], par, B, H, W, comp);
    double *dst = d->convolve[c] ? conv : model;
    if (d->convolve[c]) any_conv = 1;
    for (size_t t = 0; t < N; ++t) dst[t] += comp[t];
  }
  if (any_conv) {
    /* model currently holds the unconvolved part; add the correlated part */
    or_correlate(conv, H, W, psf, K, comp);
    for (size_t t = 0; t < N; ++t) model[t] += comp[t];
  }
}

/* Eq. (chinu): chi^2 = sum Omega (D - M)^2 / sigma^2, Omega = (mask == 0). */
double or_chi2_one(const double *model, const double *image, const double *sigma,
                   const unsigned char *mask, size_t N) {
  double s = 0.0;
  for (size_t t = 0; t < N; ++t) {
    if (mask && mask[t]) continue;
    double r = image[t] - model[t];
    s += r * r / (sigma[t] * sigma[t]);
  }
  return s;
}

/* Internal (fitted) coordinate of a slot: ln p for log slots, p otherwise. */
static double or_to_u(const or_desc *d, int s, double p) { return d->is_log[s] ? log(p) : p; }
static double or_from_u(const or_desc *d, int s, double u) { return d->is_log[s] ? exp(u) : u; }

/* Central-difference Jacobian dM/du_s for every free slot s (in slot order),
 * u the internal coordinate when `internal` is set, else the physical one.
 * J is [n_free][H*W].  work must hold 4*H*W doubles. */
void or_jacobian_one(const or_desc *d, const double *p, int H, int W, const double *psf, int K,
                     int internal, double *J, double *work) {
  size_t N = (size_t)H * W;
  double pp[OR_MAX_SLOTS];
  double *mp = work, *mm = work + N, *w2 = work + 2 * N;
  int f = 0;
  for (int s = 0; s < d->n_slots; ++s) {
    if (!d->is_free[s]) continue;
    int lg = internal && d->is_log[s];
    double u = lg ? log(p[s]) : p[s];
    double h = lg ? 1e-6 : 1e-6 * fmax(fabs(u), 1.0);
    memcpy(pp, p, sizeof(double) * d->n_slots);
    pp[s] = lg ? exp(u + h) : u + h;
    or_model_one(d, pp, H, W, psf, K, mp, w2);
    pp[s] = lg ? exp(u - h) : u - h;
    or_model_one(d, pp, H, W, psf, K, mm, w2);
    for (size_t t = 0; t < N; ++t) J[(size_t)f * N + t] = (mp[t] - mm[t]) / (2.0 * h);
    ++f;
  }
}

/* Cholesky factorisation in place (lower triangle), n x n row-major.
 * Returns 0 on success, -1 if the matrix is not positive definite. */
static int or_cholesky(double *A, int n) {
  for (int j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (int k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
    if (!(s > 0.0)) return -1;
    double l = sqrt(s);
    A[j * n + j] = l;
    for (int i = j + 1; i < n; ++i) {
      double t = A[i * n + j];
      for (int k = 0; k < j; ++k) t -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = t / l;
    }
  }
  return 0;
}

/* Solve L L^T x = b with the factor from or_cholesky. */
static void or_chol_solve(const double *L, int n, const double *b, double *x) {
  double y[OR_MAX_SLOTS];
  for (int i = 0; i < n; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[i * n + k] * y[k];
    y[i] = s / L[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
    x[i] = s / L[i * n + i];
  }
}

/* Gauss-Newton normal equations at p: chi^2, A = J^T W J, g = J^T W r with
 * r = D - M and J taken in internal coordinates.  Returns chi^2. */
static double or_normal_eq(const or_desc *d, const double *p, int H, int W, const double *psf, int K,
                           const double *image, const double *sigma, const unsigned char *mask,
                           int nf, double *A, double *g, double *J, double *model, double *work) {
  size_t N = (size_t)H * W;
  or_model_one(d, p, H, W, psf, K, model, work);
  double chi2 = or_chi2_one(model, image, sigma, mask, N);
  or_jacobian_one(d, p, H, W, psf, K, 1, J, work);
  for (int a = 0; a < nf; ++a) {
    g[a] = 0.0;
    for (int b = 0; b < nf; ++b) A[a * nf + b] = 0.0;
  }
  for (size_t t = 0; t < N; ++t) {
    if (mask && mask[t]) continue;
    double w = 1.0 / (sigma[t] * sigma[t]);
    double r = image[t] - model[t];
    for (int a = 0; a < nf; ++a) {
      double ja = J[(size_t)a * N + t];
      g[a] += w * ja * r;
      for (int b = 0; b < nf; ++b) A[a * nf + b] += w * ja * J[(size_t)b * N + t];
    }
  }
  return chi2;
}

static void or_clamp(const or_desc *d, double *p) {
  for (int s = 0; s < d->n_slots; ++s) {
    if (p[s] < d->lo[s]) p[s] = d->lo[s];
    if (p[s] > d->hi[s]) p[s] = d->hi[s];
  }
}

/* Indices of a component's scale-length parameters (r_e, r_s, r_out, r_c and
 * r_t, FWHM); returns how many. */
static int or_scale_params(int kind, int *idx) {
  switch (kind) {
    case OR_SERSIC: case OR_EXPDISK: case OR_FERRER: case OR_GAUSSIAN: case OR_MOFFAT:
      idx[0] = 5;
      return 1;
    case OR_KING:
      idx[0] = 5;
      idx[1] = 6;
      return 2;
    default:
      return 0;
  }
}

/* Role of parameter k of a component: 1 axis ratio, 2 position angle, 3 scale length, 0 other. */
static int or_flat(int kind) { return kind == OR_SKY || kind == OR_TSKY; }

static int or_role(int kind, int k) {
  if (or_flat(kind)) return 0;
  if (k == 2) return 1;
  if (k == 3) return 2;
  int idx[2], n = or_scale_params(kind, idx);
  for (int i = 0; i < n; ++i)
    if (idx[i] == k) return 3;
  return 0;
}

/* An axis ratio q > 1 describes the same ellipse as 1/q with the position angle
 * turned by pi/2 and every scale length multiplied by q: with X' = Y and
 * Y' = -X, sqrt(X'^2 + (Y'/(1/q))^2) = q sqrt(X^2 + (Y/q)^2), so a profile of
 * r / r_s is unchanged when r_s becomes q r_s.  Each q slot above 1 is rewritten
 * that way, provided every slot the affected components use as axis ratio,
 * position angle or scale length is used in that same role only by components
 * sharing the q slot.  Returns the number of q slots rewritten. */
static int or_canonical_q(const or_desc *d, double *p) {
  int changed = 0;
  for (int c = 0; c < d->n_comp; ++c) {
    if (or_flat(d->kind[c])) continue;
    int qs = d->slot[c][2];
    if (!(p[qs] > 1.0)) continue;
    int ok = 1;
    /* every use of a slot that some component of this q group uses as q, pa or scale */
    for (int c1 = 0; c1 < d->n_comp && ok; ++c1) {
      if (or_flat(d->kind[c1]) || d->slot[c1][2] != qs) continue;
      int np1 = or_n_params(d->kind[c1]);
      for (int k1 = 0; k1 < np1 && ok; ++k1) {
        int r1 = or_role(d->kind[c1], k1);
        if (r1 == 0) continue;
        int s1 = d->slot[c1][k1];
        for (int c2 = 0; c2 < d->n_comp && ok; ++c2) {
          int np2 = or_n_params(d->kind[c2]);
          for (int k2 = 0; k2 < np2; ++k2) {
            if (d->slot[c2][k2] != s1) continue;
            if (or_flat(d->kind[c2]) || d->slot[c2][2] != qs || or_role(d->kind[c2], k2) != r1) ok = 0;
          }
        }
      }
    }
    if (!ok) continue;
    double q = p[qs];
    int done[OR_MAX_SLOTS] = {0};
    for (int c1 = 0; c1 < d->n_comp; ++c1) {
      if (or_flat(d->kind[c1]) || d->slot[c1][2] != qs) continue;
      int pas = d->slot[c1][3];
      if (!done[pas]) { p[pas] += 0.5 * M_PI; done[pas] = 1; }
      int idx[2], n = or_scale_params(d->kind[c1], idx);
      for (int i = 0; i < n; ++i) {
        int ss = d->slot[c1][idx[i]];
        if (!done[ss]) { p[ss] *= q; done[ss] = 1; }
      }
    }
    p[qs] = 1.0 / q;
    ++changed;
  }
  return changed;
}

/* Slots that some radial component uses as its position angle. */
static void or_pa_slots(const or_desc *d, int *is_pa) {
  for (int s = 0; s < OR_MAX_SLOTS; ++s) is_pa[s] = 0;
  for (int c = 0; c < d->n_comp; ++c)
    if (!or_flat(d->kind[c])) is_pa[d->slot[c][3]] = 1;
}

/* held[a] = 1 for a free parameter that sits on a bound while chi^2 falls
 * beyond it (g = J^T W r is the descent direction): at its lower bound with
 * g_a < 0, or at its upper bound with g_a > 0.  A held parameter does not move
 * in the next step. */
static void or_held(const or_desc *d, const int *fidx, int nf, const double *p, const double *g, int *held) {
  for (int a = 0; a < nf; ++a) {
    int s = fidx[a];
    held[a] = (p[s] <= d->lo[s] && g[a] < 0.0) || (p[s] >= d->hi[s] && g[a] > 0.0);
  }
}

/* The linear system of a step over the parameters not held:
 * M = A + lambda max(A_aa, 1e-12 max diag A) on the diagonal (lambda = 0: the
 * 1e-12 max diag A term alone), with the rows and columns of held parameters
 * replaced by those of the identity; rhs r = g with zeros at held parameters. */
static void or_step_system(const double *A, const double *g, int nf, double lambda, const int *held, double *M,
                           double *r) {
  double dmax = 0.0;
  for (int a = 0; a < nf; ++a) dmax = fmax(dmax, A[a * nf + a]);
  double dfloor = 1e-12 * dmax;
  for (int a = 0; a < nf; ++a) {
    for (int b = 0; b < nf; ++b)
      M[a * nf + b] = (held[a] || held[b]) ? (a == b ? 1.0 : 0.0) : A[a * nf + b];
    if (!held[a]) M[a * nf + a] += lambda > 0.0 ? lambda * fmax(A[a * nf + a], dfloor) : dfloor;
    r[a] = held[a] ? 0.0 : g[a];
  }
}

/* Gauss-Newton decrement g^T A^-1 g over the parameters not held: the chi^2
 * reduction a full Gauss-Newton step predicts from the current point (A
 * regularised by 1e-12 max(diag A) on the diagonal).  Negative when A cannot
 * be factorised. */
static double or_gn_decrement(const double *A, const double *g, int nf, const int *held) {
  double M[OR_MAX_SLOTS * OR_MAX_SLOTS], r[OR_MAX_SLOTS], x[OR_MAX_SLOTS];
  or_step_system(A, g, nf, 0.0, held, M, r);
  if (or_cholesky(M, nf) != 0) return -1.0;
  or_chol_solve(M, nf, r, x);
  double s = 0.0;
  for (int a = 0; a < nf; ++a) s += r[a] * x[a];
  return s;
}

/*
 * Levenberg-Marquardt fit of one galaxy, in internal coordinates u.
 *   1. Evaluate chi^2, A, g at the (clamped) start; this is iteration 1.
 *   2. Damped step: solve (A + lambda diag(A)) delta = g by Cholesky, the
 *      diagonal floored at 1e-12 max(diag A); a failed factorisation
 *      multiplies lambda by lambda_up and retries (SINGULAR past lambda_max).
 *      A free parameter on a bound with the descent direction g pointing out
 *      of the box is held (its delta is 0): steps 2, 5 and 7 solve over the
 *      other parameters (or_held, or_step_system).
 *   3. Trial p' = clamp(from_u(u + delta)); evaluate it (one iteration).
 *   4. The step is "small" when every internal step satisfies
 *      |u'_s - u_s| <= xtol (|u_s| + xtol).  Its predicted decrease is
 *      pred = 2 g^T delta - delta^T A delta (the quadratic model of chi^2),
 *      taken as infinite when the clamp moved p'; the step is "resolved" when
 *      pred >= 1e-7 chi^2.
 *      chi^2' < chi^2, or an unresolved step with chi^2' <= chi^2 (1 + 1e-7):
 *      accept, lambda = max(lambda*lambda_down, lambda_min); CONVERGED if the
 *      step's decrease -- (chi^2 - chi^2')/chi^2 when resolved, pred/chi^2 when
 *      not -- is below tol, or the step was small.
 *      Otherwise reject: CONVERGED at the kept point if the step was small,
 *      else lambda *= lambda_up and STALLED past lambda_max.
 *   5. At the start and after every accepted step: CONVERGED when the
 *      Gauss-Newton decrement g^T A^-1 g <= gtol chi^2 (no step can gain more).
 *   6. MAX_ITER once max_iter evaluations have been spent.
 *   7. With polish, a fit that ended CONVERGED with evaluations to spare takes
 *      one undamped Gauss-Newton step delta = A^-1 g from its best point (diag
 *      A floored at 1e-12 max diag A), p' = clamp(from_u(u + delta)), and
 *      evaluates it (one iteration); p' replaces the best point unless its
 *      chi^2 is non-finite or above the best by more than 1e-6 relative.
 *   8. The damping starts at *lam_io instead of lambda0 when given (> 0,
 *      finite), and its final value is written back: with canonical = 0 the
 *      best point is returned as held, so that a fit stopped at max_iter can
 *      be resumed (the first evaluation repeats the best point's A, g, chi^2).
 * At exit (canonical = 1) an axis ratio above 1 is rewritten as its reciprocal (or_canonical_q).
 * The covariance of Sec. 5.2 is taken from A at the best point; for a log
 * slot sigma_p = p sigma_u.  Position angles are wrapped to [0, pi) at exit.
 */
static void or_fit_one(const or_desc *d, const or_opts *o, double *p, int H, int W,
                       const double *psf, int K, const double *image, const double *sigma,
                       const unsigned char *mask, double *chi2_out, int *dof_out, int *iters_out,
                       int *status_out, double *sigma_p, double *lam_io) {
  size_t N = (size_t)H * W;
  int nf = 0, fidx[OR_MAX_SLOTS];
  for (int s = 0; s < d->n_slots; ++s)
    if (d->is_free[s]) fidx[nf++] = s;
  long nused = 0;
  int bad = 0;
  for (size_t t = 0; t < N; ++t) {
    if (mask && mask[t]) continue;
    ++nused;
    if (!(sigma[t] > 0.0) || !isfinite(sigma[t]) || !isfinite(image[t])) bad = 1;
  }
  *dof_out = (int)(nused - nf);
  *iters_out = 0;
  *chi2_out = NAN;
  if (sigma_p)
    for (int s = 0; s < d->n_slots; ++s) sigma_p[s] = 0.0;
  if (bad) { *status_out = OR_BAD_INPUT; return; }
  if (nused - nf <= 0) { *status_out = OR_NO_DOF; return; }

  double *J = malloc(sizeof(double) * nf * N);
  double *model = malloc(sizeof(double) * N);
  double *work = malloc(sizeof(double) * 4 * N);
  double A[OR_MAX_SLOTS * OR_MAX_SLOTS], g[OR_MAX_SLOTS];
  double At[OR_MAX_SLOTS * OR_MAX_SLOTS], gt[OR_MAX_SLOTS];
  double M[OR_MAX_SLOTS * OR_MAX_SLOTS], delta[OR_MAX_SLOTS];
  double pt[OR_MAX_SLOTS];

  or_clamp(d, p);
  double chi2 = or_normal_eq(d, p, H, W, psf, K, image, sigma, mask, nf, A, g, J, model, work);
  int it = 1;
  int status = OR_RUNNING;
  double lambda = (lam_io && *lam_io > 0.0 && isfinite(*lam_io)) ? *lam_io : o->lambda0;
  if (!isfinite(chi2)) status = OR_NONFINITE;
  else if (chi2 == 0.0) status = OR_CONVERGED;
  int held[OR_MAX_SLOTS];
  double rhs[OR_MAX_SLOTS];
  if (status == OR_RUNNING) {
    or_held(d, fidx, nf, p, g, held);
    double gn = or_gn_decrement(A, g, nf, held);
    if (gn >= 0.0 && gn <= o->gtol * chi2) status = OR_CONVERGED;
  }

  while (status == OR_RUNNING) {
    if (it >= o->max_iter) { status = OR_MAX_ITER; break; }
    or_held(d, fidx, nf, p, g, held);
    for (;;) {
      or_step_system(A, g, nf, lambda, held, M, rhs);
      if (or_cholesky(M, nf) == 0) break;
      lambda *= o->lambda_up;
      if (lambda > o->lambda_max) { status = OR_SINGULAR; break; }
    }
    if (status != OR_RUNNING) break;
    or_chol_solve(M, nf, rhs, delta);
    memcpy(pt, p, sizeof(double) * d->n_slots);
    for (int a = 0; a < nf; ++a) {
      int s = fidx[a];
      pt[s] = or_from_u(d, s, or_to_u(d, s, p[s]) + delta[a]);
    }
    double pred = 0.0;
    for (int a = 0; a < nf; ++a) {
      double ad = 0.0;
      for (int b = 0; b < nf; ++b) ad += A[a * nf + b] * delta[b];
      pred += delta[a] * (2.0 * g[a] - ad);
    }
    for (int s = 0; s < d->n_slots; ++s)
      if (pt[s] < d->lo[s] || pt[s] > d->hi[s]) pred = INFINITY;
    or_clamp(d, pt);
    double chi2t = or_normal_eq(d, pt, H, W, psf, K, image, sigma, mask, nf, At, gt, J, model, work);
    ++it;
    int small = 1;
    for (int a = 0; a < nf; ++a) {
      int s = fidx[a];
      double u0 = or_to_u(d, s, p[s]), u1 = or_to_u(d, s, pt[s]);
      if (fabs(u1 - u0) > o->xtol * (fabs(u0) + o->xtol)) small = 0;
    }
    int resolved = pred >= 1e-7 * chi2;
    if (isfinite(chi2t) && (chi2t < chi2 || (!resolved && chi2t <= chi2 * (1.0 + 1e-7)))) {
      double act = resolved ? (chi2 - chi2t) / chi2 : fmax(pred, 0.0) / chi2;
      memcpy(p, pt, sizeof(double) * d->n_slots);
      memcpy(A, At, sizeof(double) * nf * nf);
      memcpy(g, gt, sizeof(double) * nf);
      chi2 = chi2t;
      lambda = fmax(lambda * o->lambda_down, o->lambda_min);
      if (act < o->tol || small || chi2 == 0.0) status = OR_CONVERGED;
      if (status == OR_RUNNING) {
        or_held(d, fidx, nf, p, g, held);
        double gn = or_gn_decrement(A, g, nf, held);
        if (gn >= 0.0 && gn <= o->gtol * chi2) status = OR_CONVERGED;
      }
    } else if (small) {
      status = OR_CONVERGED; /* the damped step is below resolution: nothing left to gain */
    } else {
      lambda *= o->lambda_up;
      if (lambda > o->lambda_max) status = OR_STALLED;
    }
  }

  if (status == OR_CONVERGED && o->polish && it < o->max_iter && chi2 > 0.0) {
    or_held(d, fidx, nf, p, g, held);
    or_step_system(A, g, nf, 0.0, held, M, rhs);
    if (or_cholesky(M, nf) == 0) {
      or_chol_solve(M, nf, rhs, delta);
      memcpy(pt, p, sizeof(double) * d->n_slots);
      for (int a = 0; a < nf; ++a) {
        int s = fidx[a];
        pt[s] = or_from_u(d, s, or_to_u(d, s, p[s]) + delta[a]);
      }
      or_clamp(d, pt);
      double chi2t = or_normal_eq(d, pt, H, W, psf, K, image, sigma, mask, nf, At, gt, J, model, work);
      ++it;
      if (isfinite(chi2t) && chi2t <= chi2 * (1.0 + 1e-6)) {
        memcpy(p, pt, sizeof(double) * d->n_slots);
        memcpy(A, At, sizeof(double) * nf * nf);
        memcpy(g, gt, sizeof(double) * nf);
        chi2 = chi2t;
      }
    }
  }

  *chi2_out = chi2;
  *iters_out = it;
  *status_out = status;
  /* canonical axis ratios (q <= 1); the covariance is then taken at the rewritten
   * point from a fresh finite-difference Jacobian */
  if (lam_io) *lam_io = lambda;
  if (status != OR_NONFINITE && o->canonical && or_canonical_q(d, p) > 0)
    or_normal_eq(d, p, H, W, psf, K, image, sigma, mask, nf, A, g, J, model, work);
  if (sigma_p && status != OR_NONFINITE) {
    /* covariance: diag of A^-1 column by column through the Cholesky factor */
    memcpy(M, A, sizeof(double) * nf * nf);
    if (or_cholesky(M, nf) == 0) {
      for (int a = 0; a < nf; ++a) {
        double e[OR_MAX_SLOTS], x[OR_MAX_SLOTS];
        for (int b = 0; b < nf; ++b) e[b] = (a == b) ? 1.0 : 0.0;
        or_chol_solve(M, nf, e, x);
        int s = fidx[a];
        double su = sqrt(x[a]);
        sigma_p[s] = d->is_log[s] ? p[s] * su : su;
      }
    } else {
      for (int a = 0; a < nf; ++a) sigma_p[fidx[a]] = NAN;
    }
  }
  int is_pa[OR_MAX_SLOTS];
  or_pa_slots(d, is_pa);
  for (int s = 0; s < d->n_slots; ++s)
    if (is_pa[s] && o->canonical) p[s] -= M_PI * floor(p[s] / M_PI);
  free(J);
  free(model);
  free(work);
}

/* ------------------------------------------------------------------------ */
/* Batch entry points (equal-size stamps; galaxies are independent).          */
/* ------------------------------------------------------------------------ */

int or_model_batch(const or_desc *d, int G, int H, int W, int K, const double *params,
                   const double *psf, double *model) {
  size_t N = (size_t)H * W;
#pragma omp parallel for schedule(dynamic, 1)
  for (int gi = 0; gi < G; ++gi) {
    double *work = malloc(sizeof(double) * 2 * N);
    or_model_one(d, params + (size_t)gi * d->n_slots, H, W, psf + (size_t)gi * K * K, K,
                 model + (size_t)gi * N, work);
    free(work);
  }
  return 0;
}

int or_component_images_batch(const or_desc *d, int G, int H, int W, int K, const double *params,
                              const double *psf, double *comp) {
  /* Each component's own contribution to the model: correlated with the PSF
   * when the component is convolved.  comp is [G][n_comp][H*W]. */
  size_t N = (size_t)H * W;
#pragma omp parallel for schedule(dynamic, 1)
  for (int gi = 0; gi < G; ++gi) {
    double *tmp = malloc(sizeof(double) * N);
    double par[9];
    const double *p = params + (size_t)gi * d->n_slots;
    for (int c = 0; c < d->n_comp; ++c) {
      double *dst = comp + ((size_t)gi * d->n_comp + c) * N;
      double B = or_gather(d, c, p, par);
      if (d->convolve[c]) {
        or_component_image_box(d->kind[c], par, B, H, W, tmp);
        or_correlate(tmp, H, W, psf + (size_t)gi * K * K, K, dst);
      } else {
        or_component_image_box(d->kind[c], par, B, H, W, dst);
      }
    }
    free(tmp);
  }
  return 0;
}

int or_chi2_batch(const or_desc *d, int G, int H, int W, int K, const double *params,
                  const double *psf, const double *image, const double *sigma,
                  const unsigned char *mask, double *chi2) {
  size_t N = (size_t)H * W;
#pragma omp parallel for schedule(dynamic, 1)
  for (int gi = 0; gi < G; ++gi) {
    double *model = malloc(sizeof(double) * N);
    double *work = malloc(sizeof(double) * 2 * N);
    or_model_one(d, params + (size_t)gi * d->n_slots, H, W, psf + (size_t)gi * K * K, K, model, work);
    chi2[gi] = or_chi2_one(model, image + (size_t)gi * N, sigma + (size_t)gi * N,
                           mask ? mask + (size_t)gi * N : NULL, N);
    free(model);
    free(work);
  }
  return 0;
}

int or_jacobian_batch(const or_desc *d, int G, int H, int W, int K, const double *params,
                      const double *psf, int internal, double *J) {
  size_t N = (size_t)H * W;
  int nf = 0;
  for (int s = 0; s < d->n_slots; ++s) nf += d->is_free[s] ? 1 : 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int gi = 0; gi < G; ++gi) {
    double *work = malloc(sizeof(double) * 4 * N);
    or_jacobian_one(d, params + (size_t)gi * d->n_slots, H, W, psf + (size_t)gi * K * K, K, internal,
                    J + (size_t)gi * nf * N, work);
    free(work);
  }
  return 0;
}

/* Canonical form of a parameter vector (see or_canonical_q), exposed for tests. */
int or_canonicalize(const or_desc *d, double *p) { return or_canonical_q(d, p); }

int or_fit_batch(const or_desc *d, const or_opts *o, int G, int H, int W, int K, double *params,
                 const double *psf, const double *image, const double *sigma,
                 const unsigned char *mask, double *chi2, int *dof, int *iters, int *status,
                 double *sigma_p) {
  size_t N = (size_t)H * W;
#pragma omp parallel for schedule(dynamic, 1)
  for (int gi = 0; gi < G; ++gi) {
    or_fit_one(d, o, params + (size_t)gi * d->n_slots, H, W, psf + (size_t)gi * K * K, K,
               image + (size_t)gi * N, sigma + (size_t)gi * N, mask ? mask + (size_t)gi * N : NULL,
               chi2 + gi, dof + gi, iters + gi, status + gi,
               sigma_p ? sigma_p + (size_t)gi * d->n_slots : NULL,
               o->lambda_inout ? o->lambda_inout + gi : NULL);
  }
  return 0;
}

int or_max_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
