// gm_profiles.cuh -- per-galaxy set-up (FP64) and per-pixel light profiles with
// their analytic parameter derivatives (FP32) for the fused kernels.
//
// Profiles follow Sec. 4.1-4.2 of arxiv 2404.07780: the elliptical radius of
// Eqs. (r)-(rmin) with B = 0, and Eqs. (sersic-intensity), (expdisk_I),
// (ferrer_I), (BE_S) (bracket read so that I(0) = I0), (gaussion_I),
// (moffat_I)+(moffat_rd) and (sky_I).  Derivatives are the chain rule through
// the radius:
//   dr/dx0 = (-X c + (Y/q^2) s)/r     dr/dy0 = (-X s - (Y/q^2) c)/r
//   dr/dq  = -Y^2/(q^3 r)             dr/dpa = X Y (1 - 1/q^2)/r
// with X = c dx + s dy, Y = -s dx + c dy, c = cos pa, s = sin pa, and r
// floored at 1e-4 px (geometric derivatives vanish under the floor).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <math_constants.h>
#include <stdint.h>

namespace gm {

constexpr int kMaxComp = 8;
constexpr int kMaxSlots = 24;  // parameter slots of a model
constexpr int kMaxFree = 16;   // free (fitted) parameters of a model
constexpr int kCC = 20;          // FP32 constants per component per galaxy (a multiple of 4)
constexpr float kRFloor = 1e-4f;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr double kPiD = 3.14159265358979323846;

enum Kind { SERSIC = 1, EXPDISK = 2, FERRER = 3, KING = 4, GAUSSIAN = 5, MOFFAT = 6, SKY = 7, TSKY = 8 };

// Flag on the kind a tile kernel passes to eval_component: the amplitude slot
// holds a magnitude (the chain-rule constants are in the component's cc).
constexpr int kMagFlag = 16;
// Flag for a boxy radius (exponent p = B + 2 in cc[16]).
constexpr int kBoxFlag = 32;

// Flat and tilted sky: no centre, axis ratio or position angle.
__host__ __device__ inline bool is_flat(int kind) { return kind == SKY || kind == TSKY; }

__host__ __device__ inline int n_params(int kind) {
  switch (kind) {
    case SERSIC: return 7;
    case EXPDISK: return 6;
    case FERRER: return 8;
    case KING: return 8;
    case GAUSSIAN: return 6;
    case MOFFAT: return 7;
    case SKY: return 1;
    case TSKY: return 3;
    default: return -1;
  }
}

// ---------------------------------------------------------------------------
// nu_n of the Sersic profile (Sec. 4.1): the root of P(2n, x) = 1/2, i.e. the
// radius r_e encloses half of the light.  P is the regularised lower
// incomplete gamma function, summed as
//   P(a, x) = pref * sum_k t_k,   pref = x^a e^-x / Gamma(a),
//   t_0 = 1/a,  t_k = t_{k-1} x / (a + k),
// which converges geometrically below x = a, where the root lies.  Newton's
// method on x starts from the asymptotic expansion of Ciotti & Bertin (1999)
// for n >= 0.36 and from the polynomial fit of MacArthur, Courteau & Holtzman
// (2003) below; dP/dx = pref / x.
//
// dnu/dn follows from differentiating P(2n, nu(n)) = 1/2:
//   dnu/dn = -2 (dP/da) / (dP/dx),
//   dP/da  = P ln x - pref * sum_k t_k psi(a + k + 1),
// with psi(a+k+1) = psi(a+1) + sum_{j=1..k} 1/(a+j) accumulated along the
// series and psi(a+1) from the recurrence psi(z) = psi(z+1) - 1/z up to
// z >= 10 and the asymptotic (Bernoulli) expansion there.
// ---------------------------------------------------------------------------
__device__ inline double digamma_pos(double z) {
  double acc = 0.0;
  while (z < 10.0) {
    acc -= 1.0 / z;
    z += 1.0;
  }
  const double iz = 1.0 / z, iz2 = iz * iz;
  // ln z - 1/(2z) - B2/(2 z^2) - B4/(4 z^4) - ... with B2 = 1/6, B4 = -1/30,
  // B6 = 1/42, B8 = -1/30, B10 = 5/66
  const double tail = iz2 * (1.0 / 12.0 - iz2 * (1.0 / 120.0 - iz2 * (1.0 / 252.0 - iz2 * (1.0 / 240.0 - iz2 / 132.0))));
  return acc + log(z) - 0.5 * iz - tail;
}

// sum_k t_k (and, when s1 != nullptr, sum_k t_k psi(a+k+1) given psi(a+1))
__device__ inline double gamma_series(double a, double x, double psi1, double* s1) {
  double t = 1.0 / a, s0 = t, psi = psi1, acc1 = t * psi;
  for (int k = 1; k < 4000; ++k) {
    const double ik = __drcp_rn(a + k);
    t *= x * ik;
    s0 += t;
    if (s1) {
      psi += ik;
      acc1 += t * psi;
    }
    if (t < s0 * 1e-17) break;
  }
  if (s1) *s1 = acc1;
  return s0;
}

__device__ inline void sersic_nu_dnu(double n, double* nu_out, double* dnu_out) {
  const double a = 2.0 * n;
  double x;
  if (n >= 0.36) {
    const double in = 1.0 / n;
    x = 2.0 * n - 1.0 / 3.0 +
        in * (4.0 / 405.0 + in * (46.0 / 25515.0 + in * (131.0 / 1148175.0 - in * (2194697.0 / 30690717750.0))));
  } else {
    x = 0.01945 + n * (-0.8902 + n * (10.95 + n * (-19.67 + n * 13.43)));
    if (!(x > 0.0)) x = 0.5 * a;
  }
  const double lga = lgamma(a);
  for (int it = 0; it < 60; ++it) {
    const double pref = exp(a * log(x) - x - lga);
    const double f = pref * gamma_series(a, x, 0.0, nullptr) - 0.5;
    double xn = x - f * x / pref;  // Newton: dP/dx = pref / x
    if (!(xn > 0.0)) xn = 0.5 * x;
    const double dx = fabs(xn - x);
    x = xn;
    if (dx <= 1e-14 * x) break;
  }
  const double lx = log(x);
  const double pref = exp(a * lx - x - lga);
  double s1 = 0.0;
  const double s0 = gamma_series(a, x, digamma_pos(a + 1.0), &s1);
  const double P = pref * s0;
  const double dPda = P * lx - pref * s1;
  *nu_out = x;
  *dnu_out = -2.0 * dPda * x / pref;
}

#ifdef GM_HOST_TU
// nu_n and d nu/dn at kNuNodes nodes n_i = kNuN0 + i kNuH (n from 0.2 to 10.2),
// solved by sersic_nu_dnu once per device (k_nu_table, then k_nu_ready sets
// the flag).  Inside the node range setup_component interpolates them: the
// cubic Hermite polynomial of the node values and slopes gives nu_n, its
// derivative d nu/dn; both agree with the direct solve to ~1e-10 and ~1e-7
// relative, far below the FP32 constants they feed.  Outside the range, and
// until the flag is set, the direct solve runs.  The solve is ~40 % of an LM
// step, which is latency-bound (one thread per galaxy).
constexpr int kNuNodes = 4096;
constexpr double kNuN0 = 0.2, kNuH = 10.0 / (kNuNodes - 1);
__device__ double g_nu_tab[2 * kNuNodes];
__device__ int g_nu_ready;

__global__ void k_nu_table() {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNuNodes; i += gridDim.x * blockDim.x) {
    double nu, dnu;
    sersic_nu_dnu(kNuN0 + i * kNuH, &nu, &dnu);
    g_nu_tab[2 * i] = nu;
    g_nu_tab[2 * i + 1] = dnu;
  }
}
__global__ void k_nu_ready() { g_nu_ready = 1; }

__device__ inline void sersic_nu_dnu_fast(double n, double* nu_out, double* dnu_out) {
  const double t = (n - kNuN0) * (1.0 / kNuH);
  if (g_nu_ready && t >= 0.0 && t < (double)(kNuNodes - 1)) {
    const int i = (int)t;
    const double s = t - i, s2 = s * s, s3 = s2 * s;
    const double y0 = g_nu_tab[2 * i], m0 = g_nu_tab[2 * i + 1] * kNuH;
    const double y1 = g_nu_tab[2 * i + 2], m1 = g_nu_tab[2 * i + 3] * kNuH;
    *nu_out = (2.0 * s3 - 3.0 * s2 + 1.0) * y0 + (s3 - 2.0 * s2 + s) * m0 + (3.0 * s2 - 2.0 * s3) * y1 +
              (s3 - s2) * m1;
    *dnu_out = ((6.0 * s2 - 6.0 * s) * y0 + (3.0 * s2 - 4.0 * s + 1.0) * m0 + (6.0 * s - 6.0 * s2) * y1 +
                (3.0 * s2 - 2.0 * s) * m1) * (1.0 / kNuH);
    return;
  }
  sersic_nu_dnu(n, nu_out, dnu_out);
}
#endif  // GM_HOST_TU


// ---------------------------------------------------------------------------
// Per-component constants (FP32), computed in FP64 from the parameters.
//   [0] xi (int bits) [1] yi (int bits) [2] xf [3] yf : dx = (j + xi) + xf,
//       dy = (yi - i) + yf, an exact split of x_j - x0 and y_i - y0 so that
//       the pixel offset keeps full FP32 precision far from the origin
//   [4] cos pa [5] sin pa [6] 1/q [7] q   [8..15] kind specific:
//   SERSIC   Ie, 1/Re, 1/n, nu, dnu/dn
//   EXPDISK  I0, 1/rs
//   FERRER   I0, 1/rout, a, 2 - b
//   KING     I0, 1/rc, alpha, A_t, dA_t/drc, dA_t/drt, dA_t/dalpha, rt
//            with A(r) = (1 + (r/rc)^2)^(-1/alpha), A_t = A(rt)
//   GAUSSIAN I0, 1/sigma^2, 1/fwhm
//   MOFFAT   I0, 1/rd, n, d ln rd / dn, 1/fwhm
//   SKY      Isky
//   TSKY     Isky, kx, ky; cc[0] = 0.5 - W/2, cc[1] = H/2 - 0.5 (pixel (i, j) lies at
//            x - W/2 = j + cc[0], y - H/2 = cc[1] - i)
// ---------------------------------------------------------------------------
// Magnitude mode (mag = 1, par[4] = m): the amplitude is the one giving the total
// flux F = 10^(-0.4 (m - m0)) (Eqs. sersicLtot, expdiskI0, ferrerI0, moffatI0,
// r_box = 1; the Gaussian's flux 2 pi q sigma^2 I0), and the free cc entries
// hold d ln(amplitude) / d p for the shape parameters p it depends on:
//   SERSIC   cc[13] q, cc[14] Re, cc[15] n
//   EXPDISK  cc[13] q, cc[14] rs
//   FERRER   cc[12] q, cc[13] rout, cc[14] a, cc[15] b
//   GAUSSIAN cc[13] q, cc[14] fwhm
//   MOFFAT   cc[13] q, cc[14] fwhm, cc[15] n
// Boxiness (box = 1, B = par[n_params(kind)]): cc[16] = p = B + 2, and in
// magnitude mode the amplitude carries r_box (Eq. rbox) and cc[17] = d ln r_box / dB.
__device__ inline void setup_component(int kind, const double* par, int H, int W, int mag, double m0, int box,
                                       float* cc) {
  for (int k = 0; k < kCC; ++k) cc[k] = 0.f;
  if (kind == SKY) {
    cc[8] = (float)par[0];
    return;
  }
  if (kind == TSKY) {
    cc[0] = (float)(0.5 - 0.5 * W);
    cc[1] = (float)(0.5 * H - 0.5);
    cc[8] = (float)par[0];
    cc[9] = (float)par[1];
    cc[10] = (float)par[2];
    return;
  }
  const double x0 = par[0], y0 = par[1], q = par[2], pa = par[3];
  const double sx = 0.5 - x0;
  const double sxi = floor(sx);
  const double ty = (double)H - 0.5 - y0;
  const double tyi = floor(ty);
  cc[0] = __int_as_float((int)sxi);
  cc[1] = __int_as_float((int)tyi);
  cc[2] = (float)(sx - sxi);
  cc[3] = (float)(ty - tyi);
  cc[4] = (float)cos(pa);
  cc[5] = (float)sin(pa);
  cc[6] = (float)(1.0 / q);
  cc[7] = (float)q;
  double lnF = mag ? -0.4 * log(10.0) * (par[4] - m0) : 0.0;  // ln of the total flux
  if (box) {
    const double p = par[n_params(kind)] + 2.0, a = 1.0 / p;
    cc[16] = (float)p;
    if (mag) {
      // r_box = pi p / (2 beta(a, a)), beta(a, a) = Gamma(a)^2 / Gamma(2a)
      lnF += log(kPiD * p / 2.0) - (2.0 * lgamma(a) - lgamma(2.0 * a));
      cc[17] = (float)(1.0 / p + 2.0 * (digamma_pos(a) - digamma_pos(2.0 * a)) / (p * p));
    }
  }
  switch (kind) {
    case SERSIC: {
      const double n = par[6];
      cc[8] = (float)par[4];
      cc[9] = (float)(1.0 / par[5]);
      cc[10] = (float)(1.0 / n);
      double nu, dnu;
#ifdef GM_HOST_TU
      sersic_nu_dnu_fast(n, &nu, &dnu);
#else
      sersic_nu_dnu(n, &nu, &dnu);
#endif
      cc[11] = (float)nu;
      cc[12] = (float)dnu;
      if (mag) {
        const double re = par[5];
        cc[8] = (float)exp(2.0 * n * log(nu) + lnF - log(2.0 * kPiD * q * re * re * n) - lgamma(2.0 * n) - nu);
        cc[13] = (float)(-1.0 / q);
        cc[14] = (float)(-2.0 / re);
        cc[15] = (float)(2.0 * log(nu) + 2.0 * n * dnu / nu - 1.0 / n - 2.0 * digamma_pos(2.0 * n) - dnu);
      }
      break;
    }
    case EXPDISK:
      cc[8] = (float)par[4];
      cc[9] = (float)(1.0 / par[5]);
      if (mag) {
        cc[8] = (float)(exp(lnF) / (2.0 * kPiD * q * par[5] * par[5]));
        cc[13] = (float)(-1.0 / q);
        cc[14] = (float)(-2.0 / par[5]);
      }
      break;
    case FERRER:
      cc[8] = (float)par[4];
      cc[9] = (float)(1.0 / par[5]);
      cc[10] = (float)par[6];
      cc[11] = (float)(2.0 - par[7]);
      if (mag) {
        const double rout = par[5], a = par[6], b = par[7], cb = 1.0 + 2.0 / (2.0 - b);
        const double lnbeta = lgamma(a) + lgamma(cb) - lgamma(a + cb);
        const double psi_acb = digamma_pos(a + cb);
        cc[8] = (float)exp(lnF - log(kPiD * q * rout * rout * a) - lnbeta);
        cc[12] = (float)(-1.0 / q);
        cc[13] = (float)(-2.0 / rout);
        cc[14] = (float)(-1.0 / a - (digamma_pos(a) - psi_acb));
        cc[15] = (float)(-(digamma_pos(cb) - psi_acb) * 2.0 / ((2.0 - b) * (2.0 - b)));
      }
      break;
    case KING: {
      const double rc = par[5], rt = par[6], al = par[7];
      const double xt2 = (rt / rc) * (rt / rc);
      const double vt = 1.0 + xt2;
      const double At = pow(vt, -1.0 / al);
      cc[8] = (float)par[4];
      cc[9] = (float)(1.0 / rc);
      cc[10] = (float)al;
      cc[11] = (float)At;
      cc[12] = (float)(2.0 * xt2 / (al * rc) * At / vt);       // dA_t/drc
      cc[13] = (float)(-2.0 * rt / (al * rc * rc) * At / vt);  // dA_t/drt
      cc[14] = (float)(At * log(vt) / (al * al));              // dA_t/dalpha
      cc[15] = (float)rt;
      break;
    }
    case GAUSSIAN: {
      const double fw = par[5];
      const double sig = fw / (2.0 * sqrt(2.0 * log(2.0)));
      cc[8] = (float)par[4];
      cc[9] = (float)(1.0 / (sig * sig));
      cc[10] = (float)(1.0 / fw);
      if (mag) {
        cc[8] = (float)(exp(lnF) / (2.0 * kPiD * q * sig * sig));
        cc[13] = (float)(-1.0 / q);
        cc[14] = (float)(-2.0 / fw);
      }
      break;
    }
    case MOFFAT: {
      const double fw = par[5], n = par[6];
      const double t = exp2(1.0 / n);
      const double rd = fw / (2.0 * sqrt(t - 1.0));
      cc[8] = (float)par[4];
      cc[9] = (float)(1.0 / rd);
      cc[10] = (float)n;
      cc[11] = (float)(t * log(2.0) / (2.0 * n * n * (t - 1.0)));  // d ln rd / dn
      cc[12] = (float)(1.0 / fw);
      if (mag) {
        cc[8] = (float)((n - 1.0) * exp(lnF) / (kPiD * q * rd * rd));
        cc[13] = (float)(-1.0 / q);
        cc[14] = (float)(-2.0 / fw);
        cc[15] = (float)(1.0 / (n - 1.0) - 2.0 * t * log(2.0) / (2.0 * n * n * (t - 1.0)));
      }
      break;
    }
    default:
      break;
  }
}

// ---------------------------------------------------------------------------
// One component at stamp pixel (i, j): value and d value / d p_k for each of
// the component's parameters (physical units, order of the ABI header).
// ---------------------------------------------------------------------------
// kExt = false is the plain instance (no magnitude, no boxiness): the hot path of
// most models, kept free of the extras' instructions.
template <bool kExt>
__device__ __forceinline__ float eval_component_t(int kind, const float* __restrict__ cc, int i, int j,
                                                  float (&d)[8]) {
  const bool mag = kExt && (kind & kMagFlag), box = kExt && (kind & kBoxFlag);
  kind &= kMagFlag - 1;
  if (kind == SKY) {
    d[0] = 1.f;
    return cc[8];
  }
  if (kind == TSKY) {
    const float xs = (float)j + cc[0], ys = cc[1] - (float)i;
    d[0] = 1.f;
    d[1] = xs;
    d[2] = ys;
    return fmaf(cc[9], xs, fmaf(cc[10], ys, cc[8]));
  }
  const float dx = (float)(j + __float_as_int(cc[0])) + cc[2];
  const float dy = (float)(__float_as_int(cc[1]) - i) + cc[3];
  const float c = cc[4], s = cc[5], iq = cc[6], q = cc[7];
  const float X = fmaf(c, dx, s * dy);
  const float Y = fmaf(-s, dx, c * dy);
  const float Yq = Y * iq;
  // r and its derivatives in X, Y/q and (boxy) the exponent p = B + 2
  float r, ir, rX, rY, rB = 0.f;
  bool floored;
  if (!box) {
    r = sqrtf(fmaf(X, X, Yq * Yq));
    floored = r < kRFloor;
    if (floored) r = kRFloor;
    ir = 1.f / r;
    rX = rY = 0.f;  // unused: the elliptical radius takes dr/dX = X/r, dr/d(Y/q) = (Y/q)/r below
  } else {
    // r = (|X|^p + |Y/q|^p)^(1/p); dr/dX = r |X|^p / (S X); dr/dp = r (-ln S / p^2 + sum |x|^p ln|x| / (p S))
    const float p = cc[16], ip = 1.f / p;
    const float ax = fabsf(X), ay = fabsf(Yq);
    const float lx = log2f(ax), ly = log2f(ay);
    const float tx = ax > 0.f ? exp2f(p * lx) : 0.f, ty = ay > 0.f ? exp2f(p * ly) : 0.f;
    const float S = tx + ty;
    const float lS = log2f(S);
    r = exp2f(lS * ip);
    floored = !(r >= kRFloor);
    if (floored) {
      r = kRFloor;
      rX = rY = 0.f;
    } else {
      const float iS = 1.f / S;
      rX = ax > 0.f ? r * tx * iS / X : 0.f;
      rY = ay > 0.f ? r * ty * iS / Yq : 0.f;
      const float tl = (ax > 0.f ? tx * lx : 0.f) + (ay > 0.f ? ty * ly : 0.f);
      rB = r * kLn2 * ip * fmaf(tl, iS, -lS * ip);
    }
    ir = 1.f / r;
  }
  float val = 0.f, dIdr = 0.f;
  switch (kind) {
    case SERSIC: {
      const float Ie = cc[8], iRe = cc[9], in = cc[10], nu = cc[11], dnu = cc[12];
      const float lt = log2f(r * iRe);            // log2(r / Re)
      const float u = exp2f(lt * in);             // (r / Re)^(1/n)
      const float e = exp2f(-nu * (u - 1.f) * kLog2e);
      val = Ie * e;
      const float vu = val * nu * u * in;         // I nu u / n
      dIdr = -vu * ir;
      d[4] = e;                                   // dI/dIe
      d[5] = vu * iRe;                            // dI/dRe
      d[6] = val * fmaf(-dnu, u - 1.f, nu * u * lt * kLn2 * in * in);  // dI/dn
      break;
    }
    case EXPDISK: {
      const float I0 = cc[8], irs = cc[9];
      const float e = exp2f(-r * irs * kLog2e);
      val = I0 * e;
      dIdr = -val * irs;
      d[4] = e;
      d[5] = val * r * irs * irs;
      break;
    }
    case FERRER: {
      const float I0 = cc[8], irout = cc[9], a = cc[10], ex = cc[11];
      const float x = r * irout;
      float sv = 0.f, gg = 0.f;
      if (x < 1.f) {
        sv = exp2f(ex * log2f(x));                // (r/rout)^(2-b)
        gg = 1.f - sv;
      }
      if (gg > 0.f) {
        const float lg = log2f(gg);
        const float ga1 = exp2f((a - 1.f) * lg);  // g^(a-1)
        val = I0 * ga1 * gg;
        const float t = a * I0 * ga1 * ex * sv;
        dIdr = -t * ir;
        d[4] = ga1 * gg;
        d[5] = t * irout;                         // dI/drout
        d[6] = val * lg * kLn2;                   // dI/da
        d[7] = a * I0 * ga1 * sv * log2f(x) * kLn2;  // dI/db
      } else {
        d[4] = d[5] = d[6] = d[7] = 0.f;
      }
      break;
    }
    case KING: {
      const float I0 = cc[8], irc = cc[9], al = cc[10], At = cc[11];
      const float dAt_rc = cc[12], dAt_rt = cc[13], dAt_al = cc[14], rt = cc[15];
      const float x2 = r * irc * r * irc;
      const float v = 1.f + x2;
      const float lv = log2f(v);
      const float A = exp2f(-lv / al);
      const float D = A - At, N = 1.f - At;
      const float f = D / N;
      if (r < rt && f > 0.f) {
        const float lf = log2f(f);
        const float fa1 = exp2f((al - 1.f) * lf);   // f^(alpha-1)
        val = I0 * fa1 * f;
        const float k = I0 * al * fa1 / N;          // dI/dA at fixed A_t
        const float iN = 1.f / N;
        dIdr = k * (-2.f * r * irc * irc / al) * A / v;
        const float dA_rc = 2.f * x2 * irc / al * A / v;
        d[4] = fa1 * f;
        d[5] = k * ((dA_rc - dAt_rc) + D * iN * dAt_rc);
        d[6] = k * dAt_rt * (A - 1.f) * iN;
        const float dA_al = A * lv * kLn2 / (al * al);
        d[7] = val * lf * kLn2 + k * ((dA_al - dAt_al) + D * iN * dAt_al);
      } else {
        d[4] = d[5] = d[6] = d[7] = 0.f;
      }
      break;
    }
    case GAUSSIAN: {
      const float I0 = cc[8], is2 = cc[9], ifw = cc[10];
      const float e = exp2f(-0.5f * r * r * is2 * kLog2e);
      val = I0 * e;
      dIdr = -val * r * is2;
      d[4] = e;
      d[5] = val * r * r * is2 * ifw;
      break;
    }
    case MOFFAT: {
      const float I0 = cc[8], ird = cc[9], n = cc[10], dlrd = cc[11], ifw = cc[12];
      const float w = r * ird;
      const float v = fmaf(w, w, 1.f);
      const float lv = log2f(v);
      const float e = exp2f(-n * lv);
      val = I0 * e;
      const float t = 2.f * n * val * w * w / v;     // rd dI/drd
      dIdr = -t * ir;
      d[4] = e;
      d[5] = t * ifw;                                // dI/dfwhm
      d[6] = -val * lv * kLn2 + t * dlrd;            // dI/dn
      break;
    }
    default:
      break;
  }
  if (floored) {
    d[0] = d[1] = d[2] = d[3] = 0.f;
  } else {
    // X = c dx + s dy, Y/q = (-s dx + c dy)/q: d/dx0 = (-c, s/q), d/dy0 = (-s, -c/q),
    // d/dq = (0, -Y/q^2), d/dpa = (Y, -X/q)
    if (!box) {
      const float gr = dIdr * ir;                   // (dI/dr) / r
      d[0] = gr * fmaf(-X, c, Yq * s * iq);         // dI/dx0
      d[1] = gr * fmaf(-X, s, -Yq * c * iq);        // dI/dy0
      d[2] = gr * (-Yq * Yq * iq);                  // dI/dq
      d[3] = gr * (X * Yq * (q - iq));              // dI/dpa
    } else {
      const float gX = dIdr * rX, gY = dIdr * rY;
      d[0] = fmaf(-gX, c, gY * s * iq);
      d[1] = fmaf(-gX, s, -gY * c * iq);
      d[2] = -gY * Yq * iq;
      d[3] = fmaf(gX, q * Yq, -gY * X * iq);
    }
  }
  if (box) {
    // dI/dB = dI/dp (rB is zero on the floor), plus I d ln(r_box)/dB with a magnitude.
    // B follows the profile's own parameters: slot 6 (exponential, Gaussian) or 7
    // (Sersic, Moffat).  The slot is picked by compile-time indices so that d stays
    // in registers.
    float dB = dIdr * rB;
    if (mag) dB = fmaf(val, cc[17], dB);
    const bool at6 = kind == EXPDISK || kind == GAUSSIAN;
    if (at6) d[6] = dB;
    else d[7] = dB;
  }
  if (mag) {
    // amplitude A(m, shape): dI/dm = I d ln A / dm, and dI/dp gains I d ln A / dp
    d[4] = -0.92103403719761836f * val;  // -0.4 ln 10
    switch (kind) {
      case FERRER:
        d[2] = fmaf(val, cc[12], d[2]);
        d[5] = fmaf(val, cc[13], d[5]);
        d[6] = fmaf(val, cc[14], d[6]);
        d[7] = fmaf(val, cc[15], d[7]);
        break;
      case SERSIC:
      case MOFFAT:
        d[6] = fmaf(val, cc[15], d[6]);
        d[2] = fmaf(val, cc[13], d[2]);
        d[5] = fmaf(val, cc[14], d[5]);
        break;
      default:  // EXPDISK, GAUSSIAN
        d[2] = fmaf(val, cc[13], d[2]);
        d[5] = fmaf(val, cc[14], d[5]);
        break;
    }
  }
  return val;
}

// The kind carries the magnitude and boxiness flags; the test is uniform across a
// warp (one component at a time), so only one instance runs.
__device__ __forceinline__ float eval_component(int kind, const float* __restrict__ cc, int i, int j,
                                                float (&d)[8]) {
  if (kind & (kMagFlag | kBoxFlag)) return eval_component_t<true>(kind, cc, i, j, d);
  return eval_component_t<false>(kind, cc, i, j, d);
}

}  // namespace gm
