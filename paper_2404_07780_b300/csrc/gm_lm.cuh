// gm_lm.cuh -- per-galaxy kernels around the fused pass: input validation,
// set-up of the per-component constants, the Levenberg-Marquardt step (FP64
// Cholesky on the damped normal equations) and the final outputs with the
// covariance uncertainty sigma_p = sqrt(diag[(J^T W J)^-1]) of Sec. 5.2 of
// arxiv 2404.07780.
#pragma once

#include "gm_geom.cuh"
#include "gm_profiles.cuh"

namespace gm {

constexpr int ST_RUNNING = 0, ST_CONVERGED = 1, ST_MAX_ITER = 2, ST_STALLED = 3, ST_SINGULAR = 4,
              ST_NONFINITE = 5, ST_BAD_INPUT = 6, ST_NO_DOF = 7;
// Internal: CONVERGED, with the final Gauss-Newton step queued for evaluation
// (never an output: the next pass evaluates it and the step resolves it).
constexpr int ST_POLISH = 16;
// The final step's point is kept unless its chi^2 exceeds the best by more than
// this (relative): far above the FP32 rounding of chi^2, far below any real loss.
constexpr double kPolishSlack = 1e-6;
// chi^2 changes below this fraction of chi^2 are not resolved by the tile sums of
// FP32 pixel terms (their rounding is ~1e-8 relative): a step whose predicted
// decrease is smaller is judged by its prediction, not by the measured change.
constexpr double kChi2Res = 1e-7;

constexpr int kMaxAcc = 1 + kMaxFree + kMaxFree * (kMaxFree + 1) / 2;

// Components sharing one axis-ratio slot whose geometry can be rewritten from
// q > 1 to 1/q (position angles + pi/2, scale lengths x q): same image.
struct CanonGroup {
  int q_slot;
  int n_pa, pa[kMaxComp];
  int n_scale, scale[2 * kMaxComp];
};

// Model description as the per-galaxy kernels need it.
struct DescDev {
  int n_comp;
  int kind[kMaxComp];
  int np[kMaxComp];
  int slot[kMaxComp][8];
  int n_slots;
  int P;                       // free slots
  int free_slot[kMaxFree];     // accumulator order -> slot
  int is_log[kMaxSlots];
  int is_pa[kMaxSlots];        // slot is some radial component's position angle
  double lo[kMaxSlots], hi[kMaxSlots];
  int n_canon;
  CanonGroup canon[kMaxComp];
  int mag[kMaxComp];           // amplitude slot holds a magnitude ...
  double mag_zero[kMaxComp];   // ... with this zero point
  int box[kMaxComp];           // boxiness B follows the profile's parameters
};

struct LMOpts {
  double tol, xtol, gtol;
  int max_iter;
  double lambda0, lambda_up, lambda_down, lambda_min, lambda_max;
  int polish;  // one final Gauss-Newton step after CONVERGED
  int canonical;         // rewrite q > 1 and wrap position angles at exit
  double* lambda_inout;  // [G] starting damping in (when > 0 and finite), final damping out; or nullptr
};

// Per-galaxy LM state, struct of arrays in the caller's workspace.
struct LMState {
  double* p_b;     // [G][S] best point
  double* p_t;     // [G][S] point being evaluated
  double* A_b;     // [G][P(P+1)/2] J^T W J at p_b (internal coordinates, packed upper)
  double* g_b;     // [G][P] J^T W r at p_b
  double* chi2_b;  // [G]
  double* lam;     // [G]
  double* pred;    // [G] chi^2 decrease the quadratic model predicts for the pending step (inf: clamped)
  int* it;         // [G] evaluations done
  int* status;     // [G]
  int* nused;      // [G] unmasked pixels
  int* bad;        // [G] bad sigma / image on a used pixel
  int* list[2];    // active galaxies, double-buffered by iteration parity
  int* count[2];
  int2* items[2];  // their (galaxy, tile) items, same parity
  int* icount[2];
  unsigned long long* evals;  // [3]: galaxies evaluated over the passes, converged, iterations
};

__device__ inline void setup_galaxy(const DescDev& D, const double* p, int H, int W, int use_log, float* cc,
                                    float* scale) {
  double par[8];
  for (int c = 0; c < D.n_comp; ++c) {
    for (int k = 0; k < D.np[c]; ++k) par[k] = p[D.slot[c][k]];  // D.np includes B when boxy
    setup_component(D.kind[c], par, H, W, D.mag[c], D.mag_zero[c], D.box[c], cc + c * kCC);
  }
  for (int s = 0; s < D.n_slots; ++s) scale[s] = (use_log && D.is_log[s]) ? (float)p[s] : 1.f;
}

#ifdef GM_HOST_TU
// Constants for every galaxy from caller parameters (gm_model, gm_chi2_grad).
// Stamp heights from geo, or H for every galaxy when geo is nullptr.
__global__ void k_setup(const __grid_constant__ DescDev D, int G, const GalGeom* __restrict__ geo, int H, int W,
                        const double* __restrict__ params, int use_log, float* cconst, float* scale) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  setup_galaxy(D, params + (size_t)g * D.n_slots, geo ? geo[g].H : H, geo ? geo[g].W : W, use_log,
               cconst + (size_t)g * D.n_comp * kCC, scale + (size_t)g * scale_stride(D.n_slots));
}
#endif  // GM_HOST_TU

#ifdef GM_HOST_TU
// Used-pixel count and bad-input flag per galaxy (one block per galaxy, strided).
__global__ void k_validate(int G, const GalGeom* __restrict__ geo, const float* __restrict__ image,
                           const float* __restrict__ sigma, const uint8_t* __restrict__ mask, int* nused, int* bad) {
  __shared__ int s_n[32], s_b[32];
  for (int g = blockIdx.x; g < G; g += gridDim.x) {
    const size_t HW = (size_t)geo[g].H * geo[g].W, base = (size_t)geo[g].pix;
    int n = 0, b = 0;
    for (size_t t = threadIdx.x; t < HW; t += blockDim.x) {
      const size_t gp = base + t;
      if (mask && mask[gp]) continue;
      ++n;
      const float s = sigma[gp], d = image[gp];
      if (!(s > 0.f) || !isfinite(s) || !isfinite(d)) b = 1;
    }
    for (int o = 16; o > 0; o >>= 1) {
      n += __shfl_xor_sync(0xffffffffu, n, o);
      b |= __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
      s_n[warp] = n;
      s_b[warp] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int tn = 0, tb = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        tn += s_n[w];
        tb |= s_b[w];
      }
      nused[g] = tn;
      bad[g] = tb;
    }
    __syncthreads();
  }
}
#endif  // GM_HOST_TU

__device__ inline double to_u(const DescDev& D, int s, double p) { return D.is_log[s] ? log(p) : p; }
__device__ inline double from_u(const DescDev& D, int s, double u) { return D.is_log[s] ? exp(u) : u; }

__device__ inline void clamp_slots(const DescDev& D, double* p) {
  for (int s = 0; s < D.n_slots; ++s) p[s] = fmin(fmax(p[s], D.lo[s]), D.hi[s]);
}

// Queue galaxy g and its tiles for the pass of list `l`.
__device__ inline void queue_galaxy(const LMState& S, int l, int g, const GalGeom& geo) {
  const int pos = atomicAdd(S.count[l], 1);
  S.list[l][pos] = g;
  const int nt = geo.n_tiles;
  const int ipos = atomicAdd(S.icount[l], nt);
  for (int t = 0; t < nt; ++t) S.items[l][ipos + t] = make_int2(g, t);
}

#ifdef GM_HOST_TU
// Start of a fit: clamp the start point, set status from the validation and
// queue the galaxies that can be fitted, in the processing order `order`
// (most expensive first).
__global__ void k_lm_init(const __grid_constant__ DescDev D, LMState S, LMOpts O, int G,
                          const GalGeom* __restrict__ geo, const int* __restrict__ order,
                          const double* __restrict__ params0, float* cconst, float* scale) {
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= G) return;
  const int g = order[pos];
  const int NS = D.n_slots, P = D.P;
  double* pb = S.p_b + (size_t)g * NS;
  double* pt = S.p_t + (size_t)g * NS;
  for (int s = 0; s < NS; ++s) pb[s] = params0[(size_t)g * NS + s];
  clamp_slots(D, pb);
  for (int s = 0; s < NS; ++s) pt[s] = pb[s];
  S.it[g] = 0;
  const double li = O.lambda_inout ? O.lambda_inout[g] : 0.0;
  S.lam[g] = (li > 0.0 && isfinite(li)) ? li : O.lambda0;
  S.chi2_b[g] = CUDART_NAN;
  int st = ST_RUNNING;
  if (S.bad[g]) st = ST_BAD_INPUT;
  else if (S.nused[g] - P <= 0) st = ST_NO_DOF;
  S.status[g] = st;
  if (st == ST_RUNNING) {
    setup_galaxy(D, pt, geo[g].H, geo[g].W, 1, cconst + (size_t)g * D.n_comp * kCC,
                 scale + (size_t)g * scale_stride(NS));
    queue_galaxy(S, 0, g, geo[g]);
  }
}
#endif  // GM_HOST_TU

// Entry (f, h) of a row-major packed upper triangle of a symmetric P x P matrix.
__device__ inline double packed(const double* Ap, int P, int f, int h) {
  if (f > h) {
    const int t = f;
    f = h;
    h = t;
  }
  return Ap[f * P - (f * (f - 1)) / 2 + (h - f)];
}

#ifdef GM_HOST_TU
// ---------------------------------------------------------------------------
// Warp-cooperative pieces of the LM step (one warp per galaxy).  Matrices are
// P x P row-major in shared memory; lane f owns row / parameter f (P <= 16).
// ---------------------------------------------------------------------------
constexpr unsigned kFull = 0xffffffffu;

__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// In-place Cholesky (lower triangle) of M, column by column: lanes i >= j form
// their entry of column j at once.  The pivot is l_jj = d rsqrt(d) and the
// entries below it are multiplied by rsqrt(d), which is also kept in dinv[j]
// for the solves: an FP64 square root or division is a long chain of FP64
// instructions at sm_103a's FP64 issue rate, on the critical path of every
// column, and rsqrt is one approximation and a short refinement.  false (on
// every lane) if M is not positive definite.
__device__ inline bool warp_cholesky(double* M, double* dinv, int P, int lane) {
  for (int j = 0; j < P; ++j) {
    double t = 0.0;
    if (lane >= j && lane < P) {
      t = M[lane * P + j];
      for (int k = 0; k < j; ++k) t -= M[lane * P + k] * M[j * P + k];
    }
    const double d = __shfl_sync(kFull, t, j);
    if (!(d > 0.0)) return false;
    const double il = rsqrt(d);
    if (lane == j) {
      M[j * P + j] = d * il;
      dinv[j] = il;
    } else if (lane > j && lane < P) {
      M[lane * P + j] = t * il;
    }
    __syncwarp();
  }
  return true;
}

// Solve L L^T x = b (L and dinv from warp_cholesky); b and x are lane-owned
// (entry f on lane f); returns x on every lane f < P.
__device__ inline double warp_chol_solve(const double* L, const double* dinv, int P, int lane, double b) {
  double r = b, y = 0.0;
  for (int i = 0; i < P; ++i) {  // forward: y_i = (b_i - sum_{k<i} L_ik y_k) / L_ii
    const double yi = __shfl_sync(kFull, r, i) * dinv[i];
    if (lane == i) y = yi;
    if (lane > i && lane < P) r -= L[lane * P + i] * yi;
  }
  r = y;
  double x = 0.0;
  for (int i = P - 1; i >= 0; --i) {  // back: x_i = (y_i - sum_{k>i} L_ki x_k) / L_ii
    const double xi = __shfl_sync(kFull, r, i) * dinv[i];
    if (lane == i) x = xi;
    if (lane < i) r -= L[i * P + lane] * xi;
  }
  return x;
}

// The system of a step, lane f writing row f of M and returning r_f: M = A with
// lam max(A_ff, 1e-12 max diag A) added on the diagonal (lam = 0: 1e-12 max diag
// A alone), the rows and columns of held parameters (bits of `held`) replaced by
// the identity; r = g with zeros at held parameters.
__device__ inline double warp_step_system(const double* Ap, const double* g, int P, double lam, unsigned held,
                                          double* M, int lane) {
  double dmax = 0.0;
  for (int f = 0; f < P; ++f) dmax = fmax(dmax, packed(Ap, P, f, f));
  const double dfloor = 1e-12 * dmax;
  double r = 0.0;
  if (lane < P) {
    const int f = lane;
    const bool hf = (held >> f) & 1u;
    for (int h = 0; h < P; ++h)
      M[f * P + h] = (hf || ((held >> h) & 1u)) ? (f == h ? 1.0 : 0.0) : packed(Ap, P, f, h);
    if (!hf) M[f * P + f] += lam > 0.0 ? lam * fmax(packed(Ap, P, f, f), dfloor) : dfloor;
    r = hf ? 0.0 : g[f];
  }
  __syncwarp();
  return r;
}

// setup_galaxy() by the lanes: lane c sets up component c, lanes s the slot scales.
__device__ inline void warp_setup_galaxy(const DescDev& D, const double* p, int H, int W, float* cc, float* scale,
                                         int lane) {
  if (lane < D.n_comp) {
    double par[8];
    for (int k = 0; k < D.np[lane]; ++k) par[k] = p[D.slot[lane][k]];
    setup_component(D.kind[lane], par, H, W, D.mag[lane], D.mag_zero[lane], D.box[lane], cc + lane * kCC);
  }
  for (int s = lane; s < D.n_slots; s += 32) scale[s] = D.is_log[s] ? (float)p[s] : 1.f;
}

// queue_galaxy() by the lanes: lane 0 takes the list and item positions, every lane writes items.
__device__ inline void warp_queue_galaxy(const LMState& S, int l, int g, const GalGeom& geo, int lane) {
  const int nt = geo.n_tiles;
  int ipos = 0;
  if (lane == 0) {
    const int pos = atomicAdd(S.count[l], 1);
    S.list[l][pos] = g;
    ipos = atomicAdd(S.icount[l], nt);
  }
  ipos = __shfl_sync(kFull, ipos, 0);
  for (int t = lane; t < nt; t += 32) S.items[l][ipos + t] = make_int2(g, t);
}

// pt = clamp(from_u(to_u(pb) + delta)) by the lanes (delta lane-owned), with the
// galaxy's constants for it; returns whether the clamp moved a slot.
__device__ inline bool warp_trial_point(const DescDev& D, const double* pb, double* pt, double delta, int lane) {
  const int NS = D.n_slots, P = D.P;
  for (int s = lane; s < NS; s += 32) pt[s] = pb[s];
  __syncwarp();
  if (lane < P) {
    const int s = D.free_slot[lane];
    pt[s] = from_u(D, s, to_u(D, s, pb[s]) + delta);
  }
  __syncwarp();
  bool out = false;
  for (int s = lane; s < NS; s += 32) {
    out = out || pt[s] < D.lo[s] || pt[s] > D.hi[s];
    pt[s] = fmin(fmax(pt[s], D.lo[s]), D.hi[s]);
  }
  __syncwarp();
  return __any_sync(kFull, out);
}

// One LM step for every galaxy evaluated in this iteration (list `cur`):
// sum the tile partials of the pass, accept or reject the evaluated point,
// test convergence, solve the damped normal equations for the next trial point
// and queue the galaxy for the next pass (list `cur ^ 1`).  The rules are the
// ones the FP64 oracle states: accept when chi^2 drops -- or, for a step whose
// predicted decrease is below kChi2Res chi^2, unless chi^2 rose by more than
// kChi2Res chi^2, the step's decrease then taken as the predicted one (not
// clamped steps); CONVERGED when an
// accepted step lowers chi^2 by less than tol relative, any evaluated step
// is below xtol, or the Gauss-Newton decrement at the best point is at most
// gtol chi^2; STALLED / SINGULAR past lambda_max; MAX_ITER at max_iter.
// Free parameters on a bound whose descent direction leaves the box are held
// (zero step) in the damped solve, the decrement and the final step.
// With O.polish, a galaxy that reaches CONVERGED before max_iter queues one
// undamped Gauss-Newton step from its best point instead of stopping; the
// next step call adopts that point unless its chi^2 is non-finite or above
// the best by more than kPolishSlack relative (FP32-accumulated chi^2 cannot
// resolve the last decreases towards the minimum; the gradient can).
// One warp per active galaxy, kLmGals galaxies per block: the lanes sum the
// tile partials (entry e over the galaxy's tiles in tile order: deterministic),
// form the Cholesky factor a column at a time, and split the per-parameter,
// per-component and per-tile work; the scalar decisions are taken alike by
// every lane.
constexpr int kLmWarps = 4;   // warps per block of k_chi2_grad_finish (one galaxy per warp)
constexpr int kLmGals = 4;    // galaxies (warps) per block of k_lm_step

__global__ void __launch_bounds__(32 * kLmGals) k_lm_step(const __grid_constant__ DescDev D, LMState S, LMOpts O,
                                                         int cur, const GalGeom* __restrict__ geo,
                                                         const double* __restrict__ partial, float* cconst,
                                                         float* scale) {
  __shared__ double s_acc[kLmGals][kMaxAcc];
  __shared__ double s_M[kLmGals][kMaxFree * kMaxFree];
  __shared__ double s_dinv[kLmGals][kMaxFree];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int gi = blockIdx.x * kLmGals + wl;
  const int n_cur = *S.count[cur];
  if (gi == 0 && lane == 0) atomicAdd(S.evals, (unsigned long long)n_cur);
  if (gi >= n_cur) return;
  const int NS = D.n_slots, P = D.P, NAp = P * (P + 1) / 2, NA = 1 + P + NAp;
  const int g = S.list[cur][gi];
  double* acc = s_acc[wl];
  double* M = s_M[wl];
  double* dinv = s_dinv[wl];
  {
    const int n_tiles = geo[g].n_tiles;
    const double* pp = partial + (size_t)geo[g].tile0 * NA;
    for (int e = lane; e < NA; e += 32) {
      double a = 0.0;
      for (int t = 0; t < n_tiles; ++t) a += pp[(size_t)t * NA + e];
      acc[e] = a;
    }
  }
  __syncwarp();

  double* pb = S.p_b + (size_t)g * NS;
  double* pt = S.p_t + (size_t)g * NS;
  double* Ab = S.A_b + (size_t)g * NAp;
  double* gb = S.g_b + (size_t)g * P;
  const double chi2_t = acc[0];
  float* ccg = cconst + (size_t)g * D.n_comp * kCC;
  float* scg = scale + (size_t)g * scale_stride(NS);

  // adopt the evaluated point and its normal equations as the best
  auto adopt = [&]() {
    for (int s = lane; s < NS; s += 32) pb[s] = pt[s];
    for (int f = lane; f < P; f += 32) gb[f] = acc[1 + f];
    for (int e = lane; e < NAp; e += 32) Ab[e] = acc[1 + P + e];
  };

  int st = ST_RUNNING;
  const int it = S.it[g] + 1;
  double lam = S.lam[g];
  const double chi2_b = S.chi2_b[g];
  const int status_in = S.status[g];
  __syncwarp();
  if (lane == 0) S.it[g] = it;
  bool accepted = false;
  if (status_in == ST_POLISH) {
    // the final Gauss-Newton step's point, evaluated: it becomes the result unless
    // its chi^2 is non-finite or above the best by more than the slack
    if (isfinite(chi2_t) && chi2_t <= chi2_b * (1.0 + kPolishSlack)) {
      adopt();
      if (lane == 0) S.chi2_b[g] = chi2_t;
    }
    if (lane == 0) S.status[g] = ST_CONVERGED;
    return;
  }
  if (it == 1) {
    if (!isfinite(chi2_t)) {
      st = ST_NONFINITE;
    } else {
      adopt();
      if (lane == 0) S.chi2_b[g] = chi2_t;
      accepted = true;
      if (chi2_t == 0.0) st = ST_CONVERGED;
    }
  } else {
    bool big = false;
    if (lane < P) {
      const int s = D.free_slot[lane];
      const double u0 = to_u(D, s, pb[s]), u1 = to_u(D, s, pt[s]);
      big = fabs(u1 - u0) > O.xtol * (fabs(u0) + O.xtol);
    }
    const bool small = !__any_sync(kFull, big);
    // a step whose predicted decrease is below the resolution of chi^2 is accepted unless
    // chi^2 rose by more than that resolution, and its decrease is the predicted one
    const double pred = S.pred[g];
    const bool resolved = pred >= kChi2Res * chi2_b;
    if (isfinite(chi2_t) && (chi2_t < chi2_b || (!resolved && chi2_t <= chi2_b * (1.0 + kChi2Res)))) {
      const double act = resolved ? (chi2_b - chi2_t) / chi2_b : fmax(pred, 0.0) / chi2_b;
      __syncwarp();
      adopt();
      if (lane == 0) S.chi2_b[g] = chi2_t;
      lam = fmax(lam * O.lambda_down, O.lambda_min);
      accepted = true;
      if (act < O.tol || small || chi2_t == 0.0) st = ST_CONVERGED;
    } else if (small) {
      st = ST_CONVERGED;
    } else {
      lam *= O.lambda_up;
      if (lam > O.lambda_max) st = ST_STALLED;
    }
  }
  __syncwarp();
  const double chi2_best = accepted ? chi2_t : chi2_b;

  // parameters held at a bound for the next step (bit f), from the best point
  bool hb = false;
  if (lane < P) {
    const int s = D.free_slot[lane];
    hb = (pb[s] <= D.lo[s] && gb[lane] < 0.0) || (pb[s] >= D.hi[s] && gb[lane] > 0.0);
  }
  const unsigned held = __ballot_sync(kFull, hb) & ((1u << P) - 1u);
  const double gf = lane < P ? gb[lane] : 0.0;

  if (st == ST_RUNNING && accepted) {
    // Gauss-Newton decrement g^T A^-1 g over the parameters not held.  The system matrix is
    // positive definite, so g^T A^-1 g >= |g|^2 / lambda_max >= |g|^2 / trace: while that bound
    // is above the threshold the test cannot pass, and the factorisation is skipped (the
    // sums are the same in every lane, so the warp takes one branch)
    const double r = warp_step_system(Ab, gb, P, 0.0, held, M, lane);
    const double r2 = warp_sum(r * r), tr = warp_sum(lane < P ? M[lane * P + lane] : 0.0);
    if (!(r2 > O.gtol * chi2_best * tr) && warp_cholesky(M, dinv, P, lane)) {
      const double x = warp_chol_solve(M, dinv, P, lane, r);
      const double gn = warp_sum(lane < P ? r * x : 0.0);
      if (gn >= 0.0 && gn <= O.gtol * chi2_best) st = ST_CONVERGED;
    }
  }
  if (st == ST_RUNNING && it >= O.max_iter) st = ST_MAX_ITER;
  if (st == ST_CONVERGED && O.polish && it < O.max_iter && chi2_best > 0.0) {
    // final Gauss-Newton step from the best point: delta = A^-1 g with the diagonal
    // floored as in the damped solve, evaluated in the next pass
    const double r = warp_step_system(Ab, gb, P, 0.0, held, M, lane);
    if (warp_cholesky(M, dinv, P, lane)) {
      const double delta = warp_chol_solve(M, dinv, P, lane, r);
      warp_trial_point(D, pb, pt, delta, lane);
      warp_setup_galaxy(D, pt, geo[g].H, geo[g].W, ccg, scg, lane);
      warp_queue_galaxy(S, cur ^ 1, g, geo[g], lane);
      st = ST_POLISH;
    }
  }
  if (st == ST_RUNNING) {
    double r = 0.0;
    for (;;) {
      r = warp_step_system(Ab, gb, P, lam, held, M, lane);
      if (warp_cholesky(M, dinv, P, lane)) break;
      lam *= O.lambda_up;
      if (lam > O.lambda_max) {
        st = ST_SINGULAR;
        break;
      }
    }
    if (st == ST_RUNNING) {
      const double delta = warp_chol_solve(M, dinv, P, lane, r);
      // predicted decrease 2 g^T delta - delta^T A delta (every lane's delta_h by shuffles)
      double ad = 0.0;
      for (int h = 0; h < P; ++h) {
        const double dh = __shfl_sync(kFull, delta, h);
        if (lane < P) ad += packed(Ab, P, lane, h) * dh;
      }
      double pred = warp_sum(lane < P ? delta * (2.0 * gf - ad) : 0.0);
      if (warp_trial_point(D, pb, pt, delta, lane)) pred = CUDART_INF;  // clamped: judged by chi^2
      if (lane == 0) S.pred[g] = pred;
      warp_setup_galaxy(D, pt, geo[g].H, geo[g].W, ccg, scg, lane);
      warp_queue_galaxy(S, cur ^ 1, g, geo[g], lane);
    }
  }
  if (lane == 0) {
    S.lam[g] = lam;
    S.status[g] = st;
  }
}
#endif  // GM_HOST_TU

#ifdef GM_HOST_TU
// Outputs of a fit: best point, chi^2, degrees of freedom, evaluations, status
// and the covariance error bars sqrt(diag[(J^T W J)^-1]) (Sec. 5.2).  An axis
// ratio above 1 is rewritten as 1/q with its position angles turned by pi/2
// and its scale lengths multiplied by q (the same image), and the covariance
// is carried along: Sigma' = T Sigma T^T with T the Jacobian of the rewrite.
// Position angles are wrapped to [0, pi).  One warp per galaxy, as k_lm_step:
// lane f solves for column f of the inverse (its own forward and back
// substitution, with the factor's reciprocal pivots) and forms row f of the
// products; the rewrite of the point itself (a few groups, in order) is lane
// 0's.
__global__ void __launch_bounds__(32 * kLmGals) k_lm_finish(const __grid_constant__ DescDev D, LMState S, int G,
                                                           int canonical, double* lambda_out, double* params_out,
                                                           double* chi2_out, int* dof_out, int* iters_out,
                                                           int* status_out, double* sigma_p_out) {
  __shared__ double s_M[kLmGals][kMaxFree * kMaxFree];  // Cholesky factor, then T Sigma
  __shared__ double s_dinv[kLmGals][kMaxFree];          // 1 / the factor's diagonal
  __shared__ double s_C[kLmGals][kMaxFree * kMaxFree];  // Sigma
  __shared__ double s_T[kLmGals][kMaxFree * kMaxFree];  // Jacobian of the q > 1 rewrite
  __shared__ double s_p[kLmGals][kMaxSlots];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int g = blockIdx.x * kLmGals + wl;
  if (g >= G) return;
  const int NS = D.n_slots, P = D.P;
  const double pi = 3.14159265358979323846;
  double* p = s_p[wl];
  double* M = s_M[wl];
  double* dinv = s_dinv[wl];
  double* cov = s_C[wl];
  double* T = s_T[wl];
  for (int s = lane; s < NS; s += 32) p[s] = S.p_b[(size_t)g * NS + s];
  if (lane == 0) {
    chi2_out[g] = S.chi2_b[g];
    dof_out[g] = S.nused[g] - P;
    iters_out[g] = S.it[g];
    status_out[g] = S.status[g];
    if (lambda_out) lambda_out[g] = S.lam[g];
  }
  const bool evaluated = S.it[g] > 0 && S.status[g] != ST_NONFINITE;
  __syncwarp();

  // covariance of the free parameters in physical units at the best point
  bool have_cov = false;
  if (sigma_p_out && evaluated) {
    const double* Ab = S.A_b + (size_t)g * (P * (P + 1) / 2);
    if (lane < P)
      for (int h = 0; h < P; ++h) M[lane * P + h] = packed(Ab, P, lane, h);
    __syncwarp();
    if (warp_cholesky(M, dinv, P, lane)) {
      have_cov = true;
      if (lane < P) {
        const int f = lane;
        double y[kMaxFree], x[kMaxFree];
        for (int i = 0; i < P; ++i) {
          double t = (i == f) ? 1.0 : 0.0;
          for (int k = 0; k < i; ++k) t -= M[i * P + k] * y[k];
          y[i] = t * dinv[i];
        }
        for (int i = P - 1; i >= 0; --i) {
          double t = y[i];
          for (int k = i + 1; k < P; ++k) t -= M[k * P + i] * x[k];
          x[i] = t * dinv[i];
        }
        for (int h = 0; h < P; ++h) cov[h * P + f] = x[h];
      }
      __syncwarp();
      if (lane < P) {
        const int f = lane, sf = D.free_slot[f];
        const double df = D.is_log[sf] ? p[sf] : 1.0;
        for (int h = 0; h < P; ++h) {
          const int sh = D.free_slot[h];
          cov[f * P + h] *= df * (D.is_log[sh] ? p[sh] : 1.0);
        }
      }
      __syncwarp();
    }
  }

  // canonical axis ratios
  if (evaluated && canonical) {
    int any = 0;
    if (lane == 0) {
      int fidx[kMaxSlots];
      for (int s = 0; s < NS; ++s) fidx[s] = -1;
      for (int f = 0; f < P; ++f) fidx[D.free_slot[f]] = f;
      for (int f = 0; f < P * P; ++f) T[f] = 0.0;
      for (int f = 0; f < P; ++f) T[f * P + f] = 1.0;
      for (int k = 0; k < D.n_canon; ++k) {
        const CanonGroup& cg = D.canon[k];
        const double q = p[cg.q_slot];
        if (!(q > 1.0)) continue;
        any = 1;
        const int fq = fidx[cg.q_slot];
        for (int i = 0; i < cg.n_scale; ++i) {
          const int ss = cg.scale[i];
          const int fs = fidx[ss];
          if (fs >= 0) {
            T[fs * P + fs] = q;
            if (fq >= 0) T[fs * P + fq] = p[ss];
          }
          p[ss] *= q;
        }
        for (int i = 0; i < cg.n_pa; ++i) p[cg.pa[i]] += 0.5 * pi;
        if (fq >= 0) T[fq * P + fq] = -1.0 / (q * q);
        p[cg.q_slot] = 1.0 / q;
      }
    }
    any = __shfl_sync(kFull, any, 0);
    __syncwarp();
    if (any && have_cov) {  // cov <- T cov T^T, row f on lane f
      if (lane < P) {
        const int f = lane;
        for (int h = 0; h < P; ++h) {
          double acc = 0.0;
          for (int k = 0; k < P; ++k) acc += T[f * P + k] * cov[k * P + h];
          M[f * P + h] = acc;
        }
      }
      __syncwarp();
      if (lane < P) {
        const int f = lane;
        for (int h = 0; h < P; ++h) {
          double acc = 0.0;
          for (int k = 0; k < P; ++k) acc += M[f * P + k] * T[h * P + k];
          cov[f * P + h] = acc;
        }
      }
      __syncwarp();
    }
  }

  for (int s = lane; s < NS; s += 32) {
    double v = p[s];
    if (D.is_pa[s] && canonical) v -= pi * floor(v / pi);
    params_out[(size_t)g * NS + s] = v;
  }
  if (sigma_p_out) {
    double* sp = sigma_p_out + (size_t)g * NS;
    for (int s = lane; s < NS; s += 32) sp[s] = 0.0;
    __syncwarp();
    if (lane < P) sp[D.free_slot[lane]] = have_cov ? sqrt(cov[lane * P + lane]) : CUDART_NAN;
  }
  if (lane == 0) {
    if (S.status[g] == ST_CONVERGED) atomicAdd(S.evals + 1, 1ull);
    atomicAdd(S.evals + 2, (unsigned long long)S.it[g]);
  }
}
#endif  // GM_HOST_TU

#ifdef GM_HOST_TU
// gm_chi2_grad outputs from the tile partials (physical coordinates).
// One warp per galaxy, as k_lm_step: tile sums by the lanes, outputs by lane 0.
__global__ void __launch_bounds__(32 * kLmWarps) k_chi2_grad_finish(const __grid_constant__ DescDev D, int G,
                                                                     const GalGeom* __restrict__ geo,
                                                                     const double* __restrict__ partial,
                                                                     const int* __restrict__ err, double* chi2,
                                                                     double* grad, double* jtj) {
  __shared__ double s_acc[kLmWarps][kMaxAcc];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int g = blockIdx.x * kLmWarps + wl;
  if (g >= G) return;
  const int NS = D.n_slots, P = D.P, NAp = P * (P + 1) / 2, NA = 1 + P + NAp;
  if (*err) {
    // a tile load timed out: some partial sums were never written, so every output is NaN
    for (int e = lane; e < NS * NS; e += 32) {
      if (e == 0) chi2[g] = CUDART_NAN;
      if (grad && e < NS) grad[(size_t)g * NS + e] = CUDART_NAN;
      if (jtj) jtj[(size_t)g * NS * NS + e] = CUDART_NAN;
    }
    return;
  }
  const int n_tiles = geo[g].n_tiles;
  const double* pp = partial + (size_t)geo[g].tile0 * NA;
  for (int e = lane; e < NA; e += 32) {
    double a = 0.0;
    for (int t = 0; t < n_tiles; ++t) a += pp[t * NA + e];
    s_acc[wl][e] = a;
  }
  __syncwarp();
  if (lane != 0) return;
  const double* acc = s_acc[wl];
  chi2[g] = acc[0];
  if (grad) {
    double* gr = grad + (size_t)g * NS;
    for (int s = 0; s < NS; ++s) gr[s] = 0.0;
    for (int f = 0; f < P; ++f) gr[D.free_slot[f]] = -2.0 * acc[1 + f];
  }
  if (jtj) {
    double* J = jtj + (size_t)g * NS * NS;
    for (int s = 0; s < NS * NS; ++s) J[s] = 0.0;
    for (int f = 0; f < P; ++f)
      for (int h = 0; h < P; ++h) J[D.free_slot[f] * NS + D.free_slot[h]] = packed(acc + 1 + P, P, f, h);
  }
}
#endif  // GM_HOST_TU

#ifdef GM_HOST_TU
// ---------------------------------------------------------------------------
// gradient-descent (Adam) fit on the adjoint gradient
// ---------------------------------------------------------------------------
struct AdamState {
  double* m;          // [G][S] first moment, internal coordinates (ln p for log slots)
  double* v;          // [G][S] second moment
  double* scale;      // [G][S] step scale: 1 for log slots, max(|p0|, 1) otherwise
  double* best;       // [G][S] lowest-chi^2 point evaluated (the caller's params)
  double* best_chi2;  // [G]
};

__global__ void k_adam_init(const __grid_constant__ DescDev D, int G, double* params, double* cur, AdamState S) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  const int NS = D.n_slots;
  double* p = params + (size_t)g * NS;
  clamp_slots(D, p);
  for (int s = 0; s < NS; ++s) {
    cur[(size_t)g * NS + s] = p[s];
    S.m[(size_t)g * NS + s] = 0.0;
    S.v[(size_t)g * NS + s] = 0.0;
    S.scale[(size_t)g * NS + s] = D.is_log[s] ? 1.0 : fmax(fabs(p[s]), 1.0);
  }
  S.best_chi2[g] = CUDART_INF;
}

__device__ inline void adam_keep_best(const DescDev& D, int g, const double* cur, double chi2, const AdamState& S) {
  const int NS = D.n_slots;
  if (isfinite(chi2) && chi2 < S.best_chi2[g]) {
    S.best_chi2[g] = chi2;
    for (int s = 0; s < NS; ++s) S.best[(size_t)g * NS + s] = cur[(size_t)g * NS + s];
  }
}

// Keep the evaluated point if it is the best so far, then one Adam step (bias-corrected,
// c1 = 1 - beta1^t, c2 = 1 - beta2^t) in internal coordinates, clamped to the bounds.
__global__ void k_adam_step(const __grid_constant__ DescDev D, int G, double* cur, const double* __restrict__ grad,
                            const double* __restrict__ chi2, AdamState S, double lr, double b1, double b2, double eps,
                            double c1, double c2, int last) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  const int NS = D.n_slots;
  adam_keep_best(D, g, cur, chi2[g], S);
  double* p = cur + (size_t)g * NS;
  for (int f = 0; f < D.P; ++f) {
    const int s = D.free_slot[f];
    const size_t e = (size_t)g * NS + s;
    const double gp = grad[e];
    const double gu = D.is_log[s] ? gp * p[s] : gp;  // d chi^2 / du
    const double m = b1 * S.m[e] + (1.0 - b1) * gu;
    const double v = b2 * S.v[e] + (1.0 - b2) * gu * gu;
    S.m[e] = m;
    S.v[e] = v;
    const double du = lr * S.scale[e] * (m / c1) / (sqrt(v / c2) + eps);
    p[s] = from_u(D, s, to_u(D, s, p[s]) - du);
  }
  clamp_slots(D, p);
  (void)last;
}

// The final evaluation, then the best point in canonical form: an axis ratio
// above 1 rewritten as 1/q with the position angles turned by pi/2 and the
// scale lengths times q (the same image), position angles wrapped to [0, pi).
__global__ void k_adam_finish(const __grid_constant__ DescDev D, int G, const double* cur,
                              const double* __restrict__ chi2, AdamState S) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  adam_keep_best(D, g, cur, chi2[g], S);
  const double pi = 3.14159265358979323846;
  double* p = S.best + (size_t)g * D.n_slots;
  for (int k = 0; k < D.n_canon; ++k) {
    const CanonGroup& cg = D.canon[k];
    const double q = p[cg.q_slot];
    if (!(q > 1.0)) continue;
    for (int i = 0; i < cg.n_scale; ++i) p[cg.scale[i]] *= q;
    for (int i = 0; i < cg.n_pa; ++i) p[cg.pa[i]] += 0.5 * pi;
    p[cg.q_slot] = 1.0 / q;
  }
  for (int s = 0; s < D.n_slots; ++s)
    if (D.is_pa[s]) p[s] -= pi * floor(p[s] / pi);
}
#endif  // GM_HOST_TU

}  // namespace gm
