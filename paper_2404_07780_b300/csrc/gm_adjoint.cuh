// gm_adjoint.cuh -- chi^2 and its gradient by the adjoint of the PSF
// correlation: two single-channel correlations per pass, whatever the number
// of free parameters.
//
// With M = P (*) I_conv + I_unconv (cross-correlation with zero padding) and
// r = D - M, w = Omega / sigma^2 (Eq. chinu of arxiv 2404.07780):
//   d chi^2 / dp = -2 sum_pix w r dM/dp
//                = -2 [ sum_pix' (dI_conv/dp)(pix') v(pix') + sum_pix w r dI_unconv/dp ],
//   v = P^T (w r),
// and the adjoint of the same-size zero-padded correlation is the same-size
// zero-padded correlation with the PSF flipped in both axes
// (sum_ab P[a,b] u[i-a+c, j-b+c] = sum_a'b' P[K-1-a', K-1-b'] u[i+a'-c, j+b'-c]).
//
// Each pass is five kernels:
//   k_profile_pairs   I_conv of two galaxies per pixel into one pair plane
//   k_adjoint<RESID>  correlate the I_conv plane with the pair's PSFs -> M_conv plane
//   k_adj_resid       M = M_conv + the unconvolved components, u = w r written over
//                     M_conv; chi^2 and sum u dI_unconv/dp per tile
//   k_adjoint<GRAD>   correlate the u plane with the PSFs flipped -> v plane
//   k_adj_deriv       the convolved profiles' derivatives at every pixel: sum
//                     v dI_conv/dp per tile
// The correlations are bound by the FMA pipe, the pixel kernels by instruction
// issue (profile code per pixel, component and galaxy); kept apart, each runs at
// its own limit with the registers and occupancy it needs (inside the
// correlation kernel the epilogues doubled its instructions per window and held
// the registers of both phases).  The planes between them cost one write and one
// read of 8 bytes per pixel pair.
// Two galaxies share one f32x2 lane pair: the plane holds (galaxy 2k, galaxy
// 2k+1) and the PSF pair is (P_2k[a,b], P_2k+1[a,b]), so every packed FMA does
// useful work although each galaxy has a single channel.  Windows are loaded
// by TMA exactly as in the fused pass (gm_fused.cuh).
#pragma once

#include "gm_fused.cuh"
#include "gm_lm.cuh"

namespace gm {

enum AdjMode { ADJ_RESID = 0, ADJ_GRAD = 1 };

template <int N>
__device__ __forceinline__ void swap_rows(float (&a)[2][N]) {
#pragma unroll
  for (int e = 0; e < N; ++e) {
    const float t = a[0][e];
    a[0][e] = a[1][e];
    a[1][e] = t;
  }
}

// a[k] <- a[(k + S) mod N]
template <int S, int N>
__device__ __forceinline__ void rotate_left(float (&a)[N]) {
  float t[N];
#pragma unroll
  for (int k = 0; k < N; ++k) t[k] = a[(k + S) % N];
#pragma unroll
  for (int k = 0; k < N; ++k) a[k] = t[k];
}

struct AdjArgs {
  CUtensorMap tmap;          // input pair planes [(G+1)/2][H][2*Wp] FP32
  int G, H, W, Wp, K, cpad, tiles_x, n_tiles, rw, plane;
  const float* psf;
  float* out_planes;         // output pair planes [(G+1)/2][H][Wp] float2
  int* err;
  unsigned wait_polls;       // polls of a window wait before it gives up (kWaitTries)
  int starve;                // test of the timeout path: block 0 issues no load for its first window
  int off_psf, off_in, off_bar;
};

#ifdef GM_HOST_TU
// I_conv of galaxies 2k and 2k+1 (the second zero past the end) into pair plane k.
__global__ void __launch_bounds__(256) k_profile_pairs(const __grid_constant__ ProfileArgs A) {
  __shared__ float s_cc[2][kMaxComp * kCC];
  const ChanMap& m = A.m;
  const int tid = threadIdx.x;
  const int per_pair = (A.H * A.Wp + 255) / 256;
  const int n_pairs = (A.G + 1) / 2;
  for (int blk = blockIdx.x; blk < n_pairs * per_pair; blk += gridDim.x) {
    const int gp = blk / per_pair, chunk = blk - gp * per_pair;
    __syncthreads();
    for (int t = tid; t < 2 * m.n_comp * kCC; t += 256) {
      const int h = t / (m.n_comp * kCC), e = t - h * (m.n_comp * kCC);
      const int g = 2 * gp + h;
      s_cc[h][e] = (g < A.G) ? A.cconst[(size_t)g * m.n_comp * kCC + e] : 0.f;
    }
    __syncthreads();
    const int pix = chunk * 256 + tid;
    if (pix >= A.H * A.Wp) continue;
    const int i = pix / A.Wp, j = pix - (pix / A.Wp) * A.Wp;
    float v[2] = {0.f, 0.f};
    if (j < A.W) {
      for (int h = 0; h < 2; ++h) {
        if (2 * gp + h >= A.G) continue;
        for (int cm = 0; cm < m.n_comp; ++cm) {
          if (!m.conv[cm]) continue;
          float d[8];
          v[h] += eval_component(m.kind[cm], s_cc[h] + cm * kCC, i, j, d);
        }
      }
    }
    reinterpret_cast<float2*>(A.planes)[((size_t)gp * A.H + i) * A.Wp + j] = make_float2(v[0], v[1]);
  }
}
#endif  // GM_HOST_TU

__device__ __forceinline__ void adj_issue(const AdjArgs& A, float2* s_in, u64* bar, int item) {
  const int gp = item / A.n_tiles, tile = item - gp * A.n_tiles;
  const int i0 = (tile / A.tiles_x) * kTile, j0 = (tile % A.tiles_x) * kTile;
  const int c = (A.K - 1) / 2;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_expect_tx(bar, (unsigned)(kTile + A.K - 1) * A.rw * 8u);
  tma_load_3d(s_in, &A.tmap, 2 * (j0 - c - A.cpad), i0 - c, gp, bar);
}

// Correlation of one pair plane with the pair's PSFs (RESID: P as given; GRAD: P
// flipped in both axes, the adjoint), written to the output pair plane.  Items
// are (galaxy pair, 32 x 32 tile); each block takes a contiguous range of them,
// so a pair's tiles run back to back and its PSF pair is staged once for them.
template <int MODE>
__global__ void __launch_bounds__(128, 4) k_adjoint(const __grid_constant__ AdjArgs A) {
  extern __shared__ __align__(128) unsigned char smem[];
  u64* s_psf = reinterpret_cast<u64*>(smem + A.off_psf);
  float2* s_in = reinterpret_cast<float2*>(smem + A.off_in);
  u64* bar = reinterpret_cast<u64*>(smem + A.off_bar);
  int* s_flag = reinterpret_cast<int*>(smem + A.off_bar + 8);

  const int tid = threadIdx.x;
  const int K = A.K, c = (K - 1) / 2, K2 = K + 1;
  const int n_pairs = (A.G + 1) / 2;
  const int n_items = n_pairs * A.n_tiles;
  const int it_lo = (int)((long long)blockIdx.x * n_items / gridDim.x);
  const int it_hi = (int)((long long)(blockIdx.x + 1) * n_items / gridDim.x);
  if (it_lo >= it_hi) return;
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *s_flag = 0;
  }
  __syncthreads();
  bool inflight = false;  // thread 0: a window load is outstanding on the mbarrier
  if (tid == 0 && !(A.starve && blockIdx.x == 0)) {
    adj_issue(A, s_in, bar, it_lo);
    inflight = true;
  }
  unsigned phase = 0;
  const int lane = tid & 31, wig = tid >> 5;
  const int row = wig * 8 + (lane & 7), col0 = (lane >> 3) * 8;
  const int row0 = wig * 8;

  int staged = -1;  // galaxy pair whose PSF pair is in shared memory
  for (int item = it_lo; item < it_hi; ++item) {
    const int gp = item / A.n_tiles, tile = item - gp * A.n_tiles;
    const int g0 = 2 * gp, g1 = 2 * gp + 1;
    const bool has1 = g1 < A.G;
    const int i0 = (tile / A.tiles_x) * kTile, j0 = (tile % A.tiles_x) * kTile;

    __syncthreads();  // the previous item is done with s_psf
    if (gp != staged) {
      staged = gp;
      for (int t = tid; t < K * K2; t += blockDim.x) {
        const int a = t / K2, bb = t - a * K2;
        const int b = bb - A.cpad;
        float v0 = 0.f, v1 = 0.f;
        if (b >= 0 && b < K) {
          const int src = (MODE == ADJ_RESID) ? a * K + b : (K - 1 - a) * K + (K - 1 - b);
          v0 = A.psf[(size_t)g0 * K * K + src];
          v1 = has1 ? A.psf[(size_t)g1 * K * K + src] : 0.f;
        }
        s_psf[t] = pack2(v0, v1);
      }
    }
    const int a_lo = max(0, c - i0 - row0 - 7);
    const int a_hi = min(K, c - i0 + A.H - row0);

    if (tid == 0) {
      if (mbar_wait_bounded(bar, phase, A.wait_polls)) inflight = false;
      else *s_flag = 1;
    }
    __syncthreads();
    if (*s_flag) {
      if (tid == 0) {
        atomicExch(A.err, 1);
        if (inflight) mbar_wait_bounded(bar, phase);  // let the copy in flight land before leaving
      }
      return;
    }
    mbar_try_wait(bar, phase);
    phase ^= 1u;
    u64 acc[1][8];
    correlate_pairs<1>(acc, s_in, s_psf, 0, A.plane, A.rw, K, row, col0, a_lo, a_hi, col_all(K));
    __syncthreads();  // every warp is done reading the window
    if (tid == 0 && item + 1 < it_hi) {
      adj_issue(A, s_in, bar, item + 1);
      inflight = true;
    }
    const int i = i0 + row;
    if (i < A.H) {
      float2* out = reinterpret_cast<float2*>(A.out_planes) + ((size_t)gp * A.H + i) * A.Wp;
#pragma unroll
      for (int rx = 0; rx < 8; ++rx) {
        const int j = j0 + col0 + rx;
        float x, y;
        unpack2(acc[0][rx], x, y);
        if (j < A.Wp) out[j] = make_float2(x, y);
      }
    }
  }
}

// Arguments of k_adj_resid and k_adj_deriv (equal stamps).
struct PixArgs {
  ChanMap m;
  int acc_of[kMaxComp][8];    // k_adj_resid: accumulator of d/dp_k of an unconvolved comp c, k_adj_deriv:
                              // of a convolved one (-1 none)
  int G, H, W, Wp, tiles_x, n_tiles;
  const float* image;
  const float* sigma;
  const uint8_t* mask;
  const float* cconst;        // [G][n_comp][kCC]
  float* planes;              // [(G+1)/2][H][Wp] float2: k_adj_resid reads M_conv and writes u = w r in
                              // place; k_adj_deriv reads v
  double* partial;            // [G][pix_parts(H, W)][1 + P]: the galaxy's sums over each part of its stamp
};

constexpr int kPixThreads = 256;
constexpr int kPixPerThread = 4;  // pixels per thread in one chunk of a pixel kernel
constexpr int kPixPart = 2 * kPixThreads * kPixPerThread;  // pixels of a stamp per block (FP32 sums of <= 8
                                                           // terms per thread before the block sum)

__host__ __device__ inline int pix_parts(int H, int W) { return (H * W + kPixPart - 1) / kPixPart; }

// The pair's sums over one part of the stamp into its partials: warp sums by
// recursive halving, then the compensated sum over the warps in warp order
// (deterministic).
template <int NA>
__device__ __forceinline__ void pix_pair_sums(const PixArgs& A, float (&red)[2][NA], float* s_red, int g0, int part,
                                              int n_parts) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float flat[2 * NA];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int e = 0; e < NA; ++e) flat[h * NA + e] = red[h][e];
  warp_sum_scatter(flat, lane, [&](int t, float v) { s_red[warp * 2 * NA + t] = v; });
  __syncthreads();
  for (int t = tid; t < 2 * NA; t += kPixThreads) {
    const int h = t / NA, e = t - h * NA;
    const int g = g0 + h;
    if (g >= A.G) continue;
    A.partial[((size_t)g * n_parts + part) * NA + e] = compensated_sum(s_red + h * NA + e, 2 * NA, kPixThreads / 32);
  }
}

// red[0][1 + f] += sd[k] for the accumulator f of each of the component's np derivatives
// (a compare-select over the P free parameters keeps red in registers)
template <int P, int NA>
__device__ __forceinline__ void scatter_sums(float (&red)[2][NA], const int (&acc_of)[8], int np,
                                             const float (&sd)[8]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if (k >= np) break;
    const int f = acc_of[k];
#pragma unroll
    for (int ff = 0; ff < P; ++ff)
      if (ff == f) red[0][1 + ff] += sd[k];
  }
}

// For the components with conv[cm] == conv: red[h][1 + f] += sum over the chunk's
// pixels of wt[h][q] dI_cm/dp_k (f the accumulator of slot k).  The galaxies run as a
// loop over row 0 of each [2][.] array, the rows swapped after each galaxy, and the
// pixels as a loop that rotates row 0 (compile-time indices: registers; one copy of
// the profile code).
template <int P, int NA>
__device__ __forceinline__ void chunk_deriv_sums(const PixArgs& A, const float* s_cc, int ncc, bool has1,
                                                 const int (&pi)[kPixPerThread], const int (&pj)[kPixPerThread],
                                                 float (&wt)[2][kPixPerThread], float (&red)[2][NA], bool conv) {
  const ChanMap& m = A.m;
  for (int cm = 0; cm < m.n_comp; ++cm) {
    if ((m.conv[cm] != 0) != conv) continue;
    const int np = m.np[cm];
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      if (h == 0 || has1) {
        const float* cc = s_cc + h * ncc + cm * kCC;
        float sd[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
        for (int q = 0; q < kPixPerThread; ++q) {
          if (pi[q] >= 0) {
            float d[8];
            eval_component(m.kind[cm], cc, pi[q], pj[q], d);
#pragma unroll
            for (int k = 0; k < 8; ++k)
              if (k < np) sd[k] = fmaf(wt[0][0], d[k], sd[k]);
          }
          rotate_left<1>(wt[0]);
        }
        scatter_sums<P>(red, A.acc_of[cm], np, sd);
      }
      swap_rows(wt);
      swap_rows(red);
    }
  }
}

// chunk_deriv_sums for a lone flat sky (ChanMap::sky_comp): its one derivative is
// 1 at every pixel, so the sums are the weights' own, added in the same order.
template <int P, int NA>
__device__ __forceinline__ void chunk_sky_sums(const PixArgs& A, int sky, bool has1, const int (&pi)[kPixPerThread],
                                               float (&wt)[2][kPixPerThread], float (&red)[2][NA]) {
#pragma unroll 1
  for (int h = 0; h < 2; ++h) {
    if (h == 0 || has1) {
      float sd[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
      for (int q = 0; q < kPixPerThread; ++q) {
        if (pi[q] >= 0) sd[0] = fmaf(wt[0][0], 1.f, sd[0]);
        rotate_left<1>(wt[0]);
      }
      scatter_sums<P>(red, A.acc_of[sky], 1, sd);
    }
    swap_rows(wt);
    swap_rows(red);
  }
}

// Residuals of one galaxy pair, one block of 256 threads per kPixPart pixels of the
// stamp, in chunks of 4 pixels per thread (pixel p, row-major, on thread p % 256:
// each warp reads consecutive pixels): M = M_conv + the unconvolved components,
// r = D - M, u = w r (0 for masked pixels) written over M_conv, and the pair's
// chi^2 and sum u dI_unconv/dp.
template <int P>
__global__ void __launch_bounds__(kPixThreads, 2) k_adj_resid(const __grid_constant__ PixArgs A) {
  constexpr int NA = 1 + P;
  __shared__ float s_cc[2 * kMaxComp * kCC];
  __shared__ float s_red[(kPixThreads / 32) * 2 * NA];
  const ChanMap& m = A.m;
  const int tid = threadIdx.x;
  const int ncc = m.n_comp * kCC;
  const int HW = A.H * A.W, n_parts = pix_parts(A.H, A.W);
  const int gp = blockIdx.x / n_parts, part = blockIdx.x - gp * n_parts;
  const int g0 = 2 * gp;
  const bool has1 = g0 + 1 < A.G;
  const int p_end = min(HW, (part + 1) * kPixPart);
  float2* planes = reinterpret_cast<float2*>(A.planes);
  for (int t = tid; t < 2 * ncc; t += kPixThreads) s_cc[t] = (t < ncc || has1) ? A.cconst[(size_t)g0 * ncc + t] : 0.f;
  if ((A.W & 1) && part == 0)  // the pad column of an odd width: u = 0, the zero padding of the next correlation
    for (int i = tid; i < A.H; i += kPixThreads) planes[((size_t)gp * A.H + i) * A.Wp + A.W] = make_float2(0.f, 0.f);
  __syncthreads();
  float red[2][NA];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int e = 0; e < NA; ++e) red[h][e] = 0.f;
  for (int p0 = part * kPixPart; p0 < p_end; p0 += kPixThreads * kPixPerThread) {
    // every load of the chunk first (one memory latency for all of them), then the arithmetic
    int pi[kPixPerThread], pj[kPixPerThread];
    float2 mc[kPixPerThread];
    float Dv[2][kPixPerThread], Sv[2][kPixPerThread];
    bool use[2][kPixPerThread];
#pragma unroll
    for (int q = 0; q < kPixPerThread; ++q) {
      const int p = p0 + tid + q * kPixThreads;
      const bool in = p < p_end;
      const int i = in ? p / A.W : 0, j = in ? p - i * A.W : 0;
      pi[q] = in ? i : -1;
      pj[q] = j;
      mc[q] = in ? planes[((size_t)gp * A.H + i) * A.Wp + j] : make_float2(0.f, 0.f);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const size_t gpx = (size_t)(g0 + h) * HW + p;
        use[h][q] = in && (h == 0 || has1);
        Dv[h][q] = use[h][q] ? __ldg(A.image + gpx) : 0.f;
        Sv[h][q] = use[h][q] ? __ldg(A.sigma + gpx) : 1.f;
        if (use[h][q] && A.mask && __ldg(A.mask + gpx)) use[h][q] = false;
      }
    }
    float uu[2][kPixPerThread];
#pragma unroll
    for (int q = 0; q < kPixPerThread; ++q) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uu[h][q] = 0.f;
        if (!use[h][q]) continue;
        float Mv = h ? mc[q].y : mc[q].x;
        if (m.sky_comp >= 0) {  // a lone flat sky: its level, without evaluating the component
          Mv += s_cc[h * ncc + m.sky_comp * kCC + 8];
        } else {
          for (int cm = 0; cm < m.n_comp; ++cm) {
            if (m.conv[cm]) continue;
            float d[8];
            Mv += eval_component(m.kind[cm], s_cc + h * ncc + cm * kCC, pi[q], pj[q], d);
          }
        }
        const float isg = 1.f / Sv[h][q];
        const float rr = (Dv[h][q] - Mv) * isg;
        red[h][0] = fmaf(rr, rr, red[h][0]);
        uu[h][q] = rr * isg;
      }
      if (pi[q] >= 0) planes[((size_t)gp * A.H + pi[q]) * A.Wp + pj[q]] = make_float2(uu[0][q], uu[1][q]);
    }
    if (m.sky_comp >= 0) chunk_sky_sums<P>(A, m.sky_comp, has1, pi, uu, red);
    else if (m.any_unconv) chunk_deriv_sums<P>(A, s_cc, ncc, has1, pi, pj, uu, red, false);
  }
  pix_pair_sums(A, red, s_red, g0, part, n_parts);
}

// sum over the stamp of v dI_conv/dp for both galaxies of a pair, one block of 256
// threads per kPixPart pixels of the stamp, in chunks of 4 pixels per thread as in
// k_adj_resid.  Each thread keeps its 2 (1 + P) sums in a row of shared memory
// indexed by parameter (an odd row pitch: the lanes of a warp hit distinct banks),
// so adding a derivative's sum costs one shared-memory update instead of a
// compare-select over the P accumulators.
template <int P>
__global__ void __launch_bounds__(kPixThreads, 3) k_adj_deriv(const __grid_constant__ PixArgs A) {
  constexpr int NA = 1 + P, RP = 2 * NA + 1;
  __shared__ float s_cc[2 * kMaxComp * kCC];
  __shared__ float s_red[(kPixThreads / 32) * 2 * NA];
  __shared__ float s_sum[kPixThreads * RP];
  const ChanMap& m = A.m;
  const int tid = threadIdx.x;
  const int ncc = m.n_comp * kCC;
  const int HW = A.H * A.W, n_parts = pix_parts(A.H, A.W);
  const int gp = blockIdx.x / n_parts, part = blockIdx.x - gp * n_parts;
  const int g0 = 2 * gp;
  const bool has1 = g0 + 1 < A.G;
  const int p_end = min(HW, (part + 1) * kPixPart);
  for (int t = tid; t < 2 * ncc; t += kPixThreads) s_cc[t] = (t < ncc || has1) ? A.cconst[(size_t)g0 * ncc + t] : 0.f;
  float* my = s_sum + tid * RP;
#pragma unroll
  for (int e = 0; e < 2 * NA; ++e) my[e] = 0.f;
  __syncthreads();
  for (int p0 = part * kPixPart; p0 < p_end; p0 += kPixThreads * kPixPerThread) {
    int pi[kPixPerThread], pj[kPixPerThread];
    float vv[2][kPixPerThread];
#pragma unroll
    for (int q = 0; q < kPixPerThread; ++q) {
      const int p = p0 + tid + q * kPixThreads;
      const bool in = p < p_end;
      const int i = in ? p / A.W : 0, j = in ? p - i * A.W : 0;
      pi[q] = in ? i : -1;
      pj[q] = j;
      const float2 v = in ? reinterpret_cast<const float2*>(A.planes)[((size_t)gp * A.H + i) * A.Wp + j]
                          : make_float2(0.f, 0.f);
      vv[0][q] = v.x;
      vv[1][q] = v.y;
    }
    for (int cm = 0; cm < m.n_comp; ++cm) {
      if (!m.conv[cm]) continue;
      const int np = m.np[cm];
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        if (h == 0 || has1) {
          const float* cc = s_cc + h * ncc + cm * kCC;
          float sd[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
          for (int q = 0; q < kPixPerThread; ++q) {
            if (pi[q] >= 0) {
              float d[8];
              eval_component(m.kind[cm], cc, pi[q], pj[q], d);
#pragma unroll
              for (int k = 0; k < 8; ++k)
                if (k < np) sd[k] = fmaf(vv[0][0], d[k], sd[k]);
            }
            rotate_left<1>(vv[0]);
          }
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            if (k >= np) break;
            const int f = A.acc_of[cm][k];
            if (f >= 0) my[h * NA + 1 + f] += sd[k];
          }
        }
        swap_rows(vv);
      }
    }
  }
  float red[2][NA];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int e = 0; e < NA; ++e) red[h][e] = my[h * NA + e];
  pix_pair_sums(A, red, s_red, g0, part, n_parts);
}

#ifdef GM_HOST_TU
// chi^2 and d chi^2/dp = -2 (unconvolved + convolved terms) from the two passes' partials.
// A tile load that timed out (*err set) leaves partial sums unwritten: every output is NaN then.
__global__ void k_adjoint_finish(const __grid_constant__ DescDev D, int G, int n_tiles,
                                 const double* __restrict__ part_resid, const double* __restrict__ part_adj,
                                 const int* __restrict__ err, double* chi2, double* grad) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  const int P = D.P, n_slots = D.n_slots;
  if (*err) {
    chi2[g] = CUDART_NAN;
    if (grad)
      for (int s = 0; s < n_slots; ++s) grad[(size_t)g * n_slots + s] = CUDART_NAN;
    return;
  }
  const int* free_slot = D.free_slot;
  const int NA = 1 + P;
  double acc[1 + kMaxFree];
  for (int e = 0; e < NA; ++e) acc[e] = 0.0;
  for (int t = 0; t < n_tiles; ++t)
    for (int e = 0; e < NA; ++e)
      acc[e] += part_resid[((size_t)g * n_tiles + t) * NA + e] + (e > 0 ? part_adj[((size_t)g * n_tiles + t) * NA + e] : 0.0);
  chi2[g] = acc[0];
  if (grad) {
    for (int s = 0; s < n_slots; ++s) grad[(size_t)g * n_slots + s] = 0.0;
    for (int f = 0; f < P; ++f) grad[(size_t)g * n_slots + free_slot[f]] = -2.0 * acc[1 + f];
  }
}
#endif  // GM_HOST_TU

}  // namespace gm
