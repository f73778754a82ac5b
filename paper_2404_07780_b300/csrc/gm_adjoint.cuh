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
// Each pass is three kernels:
//   k_profile_pairs   I_conv of two galaxies per pixel into one pair plane
//   k_adjoint<RESID>  correlate I_conv with P -> M, add the unconvolved part,
//                     write u = w r into a second pair plane; chi^2 and the
//                     unconvolved gradient terms per tile
//   k_adjoint<ADJ>    correlate u with the flipped P -> v, evaluate the
//                     convolved profiles' derivatives at the pixel and
//                     accumulate sum v dI/dp per tile
// Two galaxies share one f32x2 lane pair: the plane holds (galaxy 2k, galaxy
// 2k+1) and the PSF pair is (P_2k[a,b], P_2k+1[a,b]), so every packed FMA does
// useful work although each galaxy has a single channel.  Windows are loaded
// by TMA exactly as in the fused pass (gm_fused.cuh).
#pragma once

#include "gm_fused.cuh"
#include "gm_lm.cuh"

namespace gm {

enum AdjMode { ADJ_RESID = 0, ADJ_GRAD = 1 };

// Pixels of a thread's row of 8 that one iteration of the epilogue loop evaluates.
// Smaller is faster on the 15-parameter bulge+bar+nucleus pass: 7.34 and 7.68 ms for
// 1 and 2 pixels; with strided tiles, 7.84, 8.22 and 8.44 ms for 2, 4 and 8.  The
// instruction footprint outweighs the lost overlap of independent pixels, as the
// kernel has 12 warps per SM to interleave.
constexpr int kEpiPx = 1;

template <int N>
__device__ __forceinline__ void swap_rows(float (&a)[2][N]) {
#pragma unroll
  for (int e = 0; e < N; ++e) {
    const float t = a[0][e];
    a[0][e] = a[1][e];
    a[1][e] = t;
  }
}

// Image D and 1/sigma of 8 consecutive pixels of one stamp row starting at element
// base, n_in of them inside the stamp (n_in may be below 1 or above 8): two float4
// loads per array when the row holds all 8 and both addresses are 16-byte aligned,
// one 8-byte mask load when that is aligned, else element by element within the row.
// Bit k of excl is set for a pixel outside the stamp or masked (mask byte nonzero);
// such a pixel gets D = 0 and 1/sigma = 0 and no sigma is divided for it.
__device__ __forceinline__ void load_row8(const float* __restrict__ image, const float* __restrict__ sigma,
                                          const uint8_t* __restrict__ mask, size_t base, int n_in,
                                          float (&D)[8], float (&isg)[8], unsigned& excl) {
  const float* ip = image + base;
  const float* sp = sigma + base;
  float S[8];
  const bool full = n_in >= 8;
  if (full && ((reinterpret_cast<uintptr_t>(ip) | reinterpret_cast<uintptr_t>(sp)) & 15) == 0) {
    const float4 a0 = __ldg(reinterpret_cast<const float4*>(ip)), a1 = __ldg(reinterpret_cast<const float4*>(ip) + 1);
    const float4 s0 = __ldg(reinterpret_cast<const float4*>(sp)), s1 = __ldg(reinterpret_cast<const float4*>(sp) + 1);
    D[0] = a0.x; D[1] = a0.y; D[2] = a0.z; D[3] = a0.w; D[4] = a1.x; D[5] = a1.y; D[6] = a1.z; D[7] = a1.w;
    S[0] = s0.x; S[1] = s0.y; S[2] = s0.z; S[3] = s0.w; S[4] = s1.x; S[5] = s1.y; S[6] = s1.z; S[7] = s1.w;
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      D[k] = k < n_in ? __ldg(ip + k) : 0.f;
      S[k] = k < n_in ? __ldg(sp + k) : 1.f;
    }
  }
  unsigned ex = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (k >= n_in) ex |= 1u << k;
  if (mask) {
    const uint8_t* mp = mask + base;
    if (full && (reinterpret_cast<uintptr_t>(mp) & 7) == 0) {
      const uint2 mv = __ldg(reinterpret_cast<const uint2*>(mp));
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if ((mv.x >> (8 * k)) & 0xffu) ex |= 1u << k;
        if ((mv.y >> (8 * k)) & 0xffu) ex |= 1u << (k + 4);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (k < n_in && __ldg(mp + k)) ex |= 1u << k;
    }
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const bool off = (ex >> k) & 1u;
    isg[k] = off ? 0.f : 1.f / S[k];
    if (off) D[k] = 0.f;
  }
  excl = ex;
}

// a[k] <- a[(k + S) mod 8]
template <int S>
__device__ __forceinline__ void rotate_left(float (&a)[8]) {
  float t[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) t[k] = a[(k + S) & 7];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = t[k];
}

struct AdjArgs {
  CUtensorMap tmap;          // input pair planes [(G+1)/2][H][2*Wp] FP32
  ChanMap m;
  int P;                     // free slots (accumulator order)
  int conv_acc[kMaxComp][8]; // accumulator of d/dp_k of a convolved comp c (-1 none)
  int unconv_acc[kMaxComp][8];  // same for unconvolved comps
  int nacc;                  // 1 + P
  int G, H, W, Wp, K, cpad, tiles_x, n_tiles, rw, plane;
  const float* image;
  const float* sigma;
  const uint8_t* mask;
  const float* psf;
  const float* cconst;
  float* u_planes;           // RESID: output pair planes of u = w r
  double* partial;           // [G][n_tiles][nacc]: RESID writes [0] chi^2 and unconvolved terms,
                             //                     ADJ adds the convolved terms to a second copy
  int* err;
  unsigned wait_polls;       // polls of a window wait before it gives up (kWaitTries)
  int starve;                // test of the timeout path: block 0 issues no load for its first window
  int off_psf, off_in, off_cc, off_red, off_bar;
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

template <int MODE, int P>
__global__ void __launch_bounds__(128, 3) k_adjoint(const __grid_constant__ AdjArgs A) {
  extern __shared__ __align__(128) unsigned char smem[];
  u64* s_psf = reinterpret_cast<u64*>(smem + A.off_psf);
  float2* s_in = reinterpret_cast<float2*>(smem + A.off_in);
  float* s_cc = reinterpret_cast<float*>(smem + A.off_cc);
  float* s_red = reinterpret_cast<float*>(smem + A.off_red);
  u64* bar = reinterpret_cast<u64*>(smem + A.off_bar);
  int* s_flag = reinterpret_cast<int*>(smem + A.off_bar + 8);
  const ChanMap& m = A.m;
  constexpr int NA = 1 + P;

  const int tid = threadIdx.x;
  const int K = A.K, c = (K - 1) / 2, K2 = K + 1;
  const int n_pairs = (A.G + 1) / 2;
  const int n_items = n_pairs * A.n_tiles;
  // Each block takes a contiguous range of items: the tiles of one galaxy pair run
  // back to back on it, and the pair's PSF and constants are staged once for them.
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
  const int ncc = m.n_comp * kCC;

  int staged = -1;  // galaxy pair whose PSF and constants are in shared memory
  for (int item = it_lo; item < it_hi; ++item) {
    const int gp = item / A.n_tiles, tile = item - gp * A.n_tiles;
    const int g0 = 2 * gp, g1 = 2 * gp + 1;
    const bool has1 = g1 < A.G;
    const int i0 = (tile / A.tiles_x) * kTile, j0 = (tile % A.tiles_x) * kTile;

    __syncthreads();  // the previous item is done with s_psf, s_cc, s_red
    if (gp != staged) {
      staged = gp;
      for (int t = tid; t < 2 * ncc; t += blockDim.x) {
        const int h = t / ncc, e = t - h * ncc;
        const int g = g0 + h;
        s_cc[t] = (g < A.G) ? A.cconst[(size_t)g * ncc + e] : 0.f;
      }
      for (int t = tid; t < K * K2; t += blockDim.x) {
        const int a = t / K2, bb = t - a * K2;
        const int b = bb - A.cpad;
        float v0 = 0.f, v1 = 0.f;
        if (b >= 0 && b < K) {
          // RESID correlates with P, ADJ with P flipped in both axes (the adjoint)
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
    correlate_pairs<1>(acc, s_in, s_psf, 0, A.plane, A.rw, K, row, col0, a_lo, a_hi);
    __syncthreads();  // every warp is done reading the window
    if (tid == 0 && item + 1 < it_hi) {
      adj_issue(A, s_in, bar, item + 1);
      inflight = true;
    }

    // ---- epilogue: this thread's 8 pixels, both galaxies, straight from registers ----
    // Code size decides its speed: eval_component is a large inline body, and a fully
    // unrolled epilogue (2 galaxies x 8 pixels of it) misses the instruction cache.  The
    // galaxies of the pair therefore run as a loop over h that works on row 0 of each
    // [2][.] array and swaps the rows after each galaxy, and the 8 pixels as a loop of
    // kEpiPx-pixel chunks that works on entries 0..kEpiPx-1 and rotates the row by kEpiPx
    // after each chunk; every index stays a compile-time constant (registers), and both
    // the swaps and the full turn of rotations leave the arrays in their starting order.
    float red[2][NA];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int e = 0; e < NA; ++e) red[h][e] = 0.f;
    const int i = i0 + row;
    float vv[2][8];
#pragma unroll
    for (int rx = 0; rx < 8; ++rx) unpack2(acc[0][rx], vv[0][rx], vv[1][rx]);
    // Each gradient term is a sum over pixels of a weight times dI/dp_k.  The
    // accumulator of (component, k) is run-time data, and a compare-select over the
    // free parameters keeps red[] in registers; it is paid once per component and
    // galaxy: the thread first sums each derivative over its 8 pixels.
    auto scatter = [&](const int (&acc_of)[8], int np, const float (&sd)[8]) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (k >= np) break;
        const int f = acc_of[k];
#pragma unroll
        for (int ff = 0; ff < P; ++ff)
          if (ff == f) red[0][1 + ff] += sd[k];
      }
    };
    // sum over the 8 pixels of wt * dI_cm/dp_k for the components cm that are (not) convolved
    auto deriv_sums = [&](float (&wt)[2][8], bool conv) {
      for (int cm = 0; cm < m.n_comp; ++cm) {
        if ((m.conv[cm] != 0) != conv) continue;
        const int np = m.np[cm];
        const float* cc = s_cc + cm * kCC;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          if (h == 0 || has1) {
            float sd[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
            for (int rb = 0; rb < 8; rb += kEpiPx) {
#pragma unroll
              for (int q = 0; q < kEpiPx; ++q) {
                const int j = j0 + col0 + rb + q;
                if (i < A.H && j < A.W) {
                  float d[8];
                  eval_component(m.kind[cm], cc + h * ncc, i, j, d);
#pragma unroll
                  for (int k = 0; k < 8; ++k)
                    if (k < np) sd[k] = fmaf(wt[0][q], d[k], sd[k]);
                }
              }
              rotate_left<kEpiPx>(wt[0]);
            }
            scatter(conv ? A.conv_acc[cm] : A.unconv_acc[cm], np, sd);
          }
          swap_rows(wt);
          swap_rows(red);
        }
      }
    };
    if (MODE == ADJ_RESID) {
      float wr[2][8];  // w r = (D - M) / sigma^2 per pixel; 0 outside the stamp or masked
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        const int g = g0 + h;
        // D and 1/sigma of this galaxy's 8 pixels, loaded before the pixel loop
        float Dv[8], Iv[8];
        unsigned excl = 0xffu;  // bit k: pixel k is not used (masked, outside the stamp)
        if ((h == 0 || has1) && i < A.H) {
          load_row8(A.image, A.sigma, A.mask, ((size_t)g * A.H + i) * A.W + j0 + col0, A.W - (j0 + col0), Dv, Iv,
                    excl);
        } else {
#pragma unroll
          for (int k = 0; k < 8; ++k) Dv[k] = Iv[k] = 0.f;
        }
#pragma unroll 1
        for (int rb = 0; rb < 8; rb += kEpiPx) {
#pragma unroll
          for (int q = 0; q < kEpiPx; ++q) {
            const int j = j0 + col0 + rb + q;
            float uu = 0.f;
            if (!((excl >> q) & 1u)) {
              float Mv = vv[0][q];
              for (int cm = 0; cm < m.n_comp; ++cm) {
                if (m.conv[cm]) continue;
                float d[8];
                Mv += eval_component(m.kind[cm], s_cc + h * ncc + cm * kCC, i, j, d);
              }
              const float rr = (Dv[q] - Mv) * Iv[q];
              red[0][0] = fmaf(rr, rr, red[0][0]);
              uu = rr * Iv[q];
            }
            wr[0][q] = uu;
          }
          rotate_left<kEpiPx>(vv[0]);
          rotate_left<kEpiPx>(wr[0]);
          rotate_left<kEpiPx>(Dv);
          rotate_left<kEpiPx>(Iv);
          excl >>= kEpiPx;
        }
        swap_rows(vv);
        swap_rows(wr);
        swap_rows(red);
      }
#pragma unroll
      for (int rx = 0; rx < 8; ++rx) {
        const int j = j0 + col0 + rx;
        if (i < A.H && j < A.Wp)
          reinterpret_cast<float2*>(A.u_planes)[((size_t)gp * A.H + i) * A.Wp + j] = make_float2(wr[0][rx], wr[1][rx]);
      }
      deriv_sums(wr, false);
    } else {
      deriv_sums(vv, true);
    }
    // ---- block reduction: warp sums (recursive halving), then across the 4 warps, FP64 per tile ----
    {
      float flat[2 * NA];
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int e = 0; e < NA; ++e) flat[h * NA + e] = red[h][e];
      warp_sum_scatter(flat, lane, [&](int t, float v) { s_red[wig * 2 * NA + t] = v; });
    }
    __syncthreads();
    for (int t = tid; t < 2 * NA; t += blockDim.x) {
      const int h = t / NA, e = t - h * NA;
      const int g = g0 + h;
      if (g >= A.G) continue;
      double s = 0.0;
      for (int w = 0; w < 4; ++w) s += (double)s_red[(w * 2 + h) * NA + e];
      A.partial[((size_t)g * A.n_tiles + tile) * NA + e] = s;
    }
  }
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
