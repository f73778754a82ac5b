// gm_fused.cuh -- the fused per-tile kernel: light profiles + analytic
// derivatives on the tile and its PSF halo (in shared memory), multi-channel
// direct PSF correlation in FP32 (packed f32x2 FMAs), residual, weights and the
// per-tile reduction of chi^2, J^T W r and J^T W J.
//
// Work item = (galaxy, 32x32 output tile).  A persistent grid strides over the
// items of the galaxies still being fitted.  Per item:
//   1. PSF (as (p, p) pairs), per-galaxy constants and slot scales -> smem.
//   2. Profile phase: every pixel of the (32+K-1)^2 input window that lies in
//      the stamp gets the summed convolved components (channel 0) and one
//      derivative channel per free parameter of a convolved component; zero
//      outside the stamp (the zero padding of conv2d "same").  Channels are
//      stored as interleaved pairs so that one f32x2 FMA serves two channels.
//   3. Correlation: each thread owns 8 adjacent output pixels of one row and 2
//      channel pairs; for every PSF row it slides a 10-entry register window
//      along the input row (one 16-byte shared load per 2 taps per pair, one
//      16-byte PSF load per 2 taps) and issues 16 f32x2 FMAs per tap pair and
//      channel pair.  PSF rows whose input rows lie wholly outside the stamp
//      for the warp are skipped.
//   4. Unconvolved components (the sky) are added at the output pixels.
//   5. NORMAL mode: r = D - M, w = Omega/sigma^2 per pixel, FP32 accumulation
//      of chi^2, J^T W r and J^T W J per thread, warp shuffles, a cross-warp
//      sum, one FP64 partial per tile written to global memory.
//      MODEL mode: the model (and per-component images) written out.
//
// The correlation is M[i,j] = sum_ab P[a,b] I[i+a-c, j+b-c] (cross-correlation,
// torch conv2d semantics, App. C of arxiv 2404.07780).
#pragma once

#include "gm_profiles.cuh"

namespace gm {

constexpr int kTile = 32;          // output tile is kTile x kTile
constexpr int kTilePix = kTile * kTile;
constexpr int kMaxConvCh = 8;      // channels one pass correlates (4 pairs)
constexpr int kGroupThreads = 128; // threads per channel-pair group (32 rows x 4 col-blocks)

enum Mode { MODE_MODEL = 0, MODE_NORMAL = 1 };

struct FusedArgs {
  // model description (uniform over the batch)
  int n_comp;
  int kind[kMaxComp];
  int conv[kMaxComp];
  int np[kMaxComp];
  int slot[kMaxComp][8];         // parameter k of comp c -> slot
  int chan[kMaxComp][8];         // d/dp_k of comp c -> s_out channel (-1: not needed)
  int comp_chan[kMaxComp];       // MODEL mode: channel holding comp c's own image (-1: none)
  int any_unconv;
  int nch_conv;                  // correlated channels (<= kMaxConvCh)
  int ncp;                       // channel pairs = ceil(nch_conv / 2)
  int nch_tot;                   // channels in s_out
  int n_slots;
  int nacc;                      // accumulators per tile (NORMAL)
  // batch
  int G, H, W, K, tiles_x, n_tiles, rw;
  const float* image;
  const float* sigma;
  const uint8_t* mask;
  const float* psf;
  // per-galaxy constants
  const float* cconst;           // [G][n_comp][kCC]
  const float* scale;            // [G][n_slots]
  // work list: galaxies list[0 .. *count); list == nullptr -> all G
  const int* list;
  const int* count;
  // outputs
  double* partial;               // [G][n_tiles][nacc]
  float* model_out;              // [G][H][W]
  float* comp_out;               // [G][n_comp][H][W] or nullptr
  // shared-memory carve-up (bytes)
  int off_psf, off_in, off_out, off_cc, off_scale, off_red;
};

typedef unsigned long long u64;

__device__ __forceinline__ u64 ffma2(u64 a, u64 b, u64 c) {
  u64 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

__device__ __forceinline__ u64 pack2(float x, float y) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}

__device__ __forceinline__ void unpack2(u64 v, float& x, float& y) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(v));
}

// One 2-tap chunk of the sliding-window correlation.  R is the ring rotation:
// window element e (input column b + e relative to the thread's first column)
// lives in w[q][(2R + e) % 10].  Elements 0..7 are present on entry; elements 8
// and 9 are loaded here.
template <int CP, int R>
__device__ __forceinline__ void corr_chunk(u64 (&acc)[CP][8], u64 (&w)[CP][10],
                                           const float2* const (&irow)[CP], const u64* prow, int b) {
  constexpr int L = (2 * R + 8) % 10;
#pragma unroll
  for (int q = 0; q < CP; ++q) {
    const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(irow[q] + b + 8);
    w[q][L] = v.x;
    w[q][L + 1] = v.y;
  }
  const ulonglong2 pp = *reinterpret_cast<const ulonglong2*>(prow + b);
#pragma unroll
  for (int q = 0; q < CP; ++q) {
#pragma unroll
    for (int rx = 0; rx < 8; ++rx) acc[q][rx] = ffma2(pp.x, w[q][(2 * R + rx) % 10], acc[q][rx]);
#pragma unroll
    for (int rx = 0; rx < 8; ++rx) acc[q][rx] = ffma2(pp.y, w[q][(2 * R + 1 + rx) % 10], acc[q][rx]);
  }
}

// Correlate CP channel pairs for one thread's 8 output pixels over PSF rows
// [a_lo, a_hi).  s_in is [ncp][HH][rw] float2, s_psf is [K][K+1] (p, p) pairs.
template <int CP>
__device__ __forceinline__ void correlate_pairs(u64 (&acc)[CP][8], const float2* s_in, const u64* s_psf,
                                                int cp0, int HH, int rw, int K, int row, int col0,
                                                int a_lo, int a_hi) {
#pragma unroll
  for (int q = 0; q < CP; ++q)
#pragma unroll
    for (int rx = 0; rx < 8; ++rx) acc[q][rx] = 0ull;
  const int K2 = K + 1;
  const int nch = K2 >> 1;        // 2-tap chunks per PSF row
  const int nsc = nch / 5;        // full 5-chunk rotations
  const int tail = nch - 5 * nsc;
  for (int a = a_lo; a < a_hi; ++a) {
    const u64* prow = s_psf + a * K2;
    const float2* irow[CP];
#pragma unroll
    for (int q = 0; q < CP; ++q) irow[q] = s_in + ((size_t)(cp0 + q) * HH + row + a) * rw + col0;
    u64 w[CP][10];
#pragma unroll
    for (int q = 0; q < CP; ++q) {
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(irow[q] + e);
        w[q][e] = v.x;
        w[q][e + 1] = v.y;
      }
    }
    int b = 0;
    for (int sc = 0; sc < nsc; ++sc) {
      corr_chunk<CP, 0>(acc, w, irow, prow, b);
      corr_chunk<CP, 1>(acc, w, irow, prow, b + 2);
      corr_chunk<CP, 2>(acc, w, irow, prow, b + 4);
      corr_chunk<CP, 3>(acc, w, irow, prow, b + 6);
      corr_chunk<CP, 4>(acc, w, irow, prow, b + 8);
      b += 10;
    }
    if (tail > 0) corr_chunk<CP, 0>(acc, w, irow, prow, b);
    if (tail > 1) corr_chunk<CP, 1>(acc, w, irow, prow, b + 2);
    if (tail > 2) corr_chunk<CP, 2>(acc, w, irow, prow, b + 4);
    if (tail > 3) corr_chunk<CP, 3>(acc, w, irow, prow, b + 6);
  }
}

template <int CP>
__device__ __forceinline__ void store_pairs(const u64 (&acc)[CP][8], float* s_out, int cp0, int nch_conv,
                                            int row, int col0) {
#pragma unroll
  for (int q = 0; q < CP; ++q) {
    const int ch = 2 * (cp0 + q);
#pragma unroll
    for (int rx = 0; rx < 8; ++rx) {
      float x, y;
      unpack2(acc[q][rx], x, y);
      const int pix = row * kTile + col0 + rx;
      s_out[ch * kTilePix + pix] = x;
      if (ch + 1 < nch_conv) s_out[(ch + 1) * kTilePix + pix] = y;
    }
  }
}

// Accumulate J^T W J (packed upper triangle), J^T W r and chi^2 for P free
// parameters over this thread's pixels of the tile, reduce over the block and
// write the tile's FP64 partial sums.
template <int P>
__device__ __forceinline__ void reduce_tile(const FusedArgs& A, const float* s_out, float* s_red,
                                            int g, int tile, int i0, int j0) {
  constexpr int NA = 1 + P + P * (P + 1) / 2;
  float acc[NA];
#pragma unroll
  for (int e = 0; e < NA; ++e) acc[e] = 0.f;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const size_t base = (size_t)g * A.H * A.W;
  for (int pix = tid; pix < kTilePix; pix += nthr) {
    const int i = i0 + pix / kTile, j = j0 + pix % kTile;
    if (i >= A.H || j >= A.W) continue;
    const size_t gp = base + (size_t)i * A.W + j;
    if (A.mask && A.mask[gp]) continue;
    const float isg = 1.f / A.sigma[gp];
    const float rr = (A.image[gp] - s_out[pix]) * isg;  // (D - M) / sigma
    acc[0] = fmaf(rr, rr, acc[0]);
    float jw[P > 0 ? P : 1];
#pragma unroll
    for (int f = 0; f < P; ++f) jw[f] = s_out[(1 + f) * kTilePix + pix] * isg;  // J / sigma
#pragma unroll
    for (int f = 0; f < P; ++f) acc[1 + f] = fmaf(jw[f], rr, acc[1 + f]);
    int e = 1 + P;
#pragma unroll
    for (int f = 0; f < P; ++f)
#pragma unroll
      for (int h = f; h < P; ++h) {
        acc[e] = fmaf(jw[f], jw[h], acc[e]);
        ++e;
      }
  }
  const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
#pragma unroll
  for (int e = 0; e < NA; ++e) {
    float v = acc[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_red[warp * NA + e] = v;
  }
  __syncthreads();
  for (int e = tid; e < NA; e += nthr) {
    double s = 0.0;
    for (int w = 0; w < nwarp; ++w) s += (double)s_red[w * NA + e];
    A.partial[((size_t)g * A.n_tiles + tile) * NA + e] = s;
  }
}

// CPT = channel pairs per thread: 1 (128 threads per pair, up to 512 threads,
// more warps to hide latency) or 2 (fewer, fatter threads; used when the
// reduction of many free parameters needs more registers).
template <int MODE, int P, int CPT>
__global__ void __launch_bounds__(CPT == 1 ? 512 : 256, 1) k_fused(const __grid_constant__ FusedArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  u64* s_psf = reinterpret_cast<u64*>(smem + A.off_psf);
  float2* s_in = reinterpret_cast<float2*>(smem + A.off_in);
  float* s_out = reinterpret_cast<float*>(smem + A.off_out);
  float* s_cc = reinterpret_cast<float*>(smem + A.off_cc);
  float* s_scale = reinterpret_cast<float*>(smem + A.off_scale);
  float* s_red = reinterpret_cast<float*>(smem + A.off_red);

  const int tid = threadIdx.x, nthr = blockDim.x;
  const int K = A.K, c = (K - 1) / 2, K2 = K + 1;
  const int HH = kTile + K - 1, WW = kTile + K - 1, rw = A.rw;
  const int n_gal = A.list ? *A.count : A.G;
  const int n_items = n_gal * A.n_tiles;

  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int gi = item / A.n_tiles, tile = item - gi * A.n_tiles;
    const int g = A.list ? A.list[gi] : gi;
    const int i0 = (tile / A.tiles_x) * kTile, j0 = (tile % A.tiles_x) * kTile;

    __syncthreads();  // the previous item is done with shared memory
    for (int t = tid; t < A.n_comp * kCC; t += nthr) s_cc[t] = A.cconst[(size_t)g * A.n_comp * kCC + t];
    for (int t = tid; t < A.n_slots; t += nthr) s_scale[t] = A.scale[(size_t)g * A.n_slots + t];
    for (int t = tid; t < K * K2; t += nthr) {
      const int a = t / K2, b = t - a * K2;
      const float v = (b < K) ? A.psf[(size_t)g * K * K + a * K + b] : 0.f;
      s_psf[t] = pack2(v, v);
    }
    __syncthreads();

    // ---- 2. profile phase over the input window (zero outside the stamp) ----
    const size_t pstride = (size_t)HH * rw * 2;  // floats between channel pairs
    for (int hp = tid; hp < HH * rw; hp += nthr) {
      const int hr = hp / rw, hc = hp - hr * rw;
      const int i = i0 + hr - c, j = j0 + hc - c;
      float* px = reinterpret_cast<float*>(s_in + (size_t)hr * rw + hc);
      for (int cp = 0; cp < A.ncp; ++cp) {
        px[cp * pstride] = 0.f;
        px[cp * pstride + 1] = 0.f;
      }
      if (hc >= WW || i < 0 || i >= A.H || j < 0 || j >= A.W) continue;
      for (int cm = 0; cm < A.n_comp; ++cm) {
        if (!A.conv[cm]) continue;
        float d[8];
        const float v = eval_component(A.kind[cm], s_cc + cm * kCC, i, j, d);
        px[0] += v;
        if (MODE == MODE_MODEL) {
          const int ch = A.comp_chan[cm];
          if (ch >= 0) px[(ch >> 1) * pstride + (ch & 1)] += v;
        } else {
          for (int k = 0; k < A.np[cm]; ++k) {
            const int ch = A.chan[cm][k];
            if (ch >= 0) px[(ch >> 1) * pstride + (ch & 1)] += d[k] * s_scale[A.slot[cm][k]];
          }
        }
      }
    }
    __syncthreads();

    // ---- 3. correlation: group = 4 warps = CPT channel pairs ----
    const int grp = tid / kGroupThreads;
    const int cp0 = CPT * grp;
    const int npair = min(CPT, A.ncp - cp0);
    const int t = tid - grp * kGroupThreads;
    const int lane = t & 31, wig = t >> 5;
    const int row = wig * 8 + (lane & 7), col0 = (lane >> 3) * 8;
    // PSF rows whose 8 input rows (for this warp) all fall outside the stamp are skipped
    const int row0 = wig * 8;
    const int a_lo = max(0, c - i0 - row0 - 7);
    const int a_hi = min(K, c - i0 + A.H - row0);
    u64 acc2[2][8];
    u64 acc1[1][8];
    if (CPT == 2 && npair == 2) correlate_pairs<2>(acc2, s_in, s_psf, cp0, HH, rw, K, row, col0, a_lo, a_hi);
    else if (npair == 1) correlate_pairs<1>(acc1, s_in, s_psf, cp0, HH, rw, K, row, col0, a_lo, a_hi);
    __syncthreads();  // s_out aliases s_in
    if (CPT == 2 && npair == 2) store_pairs<2>(acc2, s_out, cp0, A.nch_conv, row, col0);
    else if (npair == 1) store_pairs<1>(acc1, s_out, cp0, A.nch_conv, row, col0);
    __syncthreads();

    // ---- 4. unconvolved components at the output pixels ----
    for (int pix = tid; pix < kTilePix; pix += nthr) {
      for (int ch = A.nch_conv; ch < A.nch_tot; ++ch) s_out[ch * kTilePix + pix] = 0.f;
      if (!A.any_unconv) continue;
      const int i = i0 + pix / kTile, j = j0 + pix % kTile;
      if (i >= A.H || j >= A.W) continue;
      for (int cm = 0; cm < A.n_comp; ++cm) {
        if (A.conv[cm]) continue;
        float d[8];
        const float v = eval_component(A.kind[cm], s_cc + cm * kCC, i, j, d);
        s_out[pix] += v;
        if (MODE == MODE_MODEL) {
          const int ch = A.comp_chan[cm];
          if (ch >= 0) s_out[ch * kTilePix + pix] = v;
        } else {
          for (int k = 0; k < A.np[cm]; ++k) {
            const int ch = A.chan[cm][k];
            if (ch >= 0) s_out[ch * kTilePix + pix] += d[k] * s_scale[A.slot[cm][k]];
          }
        }
      }
    }
    __syncthreads();

    // ---- 5. outputs ----
    if (MODE == MODE_MODEL) {
      const size_t HW = (size_t)A.H * A.W;
      for (int pix = tid; pix < kTilePix; pix += nthr) {
        const int i = i0 + pix / kTile, j = j0 + pix % kTile;
        if (i >= A.H || j >= A.W) continue;
        const size_t off = (size_t)i * A.W + j;
        A.model_out[(size_t)g * HW + off] = s_out[pix];
        if (A.comp_out) {
          for (int cm = 0; cm < A.n_comp; ++cm)
            A.comp_out[((size_t)g * A.n_comp + cm) * HW + off] = s_out[A.comp_chan[cm] * kTilePix + pix];
        }
      }
    } else {
      reduce_tile<P>(A, s_out, s_red, g, tile, i0, j0);
    }
  }
}

}  // namespace gm
