// gm_fused.cuh -- the two kernels of one model+Jacobian pass.
//
// Work item = (galaxy, 32x32 output tile).  Stamps and PSFs may differ in size
// from galaxy to galaxy: each item looks its galaxy's geometry up in the
// GalGeom table (gm_geom.cuh).
//
// k_planes: every stamp pixel of the items' tiles gets the summed convolved
//   components (channel 0) and one derivative channel per free parameter of a
//   convolved component (NORMAL mode), or the per-component images (MODEL
//   mode), written once to the galaxy's channel-pair planes in the workspace:
//   planes[cp][i][j] = (channel 2cp, channel 2cp+1), row pitch Wp = W rounded
//   up to even (the pad column is zero).
//
// k_fused: a persistent grid takes items from an atomic queue (item b first
//   for CTA b, then gridDim.x + atomicAdd(queue, 1)); the host orders the
//   items by decreasing cost (PSF area, then stamp size), so the last items
//   handed out are the cheap ones.  Per item and per "pass" of up to four
//   channel pairs:
//     * TMA tile loads (cp.async.bulk.tensor.3d, one per pair plane, issued
//       by lane 0 of different warps) bring the (32+K-1) x rw window of every
//       pair plane of the pass into shared
//       memory, through the tensor map of the galaxy's (H, W, K) class;
//       out-of-stamp rows and columns come back as zeros, which is the zero
//       padding of conv2d(..., padding="same");
//     * each thread owns 8 adjacent output pixels of one row and CPT channel
//       pairs and runs the sliding-window correlation (one 16-byte shared
//       load per 2 taps per pair, one 16-byte load of 4 single-float PSF taps
//       per 2 chunks, the packed multipliers made by register moves, 16
//       fma.rn.f32x2 per tap pair and channel pair), summing each block of 4
//       PSF rows into a separate partial (FP32 rounding error ~3x lower than
//       one running sum; the 512-thread instances sum without); PSF rows
//       whose input rows all fall outside the stamp for the warp are skipped;
//       a pass with fewer than two pairs per group splits two pairs between
//       two or four groups by PSF rows;
//     * the next load (next pass or next item) is issued as soon as every
//       warp has finished reading the window, so it overlaps the stores and
//       the reduction.  Thread 0 claims the next item and reads its record
//       once the current item's first window has landed, while the other warps
//       correlate.
//   Then the unconvolved components (the sky) are added at the output pixels,
//   and NORMAL mode forms r = D - M, w = Omega/sigma^2 and accumulates chi^2,
//   J^T W r and J^T W J (FP32 per thread, warp shuffles, a compensated FP32
//   cross-warp sum, one FP64 partial per tile); MODEL mode writes the model and
//   component images.
//
// The correlation is M[i,j] = sum_ab P[a,b] I[i+a-c, j+b-c] (cross-correlation,
// torch conv2d semantics, App. C of arxiv 2404.07780).  The window starts at
// column j0 - c' (c' = c or c+1, c = (K-1)/2), whichever is even, so that the
// TMA start coordinate is 16-byte aligned; the PSF rows carry the matching
// shift (psf_row_floats in gm_geom.cuh; the adjoint's two-galaxy rows: K+1
// packed positions with one zero, on the left when c is odd).
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include "gm_geom.cuh"
#include "gm_profiles.cuh"

namespace gm {

constexpr int kTile = kTileSide;    // output tile is kTile x kTile
constexpr int kTilePix = kTile * kTile;
constexpr int kMaxPairs = 9;        // up to 17 correlated channels (model + 16 free parameters)
constexpr int kMaxPassPairs = 4;    // channel pairs per TMA pass
constexpr int kGroupThreads = 128;  // threads per pair group (32 rows x 4 column blocks)
constexpr int kRowBlock = 4;        // PSF rows summed into one partial accumulator
constexpr unsigned kWaitTries = 1u << 24;

enum Mode { MODE_MODEL = 0, MODE_NORMAL = 1 };

typedef unsigned long long u64;

// Model description shared by both kernels (uniform over the batch).
struct ChanMap {
  int n_comp;
  int kind[kMaxComp];
  int conv[kMaxComp];
  int np[kMaxComp];
  int slot[kMaxComp][8];     // parameter k of comp c -> slot
  int chan[kMaxComp][8];     // d/dp_k of comp c -> channel (-1: not needed)
  int comp_chan[kMaxComp];   // MODEL mode: channel holding comp c's own image (-1: none)
  int any_unconv;
  int sky_comp;              // NORMAL mode and the adjoint's residuals: the one unconvolved component
                             // when it is a flat sky (-1: none such), applied without evaluating it
  int sky_ch;                // that sky's derivative channel, the last one (-1: its level is fixed)
  int ident_comp;            // NORMAL mode: the one convolved component when its parameters are all
                             // free and own channels 1 .. np in order (-1: none such)
  int nch_conv;              // correlated channels
  int ncp;                   // channel pairs = ceil(nch_conv / 2)
  int nch_tot;               // channels at the output pixels (correlated + unconvolved-only)
  int n_slots;
};

// Arguments of the adjoint path's profile kernel (equal stamps).
struct ProfileArgs {
  ChanMap m;
  int G, H, W, Wp;
  const float* cconst;       // [G][n_comp][kCC]
  const float* scale;        // [G][n_slots]
  const int* list;           // galaxies list[0 .. *count); nullptr -> all G
  const int* count;
  float* planes;             // [G][ncp][H][Wp][2]
};

// Arguments of k_planes.
struct PlaneArgs {
  ChanMap m;
  const GalGeom* geo;        // [G]
  const int2* items;         // (galaxy, tile) items of this pass
  const int* n_items_dev;    // item count on the device (a fit's pass), or nullptr
  int n_items;               // item count when n_items_dev is nullptr
  const float* cconst;       // [G][n_comp][kCC]
  const float* scale;        // [G][n_slots]
  float* planes;             // pair planes, galaxy g from geo[g].plane
  int* zero[3];              // counters set to 0 for the next kernels (nullptr: none)
};

struct FusedArgs {
  CUtensorMap tmap;          // equal stamps: planes as a [G*ncp][H][2*Wp] FP32 tensor, box [1][32+K-1][2*rw]
  const CUtensorMap* maps;   // uneven stamps: one such map per (H, W, K) class, in global memory; else nullptr
  ChanMap m;
  int nacc;                  // accumulators per tile (NORMAL)
  int pp, passes;
  int plane;                 // float2 elements between pair planes in shared memory (a 128-byte multiple:
                             // every TMA destination must be 128-byte aligned)
  const GalGeom* geo;
  const int2* items;
  const int* n_items_dev;
  int n_items;
  int* queue;                // next item - gridDim.x (zero at launch)
  const float* image;
  const float* sigma;
  const uint8_t* mask;
  const float* psf;
  const float* psf_pad;      // [G][psf_stride]: each PSF as K rows of psf_row_floats(K) floats, laid
                             // out as in shared memory, copied into s_psf by the bulk-copy unit
  int psf_stride;            // floats per galaxy in psf_pad (a multiple of 4)
  const float* cconst;       // [G][n_comp][kCC]
  const float* scale;        // [G][scale_stride(n_slots)]
  double* partial;           // [tile0_g + tile][nacc]
  float* model_out;          // stamp g from geo[g].pix
  float* comp_out;           // [n_comp] images per stamp from n_comp * geo[g].pix, or nullptr
  int* err;                  // set to 1 when a TMA wait times out
  unsigned wait_polls;       // polls of a window wait before it gives up (kWaitTries)
  int starve;                // test of the timeout path: CTA 0 issues no load for its first window, so
                             // that wait runs out with nothing in flight
  int off_psf, off_in, off_out, off_cc, off_scale, off_red, off_bar, off_info;
};

// One item as thread 0 stages it in shared memory for the CTA.
struct ItemInfo {
  int valid, g, tile, pad;
  GalGeom geo;
};

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

// ---------------------------------------------------------------------------
// k_planes
// ---------------------------------------------------------------------------
// Work units of k_planes: a whole item (its 1024 pixels, four per thread) or, when a
// pass has so few items that their quarters fit in one wave of the grid, a quarter
// of one (256 pixels, one per thread), so that a small pass still spreads over the
// SMs; a large pass keeps whole items (the per-unit set-up costs at that size).
constexpr int kPlaneUnits = kTilePix / 256;

template <int MODE>
__global__ void __launch_bounds__(256) k_planes(const __grid_constant__ PlaneArgs A) {
  __shared__ float s_cc[kMaxComp * kCC];
  __shared__ float s_scale[kMaxSlots];
  __shared__ float s_v[256 * 2 * kMaxPairs];  // channel-major: this thread's channel ch at ch * 256 + tid
  const ChanMap& m = A.m;
  const int tid = threadIdx.x;
  if (blockIdx.x == 0 && tid < 3 && A.zero[tid]) *A.zero[tid] = 0;
  const int n = A.n_items_dev ? *A.n_items_dev : A.n_items;
  const int upi = kPlaneUnits * n <= (int)gridDim.x ? kPlaneUnits : 1;  // units per item
  float* v = s_v + tid;  // v[ch * 256]: consecutive threads, consecutive banks
  float2* out = reinterpret_cast<float2*>(A.planes);
  for (int u = blockIdx.x; u < upi * n; u += gridDim.x) {
    const int item = u / upi, r0 = u - item * upi;
    const int2 it = A.items[item];
    const int g = it.x;
    const GalGeom& G = A.geo[g];
    const int H = G.H, W = G.W, Wp = G.Wp;
    const int i0 = (it.y / G.tiles_x) * kTile, j0 = (it.y % G.tiles_x) * kTile;
    const size_t pbase = (size_t)(G.plane >> 1);
    __syncthreads();
    for (int t = tid; t < m.n_comp * kCC; t += 256) s_cc[t] = A.cconst[(size_t)g * m.n_comp * kCC + t];
    for (int t = tid; t < m.n_slots; t += 256) s_scale[t] = A.scale[(size_t)g * scale_stride(m.n_slots) + t];
    __syncthreads();
    if (MODE == MODE_NORMAL && m.ident_comp >= 0) {
      // one convolved component whose derivatives fill channels 1 .. np in order: the
      // channels stay in registers (the same values as the scatter below)
      const int cm = m.ident_comp, np = m.np[cm], kind = m.kind[cm];
      const float* cc = s_cc + cm * kCC;
      float sc[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) sc[k] = k < np ? s_scale[m.slot[cm][k]] : 0.f;
      for (int r = r0; r < kPlaneUnits; r += upi) {
        const int pix = r * 256 + tid;
        const int i = i0 + pix / kTile, j = j0 + pix % kTile;
        if (i >= H || j >= Wp) continue;
        float vr[2 * 5] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (j < W) {
          float d[8];
          vr[0] = eval_component(kind, cc, i, j, d);
#pragma unroll
          for (int k = 0; k < 8; ++k)
            if (k < np) vr[1 + k] = d[k] * sc[k];
        }
#pragma unroll
        for (int cp = 0; cp < 5; ++cp)
          if (cp < m.ncp) out[pbase + ((size_t)cp * H + i) * Wp + j] = make_float2(vr[2 * cp], vr[2 * cp + 1]);
      }
      continue;
    }
    for (int r = r0; r < kPlaneUnits; r += upi) {
      const int pix = r * 256 + tid;
      const int i = i0 + pix / kTile, j = j0 + pix % kTile;
      if (i >= H || j >= Wp) continue;
      for (int ch = 0; ch < 2 * m.ncp; ++ch) v[ch * 256] = 0.f;
      if (j < W) {
        for (int cm = 0; cm < m.n_comp; ++cm) {
          if (!m.conv[cm]) continue;
          float d[8];
          const float val = eval_component(m.kind[cm], s_cc + cm * kCC, i, j, d);
          v[0] += val;
          if (MODE == MODE_MODEL) {
            if (m.comp_chan[cm] >= 0) v[m.comp_chan[cm] * 256] += val;
          } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) {  // compile-time k keeps d in registers
              if (k >= m.np[cm]) break;
              const int ch = m.chan[cm][k];
              if (ch >= 0) v[ch * 256] += d[k] * s_scale[m.slot[cm][k]];
            }
          }
        }
      }
      for (int cp = 0; cp < m.ncp; ++cp)
        out[pbase + ((size_t)cp * H + i) * Wp + j] = make_float2(v[2 * cp * 256], v[(2 * cp + 1) * 256]);
    }
  }
}

// ---------------------------------------------------------------------------
// TMA and mbarrier helpers (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(u64* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(u64* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(u64* bar, unsigned phase) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return done != 0;
}

// Bounded wait for a phase of the mbarrier; false after `polls` polls.
__device__ __forceinline__ bool mbar_wait_bounded(u64* bar, unsigned phase, unsigned polls = kWaitTries) {
  for (unsigned t = 0; t < polls; ++t)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, u64* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<u64>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// Contiguous global -> shared copy by the bulk-copy unit (16-byte aligned, size a 16-byte multiple).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, u64* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(reinterpret_cast<u64>(src)), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Thread 0: read item `item` of this pass into *dst (valid = 0 past the end).
__device__ __forceinline__ void fetch_item(const FusedArgs& A, int n_items, int item, ItemInfo* dst) {
  if (item >= n_items) {
    dst->valid = 0;
    return;
  }
  const int2 it = A.items[item];
  dst->valid = 1;
  dst->g = it.x;
  dst->tile = it.y;
  dst->geo = A.geo[it.x];
}

// Issue the loads of pass `pass` of item I: the pass's pair-plane windows
// (copies 0 .. npairs-1) and, for pass 0, the galaxy's padded PSF rows into
// s_psf and its constants into the item's constant buffers (s_cc, s_scale of
// `slot`; copies npairs .. npairs+2), all on one mbarrier.  The calling thread
// issues copies k0, k0 + kstep, ... and, with `arrive`, makes the barrier's one
// arrival with the pass's byte count.  The copies may be spread over several
// threads (one per warp: each copy instruction holds its thread for hundreds of
// cycles) and may complete before the arrival: an mbarrier's transaction count
// may go below zero, and the phase completes only once the arrival is made and
// every byte has landed.
__device__ __forceinline__ void issue_pass(const FusedArgs& A, const ItemInfo& I, float2* s_in, u64* bar, int pass,
                                           float* s_psf, float* s_cc, float* s_scale, int k0 = 0, int kstep = 1,
                                           bool arrive = true) {
  const GalGeom& G = I.geo;
  const int K = G.K, c = (K - 1) / 2, cpad = c & 1;
  const int first = pass * A.pp;
  const int npairs = min(A.pp, A.m.ncp - first);
  const int ncopy = npairs + (pass == 0 ? 3 : 0);
  const unsigned plane_bytes = (unsigned)(kTile + K - 1) * G.rw * 8u;
  const unsigned psf_bytes = (unsigned)K * psf_row_floats(K) * 4u;
  const unsigned cc_bytes = (unsigned)A.m.n_comp * kCC * 4u;
  const unsigned sc_bytes = (unsigned)scale_stride(A.m.n_slots) * 4u;
  if (k0 < ncopy) {
    const int i0 = (I.tile / G.tiles_x) * kTile, j0 = (I.tile % G.tiles_x) * kTile;
    const CUtensorMap* map = &A.tmap;
    if (A.maps) {
      map = A.maps + G.cls;
      // the map was written to global memory by an ordinary copy: order that write before the TMA unit reads it
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<u64>(map))
                   : "memory");
    }
    // order this CTA's earlier generic-proxy reads of the buffers before the async-proxy writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const int x = 2 * (j0 - c - cpad);  // even pair index: 16-byte aligned start
    for (int k = k0; k < ncopy; k += kstep) {
      if (k < npairs) tma_load_3d(s_in + (size_t)k * A.plane, map, x, i0 - c, G.z0 + first + k, bar);
      else if (k == npairs) bulk_load(s_psf, A.psf_pad + (size_t)I.g * A.psf_stride, psf_bytes, bar);
      else if (k == npairs + 1) bulk_load(s_cc, A.cconst + (size_t)I.g * A.m.n_comp * kCC, cc_bytes, bar);
      else bulk_load(s_scale, A.scale + (size_t)I.g * scale_stride(A.m.n_slots), sc_bytes, bar);
    }
  }
  if (arrive) mbar_expect_tx(bar, plane_bytes * npairs + (pass == 0 ? psf_bytes + cc_bytes + sc_bytes : 0u));
}

// ---------------------------------------------------------------------------
// correlation
// ---------------------------------------------------------------------------
// One 2-tap chunk of the sliding-window correlation.  R is the ring rotation:
// window element e (input column b + e relative to the thread's first column)
// lives in w[q][(2R + e) % 10].  Elements 0..7 are present on entry; elements 8
// and 9 are loaded here.  pp holds the PSF pair (taps b, b+1) on entry and
// (b+2, b+3) on exit: each chunk fetches the next chunk's pair before its own
// FMAs, so no FMA waits on a shared-memory load of the tap it multiplies.
// Odd K leaves one zero tap position per padded row (K+1 positions); the half
// chunks skip it: HALF = 1 does tap b only (the row's last chunk: no loads),
// HALF = 2 tap b+1 only (the row's first chunk when the zero is in front).
template <int CP, int R, int HALF = 0>
__device__ __forceinline__ void corr_chunk(u64 (&acc)[CP][8], u64 (&w)[CP][10], ulonglong2& pp,
                                           const float2* const (&irow)[CP], const u64* prow, int b) {
  constexpr int L = (2 * R + 8) % 10;
  ulonglong2 pn = pp;
  if (HALF != 1) {
    pn = *reinterpret_cast<const ulonglong2*>(prow + b + 2);
#pragma unroll
    for (int q = 0; q < CP; ++q) {
      const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(irow[q] + b + 8);
      w[q][L] = v.x;
      w[q][L + 1] = v.y;
    }
  }
#pragma unroll
  for (int q = 0; q < CP; ++q) {
    if (HALF != 2) {
#pragma unroll
      for (int rx = 0; rx < 8; ++rx) acc[q][rx] = ffma2(pp.x, w[q][(2 * R + rx) % 10], acc[q][rx]);
    }
    if (HALF != 1) {
#pragma unroll
      for (int rx = 0; rx < 8; ++rx) acc[q][rx] = ffma2(pp.y, w[q][(2 * R + 1 + rx) % 10], acc[q][rx]);
    }
  }
  pp = pn;
}

// One PSF row into acc.  The padded row has K+1 positions, the taps at
// cpad .. cpad+K-1 (cpad = c & 1 keeps each window start 16-byte aligned):
// nf = (K-1)/2 full chunks plus one half chunk, in front (cpad = 1) or behind.
// Ten chunks per loop iteration; the last chunk may prefetch two positions past
// the row (into the next row, or the 16 slack bytes after the last one).
template <int CP>
__device__ __forceinline__ void corr_row(u64 (&acc)[CP][8], const float2* const (&irow)[CP], const u64* prow,
                                         int nf, int cpad) {
  u64 w[CP][10];
  ulonglong2 pp = *reinterpret_cast<const ulonglong2*>(prow);
  int b = 0;
  if (cpad) {
    // start the ring at rotation 4, so that the full chunks after the head half start at 0
#pragma unroll
    for (int q = 0; q < CP; ++q)
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(irow[q] + e);
        w[q][(8 + e) % 10] = v.x;
        w[q][(9 + e) % 10] = v.y;
      }
    corr_chunk<CP, 4, 2>(acc, w, pp, irow, prow, 0);
    b = 2;
  } else {
#pragma unroll
    for (int q = 0; q < CP; ++q)
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(irow[q] + e);
        w[q][e] = v.x;
        w[q][e + 1] = v.y;
      }
  }
  for (; nf >= 10; nf -= 10) {
    corr_chunk<CP, 0>(acc, w, pp, irow, prow, b);
    corr_chunk<CP, 1>(acc, w, pp, irow, prow, b + 2);
    corr_chunk<CP, 2>(acc, w, pp, irow, prow, b + 4);
    corr_chunk<CP, 3>(acc, w, pp, irow, prow, b + 6);
    corr_chunk<CP, 4>(acc, w, pp, irow, prow, b + 8);
    corr_chunk<CP, 0>(acc, w, pp, irow, prow, b + 10);
    corr_chunk<CP, 1>(acc, w, pp, irow, prow, b + 12);
    corr_chunk<CP, 2>(acc, w, pp, irow, prow, b + 14);
    corr_chunk<CP, 3>(acc, w, pp, irow, prow, b + 16);
    corr_chunk<CP, 4>(acc, w, pp, irow, prow, b + 18);
    b += 20;
  }
  if (nf >= 5) {
    corr_chunk<CP, 0>(acc, w, pp, irow, prow, b);
    corr_chunk<CP, 1>(acc, w, pp, irow, prow, b + 2);
    corr_chunk<CP, 2>(acc, w, pp, irow, prow, b + 4);
    corr_chunk<CP, 3>(acc, w, pp, irow, prow, b + 6);
    corr_chunk<CP, 4>(acc, w, pp, irow, prow, b + 8);
    b += 10;
    nf -= 5;
  }
  // nf = 0..4 full chunks left, then the tail half when the zero position is behind
  const bool tail = !cpad;
  if (nf == 0) {
    if (tail) corr_chunk<CP, 0, 1>(acc, w, pp, irow, prow, b);
    return;
  }
  corr_chunk<CP, 0>(acc, w, pp, irow, prow, b);
  if (nf == 1) {
    if (tail) corr_chunk<CP, 1, 1>(acc, w, pp, irow, prow, b + 2);
    return;
  }
  corr_chunk<CP, 1>(acc, w, pp, irow, prow, b + 2);
  if (nf == 2) {
    if (tail) corr_chunk<CP, 2, 1>(acc, w, pp, irow, prow, b + 4);
    return;
  }
  corr_chunk<CP, 2>(acc, w, pp, irow, prow, b + 4);
  if (nf == 3) {
    if (tail) corr_chunk<CP, 3, 1>(acc, w, pp, irow, prow, b + 6);
    return;
  }
  corr_chunk<CP, 3>(acc, w, pp, irow, prow, b + 6);
  if (tail) corr_chunk<CP, 4, 1>(acc, w, pp, irow, prow, b + 8);
}

// PSF rows of the fused pass in shared memory: single floats, row a of K taps
// at floats a * psf_row_floats(K) + 3 cpad + t (gm_geom.cuh).

// A chunk of the float-PSF loop: taps t0, t1 (scalars from one float4) become
// the packed multipliers by register moves.  Ring, window loads and halves as
// in corr_chunk; measured ~8 % more FMAs per clock than loading packed pairs.
template <int CP, int R, int HALF = 0>
__device__ __forceinline__ void corr_chunk_f(u64 (&acc)[CP][8], u64 (&w)[CP][10], float t0, float t1,
                                             const float2* const (&irow)[CP], int b) {
  constexpr int L = (2 * R + 8) % 10;
  if (HALF != 1) {
#pragma unroll
    for (int q = 0; q < CP; ++q) {
      const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(irow[q] + b + 8);
      w[q][L] = v.x;
      w[q][L + 1] = v.y;
    }
  }
  const u64 px = pack2(t0, t0), py = pack2(t1, t1);
#pragma unroll
  for (int q = 0; q < CP; ++q) {
    if (HALF != 2) {
#pragma unroll
      for (int rx = 0; rx < 8; ++rx) acc[q][rx] = ffma2(px, w[q][(2 * R + rx) % 10], acc[q][rx]);
    }
    if (HALF != 1) {
#pragma unroll
      for (int rx = 0; rx < 8; ++rx) acc[q][rx] = ffma2(py, w[q][(2 * R + 1 + rx) % 10], acc[q][rx]);
    }
  }
}

// Two chunks (rotations R0, R1) from the float4 cur; the next float4 is read first.
template <int CP, int R0, int R1>
__device__ __forceinline__ void corr_pair_f(u64 (&acc)[CP][8], u64 (&w)[CP][10], float4& cur, const float4* next,
                                            const float2* const (&irow)[CP], int b) {
  const float4 nx = *next;
  corr_chunk_f<CP, R0>(acc, w, cur.x, cur.y, irow, b);
  corr_chunk_f<CP, R1>(acc, w, cur.z, cur.w, irow, b + 2);
  cur = nx;
}

// The taps of a PSF row that one warp runs, from the float layout's chunk
// structure: the head half (cpad = 1: the zero position and tap 0), nf full
// 2-tap chunks starting at position 2 cpad + 4 m (m float4s of leading chunks
// skipped), the tail half (cpad = 0: tap K-1 and the zero position).  A warp
// whose 8-column range sees `lead` leading and `trail` trailing taps outside
// the stamp for every one of its pixels skips the whole chunks and halves
// among them (lead + trail < K; a warp with no tap inside runs no row).
struct ColSkip {
  int head, m, nf, tail;
};

__device__ __forceinline__ ColSkip col_skip(int K, int lead, int trail) {
  const int cpad = ((K - 1) >> 1) & 1;
  ColSkip r;
  r.head = cpad && lead == 0;
  r.m = max(0, (lead - cpad) >> 2);  // chunk 2k (k < 2m) covers taps up to cpad + 4m - 1 < lead
  r.tail = !cpad && trail == 0;
  const int nt = cpad ? trail >> 1 : max(0, (trail - 1) >> 1);  // trailing full chunks all outside
  r.nf = ((K - 1) >> 1) - 2 * r.m - nt;
  return r;
}

__device__ __forceinline__ ColSkip col_all(int K) { return col_skip(K, 0, 0); }

// One PSF row into acc from the float layout above: the head half (cpad = 1,
// the row's float 3), nf full chunks two per float4 (ten per loop iteration),
// the tail half (cpad = 0); the chunks a warp skips at the stamp's left or
// right edge are left out (cs).
template <int CP>
__device__ __forceinline__ void corr_row(u64 (&acc)[CP][8], const float2* const (&irow)[CP], const float* prow,
                                         const ColSkip& cs, int cpad) {
  u64 w[CP][10];
  const float4* pf = reinterpret_cast<const float4*>(prow);
  int b = 0;
  int nf = cs.nf;
  if (!cs.head) {
    // first full chunk at position 2 cpad + 4 m, ring at rotation 0
    b = 2 * cpad + 4 * cs.m;
    pf += cpad + cs.m;
#pragma unroll
    for (int q = 0; q < CP; ++q)
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(irow[q] + b + e);
        w[q][e] = v.x;
        w[q][e + 1] = v.y;
      }
  } else {
#pragma unroll
    for (int q = 0; q < CP; ++q)
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(irow[q] + e);
        w[q][(8 + e) % 10] = v.x;
        w[q][(9 + e) % 10] = v.y;
      }
    const float4 h = pf[0];
    corr_chunk_f<CP, 4, 2>(acc, w, 0.f, h.w, irow, 0);
    b = 2;
    ++pf;
  }
  float4 cur = pf[0];
  for (; nf >= 10; nf -= 10) {
    corr_pair_f<CP, 0, 1>(acc, w, cur, pf + 1, irow, b);
    corr_pair_f<CP, 2, 3>(acc, w, cur, pf + 2, irow, b + 4);
    corr_pair_f<CP, 4, 0>(acc, w, cur, pf + 3, irow, b + 8);
    corr_pair_f<CP, 1, 2>(acc, w, cur, pf + 4, irow, b + 12);
    corr_pair_f<CP, 3, 4>(acc, w, cur, pf + 5, irow, b + 16);
    pf += 5;
    b += 20;
  }
  // nf = 0..9 full chunks (rotations 0, 1, ...) from cur on, then the tail half
  const bool tail = cs.tail;
  if (nf == 0) {
    if (tail) corr_chunk_f<CP, 0, 1>(acc, w, cur.x, 0.f, irow, b);
    return;
  }
  if (nf == 1) {
    corr_chunk_f<CP, 0>(acc, w, cur.x, cur.y, irow, b);
    if (tail) corr_chunk_f<CP, 1, 1>(acc, w, cur.z, 0.f, irow, b + 2);
    return;
  }
  corr_pair_f<CP, 0, 1>(acc, w, cur, pf + 1, irow, b);
  if (nf == 2) {
    if (tail) corr_chunk_f<CP, 2, 1>(acc, w, cur.x, 0.f, irow, b + 4);
    return;
  }
  if (nf == 3) {
    corr_chunk_f<CP, 2>(acc, w, cur.x, cur.y, irow, b + 4);
    if (tail) corr_chunk_f<CP, 3, 1>(acc, w, cur.z, 0.f, irow, b + 6);
    return;
  }
  corr_pair_f<CP, 2, 3>(acc, w, cur, pf + 2, irow, b + 4);
  if (nf == 4) {
    if (tail) corr_chunk_f<CP, 4, 1>(acc, w, cur.x, 0.f, irow, b + 8);
    return;
  }
  if (nf == 5) {
    corr_chunk_f<CP, 4>(acc, w, cur.x, cur.y, irow, b + 8);
    if (tail) corr_chunk_f<CP, 0, 1>(acc, w, cur.z, 0.f, irow, b + 10);
    return;
  }
  corr_pair_f<CP, 4, 0>(acc, w, cur, pf + 3, irow, b + 8);
  if (nf == 6) {
    if (tail) corr_chunk_f<CP, 1, 1>(acc, w, cur.x, 0.f, irow, b + 12);
    return;
  }
  if (nf == 7) {
    corr_chunk_f<CP, 1>(acc, w, cur.x, cur.y, irow, b + 12);
    if (tail) corr_chunk_f<CP, 2, 1>(acc, w, cur.z, 0.f, irow, b + 14);
    return;
  }
  corr_pair_f<CP, 1, 2>(acc, w, cur, pf + 4, irow, b + 12);
  if (nf == 8) {
    if (tail) corr_chunk_f<CP, 3, 1>(acc, w, cur.x, 0.f, irow, b + 16);
    return;
  }
  corr_chunk_f<CP, 3>(acc, w, cur.x, cur.y, irow, b + 16);  // nf == 9
  if (tail) corr_chunk_f<CP, 4, 1>(acc, w, cur.z, 0.f, irow, b + 18);
}

// Start of PSF row a in either layout.
__device__ __forceinline__ const u64* psf_row_ptr(const u64* s_psf, int a, int K) { return s_psf + a * (K + 1); }
__device__ __forceinline__ const float* psf_row_ptr(const float* s_psf, int a, int K) {
  return s_psf + a * psf_row_floats(K);
}

// A row in either PSF layout (the packed-pair rows of the adjoint take no column skip).
template <int CP>
__device__ __forceinline__ void corr_row_any(u64 (&acc)[CP][8], const float2* const (&irow)[CP], const float* prow,
                                             const ColSkip& cs, int, int cpad) {
  corr_row<CP>(acc, irow, prow, cs, cpad);
}
template <int CP>
__device__ __forceinline__ void corr_row_any(u64 (&acc)[CP][8], const float2* const (&irow)[CP], const u64* prow,
                                             const ColSkip&, int nf, int cpad) {
  corr_row<CP>(acc, irow, prow, nf, cpad);
}

// Correlate CP pair planes (local indices lp0 .. lp0+CP-1 of the pass buffer)
// for one thread's 8 output pixels over PSF rows [a_lo, a_hi), each row's taps
// as cs gives them (float PSF rows).  With BLOCKS,
// each block of kRowBlock PSF rows is summed into its own partial first (lower
// FP32 accumulation error, at CP x 8 more registers: the 512-thread two-pair
// instances go without, to stay within 128 registers).
template <int CP, bool BLOCKS = true, class PsfT = u64>
__device__ __forceinline__ void correlate_pairs(u64 (&acc)[CP][8], const float2* s_in, const PsfT* s_psf,
                                                int lp0, int plane, int rw, int K, int row, int col0, int a_lo,
                                                int a_hi, const ColSkip& cs) {
  const u64 one2 = pack2(1.f, 1.f);
#pragma unroll
  for (int q = 0; q < CP; ++q)
#pragma unroll
    for (int rx = 0; rx < 8; ++rx) acc[q][rx] = 0ull;
  const int nf = (K - 1) >> 1;         // full 2-tap chunks per PSF row
  const int cpad = ((K - 1) >> 1) & 1;  // zero position in front of the taps
  if (!BLOCKS) {
    for (int a = a_lo; a < a_hi; ++a) {
      const float2* irow[CP];
#pragma unroll
      for (int q = 0; q < CP; ++q) irow[q] = s_in + (size_t)(lp0 + q) * plane + (size_t)(row + a) * rw + col0;
      corr_row_any<CP>(acc, irow, psf_row_ptr(s_psf, a, K), cs, nf, cpad);
    }
    return;
  }
  for (int a0 = a_lo; a0 < a_hi; a0 += kRowBlock) {
    u64 part[CP][8];
#pragma unroll
    for (int q = 0; q < CP; ++q)
#pragma unroll
      for (int rx = 0; rx < 8; ++rx) part[q][rx] = 0ull;
    const int a1 = min(a0 + kRowBlock, a_hi);
    for (int a = a0; a < a1; ++a) {
      const float2* irow[CP];
#pragma unroll
      for (int q = 0; q < CP; ++q) irow[q] = s_in + (size_t)(lp0 + q) * plane + (size_t)(row + a) * rw + col0;
      corr_row_any<CP>(part, irow, psf_row_ptr(s_psf, a, K), cs, nf, cpad);
    }
#pragma unroll
    for (int q = 0; q < CP; ++q)
#pragma unroll
      for (int rx = 0; rx < 8; ++rx) acc[q][rx] = ffma2(one2, part[q][rx], acc[q][rx]);
  }
}

// The output tile in shared memory: channel ch, pixel pix = row * kTile + col,
// at ch * kTilePix + out_idx(pix).  Each row's 4-column groups are permuted by
// XOR with (row & 7), so the 8 rows that a quarter-warp stores (same columns,
// 16 bytes per lane) fall in 8 different bank groups; a warp reading one row
// still touches 32 different banks.
static_assert(kTile == 32, "out_idx assumes 32-pixel rows");
__device__ __forceinline__ int out_idx(int pix) { return pix ^ (((pix >> 5) & 7) << 2); }

template <int CP>
__device__ __forceinline__ void store_pairs(const u64 (&acc)[CP][8], float* s_out, int cp0, int nch_conv,
                                            int row, int col0) {
  const int o0 = out_idx(row * kTile + col0), o1 = out_idx(row * kTile + col0 + 4);
#pragma unroll
  for (int q = 0; q < CP; ++q) {
    const int ch = 2 * (cp0 + q);
    float x[8], y[8];
#pragma unroll
    for (int rx = 0; rx < 8; ++rx) unpack2(acc[q][rx], x[rx], y[rx]);
    float* sx = s_out + ch * kTilePix;
    *reinterpret_cast<float4*>(sx + o0) = make_float4(x[0], x[1], x[2], x[3]);
    *reinterpret_cast<float4*>(sx + o1) = make_float4(x[4], x[5], x[6], x[7]);
    if (ch + 1 < nch_conv) {
      float* sy = sx + kTilePix;
      *reinterpret_cast<float4*>(sy + o0) = make_float4(y[0], y[1], y[2], y[3]);
      *reinterpret_cast<float4*>(sy + o1) = make_float4(y[4], y[5], y[6], y[7]);
    }
  }
}

// store_pairs for the second half of a row-split pass: adds to what the first stored.
template <int CP>
__device__ __forceinline__ void add_pairs(const u64 (&acc)[CP][8], float* s_out, int cp0, int nch_conv, int row,
                                          int col0) {
  const int o0 = out_idx(row * kTile + col0), o1 = out_idx(row * kTile + col0 + 4);
#pragma unroll
  for (int q = 0; q < CP; ++q) {
    const int ch = 2 * (cp0 + q);
    float x[8], y[8];
#pragma unroll
    for (int rx = 0; rx < 8; ++rx) unpack2(acc[q][rx], x[rx], y[rx]);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h == 1 && ch + 1 >= nch_conv) break;
      const float* v = h ? y : x;
      float4* p0 = reinterpret_cast<float4*>(s_out + (ch + h) * kTilePix + o0);
      float4* p1 = reinterpret_cast<float4*>(s_out + (ch + h) * kTilePix + o1);
      float4 a = *p0, b = *p1;
      a.x += v[0]; a.y += v[1]; a.z += v[2]; a.w += v[3];
      b.x += v[4]; b.y += v[5]; b.z += v[6]; b.w += v[7];
      *p0 = a;
      *p1 = b;
    }
  }
}

// Warp sums of N values that every lane holds, by recursive halving: at the
// level with xor mask M each lane keeps one half of its current entries (the
// upper half when its bit M is set, the odd middle entry with the lower lane)
// and adds its partner's copy of that half.  After the levels M = 16 .. 1 the
// warp sum of each entry sits in exactly one lane, where store(entry, sum) is
// called: about N shuffles instead of 5 N for a butterfly per entry.
template <int N, int M>
struct WarpScatter {
  template <class Store>
  static __device__ __forceinline__ void run(const float (&v)[N], const int (&idx)[N], int lane, Store& store) {
    constexpr int H = (N + 1) / 2;  // the lower half, with the odd middle entry
    constexpr int NP = N - H;       // entries that pair off
    const bool up = lane & M;
    float nv[H];
    int ni[H];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      const float send = up ? v[i] : v[H + i];
      const float keep = up ? v[H + i] : v[i];
      nv[i] = keep + __shfl_xor_sync(0xffffffffu, send, M);
      ni[i] = up ? idx[H + i] : idx[i];
    }
    if constexpr (H > NP) {
      nv[H - 1] = v[H - 1] + __shfl_xor_sync(0xffffffffu, v[H - 1], M);
      ni[H - 1] = up ? -1 : idx[H - 1];  // the upper lane's copy is a duplicate
    }
    WarpScatter<H, M / 2>::run(nv, ni, lane, store);
  }
};
template <int N>
struct WarpScatter<N, 0> {
  template <class Store>
  static __device__ __forceinline__ void run(const float (&v)[N], const int (&idx)[N], int, Store& store) {
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (idx[i] >= 0) store(idx[i], v[i]);
  }
};

template <int N, class Store>
__device__ __forceinline__ void warp_sum_scatter(const float (&v)[N], int lane, Store store) {
  int idx[N];
#pragma unroll
  for (int i = 0; i < N; ++i) idx[i] = i;
  WarpScatter<N, 16>::run(v, idx, lane, store);
}

// The accumulators [E0, E1) of the tile's normal equations over this thread's
// pixels (loaded by reduce_tile), then their warp sums into s_red.  Entry 0 is
// chi^2, 1..P J^T W r, then J^T W J packed by rows of its upper triangle.
template <int P, int kPx, int E0, int E1>
__device__ __forceinline__ void reduce_range(const float* s_out, float* s_red, const float (&dv)[kPx],
                                             const float (&sv)[kPx], const bool (&use)[kPx], int tid, int nthr,
                                             int lane, int warp) {
  constexpr int NA = 1 + P + P * (P + 1) / 2;
  float acc[E1 - E0];
#pragma unroll
  for (int e = 0; e < E1 - E0; ++e) acc[e] = 0.f;
#pragma unroll
  for (int k = 0; k < kPx; ++k) {
    if (!use[k]) continue;
    const int op = out_idx(tid + k * nthr);
    const float isg = 1.f / sv[k];
    const float rr = (dv[k] - s_out[op]) * isg;  // (D - M) / sigma
    if (E0 == 0) acc[0] = fmaf(rr, rr, acc[0]);
    float jw[P > 0 ? P : 1];
#pragma unroll
    for (int f = 0; f < P; ++f) jw[f] = s_out[(1 + f) * kTilePix + op] * isg;  // J / sigma
#pragma unroll
    for (int f = 0; f < P; ++f)
      if (1 + f >= E0 && 1 + f < E1) acc[1 + f - E0] = fmaf(jw[f], rr, acc[1 + f - E0]);
    int e = 1 + P;
#pragma unroll
    for (int f = 0; f < P; ++f)
#pragma unroll
      for (int h = f; h < P; ++h) {
        if (e >= E0 && e < E1) acc[e - E0] = fmaf(jw[f], jw[h], acc[e - E0]);
        ++e;
      }
  }
  warp_sum_scatter(acc, lane, [&](int e, float v) { s_red[warp * NA + E0 + e] = v; });
}

// Sum of n FP32 values v[0], v[stride], ... in that order, in FP32 with a running
// compensation term (Neumaier's variant of Kahan summation): s + c is within about
// n u^2 sum|v| of the exact sum (u = 2^-24), as close as an FP64 accumulation of the
// same values, at the FP32 rate.  FP64 arithmetic issues at a small fraction of that
// rate here, and a chain of n FP64 conversions and additions on the few summing
// threads held the whole block for about a microsecond per tile.
__device__ __forceinline__ double compensated_sum(const float* v, int stride, int n) {
  float s = v[0], c = 0.f;
  for (int w = 1; w < n; ++w) {
    const float x = v[w * stride];
    const float t = s + x;
    c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  return (double)s + (double)c;
}

// Accumulate J^T W J (packed upper triangle), J^T W r and chi^2 for P free
// parameters over this thread's pixels of the tile, reduce over the block and
// write the tile's FP64 partial sums.  NCH > 1 accumulates the entries in that
// many ranges one after the other (fewer live registers, the pixels' loads
// shared), for the 512-thread instances of many free parameters.
template <int P, int kMinThreads, int NCH = 1>
__device__ __forceinline__ void reduce_tile(const FusedArgs& A, const float* s_out, float* s_red, size_t base, int H,
                                            int W, size_t prow, int i0, int j0) {
  constexpr int NA = 1 + P + P * (P + 1) / 2;
  constexpr int kPx = kTilePix / kMinThreads;  // pixels per thread in the smallest block of the instance
  const int tid = threadIdx.x, nthr = blockDim.x;
  // every image, sigma and mask load of this thread's pixels first, so that the
  // tile waits for one memory latency rather than one per pixel (loading them
  // before the correlation instead was measured slower: registers)
  float dv[kPx], sv[kPx];
  bool use[kPx];
#pragma unroll
  for (int k = 0; k < kPx; ++k) {
    const int pix = tid + k * nthr;
    const int i = i0 + pix / kTile, j = j0 + pix % kTile;
    use[k] = pix < kTilePix && i < H && j < W;
    dv[k] = 0.f;
    sv[k] = 1.f;
    if (use[k]) {
      const size_t gp = base + (size_t)i * W + j;
      dv[k] = A.image[gp];
      sv[k] = A.sigma[gp];
      if (A.mask) use[k] = A.mask[gp] == 0;
    }
  }
  const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
  static_assert(NCH >= 1 && NCH <= 3, "one to three accumulator ranges");
  if constexpr (NCH == 1) {
    reduce_range<P, kPx, 0, NA>(s_out, s_red, dv, sv, use, tid, nthr, lane, warp);
  } else if constexpr (NCH == 2) {
    reduce_range<P, kPx, 0, NA / 2>(s_out, s_red, dv, sv, use, tid, nthr, lane, warp);
    reduce_range<P, kPx, NA / 2, NA>(s_out, s_red, dv, sv, use, tid, nthr, lane, warp);
  } else {
    reduce_range<P, kPx, 0, NA / 3>(s_out, s_red, dv, sv, use, tid, nthr, lane, warp);
    reduce_range<P, kPx, NA / 3, 2 * NA / 3>(s_out, s_red, dv, sv, use, tid, nthr, lane, warp);
    reduce_range<P, kPx, 2 * NA / 3, NA>(s_out, s_red, dv, sv, use, tid, nthr, lane, warp);
  }
  __syncthreads();
  for (int e = tid; e < NA; e += nthr) A.partial[prow * NA + e] = compensated_sum(s_red + e, NA, nwarp);
}

// ---------------------------------------------------------------------------
// k_fused
// ---------------------------------------------------------------------------
// CPT = channel pairs per thread: 1 (128 threads per pair, up to 512 threads)
// or 2 (fewer threads with the register budget the reduction of many free
// parameters needs).
// WIDE (with CPT = 2): 512 threads in four groups, launched only with 4 pairs per pass
// (groups 2k and 2k+1 split pairs 2k and 2k+1 by PSF rows) or 2 (all four groups split
// both pairs); the reduction accumulates in ranges of up to 52 entries.
template <int MODE, int P, int CPT, int WIDE>
__global__ void __launch_bounds__(CPT == 1 || WIDE ? 512 : 256, 1) k_fused(const __grid_constant__ FusedArgs A) {
  extern __shared__ __align__(128) unsigned char smem[];
  float* s_psf = reinterpret_cast<float*>(smem + A.off_psf);
  float2* s_in = reinterpret_cast<float2*>(smem + A.off_in);
  float* s_out = reinterpret_cast<float*>(smem + A.off_out);
  float* s_cc0 = reinterpret_cast<float*>(smem + A.off_cc);        // [2][n_comp * kCC], alternating per item
  float* s_scale0 = reinterpret_cast<float*>(smem + A.off_scale);  // [2][scale_stride(n_slots)]
  float* s_red = reinterpret_cast<float*>(smem + A.off_red);
  u64* bar = reinterpret_cast<u64*>(smem + A.off_bar);
  int* s_flag = reinterpret_cast<int*>(smem + A.off_bar + 8);
  ItemInfo* s_info = reinterpret_cast<ItemInfo*>(smem + A.off_info);  // [2], alternating per item
  const ChanMap& m = A.m;
  const int cc_n = m.n_comp * kCC, sc_n = scale_stride(m.n_slots);

  const int tid = threadIdx.x, nthr = blockDim.x;
  const int n_items = A.n_items_dev ? *A.n_items_dev : A.n_items;
  if ((int)blockIdx.x >= n_items) return;

  bool inflight = false;  // thread 0: a window load is outstanding on the mbarrier
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *s_flag = 0;
    fetch_item(A, n_items, blockIdx.x, &s_info[0]);
    if (!(A.starve && blockIdx.x == 0)) {
      issue_pass(A, s_info[0], s_in, bar, 0, s_psf, s_cc0, s_scale0);
      inflight = true;
    }
  }
  unsigned phase = 0;
  int slot = 0;

  const int grp = tid / kGroupThreads;
  const int t = tid - grp * kGroupThreads;
  const int lane = t & 31, wig = t >> 5;
  // warp w runs on scheduler w % 4, next to the warps of the same index in the other
  // groups.  At a stamp's top or bottom edge the row skip shortens some 8-row blocks'
  // PSF-row ranges (28, 36, 41, 41 rows for K = 41), so the blocks are dealt out such
  // that every scheduler gets the same mix: with four groups, group g takes block
  // (w + g) mod 4 (each scheduler one of every block); with two, the odd group takes
  // them in reverse order (a short and a long block per scheduler)
  const int ngroup = nthr / kGroupThreads;
  const int wb = ngroup == 4 ? (wig + grp) & 3 : (grp & 1) ? 3 - wig : wig;

  for (;;) {
    __syncthreads();  // the previous item is done with s_psf, s_cc, s_scale, s_out, s_red and s_info[slot ^ 1]
    const ItemInfo& I = s_info[slot];
    if (!I.valid) break;
    const int H = I.geo.H, W = I.geo.W, K = I.geo.K, rw = I.geo.rw;
    const int c = (K - 1) / 2;
    const int i0 = (I.tile / I.geo.tiles_x) * kTile, j0 = (I.tile % I.geo.tiles_x) * kTile;
    if (MODE == MODE_NORMAL && tid < 6 * kTile) {
      // bring the tile's image, sigma and mask rows into L1 while the CTA correlates, so
      // that the reduction's loads do not wait on DRAM: one line at each end of a row
      // segment (the segment may straddle two 128-byte lines)
      const int r = tid % kTile, which = tid / kTile;
      const int arr = which >> 1, end = which & 1;
      if (i0 + r < H && (arr < 2 || A.mask)) {
        const size_t gp = (size_t)I.geo.pix + (size_t)(i0 + r) * W + j0 + (end ? min(kTile, W - j0) - 1 : 0);
        const void* ptr = arr == 0 ? (const void*)(A.image + gp)
                        : arr == 1 ? (const void*)(A.sigma + gp) : (const void*)(A.mask + gp);
        asm volatile("prefetch.L1 [%0];" ::"l"(ptr));
      }
    }
    // this item's PSF rows (s_psf) and constants arrive with its first window
    const float* s_cc = s_cc0 + slot * cc_n;
    const float* s_scale = s_scale0 + slot * sc_n;
    // The item's lane map.  Warp block wb is 8 rows x 32 columns, and PSF rows whose
    // input rows all fall outside the stamp for the warp's 8 rows are skipped -- or, for
    // a tile whose zero padding lies in columns only (a left or right edge tile away from
    // the top and bottom), 32 rows x 8 columns, and each PSF row's taps whose input
    // columns fall outside the stamp for all of the warp's columns are skipped (col_skip)
    const bool row_pad = i0 - c < 0 || i0 + kTile - 1 + c >= H;
    const bool col_pad = j0 - c < 0 || j0 + kTile - 1 + c >= W;
    const bool by_col = col_pad && !row_pad;
    const int row = by_col ? lane : wb * 8 + (lane & 7);
    const int col0 = by_col ? wb * 8 : (lane >> 3) * 8;
    int a_lo = 0, a_hi = K;
    ColSkip cs = col_all(K);
    if (by_col) {
      const int jl = j0 + col0;
      const int lead = max(0, c - (jl + 7)), trail = max(0, K - (c + W - jl));
      if (lead + trail >= K) a_hi = 0;  // none of the warp's taps reads inside the stamp
      else cs = col_skip(K, lead, trail);
    } else {
      a_lo = max(0, c - i0 - wb * 8 - 7);
      a_hi = min(K, c - i0 + H - wb * 8);
    }

    for (int pass = 0; pass < A.passes; ++pass) {
      // wait for this pass's window (thread 0 polls with a bound, the CTA agrees)
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
      mbar_try_wait(bar, phase);  // completes at once: acquires the TMA writes for this thread
      phase ^= 1u;
      if (pass == 0 && tid == 0) {
        // claim and read the next item; its loads are issued after this item's last window.
        // Done here rather than before the wait, so that the other warps do not wait for
        // the claim's round trips: warp 0 starts correlating late, and the other warps of
        // its scheduler keep the FMA pipe busy meanwhile
        const int nxt = (int)gridDim.x + atomicAdd(A.queue, 1);
        fetch_item(A, n_items, nxt, &s_info[slot ^ 1]);
      }

      // the pass's pairs spread evenly over the groups: group q takes npass / ngroups
      // pairs, one more for the first npass % ngroups groups (at most CPT)
      const int first = pass * A.pp;
      const int npass = min(A.pp, m.ncp - first);
      const int ngroups = nthr / kGroupThreads;
      // fewer pairs than two per group: rather than one pair per thread (8 accumulators,
      // measured ~16% slower per FMA), the pass's pairs go in sets of two to gps = 2 or 4
      // groups each, which take both pairs over their part of each warp's PSF rows
      const int nsets = npass >> 1;
      const int gps = nsets > 0 ? ngroups / nsets : 0;
      const bool split = CPT == 2 && (npass & 1) == 0 && nsets * gps == ngroups && (gps == 2 || (WIDE && gps == 4));
      const int base = npass / ngroups, rem = npass - base * ngroups;
      const int npair = split ? 2 : base + (grp < rem ? 1 : 0);
      const int part = split ? grp % gps : 0;
      const int lp0 = split ? 2 * (grp / gps) : grp * base + min(grp, rem);
      const int ga_lo = split ? a_lo + part * (a_hi - a_lo) / gps : a_lo;
      const int ga_hi = split ? a_lo + (part + 1) * (a_hi - a_lo) / gps : a_hi;
      u64 acc2[2][8];
      u64 acc1[1][8];
      if (CPT == 2 && npair == 2)
        correlate_pairs<2, !WIDE>(acc2, s_in, s_psf, lp0, A.plane, rw, K, row, col0, ga_lo, ga_hi, cs);
      else if (npair == 1) correlate_pairs<1>(acc1, s_in, s_psf, lp0, A.plane, rw, K, row, col0, a_lo, a_hi, cs);
      __syncthreads();  // every warp is done reading the window
      {
        // the next window's copies, one per warp (lane 0), so that no warp is held for all
        // of them; thread 0 makes the barrier's arrival
        // (odd groups first: in a pass split by PSF rows they store after the even ones)
        const int nwarp = nthr >> 5;
        const int rank = (grp & 1) ? (ngroup - 1 - grp) >> 1 : ngroup / 2 + (ngroup - 1 - grp) / 2;
        const int k0 = (tid & 31) ? 1 << 30 : rank * 4 + 3 - wig;
        if (pass + 1 < A.passes) {
          issue_pass(A, I, s_in, bar, pass + 1, s_psf, nullptr, nullptr, k0, nwarp, tid == 0);
          inflight = tid == 0;
        } else if (s_info[slot ^ 1].valid) {
          issue_pass(A, s_info[slot ^ 1], s_in, bar, 0, s_psf, s_cc0 + (slot ^ 1) * cc_n, s_scale0 + (slot ^ 1) * sc_n,
                     k0, nwarp, tid == 0);
          inflight = tid == 0;
        }
      }
      if (split) {
        // the first part stores, the others add in turn
        if (part == 0) store_pairs<2>(acc2, s_out, first + lp0, m.nch_conv, row, col0);
        for (int q = 1; q < gps; ++q) {
          __syncthreads();
          if (part == q) add_pairs<2>(acc2, s_out, first + lp0, m.nch_conv, row, col0);
        }
      } else if (CPT == 2 && npair == 2) {
        store_pairs<2>(acc2, s_out, first + lp0, m.nch_conv, row, col0);
      } else if (npair == 1) {
        store_pairs<1>(acc1, s_out, first + lp0, m.nch_conv, row, col0);
      }
    }
    __syncthreads();

    // ---- unconvolved components at the output pixels ----
    const bool sky_fast = MODE == MODE_NORMAL && m.sky_comp >= 0;
    if (sky_fast) {
      // a lone flat sky: its level onto the model and 1 x its slot scale as its derivative
      // channel, the values the general loop below writes, without evaluating the component
      const float level = s_cc[m.sky_comp * kCC + 8];
      const int sch = m.sky_ch;
      const float dsc = sch >= 0 ? 1.f * s_scale[m.slot[m.sky_comp][0]] : 0.f;
      for (int pix = tid; pix < kTilePix; pix += nthr) {
        const int i = i0 + pix / kTile, j = j0 + pix % kTile;
        const int op = out_idx(pix);
        if (sch >= 0) s_out[sch * kTilePix + op] = (i < H && j < W) ? dsc : 0.f;
        if (i < H && j < W) s_out[op] += level;
      }
    }
    for (int pix = tid; pix < kTilePix && !sky_fast; pix += nthr) {
      const int op = out_idx(pix);
      for (int ch = m.nch_conv; ch < m.nch_tot; ++ch) s_out[ch * kTilePix + op] = 0.f;
    }
    if (m.any_unconv && !sky_fast) {
      // one component at a time: its kind, channels and scales are read once, and the
      // same thread owns the same pixels as in the loop above
      for (int cm = 0; cm < m.n_comp; ++cm) {
        if (m.conv[cm]) continue;
        const int kind = m.kind[cm];
        const float* cc = s_cc + cm * kCC;
        int chs[8];
        float scs[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          chs[k] = (MODE != MODE_MODEL && k < m.np[cm]) ? m.chan[cm][k] : -1;
          scs[k] = chs[k] >= 0 ? s_scale[m.slot[cm][k]] : 0.f;
        }
        const int own = m.comp_chan[cm];
        for (int pix = tid; pix < kTilePix; pix += nthr) {
          const int i = i0 + pix / kTile, j = j0 + pix % kTile;
          if (i >= H || j >= W) continue;
          const int op = out_idx(pix);
          float d[8];
          const float v = eval_component(kind, cc, i, j, d);
          s_out[op] += v;
          if (MODE == MODE_MODEL) {
            if (own >= 0) s_out[own * kTilePix + op] = v;
          } else {
#pragma unroll
            for (int k = 0; k < 8; ++k)  // compile-time k keeps d in registers
              if (chs[k] >= 0) s_out[chs[k] * kTilePix + op] += d[k] * scs[k];
          }
        }
      }
    }
    // no barrier here: the loops above and the outputs below touch only this thread's own
    // pixels (tid, tid + nthr, ...), and the barrier after the passes ordered the
    // correlation's stores before both

    // ---- outputs ----
    const size_t pix0 = (size_t)I.geo.pix;
    if (MODE == MODE_MODEL) {
      const size_t HW = (size_t)H * W;
      for (int pix = tid; pix < kTilePix; pix += nthr) {
        const int i = i0 + pix / kTile, j = j0 + pix % kTile;
        if (i >= H || j >= W) continue;
        const size_t off = (size_t)i * W + j;
        const int op = out_idx(pix);
        A.model_out[pix0 + off] = s_out[op];
        if (A.comp_out) {
          for (int cm = 0; cm < m.n_comp; ++cm)
            A.comp_out[(size_t)m.n_comp * pix0 + cm * HW + off] = s_out[m.comp_chan[cm] * kTilePix + op];
        }
      }
    } else {
      constexpr int NA = 1 + P + P * (P + 1) / 2;
      reduce_tile<P, WIDE ? 512 : kGroupThreads, WIDE ? (NA + 51) / 52 : 1>(A, s_out, s_red, pix0, H, W,
                                                                          (size_t)I.geo.tile0 + I.tile, i0, j0);
    }
    slot ^= 1;
  }
}

}  // namespace gm
