// gm_geom.cuh -- per-galaxy geometry of a batch whose stamps and PSFs may
// differ in size from galaxy to galaxy.
//
// Every kernel of the model+Jacobian pass works on items = (galaxy, 32x32
// output tile) and looks the galaxy's geometry up in a GalGeom table: where
// its stamp, PSF and channel-pair planes start, its sizes, where its tile
// partial sums go, and which TMA tensor map (one per distinct (H, W, K)
// class) describes its planes.  A batch of equal stamps is the one-class case
// and gets its table from k_geom_uniform on the device; an uneven batch gets
// it from the host.
#pragma once

#include <cstdint>

namespace gm {

constexpr int kTileSide = 32;

struct GalGeom {
  long long pix;    // first pixel of the stamp in image / sigma / mask / model_out
  long long psf;    // first PSF element
  long long plane;  // first float of the galaxy's pair planes: [ncp][H][Wp][2]
  int H, W, K, Wp;  // stamp rows, columns, PSF side, plane row pitch in pairs (W rounded up to even)
  int tiles_x, n_tiles, tile0, cls;  // tile columns, tiles, first tile in the partial-sum array, map class
  int z0, rw;                        // first plane in the class tensor map; window row pitch (pairs)
};
static_assert(sizeof(GalGeom) == 64, "GalGeom is one 64-byte record");

// Per-galaxy stride (floats) of the slot-scale array: n_slots rounded up to a
// multiple of 4, so every galaxy's row is a 16-byte multiple (bulk copies).
__host__ __device__ inline int scale_stride(int n_slots) { return (n_slots + 3) & ~3; }

// Shared-memory row pitch (in float2) of a (32+K-1)-row correlation window:
// >= K + 33 (the register window reads two columns past the last tap) and
// == 2 mod 4, so the 8 lanes of a quarter warp (8 consecutive rows) hit
// distinct 16-byte bank groups.
// Floats per PSF row of the fused pass (shared memory and the padded copy in the
// workspace): row a holds tap t at a * psf_row_floats(K) + 3 cpad + t with
// cpad = ((K-1)/2) & 1, zeros elsewhere.  With the window's alignment shift in
// front (cpad = 1) the taps sit 3 floats in, so that the full 2-tap chunks
// start on a 16-byte boundary and one float4 always serves two chunks;
// roundup4(K + 3) floats cover every read of a row (a multiple of 4, so rows
// and whole PSFs stay 16-byte aligned for the bulk copy).
__host__ __device__ inline int psf_row_floats(int K) { return (K + 6) & ~3; }

__host__ __device__ inline int window_pitch(int K) {
  int rw = K + 33;
  while (rw % 4 != 2) ++rw;
  return rw;
}

__host__ __device__ inline GalGeom uniform_geom(long long g, int H, int W, int K, int ncp) {
  GalGeom r;
  r.H = H;
  r.W = W;
  r.K = K;
  r.Wp = W + (W & 1);
  r.tiles_x = (W + kTileSide - 1) / kTileSide;
  r.n_tiles = r.tiles_x * ((H + kTileSide - 1) / kTileSide);
  r.pix = g * H * W;
  r.psf = g * K * K;
  r.plane = g * ncp * (long long)H * r.Wp * 2;
  r.tile0 = (int)(g * r.n_tiles);
  r.cls = 0;
  r.z0 = (int)(g * ncp);
  r.rw = window_pitch(K);
  return r;
}

#ifdef GM_HOST_TU
// Geometry table, processing order and the item list of one pass over every
// galaxy, for G equal stamps.
__global__ void k_geom_uniform(int G, int H, int W, int K, int ncp, GalGeom* geo, int* order, int2* items) {
  const int stride = gridDim.x * blockDim.x;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  for (int g = t0; g < G; g += stride) {
    geo[g] = uniform_geom(g, H, W, K, ncp);
    order[g] = g;
  }
  const int nt = ((W + kTileSide - 1) / kTileSide) * ((H + kTileSide - 1) / kTileSide);
  const long long n = (long long)G * nt;
  for (long long q = t0; q < n; q += stride) items[q] = make_int2((int)(q / nt), (int)(q % nt));
}
#endif  // GM_HOST_TU

}  // namespace gm
