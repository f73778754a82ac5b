// gm_cnn.cuh -- BF16 tensor-core kernels of the learned initialiser: a CNN of
// 3x3 stride-2 convolutions and dense layers, forward and backward.
//
// Every layer is one GEMM C[M][N] = sum_k A[M][k] B[N][k] on the 5th-generation
// tensor cores: a CTA owns a 128 x BN tile of C, accumulates it in tensor
// memory (TMEM, FP32) with tcgen05.mma.kind::f16 (BF16 inputs, one elected
// thread issues, M = 128, K = 16 per instruction), and reads it back with
// tcgen05.ld for a fused epilogue.  The operands are gathered from global
// memory by all threads -- im2col for the convolutions, transposes for the
// backward passes -- straight into shared memory in the no-swizzle K-major
// core-matrix layout the MMA descriptors describe: 8 rows x 16 bytes per core
// matrix, the 8 k-chunks of a 64-wide K slice of one 8-row group adjacent
// (leading byte offset 128 B), 8-row groups 1,024 B apart (stride byte
// offset).  Two shared-memory stages: the gather of slice s+1 overlaps the
// MMAs of slice s, whose completion tcgen05.commit signals on an mbarrier.
//
// Activations are NHWC BF16; conv weights [Co][3][3][Ci] BF16; dense weights
// [out][in] BF16; gradients of weights FP32.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

namespace gm {
namespace cnn {

typedef unsigned long long u64;
typedef __nv_bfloat16 bf16;

constexpr int kBM = 128;       // rows of a CTA tile (TMEM lanes)
constexpr int kBK = 64;        // K slice per shared-memory stage
constexpr int kThreads = 128;  // four warps: gather, one MMA issuer, epilogue by TMEM lane quarter
constexpr unsigned kWait = 1u << 26;
constexpr int kMaxSplits = 256;  // K splits of a weight-gradient GEMM (FP32 partials in the caller's workspace)

enum Op {
  DENSE_FWD = 0,       // Y[n][o]  = X[n][:] . W[o][:]                     A = X,      B = W
  DENSE_BWD_DATA = 1,  // dX[n][i] = dY[n][:] . W[:][i]                    A = dY,     B = W^T
  DENSE_BWD_W = 2,     // dW[o][i] = sum_n dY[n][o] X[n][i]                A = dY^T,   B = X^T
  CONV_FWD = 3,        // Y[b,y,x][co] = sum_{ky,kx,ci} X[b,2y+ky-1,2x+kx-1][ci] W[co][ky][kx][ci]
  CONV_BWD_DATA = 4,   // dX[b,i,j][ci] = sum_{ky,kx,co: i=2y+ky-1, j=2x+kx-1} dY[b,y,x][co] W[co][ky][kx][ci]
  CONV_BWD_W = 5,      // dW[co][ky,kx,ci] = sum_{b,y,x} dY[b,y,x][co] X[b,2y+ky-1,2x+kx-1][ci]
};

struct GemmArgs {
  int M, N, K;        // C[M][N] = sum_{k<K} A[M][k] B[N][k]
  int k_split;        // K range of one blockIdx.z (a multiple of kBK)
  const bf16* x;      // layer input (forward, weight gradient)
  const bf16* w;      // weights
  const bf16* dy;     // gradient of the layer output
  int nb, H, W, Ci, Co, Ho, Wo;  // conv geometry (NHWC input nb x H x W x Ci, output Ho x Wo x Co)
  int fin, fout;      // dense: in and out features
  const float* bias;  // [N] added in forward epilogues, or nullptr
  int relu;           // forward: max(0, .)
  const bf16* mask;   // backward data: times (mask > 0), the ReLU output of the layer below, or nullptr
  bf16* out_bf;       // [M][N] BF16, or nullptr
  float* out_f;       // [M][N] FP32 (split z at z*M*N), or nullptr
  int* err;           // set when an mbarrier wait gives up
};

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// ---------------------------------------------------------------------------
// operand gathers: 8 consecutive k of one row of A or B (zeros outside)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 zero4() { return make_uint4(0u, 0u, 0u, 0u); }

__device__ __forceinline__ uint4 pack8(const bf16 (&v)[8]) {
  uint4 r;
  r.x = (unsigned)__bfloat16_as_ushort(v[0]) | ((unsigned)__bfloat16_as_ushort(v[1]) << 16);
  r.y = (unsigned)__bfloat16_as_ushort(v[2]) | ((unsigned)__bfloat16_as_ushort(v[3]) << 16);
  r.z = (unsigned)__bfloat16_as_ushort(v[4]) | ((unsigned)__bfloat16_as_ushort(v[5]) << 16);
  r.w = (unsigned)__bfloat16_as_ushort(v[6]) | ((unsigned)__bfloat16_as_ushort(v[7]) << 16);
  return r;
}

// 8 elements p[0], p[s], ..., p[7 s] for the k still below kmax (k0 = first k)
__device__ __forceinline__ uint4 strided8(const bf16* p, long long s, int k0, int kmax) {
  bf16 v[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) v[e] = (k0 + e < kmax) ? p[e * s] : __float2bfloat16(0.f);
  return pack8(v);
}

// contiguous 8 elements when the run is aligned and complete, else element by element
__device__ __forceinline__ uint4 contig8(const bf16* p, int k0, int kmax) {
  if (k0 + 8 <= kmax && ((reinterpret_cast<uintptr_t>(p) & 15) == 0)) return *reinterpret_cast<const uint4*>(p);
  return strided8(p, 1, k0, kmax);
}

template <int OP>
__device__ __forceinline__ uint4 load_a(const GemmArgs& G, int row, int k) {
  if (row >= G.M || k >= G.K) return zero4();
  if (OP == DENSE_FWD) return contig8(G.x + (size_t)row * G.fin + k, k, G.K);
  if (OP == DENSE_BWD_DATA) return contig8(G.dy + (size_t)row * G.fout + k, k, G.K);
  if (OP == DENSE_BWD_W) return strided8(G.dy + (size_t)k * G.fout + row, G.fout, k, G.K);
  if (OP == CONV_FWD || OP == CONV_BWD_DATA) {
    // im2col row = one output (forward) or input (backward) pixel
    const int Wd = OP == CONV_FWD ? G.Wo : G.W, Hd = OP == CONV_FWD ? G.Ho : G.H;
    const int b = row / (Hd * Wd), rem = row - b * Hd * Wd, py = rem / Wd, px = rem - (rem / Wd) * Wd;
    const int C = OP == CONV_FWD ? G.Ci : G.Co;
    if (C % 8 == 0) {
      const int tap = k / C, c0 = k - tap * C, ky = tap / 3, kx = tap - 3 * (tap / 3);
      if (OP == CONV_FWD) {
        const int iy = 2 * py + ky - 1, ix = 2 * px + kx - 1;
        if (iy < 0 || iy >= G.H || ix < 0 || ix >= G.W) return zero4();
        return *reinterpret_cast<const uint4*>(G.x + (((size_t)b * G.H + iy) * G.W + ix) * G.Ci + c0);
      } else {
        const int ty = py + 1 - ky, tx = px + 1 - kx;
        if (ty < 0 || tx < 0 || (ty & 1) || (tx & 1) || ty / 2 >= G.Ho || tx / 2 >= G.Wo) return zero4();
        return *reinterpret_cast<const uint4*>(G.dy + (((size_t)b * G.Ho + ty / 2) * G.Wo + tx / 2) * G.Co + c0);
      }
    }
    bf16 v[8];  // narrow channel count (the first layer's single input channel): element by element
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      v[e] = __float2bfloat16(0.f);
      const int kk = k + e;
      if (kk >= G.K) continue;
      const int tap = kk / C, c = kk - tap * C, ky = tap / 3, kx = tap - 3 * (tap / 3);
      if (OP == CONV_FWD) {
        const int iy = 2 * py + ky - 1, ix = 2 * px + kx - 1;
        if (iy >= 0 && iy < G.H && ix >= 0 && ix < G.W) v[e] = G.x[(((size_t)b * G.H + iy) * G.W + ix) * G.Ci + c];
      } else {
        const int ty = py + 1 - ky, tx = px + 1 - kx;
        if (ty >= 0 && tx >= 0 && !(ty & 1) && !(tx & 1) && ty / 2 < G.Ho && tx / 2 < G.Wo)
          v[e] = G.dy[(((size_t)b * G.Ho + ty / 2) * G.Wo + tx / 2) * G.Co + c];
      }
    }
    return pack8(v);
  }
  // CONV_BWD_W: A[co][m] = dY[m][co]
  return strided8(G.dy + (size_t)k * G.Co + row, G.Co, k, G.K);
}

template <int OP>
__device__ __forceinline__ uint4 load_b(const GemmArgs& G, int col, int k) {
  if (col >= G.N || k >= G.K) return zero4();
  if (OP == DENSE_FWD) return contig8(G.w + (size_t)col * G.fin + k, k, G.K);
  if (OP == DENSE_BWD_DATA) return strided8(G.w + (size_t)k * G.fin + col, G.fin, k, G.K);
  if (OP == DENSE_BWD_W) return strided8(G.x + (size_t)k * G.fin + col, G.fin, k, G.K);
  if (OP == CONV_FWD) return contig8(G.w + (size_t)col * 9 * G.Ci + k, k, G.K);
  if (OP == CONV_BWD_DATA) {
    // B[ci][(tap, co)] = W[co][tap][ci]
    const int tap = k / G.Co, co = k - tap * G.Co;
    if (G.Co % 8 == 0) return strided8(G.w + ((size_t)co * 9 + tap) * G.Ci + col, (long long)9 * G.Ci, k, G.K);
    bf16 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int kk = k + e, t = kk / G.Co, c = kk - t * G.Co;
      v[e] = kk < G.K ? G.w[((size_t)c * 9 + t) * G.Ci + col] : __float2bfloat16(0.f);
    }
    return pack8(v);
  }
  // CONV_BWD_W: B[(tap, ci)][m] = X[b, 2y+ky-1, 2x+kx-1][ci] for output pixel m = (b, y, x)
  const int tap = col / G.Ci, ci = col - tap * G.Ci, ky = tap / 3, kx = tap - 3 * (tap / 3);
  bf16 v[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    v[e] = __float2bfloat16(0.f);
    const int m = k + e;
    if (m >= G.K) continue;
    const int b = m / (G.Ho * G.Wo), rem = m - b * G.Ho * G.Wo, y = rem / G.Wo, x = rem - (rem / G.Wo) * G.Wo;
    const int iy = 2 * y + ky - 1, ix = 2 * x + kx - 1;
    if (iy >= 0 && iy < G.H && ix >= 0 && ix < G.W) v[e] = G.x[(((size_t)b * G.H + iy) * G.W + ix) * G.Ci + ci];
  }
  return pack8(v);
}

// ---------------------------------------------------------------------------
// tcgen05 helpers (inline PTX)
// ---------------------------------------------------------------------------
// Shared-memory matrix descriptor, no swizzle: start address, leading byte
// offset (between the two k-adjacent core matrices of one MMA), stride byte
// offset (between 8-row groups), the fixed version bits 46-48 = 0b001.
__device__ __forceinline__ u64 smem_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
  u64 d = (u64)((saddr & 0x3FFFFu) >> 4);
  d |= (u64)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (u64)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (u64)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and B
// BF16 (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits
// 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr unsigned idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init1(u64* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test(u64* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ bool mbar_wait(u64* bar, unsigned parity) {
  for (unsigned t = 0; t < kWait; ++t)
    if (mbar_test(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(unsigned tmem, u64 adesc, u64 bdesc, unsigned idesc, unsigned accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void tc_commit(u64* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void tc_ld8(unsigned addr, float (&v)[8]) {
  unsigned r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int e = 0; e < 8; ++e) v[e] = __uint_as_float(r[e]);
}

// byte offset of the 16-byte run (row, k-chunk kc) in a rows x 64 tile
__device__ __forceinline__ unsigned core_off(int row, int kc) {
  return (unsigned)(((row >> 3) * 8 + kc) * 128 + (row & 7) * 16);
}

// ---------------------------------------------------------------------------
// the GEMM kernel
// ---------------------------------------------------------------------------
// Grid: (ceil(M/128), ceil(N/BN), splits of K).  Dynamic shared memory:
// 2 stages x (128 + BN) x 64 BF16 + barriers.
template <int OP, int BN>
__global__ void __launch_bounds__(kThreads) k_gemm(const __grid_constant__ GemmArgs G) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr int A_BYTES = kBM * kBK * 2, B_BYTES = BN * kBK * 2, STAGE = A_BYTES + B_BYTES;
  u64* bars = reinterpret_cast<u64*>(smem + 2 * STAGE);  // [0], [1]: stage MMAs done; [2]: all MMAs done
  unsigned* s_tmem = reinterpret_cast<unsigned*>(smem + 2 * STAGE + 32);
  int* s_flag = reinterpret_cast<int*>(smem + 2 * STAGE + 36);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
  const int kb = blockIdx.z * G.k_split;
  const int ke = min(G.K, kb + G.k_split);
  const int nk = ke > kb ? (ke - kb + kBK - 1) / kBK : 0;
  constexpr unsigned ncols = BN < 32 ? 32 : BN;  // TMEM columns: a power of two >= 32

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_tmem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init1(&bars[0]);
    mbar_init1(&bars[1]);
    mbar_init1(&bars[2]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *s_flag = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = *s_tmem;
  constexpr unsigned idesc = idesc_bf16(kBM, BN);

  for (int kt = 0; kt < nk; ++kt) {
    const int st = kt & 1;
    unsigned char* sa = smem + st * STAGE;
    unsigned char* sb = sa + A_BYTES;
    if (kt >= 2) {  // the MMAs that read this stage two slices ago are done
      if (tid == 0 && !mbar_wait(&bars[st], ((kt - 2) >> 1) & 1)) *s_flag = 1;
      __syncthreads();
      if (*s_flag) break;
    }
    const int k0 = kb + kt * kBK;
    // A: 128 rows x 8 k-chunks, B: BN rows x 8; consecutive threads take consecutive rows
    // of one chunk.  Every load of the slice is issued before any store, so that a thread
    // has all of them in flight at once (a load followed by its store in each loop
    // iteration waited one memory latency per chunk).
    constexpr int NA = kBM * 8 / kThreads, NB = BN * 8 / kThreads;
    static_assert(NA * kThreads == kBM * 8 && NB * kThreads == BN * 8, "whole chunks per thread");
    uint4 va[NA], vb[NB];
#pragma unroll
    for (int r = 0; r < NA; ++r) {
      const int c = tid + r * kThreads, row = c & (kBM - 1), kc = c >> 7;
      va[r] = load_a<OP>(G, m0 + row, k0 + kc * 8);
    }
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      const int c = tid + r * kThreads, row = c % BN, kc = c / BN;
      vb[r] = load_b<OP>(G, n0 + row, k0 + kc * 8);
    }
#pragma unroll
    for (int r = 0; r < NA; ++r) {
      const int c = tid + r * kThreads, row = c & (kBM - 1), kc = c >> 7;
      *reinterpret_cast<uint4*>(sa + core_off(row, kc)) = va[r];
    }
#pragma unroll
    for (int r = 0; r < NB; ++r) {
      const int c = tid + r * kThreads, row = c % BN, kc = c / BN;
      *reinterpret_cast<uint4*>(sb + core_off(row, kc)) = vb[r];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const unsigned a0 = smem_addr(sa), b0 = smem_addr(sb);
#pragma unroll
      for (int s = 0; s < kBK / 16; ++s)
        tc_mma(tmem, smem_desc(a0 + s * 256, 128, 1024), smem_desc(b0 + s * 256, 128, 1024), idesc,
               (kt > 0 || s > 0) ? 1u : 0u);
      tc_commit(&bars[st]);
    }
  }
  if (tid == 0) tc_commit(&bars[2]);  // completes when every MMA above has
  const bool ok = nk == 0 || (!*s_flag && mbar_wait(&bars[2], 0));
  if (!ok && tid == 0) atomicExch(G.err, 1);
  tc_fence_after();

  // epilogue: warp w owns TMEM lanes (tile rows) 32w .. 32w+31
  const int row = m0 + warp * 32 + lane;
  if (G.out_bf && !G.out_f && !G.mask) {
    // BF16 tile through shared memory (the operand stages are free once every MMA has
    // completed): each thread writes its row's 8-column runs, then consecutive threads
    // copy consecutive 16-byte runs of a row to global memory (coalesced)
    constexpr int PITCH = BN * 2 + 16;  // bytes per tile row; the 16-byte pad spreads rows over the banks
    static_assert(kBM * PITCH <= 2 * STAGE, "the output tile fits the operand stages");
    unsigned char* so = smem;
    for (int j = 0; j < BN; j += 8) {
      float v[8];
      if (nk > 0) tc_ld8(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)j, v);
      else {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = 0.f;
      }
      bf16 o[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int col = n0 + j + e;
        float t = v[e];
        if (G.bias && col < G.N) t += G.bias[col];
        if (G.relu) t = fmaxf(t, 0.f);
        o[e] = __float2bfloat16(t);
      }
      *reinterpret_cast<uint4*>(so + (warp * 32 + lane) * PITCH + j * 2) = pack8(o);
    }
    __syncthreads();
    if (ok) {
      for (int c = tid; c < kBM * (BN / 8); c += kThreads) {
        const int r = c / (BN / 8), ch = c - r * (BN / 8);
        const int grow = m0 + r, col = n0 + ch * 8;
        if (grow < G.M && col < G.N)  // N is a multiple of 8: a run is wholly inside or outside
          *reinterpret_cast<uint4*>(G.out_bf + (size_t)grow * G.N + col) =
              *reinterpret_cast<const uint4*>(so + r * PITCH + ch * 16);
      }
    }
  } else
  for (int j = 0; j < BN; j += 8) {
    float v[8];
    if (nk > 0) tc_ld8(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)j, v);
    else {
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = 0.f;
    }
    if (!ok || row >= G.M) continue;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int col = n0 + j + e;
      if (col >= G.N) break;
      float t = v[e];
      if (G.bias) t += G.bias[col];
      if (G.relu) t = fmaxf(t, 0.f);
      if (G.mask && !(__bfloat162float(G.mask[(size_t)row * G.N + col]) > 0.f)) t = 0.f;
      if (G.out_f) G.out_f[(size_t)blockIdx.z * G.M * G.N + (size_t)row * G.N + col] = t;
      if (G.out_bf) G.out_bf[(size_t)row * G.N + col] = __float2bfloat16(t);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

}  // namespace cnn
}  // namespace gm
