// gm_cnn_fwd.cuh -- forward layers of the learned initialiser on the TMA path.
//
// k_fwd: C[M][N] = relu(A B^T + bias) in BF16 for the 3x3 stride-2 convolutions
// with 32 or more input channels and for the hidden dense layer.  A persistent,
// warp-specialised kernel:
//   * warp 0, one thread: tensor-map copies (cp.async.bulk.tensor) of the A and B
//     slices of a tile into a ring of shared-memory stages, each signalled on its
//     "full" mbarrier by the copy's byte count;
//   * warp 1: allocates 2 x BN TMEM columns (two accumulators), and one thread
//     issues tcgen05.mma (M = 128, N = BN, K = 16 each) on each stage, whose
//     completion tcgen05.commit signals on the stage's "empty" mbarrier; the last
//     slice of a tile commits to the accumulator's "full" barrier;
//   * warps 2-5: the epilogue.  tcgen05.ld of the accumulator (warp w reads TMEM
//     lanes 32 (w % 4) ..), bias and ReLU, BF16 into a swizzled shared-memory tile,
//     the accumulator released to the MMA thread, and one tensor-map store per
//     64 columns.  With two accumulators the epilogue of tile i overlaps the MMAs
//     of tile i + 1.
// Operand layouts are the K-major swizzled ones the copies write and the MMA
// descriptors name: rows of KC BF16 (128 bytes with the 128-byte swizzle for
// KC = 64, 64 bytes with the 64-byte swizzle for KC = 32), 8-row groups 8 KC x 2
// bytes apart; the K step of 16 elements moves the start address by 32 bytes.
//
// The convolution's im2col operand needs no gather: for tap (ky, kx) and channel
// chunk c, the A slice of 128 output pixels (b, y, x) is the box of the NHWC input
// tensor at (c KC, kx - 1, 2 y0 + ky - 1, b0) with traversal stride 2 in the two
// spatial dimensions (Wo x TH x TB elements land, TH x TB images' rows of full
// width), zero-filled outside the image.  K runs over (tap, channel) in the
// order of the weights [co][3][3][ci].
//
// k_conv12: the network's first two convolutions fused for inference (below).
#pragma once

#include <cuda.h>

#include "gm_cnn.cuh"

namespace gm {
namespace cnn {

constexpr int kFwdThreads = 192;  // warp 0: copies; warp 1: TMEM and MMA; warps 2-5: epilogue
constexpr int kOutHalf = kBM * 128;  // one 64-column BF16 half of an output tile (bytes)
// Polls of one wait before it gives up: a wait lasts microseconds (one tile's copies and
// MMAs), a poll tens of nanoseconds or more.
constexpr unsigned kFwdWait = 1u << 22;
constexpr unsigned kFwdWaitSleep = 1u << 20;  // tests that may each suspend the thread (at most ~2 s in all)
constexpr int kFwdMaxN = 256;  // output columns of a layer on this path (the bias in shared memory)

struct FwdArgs {
  CUtensorMap ta;  // A: conv -- NHWC input (ci, w, h, n), box (KC, 2 Wo, 2 TH, TB), strides (1, 2, 2, 1);
                   //    dense -- (K, M, 1, 1), box (KC, 128, 1, 1)
  CUtensorMap tb;  // B: weights [N][K], box (KC, BN)
  CUtensorMap tc;  // output [M][N] BF16, box (64, 128), 128-byte swizzle
  int M, N;
  int n_ntiles;    // N / BN
  int n_tiles;     // ceil(M / 128) * n_ntiles
  int nk;          // K slices of a tile
  int conv;        // 1: A is the convolution input
  int cchunks;     // conv: channel chunks of KC per tap (ci / KC)
  int Ci;          // conv: input channels
  int P;           // conv: output pixels per image (Ho Wo; a multiple or a divisor of 128)
  int Wo;          // conv: output width (a divisor of 128)
  int stages;      // shared-memory stages of the ring
  const float* bias;  // [N] or nullptr
  int relu;
  int* err;        // set when a wait gives up
  unsigned polls;  // tests of a wait before it gives up (kFwdWaitSleep)
  int starve;      // test of the timeout path: block 0 issues no copy for its first slice
};

__device__ __forceinline__ void mbar_init_n(u64* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(u64* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(u64* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// One test of an mbarrier phase that may suspend the thread until the phase completes or
// kSleepNs nanoseconds pass, so that a waiting lane does not take issue slots from the warps
// that work beside it.
constexpr unsigned kSleepNs = 2000;
__device__ __forceinline__ bool mbar_test_sleep(u64* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity), "r"(kSleepNs)
      : "memory");
  return done != 0;
}

// Bounded wait (`polls` tests) that also gives up soon after another role of the block has
// given up.
__device__ __forceinline__ bool fwd_wait(u64* bar, unsigned parity, volatile int* abort,
                                         unsigned polls = kFwdWaitSleep) {
  for (unsigned t = 0; t < polls; ++t) {
    if (mbar_test_sleep(bar, parity)) return true;
    if ((t & 15u) == 15u && *abort) return false;
  }
  return false;
}

// Bounded wait with no early exit (the copies and MMAs in flight when a block leaves).
__device__ __forceinline__ bool fwd_drain(u64* bar, unsigned parity) {
  for (unsigned t = 0; t < kFwdWait; ++t)
    if (mbar_test(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void fwd_fail(volatile int* abort, int* err) {
  *abort = 1;
  atomicExch(err, 1);
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            u64* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<u64>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, u64* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_addr(dst)),
      "l"(reinterpret_cast<u64>(map)), "r"(c0), "r"(c1), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int c0, int c1) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   reinterpret_cast<u64>(map)),
               "r"(c0), "r"(c1), "r"(smem_addr(src))
               : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void named_sync(unsigned id, unsigned n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Barrier over n threads that returns whether any of them passed true (the same answer in all).
__device__ __forceinline__ bool named_any(unsigned id, unsigned n, bool v) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((unsigned)v), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void tc_ld16(unsigned addr, float (&v)[16]) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int e = 0; e < 16; ++e) v[e] = __uint_as_float(r[e]);
}

// Shared-memory descriptor of a K-major swizzled operand: start address, leading
// byte offset 16 (unused by these layouts), stride byte offset = one 8-row group,
// version bits 46-48 = 0b001, swizzle mode at bits 61-63 (2: 128-byte, 4: 64-byte).
template <int KC>
__device__ __forceinline__ u64 sw_desc(unsigned saddr) {
  constexpr unsigned sbo = 8u * KC * 2u;
  constexpr u64 mode = KC == 64 ? 2 : 4;
  u64 d = (u64)((saddr & 0x3FFFFu) >> 4);
  d |= (u64)1 << 16;
  d |= (u64)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (u64)1 << 46;
  d |= mode << 61;
  return d;
}

// round(max(x, 0)) to BF16 for two values, packed (x0 in the low half): the same result as
// __float2bfloat16(fmaxf(x, 0.f)) element by element, in one instruction
__device__ __forceinline__ unsigned relu_bf16x2(float x0, float x1) {
  unsigned r;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(x1), "f"(x0));
  return r;
}

// round(x) to BF16 for two values, packed (x0 in the low half)
__device__ __forceinline__ unsigned bf16x2(float x0, float x1) {
  unsigned r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(x1), "f"(x0));
  return r;
}

// 8 FP32 accumulator values + 8 biases (16-byte aligned in shared memory), ReLU, as 8 BF16
__device__ __forceinline__ uint4 bias_relu8(const float* v, const float* b) {
  const float4 b0 = *reinterpret_cast<const float4*>(b), b1 = *reinterpret_cast<const float4*>(b + 4);
  return make_uint4(relu_bf16x2(v[0] + b0.x, v[1] + b0.y), relu_bf16x2(v[2] + b0.z, v[3] + b0.w),
                    relu_bf16x2(v[4] + b1.x, v[5] + b1.y), relu_bf16x2(v[6] + b1.z, v[7] + b1.w));
}

// the same without the ReLU
__device__ __forceinline__ uint4 bias_id8(const float* v, const float* b) {
  const float4 b0 = *reinterpret_cast<const float4*>(b), b1 = *reinterpret_cast<const float4*>(b + 4);
  return make_uint4(bf16x2(v[0] + b0.x, v[1] + b0.y), bf16x2(v[2] + b0.z, v[3] + b0.w),
                    bf16x2(v[4] + b1.x, v[5] + b1.y), bf16x2(v[6] + b1.z, v[7] + b1.w));
}

// Dynamic shared memory of k_fwd<BN, KC> with `stages` stages (1,024 bytes of
// alignment slack included).
__host__ __device__ constexpr int fwd_smem_bytes(int BN, int KC, int stages) {
  return 1024 + stages * (kBM + BN) * KC * 2 + (BN / 64) * kOutHalf + kFwdMaxN * 4 + (2 * stages + 5) * 8 + 16;
}

// kTest: the instance the timeout test launches, with the poll limit and the starved slice
// of FwdArgs; the other instance waits kFwdWaitSleep tests and has no test branch (reading
// the limit from the arguments cost the layers ~20 % of their time).
template <int BN, int KC, bool kTest>
__global__ void __launch_bounds__(kFwdThreads, 1) k_fwd(const __grid_constant__ FwdArgs F) {
  const unsigned polls = kTest ? F.polls : kFwdWaitSleep;
  const bool starve = kTest && F.starve && blockIdx.x == 0;
  static_assert(KC == 32 || KC == 64, "64- or 128-byte operand rows");
  static_assert(BN % 64 == 0 && BN <= 128, "output tiles of whole 64-column halves");
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  constexpr int A_BYTES = kBM * KC * 2, B_BYTES = BN * KC * 2, STAGE = A_BYTES + B_BYTES;
  constexpr int OUT_BYTES = (BN / 64) * kOutHalf;
  constexpr unsigned ncols = 2 * BN;
  const int S = F.stages;
  unsigned char* s_out = smem + S * STAGE;
  float* s_bias = reinterpret_cast<float*>(s_out + OUT_BYTES);  // [N], zeros without a bias
  u64* full = reinterpret_cast<u64*>(s_bias + kFwdMaxN);
  u64* empty = full + S;
  u64* tfull = empty + S;
  u64* tempty = tfull + 2;
  u64* drain = tempty + 2;
  unsigned* s_tmem = reinterpret_cast<unsigned*>(drain + 1);
  volatile int* s_abort = reinterpret_cast<volatile int*>(s_tmem + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init_n(&full[s], 1);
      mbar_init_n(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init_n(&tfull[a], 1);
      mbar_init_n(&tempty[a], 128);
    }
    mbar_init_n(drain, 1);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<u64>(&F.ta)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<u64>(&F.tb)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<u64>(&F.tc)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_tmem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  for (int c = threadIdx.x; c < F.N; c += kFwdThreads) s_bias[c] = F.bias ? F.bias[c] : 0.f;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = *s_tmem;

  if (warp == 0) {
    if (lane == 0) {
      // ---- copies ----
      unsigned g = 0;  // slices issued (over every tile of this block)
      bool ok = true;
      for (int t = blockIdx.x; ok && t < F.n_tiles; t += gridDim.x) {
        const int mt = t / F.n_ntiles, n0 = (t - mt * F.n_ntiles) * BN, m0 = mt * kBM;
        int b0 = 0, y0 = 0;
        if (F.conv) {
          b0 = m0 / F.P;
          y0 = (m0 - b0 * F.P) / F.Wo;
        }
        for (int j = 0; j < F.nk; ++j, ++g) {
          const int s = (int)(g % (unsigned)S);
          if (g >= (unsigned)S && !fwd_wait(&empty[s], ((g / S) - 1) & 1u, s_abort, polls)) {
            fwd_fail(s_abort, F.err);
            ok = false;
            break;
          }
          unsigned char* sa = smem + s * STAGE;
          if (starve && g == 0) continue;  // nothing arrives on full[0]
          mbar_expect_tx(&full[s], STAGE);
          int kb;
          if (F.conv) {
            const int tap = j / F.cchunks, ch = j - tap * F.cchunks, ky = tap / 3, kx = tap - 3 * ky;
            tma_load_4d(sa, &F.ta, ch * KC, kx - 1, 2 * y0 + ky - 1, b0, &full[s]);
            kb = tap * F.Ci + ch * KC;
          } else {
            tma_load_4d(sa, &F.ta, j * KC, m0, 0, 0, &full[s]);
            kb = j * KC;
          }
          tma_load_2d(sa + A_BYTES, &F.tb, kb, n0, &full[s]);
        }
      }
      if (!ok) {  // the copies still in flight land before the block leaves (none for a starved slice)
        for (unsigned h = g > (unsigned)S ? g - S : 0u; h < g; ++h)
          if (!(starve && h == 0)) fwd_drain(&full[h % S], (h / S) & 1u);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA ----
      constexpr unsigned idesc = idesc_bf16(kBM, BN);
      unsigned g = 0;
      int i = 0;
      bool ok = true;
      for (int t = blockIdx.x; ok && t < F.n_tiles; t += gridDim.x, ++i) {
        const int acc = i & 1;
        if (i >= 2 && !fwd_wait(&tempty[acc], ((i >> 1) - 1) & 1, s_abort, polls)) {
          fwd_fail(s_abort, F.err);
          break;
        }
        tc_fence_after();
        const unsigned d = tmem + (unsigned)(acc * BN);
        for (int j = 0; j < F.nk; ++j, ++g) {
          const int s = (int)(g % (unsigned)S);
          if (!fwd_wait(&full[s], (g / S) & 1u, s_abort, polls)) {
            fwd_fail(s_abort, F.err);
            ok = false;
            break;
          }
          tc_fence_after();
          const unsigned a0 = smem_addr(smem + s * STAGE), b0 = a0 + A_BYTES;
#pragma unroll
          for (int kk = 0; kk < KC / 16; ++kk)
            tc_mma(d, sw_desc<KC>(a0 + kk * 32), sw_desc<KC>(b0 + kk * 32), idesc, (j | kk) ? 1u : 0u);
          tc_commit(&empty[s]);
        }
        if (ok) tc_commit(&tfull[acc]);
      }
      tc_commit(drain);  // arrives once every MMA issued above has completed
      fwd_drain(drain, 0);
    }
  } else {
    // ---- epilogue: 128 threads, tile row r = TMEM lane ----
    const int q = warp & 3, r = q * 32 + lane, et = threadIdx.x - 64;
    int i = 0;
    for (int t = blockIdx.x; t < F.n_tiles; t += gridDim.x, ++i) {
      const int mt = t / F.n_ntiles, n0 = (t - mt * F.n_ntiles) * BN, m0 = mt * kBM;
      const int acc = i & 1;
      bool bad = false;
      if (lane == 0) bad = !fwd_wait(&tfull[acc], (i >> 1) & 1, s_abort, polls);
      __syncwarp();
      if (named_any(1, 128, bad)) {  // the same decision in every epilogue thread
        if (bad) fwd_fail(s_abort, F.err);
        break;
      }
      tc_fence_after();
      if (et == 0) bulk_wait_read0();  // the previous tile's stores have read the staging tile
      named_sync(1, 128);
      const unsigned taddr = tmem + ((unsigned)(q * 32) << 16) + (unsigned)(acc * BN);
#pragma unroll 1
      for (int j = 0; j < BN; j += 16) {
        float v[16];
        tc_ld16(taddr + (unsigned)j, v);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float* b = s_bias + n0 + j + h * 8;
          const int c = (j >> 3) + h;  // 8-column chunk of the tile row
          unsigned char* dst = s_out + (c >> 3) * kOutHalf + r * 128 + (((c & 7) ^ (r & 7)) << 4);
          *reinterpret_cast<uint4*>(dst) = F.relu ? bias_relu8(v + h * 8, b) : bias_id8(v + h * 8, b);
        }
      }
      tc_fence_before();
      mbar_arrive(&tempty[acc]);  // the accumulator may take the next tile
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      named_sync(1, 128);
      if (et == 0) {
#pragma unroll
        for (int h = 0; h < BN / 64; ++h) tma_store_2d(&F.tc, s_out + h * kOutHalf, n0 + h * 64, m0);
        bulk_commit();
      }
    }
    if (et == 0) bulk_wait0();
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

// ---------------------------------------------------------------------------
// the first two convolutions fused (inference)
// ---------------------------------------------------------------------------
// y2 = relu(conv3x3_s2(relu(conv3x3_s2(x, w1) + b1), w2) + b2) for 64x64 single-channel
// images, with conv1 (1 -> 32 channels, 32x32) kept in shared memory.  A tile is 8 rows x 16
// columns of one image's conv2 output (16x16, 64 channels: 128 TMEM lanes).  It needs conv1
// at rows 2 y0 - 1 .. 2 y0 + 15 and columns -1 .. 31 (17 x 33 positions (rr, cc), offsets from
// the first; those at -1 are conv2's zero padding), which need input rows 4 y0 - 3 .. 4 y0 + 31 (one
// 35 x 64 tensor-map box, zero-filled above the image).  Per tile:
//   1. im2col of conv1: row p holds the 9 input values of position p and 7 zeros (K = 16,
//      no-swizzle K-major core matrices); five MMAs (M = 128, N = 32, K = 16) give conv1 for
//      640 rows in TMEM (rows past the 561 positions read whatever follows and are not used);
//   2. the conv1 rows come back through tcgen05.ld: + b1, ReLU, BF16 (zero at the padding
//      positions), each written straight into the conv2 operand rows that read it: tap (ky, kx),
//      row m = (y - y0) 16 + x holds position (2 (y - y0) + ky, 2 x + kx) (1, 2 or 4 rows per
//      position; 32 channels in a 64-byte row with the 64-byte swizzle);
//   3. 18 MMAs (N = 64, K = 16) accumulate conv2;
//   4. TMEM -> + b2, ReLU, BF16 -> swizzled staging tile -> one tensor-map store.
// conv1 is the same single K = 16 MMA per row as the gathered GEMM's (whose other K steps add
// zero products) and conv2 the same 18 K steps as k_fwd's, so the output equals the two layers
// run one after the other bit for bit.
//
// One block per SM, persistent.  20 compute warps do steps 1, 2 and 4; one control thread
// issues the input copies (two tiles ahead), both MMA stages and the stores, each on an
// mbarrier the compute warps arrive on.  Steps are pipelined across tiles: conv1's MMAs run one
// tile ahead of conv2's (two conv1 accumulators in TMEM, two sets of conv2 operands in shared
// memory), so while the tensor cores contract tile i the compute warps build tile i + 1's
// im2col and read tile i + 1's conv1 back; the epilogue runs two tiles behind (two conv2
// accumulators).  In tile i the compute warps: wait conv1(i) -> im2col(i + 1) -> epilogue(i - 2)
// -> conv1(i) back into operand set i % 2; the control thread: conv1 MMAs of tile i + 1 ->
// store of tile i - 2 -> conv2 MMAs of tile i.  Waiting for conv1(i) also covers every MMA the
// control thread issued before it (conv2 of tile i - 2), which frees operand set i % 2 and the
// im2col buffer.
constexpr int kC12Compute = 640;             // compute threads (20 warps: 5 per TMEM lane quarter)
constexpr int kC12Groups = kC12Compute / 128;  // compute warps per lane quarter
constexpr int kC12Threads = kC12Compute + 32;  // + one control warp
constexpr int kC12In = 64;                   // input side
constexpr int kC12Rows = 35;                 // input rows of a tile
constexpr int kC12Pos = 17 * 33;             // conv1 positions of a tile
constexpr int kC12Rows1 = 640;               // conv1 GEMM rows (5 MMAs of 128)
constexpr int kC12B = 0;                     // conv2 weights: 9 taps x [64][32], 64-byte swizzle
constexpr int kC12A = 9 * 4096;              // conv2 operands: 2 sets x 9 taps x [128][32], 64-byte swizzle
constexpr int kC12ASet = 9 * 8192;
constexpr int kC12X = kC12A + 2 * kC12ASet;  // input rows: 2 buffers x [35][64] BF16
constexpr int kC12XBuf = 4608;
constexpr int kC12Out = kC12X + 2 * kC12XBuf;  // output staging [128][64] BF16, 128-byte swizzle
constexpr int kC12A1 = kC12Out + kOutHalf;     // conv1 im2col [561][16], core matrices
constexpr int kC12B1 = kC12A1 + 18 * 1024;     // conv1 weights [32][16], core matrices
constexpr int kC12Bias = kC12B1 + 1024;        // b1 [32], b2 [64] FP32
constexpr int kC12Bar = kC12Bias + 512;
constexpr int kC12End = kC12Bar + 128;
// the conv1 MMAs read 640 rows of the im2col buffer: the block's shared memory must reach there
constexpr int kC12Smem = 1024 + (kC12End > kC12A1 + kC12Rows1 * 32 ? kC12End : kC12A1 + kC12Rows1 * 32);
constexpr unsigned kC12Cols = 512;  // TMEM: conv2 accumulators at 0 and 64, conv1 at 128 and 288
constexpr unsigned kC12D1 = 128, kC12D1Stride = 160;
static_assert(kC12A % 1024 == 0 && kC12X % 1024 == 0 && kC12Out % 1024 == 0 && kC12A1 % 1024 == 0 &&
                  kC12B1 % 1024 == 0 && kC12XBuf >= kC12Rows * kC12In * 2,
              "aligned regions");
static_assert((((kC12Pos - 1) >> 3) + 1) * 256 <= 18 * 1024, "the 561 im2col rows fit their buffer");
static_assert(kC12Smem <= 227 * 1024, "one block's shared memory");
static_assert(kC12D1 + 2 * kC12D1Stride <= kC12Cols, "TMEM columns");

struct Conv12Args {
  CUtensorMap tx;   // input [nb][64][64] BF16: dims (64, 64, nb), box (64, 35, 1), zero fill
  CUtensorMap tw2;  // conv2 weights [64][288] BF16: box (32, 64), 64-byte swizzle
  CUtensorMap ty;   // output [nb * 256][64] BF16: box (64, 128), 128-byte swizzle
  const bf16* w1;   // conv1 weights [32][3][3][1]
  const float* b1;  // [32] or nullptr
  const float* b2;  // [64] or nullptr
  int n_tiles;      // 2 nb
  int* err;
  unsigned polls;   // tests of a wait before it gives up (kFwdWaitSleep)
  int starve;       // test of the timeout path: block 0 issues no copy of its first input rows
};

__device__ __forceinline__ void tma_load_3d_cnn(void* dst, const CUtensorMap* map, int c0, int c1, int c2, u64* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_addr(dst)),
      "l"(reinterpret_cast<u64>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
      : "memory");
}

// byte offset of 16-byte chunk kc (0, 1) of row r in a no-swizzle K-major [rows][16] operand
__device__ __forceinline__ unsigned k16_off(int r, int kc) {
  return (unsigned)((r >> 3) * 256 + kc * 128 + (r & 7) * 16);
}

// A compute warp's wait: lane 0 polls (unless the warp has already failed), the warp learns
// the outcome; returns false on failure.
__device__ __forceinline__ bool warp_wait(u64* bar, unsigned parity, volatile int* abort, bool ok, unsigned polls) {
  bool got = ok;
  if (ok && (threadIdx.x & 31) == 0) got = fwd_wait(bar, parity, abort, polls);
  return __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
}

__device__ __forceinline__ void warp_arrive(u64* bar) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(bar);
}

// Input rows of tile t (image t / 2, output rows 8 (t % 2) ..) into an input buffer.
__device__ __forceinline__ void c12_load_x(const Conv12Args& C, unsigned char* dst, int t, u64* bar) {
  mbar_expect_tx(bar, kC12Rows * kC12In * 2);
  tma_load_3d_cnn(dst, &C.tx, 0, 32 * (t & 1) - 3, t >> 1, bar);
}

// The conv1 position (rr, cc) of im2col row p: row rr = p / 33 holds the 17 even columns cc
// first, then the 16 odd ones, so that a warp's lanes (consecutive rows) read back positions of
// one column parity, whose operand rows lie in one tap tile (no bank conflicts between lanes)
__device__ __forceinline__ void c12_pos(int p, int& rr, int& cc) {
  rr = p / 33;
  const int j = p - rr * 33;
  cc = j < 17 ? 2 * j : 2 * (j - 17) + 1;
}

// What one compute thread writes in every tile, worked out once: its im2col row (640 threads,
// 561 rows) and its two conv1 read-back jobs (10 jobs of 16 columns per TMEM lane quarter,
// block b = j / 2, columns 16 (j % 2), dealt to the quarter's five warps), each with the conv2
// operand rows its value feeds.  Position (rr, cc) feeds row (y - y0, x) of tap (ky, kx) when
// rr = 2 (y - y0) + ky and cc = 2 x + kx: ky = rr % 2 with y - y0 = rr / 2, or ky = 2 with
// y - y0 = rr / 2 - 1 (rr even); likewise for the columns.  Only the padding of conv1 row -1 at
// the top of an image depends on the tile.
struct C12Plan {
  int xo;          // im2col: byte offset of input row 2 rr, column 2 c (c = cc - 1) in the box
  unsigned a1o;    // im2col: byte offset of the row's first 16-byte chunk (the second is 128 on)
  bool row, cpos, cgt0, top;   // a row of this thread; c >= 0; c > 0; rr == 0
  unsigned tcol[2];            // read-back: TMEM column of each job
  bool jok[2], jpad[2], jtop[2];  // position exists; cc == 0 (padding); rr == 0
  int off[2][4];   // operand rows fed: byte offset (tap 8192 + m 64 + swizzled chunk of channels
                   // 16 hcol ..) of the first 8 channels in the operand set, -1 for none; the next 8
                   // channels are at off ^ 16 (the chunk index's low bit)
};

__device__ __forceinline__ C12Plan c12_plan(int ctid, int q, int grp, int lane) {
  C12Plan P;
  int rr, cc;
  P.row = ctid < kC12Pos;
  c12_pos(P.row ? ctid : 0, rr, cc);
  const int c = cc - 1;
  P.xo = 2 * rr * (kC12In * 2) + 4 * c;
  P.a1o = k16_off(P.row ? ctid : 0, 0);
  P.cpos = c >= 0;
  P.cgt0 = c > 0;
  P.top = rr == 0;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int j = grp + k * kC12Groups, b = j >> 1, hcol = j & 1;
    const int p = b * kBM + q * 32 + lane;
    P.tcol[k] = (unsigned)(32 * b + 16 * hcol);
    P.jok[k] = p < kC12Pos;
    c12_pos(P.jok[k] ? p : 0, rr, cc);
    P.jpad[k] = cc == 0;
    P.jtop[k] = rr == 0;
    const int ky0 = rr & 1, ym0 = rr >> 1, kx0 = cc & 1, xm0 = cc >> 1;
    const bool y_ok[2] = {ym0 < 8, !(rr & 1) && rr >= 2}, x_ok[2] = {xm0 < 16, !(cc & 1) && cc >= 2};
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const int oy = d >> 1, ox = d & 1;
      const int ky = oy ? 2 : ky0, kx = ox ? 2 : kx0;
      const int m = (oy ? ym0 - 1 : ym0) * 16 + (ox ? xm0 - 1 : xm0);
      P.off[k][d] = (P.jok[k] && y_ok[oy] && x_ok[ox])
                        ? (ky * 3 + kx) * 8192 + m * 64 + (((2 * hcol) ^ ((m >> 1) & 3)) << 4)
                        : -1;
    }
  }
  return P;
}

// im2col row of conv1 for a tile with first output row y0: the 9 input values of the position
// (rows 2 rr + ky of the box, columns 2 c + kx - 1) and 7 zeros
__device__ __forceinline__ void c12_im2col(const C12Plan& P, const unsigned char* X, unsigned char* A1, int y0) {
  if (!P.row) return;
  unsigned v[5] = {0u, 0u, 0u, 0u, 0u};
  if (P.cpos && !(P.top && y0 == 0)) {
    unsigned e[9];
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      const unsigned char* row = X + P.xo + ky * (kC12In * 2);
      const unsigned pair = *reinterpret_cast<const unsigned*>(row);  // columns 2c, 2c + 1
      e[ky * 3] = P.cgt0 ? *reinterpret_cast<const unsigned short*>(row - 2) : 0u;
      e[ky * 3 + 1] = pair & 0xFFFFu;
      e[ky * 3 + 2] = pair >> 16;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = e[2 * k] | (e[2 * k + 1] << 16);
    v[4] = e[8];
  }
  *reinterpret_cast<uint4*>(A1 + P.a1o) = make_uint4(v[0], v[1], v[2], v[3]);
  *reinterpret_cast<uint4*>(A1 + P.a1o + 128) = make_uint4(v[4], 0u, 0u, 0u);
}

// conv1 back from TMEM accumulator d1 (this warp's lane quarter q): + b1, ReLU, BF16 (zero at
// the padding positions), each value written into the conv2 operand rows it feeds
__device__ __forceinline__ void c12_readout(const C12Plan& P, unsigned d1, unsigned char* A2, const float* s_b1,
                                            int y0, int q, int grp) {
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    float v[16];
    tc_ld16(d1 + ((unsigned)(q * 32) << 16) + P.tcol[k], v);
    if (!P.jok[k]) continue;
    const int hcol = (grp + k * kC12Groups) & 1;
    const bool pad = P.jpad[k] || (P.jtop[k] && y0 == 0);
    const uint4 v0 = pad ? zero4() : bias_relu8(v, s_b1 + 16 * hcol);
    const uint4 v1 = pad ? zero4() : bias_relu8(v + 8, s_b1 + 16 * hcol + 8);
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const int o = P.off[k][d];
      if (o < 0) continue;
      *reinterpret_cast<uint4*>(A2 + o) = v0;
      *reinterpret_cast<uint4*>(A2 + (o ^ 16)) = v1;
    }
  }
}

template <bool kTest>  // as k_fwd's
__global__ void __launch_bounds__(kC12Threads, 1) k_conv12(const __grid_constant__ Conv12Args C) {
  const unsigned polls = kTest ? C.polls : kFwdWaitSleep;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
  u64* xfull = reinterpret_cast<u64*>(smem + kC12Bar);  // [2] input rows of a buffer landed (copy)
  u64* mma = xfull + 2;        // [2] conv2 MMAs into an accumulator done (commit)
  u64* d1 = mma + 2;           // [2] conv1 MMAs into an accumulator done (commit)
  u64* a2full = d1 + 2;        // [2] a conv2 operand set written (every compute warp)
  u64* bfull = a2full + 2;     // conv2 weights landed (copy)
  u64* a1full = bfull + 1;     // im2col written (every compute warp)
  u64* outfull = a1full + 1;   // output staging tile written (every compute warp)
  u64* outfree = outfull + 1;  // output staging tile read by its store (control thread)
  u64* drain = outfree + 1;
  unsigned* s_tmem = reinterpret_cast<unsigned*>(drain + 1);
  volatile int* s_abort = reinterpret_cast<volatile int*>(s_tmem + 1);
  float* s_b1 = reinterpret_cast<float*>(smem + kC12Bias);
  float* s_b2 = s_b1 + 32;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char* A1 = smem + kC12A1;
  unsigned char* out = smem + kC12Out;
  constexpr int kCtl = kC12Compute / 32;  // the control warp
  // this block's tiles: t_i = blockIdx.x + i gridDim.x, i < n
  const int n = (C.n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  auto tile = [&](int i) { return (int)blockIdx.x + i * (int)gridDim.x; };
  auto xbuf = [&](int i) { return smem + kC12X + (i & 1) * kC12XBuf; };
  auto aset = [&](int i) { return smem + kC12A + (i & 1) * kC12ASet; };

  if (tid == 0) {
    for (int k = 0; k < 6; ++k) mbar_init_n(&xfull[k], 1);  // xfull, mma, d1: two each
    for (int k = 0; k < 2; ++k) mbar_init_n(&a2full[k], kC12Compute / 32);
    mbar_init_n(bfull, 1);
    mbar_init_n(a1full, kC12Compute / 32);
    mbar_init_n(outfull, kC12Compute / 32);
    mbar_init_n(outfree, 1);
    mbar_init_n(drain, 1);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kCtl) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_tmem)),
                 "r"(kC12Cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // conv1 weights as the B operand (row co = the 9 taps and 7 zeros) and the biases
  if (tid < 64) {
    const int co = tid >> 1, kc = tid & 1;
    bf16 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = kc * 8 + e;
      v[e] = k < 9 ? C.w1[co * 9 + k] : __float2bfloat16(0.f);
    }
    *reinterpret_cast<uint4*>(smem + kC12B1 + k16_off(co, kc)) = pack8(v);
  } else if (tid < 64 + 96) {
    const int k = tid - 64;
    if (k < 32) s_b1[k] = C.b1 ? C.b1[k] : 0.f;
    else s_b2[k - 32] = C.b2 ? C.b2[k - 32] : 0.f;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = *s_tmem;

  if (warp == kCtl) {
    if (lane == 0) {
      // ---- control thread: copies, MMAs, stores ----
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<u64>(&C.tx)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<u64>(&C.ty)) : "memory");
      constexpr unsigned idesc2 = idesc_bf16(kBM, 64), idesc1 = idesc_bf16(kBM, 32);
      const u64 da1 = smem_desc(smem_addr(A1), 128, 256), db1 = smem_desc(smem_addr(smem + kC12B1), 128, 256);
      const u64 db2 = sw_desc<32>(smem_addr(smem + kC12B));
      auto conv1 = [&](int i) {  // the conv1 MMAs of tile i (im2col in place)
        tc_fence_after();
        const unsigned d = tmem + kC12D1 + (unsigned)((i & 1) * kC12D1Stride);
#pragma unroll
        for (int b = 0; b < kC12Rows1 / kBM; ++b)
          tc_mma(d + (unsigned)(32 * b), da1 + (u64)((b * kBM * 32) >> 4), db1, idesc1, 0u);
        tc_commit(&d1[i & 1]);
      };
      int x_issued = 0;
      bool ok = true;
      mbar_expect_tx(bfull, 9 * 4096);
      for (int tap = 0; tap < 9; ++tap) tma_load_2d(smem + kC12B + tap * 4096, &C.tw2, tap * 32, 0, bfull);
      const bool starved = kTest && C.starve && blockIdx.x == 0;  // load 0 not issued: nothing arrives on xfull[0]
      for (; x_issued < 2 && x_issued < n; ++x_issued)
        if (!(starved && x_issued == 0)) c12_load_x(C, xbuf(x_issued), tile(x_issued), &xfull[x_issued]);
      if (!fwd_wait(bfull, 0, s_abort, polls) || !fwd_wait(a1full, 0, s_abort, polls)) ok = false;
      if (ok) conv1(0);
      int i = 0;
      for (; ok && i < n; ++i) {
        if (i + 2 < n) {  // the input buffer of tile i is free: its im2col was waited for
          c12_load_x(C, xbuf(i), tile(i + 2), &xfull[i & 1]);
          ++x_issued;
        }
        if (i + 1 < n) {  // conv1 of the next tile
          if (!fwd_wait(a1full, (i + 1) & 1, s_abort, polls)) { ok = false; break; }
          conv1(i + 1);
        }
        if (i >= 2) {  // the output of tile i - 2, once its staging tile is written; the tile is
                       // handed back as soon as the store has read it
          if (!fwd_wait(outfull, i & 1, s_abort, polls)) { ok = false; break; }
          tma_store_2d(&C.ty, out, 0, tile(i - 2) * kBM);
          bulk_commit();
          bulk_wait_read0();
          mbar_arrive(outfree);
        }
        if (!fwd_wait(&a2full[i & 1], (i >> 1) & 1, s_abort, polls)) { ok = false; break; }
        tc_fence_after();
        const u64 da2 = sw_desc<32>(smem_addr(aset(i)));
#pragma unroll
        for (int tap = 0; tap < 9; ++tap)
#pragma unroll
          for (int kk = 0; kk < 2; ++kk)
            tc_mma(tmem + (unsigned)((i & 1) * 64), da2 + (u64)((tap * 8192 + kk * 32) >> 4),
                   db2 + (u64)((tap * 4096 + kk * 32) >> 4), idesc2, (tap | kk) ? 1u : 0u);
        tc_commit(&mma[i & 1]);
      }
      for (int j = i >= 2 ? i - 2 : 0; ok && j < i; ++j) {  // the last two tiles' outputs
        if (!fwd_wait(outfull, j & 1, s_abort, polls)) {
          ok = false;
          break;
        }
        tma_store_2d(&C.ty, out, 0, tile(j) * kBM);
        bulk_commit();
        bulk_wait_read0();
        mbar_arrive(outfree);
      }
      if (!ok) {
        fwd_fail(s_abort, C.err);
        for (int h = x_issued > 2 ? x_issued - 2 : 0; h < x_issued; ++h)
          if (!(starved && h == 0)) fwd_drain(&xfull[h & 1], (h >> 1) & 1);  // the input loads in flight land
      }
      tc_commit(drain);  // arrives once every MMA issued above has completed
      fwd_drain(drain, 0);
      bulk_wait0();
    }
  } else {
    // ---- compute warps ----
    const int q = warp & 3, grp = warp >> 2;  // TMEM lane quarter and column group of this warp
    const C12Plan plan = c12_plan(tid, q, grp, lane);

    // staging tile of tile number j from conv2 accumulator j % 2; the tile is free once the store
    // of tile j - 1 has read it
    auto epilogue = [&](int j, bool ok) -> bool {
      ok = warp_wait(&mma[j & 1], (j >> 1) & 1, s_abort, ok, polls);
      if (j >= 1) ok = warp_wait(outfree, (j - 1) & 1, s_abort, ok, polls);
      if (ok && grp < 4) {  // four column groups of 16
        tc_fence_after();
        const int r = q * 32 + lane;
        float v[16];
        tc_ld16(tmem + ((unsigned)(q * 32) << 16) + (unsigned)((j & 1) * 64 + grp * 16), v);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = grp * 2 + h;
          *reinterpret_cast<uint4*>(out + r * 128 + ((c ^ (r & 7)) << 4)) = bias_relu8(v + h * 8, s_b2 + c * 8);
        }
        tc_fence_before();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      if (ok) warp_arrive(outfull);
      return ok;
    };

    bool ok = true;
    if (n > 0) {  // im2col of the first tile
      ok = warp_wait(&xfull[0], 0, s_abort, ok, polls);
      if (ok) {
        c12_im2col(plan, xbuf(0), A1, 8 * (tile(0) & 1));
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        warp_arrive(a1full);
      }
    }
    int i = 0;
    for (; ok && i < n; ++i) {
      // conv1 of tile i done: so are the conv2 MMAs of tile i - 2 (issued before it), which read
      // operand set i % 2, and the im2col buffer is free
      ok = warp_wait(&d1[i & 1], (i >> 1) & 1, s_abort, ok, polls);
      if (ok && i + 1 < n) {
        ok = warp_wait(&xfull[(i + 1) & 1], ((i + 1) >> 1) & 1, s_abort, ok, polls);
        if (ok) {
          c12_im2col(plan, xbuf(i + 1), A1, 8 * (tile(i + 1) & 1));
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          warp_arrive(a1full);
        }
      }
      // the epilogue of tile i - 2 before operand set i % 2 is handed over: conv2 of tile i
      // reuses its accumulator
      if (i >= 2) ok = epilogue(i - 2, ok);
      if (ok) {
        tc_fence_after();
        c12_readout(plan, tmem + kC12D1 + (unsigned)((i & 1) * kC12D1Stride), aset(i), s_b1, 8 * (tile(i) & 1), q,
                    grp);
        tc_fence_before();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        warp_arrive(&a2full[i & 1]);
      }
    }
    for (int j = i >= 2 ? i - 2 : 0; ok && j < i; ++j) ok = epilogue(j, ok);  // the last two tiles
    if (!ok && lane == 0) fwd_fail(s_abort, C.err);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kCtl) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kC12Cols) : "memory");
  }
}

}  // namespace cnn
}  // namespace gm
