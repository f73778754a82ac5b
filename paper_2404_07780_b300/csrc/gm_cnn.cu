// gm_cnn.cu -- C ABI of the learned initialiser's layers (include/gm_cnn.h):
// BF16 tensor-core GEMMs for 3x3 stride-2 convolutions and dense layers,
// forward and backward, plus the input preparation, the loss, bias-gradient
// sums, split-K reduction and the Adam update.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <mutex>

#include "../../include/gm_cnn.h"
#include "gm_cnn.cuh"
#include "gm_cnn_fwd.cuh"

using namespace gm::cnn;

// Set by a GEMM kernel whose mbarrier wait gave up; one per device, read by gm_cnn_check_error.
static __device__ int g_cnn_flag;

namespace {

thread_local char g_cnn_err[512] = "no error";

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_cnn_err, sizeof(g_cnn_err), fmt, ap);
  va_end(ap);
  return code;
}

#define CNN_CUDA(call)                                                                          \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) return fail(GM_CNN_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define CNN_LAUNCHED(what)                                                                             \
  do {                                                                                                 \
    cudaError_t e_ = cudaGetLastError();                                                               \
    if (e_ != cudaSuccess) return fail(GM_CNN_E_CUDA, "launch %s: %s", what, cudaGetErrorString(e_)); \
  } while (0)

typedef void (*GemmKernel)(GemmArgs);

template <int OP>
GemmKernel pick(int bn) {
  if (bn == 32) return k_gemm<OP, 32>;
  if (bn == 64) return k_gemm<OP, 64>;
  return k_gemm<OP, 128>;
}

GemmKernel pick_gemm(int op, int bn) {
  switch (op) {
    case DENSE_FWD: return pick<DENSE_FWD>(bn);
    case DENSE_BWD_DATA: return pick<DENSE_BWD_DATA>(bn);
    case DENSE_BWD_W: return pick<DENSE_BWD_W>(bn);
    case CONV_FWD: return pick<CONV_FWD>(bn);
    case CONV_BWD_DATA: return pick<CONV_BWD_DATA>(bn);
    default: return pick<CONV_BWD_W>(bn);
  }
}

int tile_n(int N) { return N <= 32 ? 32 : (N <= 64 ? 64 : 128); }

int sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 148;
  return n;
}

// Device address of g_cnn_flag on the current device, looked up once per device.
int err_flag(int** out) {
  static std::mutex mu;
  static int* flags[64] = {};
  int dev = 0;
  CNN_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(GM_CNN_E_INVAL, "device ordinal %d beyond 64", dev);
  std::lock_guard<std::mutex> lock(mu);
  if (!flags[dev]) {
    void* p = nullptr;
    CNN_CUDA(cudaGetSymbolAddress(&p, g_cnn_flag));
    flags[dev] = (int*)p;
  }
  *out = flags[dev];
  return GM_CNN_OK;
}

// K splits of a GEMM: enough CTAs to cover the SMs when the M x N tiles do not.
int choose_splits(int M, int N, int K, int bn, int max_splits) {
  const int tiles = ((M + kBM - 1) / kBM) * ((N + bn - 1) / bn);
  const int want = std::max(1, (2 * sms() + tiles - 1) / tiles);
  const int by_k = std::max(1, K / (4 * kBK));
  return std::max(1, std::min({want, by_k, max_splits}));
}

// Launch one GEMM over `splits` K ranges (a multiple of kBK each); *used = the ranges launched.
int run_gemm(int op, GemmArgs G, int splits, cudaStream_t st, int* used = nullptr) {
  if (used) *used = 0;
  if (G.M <= 0 || G.N <= 0) return GM_CNN_OK;
  const int bn = tile_n(G.N);
  splits = std::max(1, splits);
  int kspl = (G.K + splits - 1) / splits;
  kspl = std::max(kBK, (kspl + kBK - 1) / kBK * kBK);
  splits = std::max(1, (G.K + kspl - 1) / kspl);
  G.k_split = kspl;
  int rc = err_flag(&G.err);
  if (rc) return rc;
  GemmKernel k = pick_gemm(op, bn);
  const int smem = 2 * (kBM + bn) * kBK * 2 + 64;
  CNN_CUDA(cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  dim3 grid((G.M + kBM - 1) / kBM, (G.N + bn - 1) / bn, splits);
  k<<<grid, kThreads, smem, st>>>(G);
  CNN_LAUNCHED("k_gemm");
  if (used) *used = splits;
  return GM_CNN_OK;
}

// ---------------------------------------------------------------------------
// forward layers on the TMA path (k_fwd) and the fused first two convolutions (k_conv12)
// ---------------------------------------------------------------------------
// cuTensorMapEncodeTiled, looked up once through the runtime (no libcuda link).
int encode_fn(PFN_cuTensorMapEncodeTiled_v12000* out) {
  static std::mutex mu;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    CNN_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !f) return fail(GM_CNN_E_CUDA, "cuTensorMapEncodeTiled is not available");
    fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
  }
  *out = fn;
  return GM_CNN_OK;
}

// BF16 tensor map: dims[0] innermost, byte strides of dims 1.., box and traversal strides.
int encode_bf16(CUtensorMap* map, int rank, const void* base, const cuuint64_t* dims, const cuuint64_t* strides,
                const cuuint32_t* box, const cuuint32_t* estr, CUtensorMapSwizzle sw) {
  PFN_cuTensorMapEncodeTiled_v12000 enc;
  int rc = encode_fn(&enc);
  if (rc) return rc;
  const CUresult cr = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void*>(base), dims,
                          strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return fail(GM_CNN_E_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
  return GM_CNN_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Every operand 16-byte aligned (NULL counts as aligned: optional operands are checked for
// presence separately); the kernels move BF16 rows in 16-byte units.
bool all16(std::initializer_list<const void*> ps) {
  for (const void* p : ps)
    if (!aligned16(p)) return false;
  return true;
}

#define CNN_ALIGNED(what, ...)                                                         \
  do {                                                                                 \
    if (!all16({__VA_ARGS__}))                                                         \
      return fail(GM_CNN_E_INVAL, "%s: operands must be 16-byte aligned", what);       \
  } while (0)

// Geometry of a convolution on the TMA path: the 128 output pixels of a tile are TH
// full-width rows of TB images.  False when the layer does not fit the path.
bool conv_tile(int H, int W, int ci, int co, int* TH, int* TB) {
  if (ci < 32 || ci % 32 != 0 || co % 64 != 0 || co > kFwdMaxN || (H & 1) || (W & 1) || H < 2 || W < 2) return false;
  const int Ho = H / 2, Wo = W / 2, P = Ho * Wo;
  if (128 % Wo != 0 || 2 * Wo > 256) return false;
  if (P >= 128) {
    if (P % 128 != 0) return false;
    *TH = 128 / Wo;
    *TB = 1;
  } else {
    if (128 % P != 0) return false;
    *TH = Ho;
    *TB = 128 / P;
  }
  return 2 * *TH <= 256 && *TB <= 256;
}

int fwd_path(int kind, int H, int W, int ci, int co, int fp32_out) {
  if (kind == 0) {
    int th = 0, tb = 0;
    return conv_tile(H, W, ci, co, &th, &tb) ? GM_CNN_PATH_TMA : GM_CNN_PATH_GATHER;
  }
  return (!fp32_out && ci >= 64 && ci % 8 == 0 && co % 64 == 0 && co <= kFwdMaxN) ? GM_CNN_PATH_TMA
                                                                                    : GM_CNN_PATH_GATHER;
}

// Shared-memory stages: as many as fit beside the output tile in ~200 KB for 128-byte
// operand rows (one block per SM); six for 64-byte rows (two blocks per SM).
int fwd_stages(int BN, int KC) {
  if (KC == 32) return 6;
  const int stage = (kBM + BN) * KC * 2;
  return std::max(2, std::min(8, (200 * 1024 - (BN / 64) * kOutHalf - 1024 - 256) / stage));
}

template <int BN, int KC>
int launch_fwd(FwdArgs& F, cudaStream_t st) {
  void (*k)(FwdArgs) = F.starve ? k_fwd<BN, KC, true> : k_fwd<BN, KC, false>;
  F.stages = fwd_stages(BN, KC);
  const int smem = fwd_smem_bytes(BN, KC, F.stages);
  CNN_CUDA(cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int occ = 0;
  CNN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kFwdThreads, smem));
  const int grid = std::max(1, std::min(F.n_tiles, sms() * std::max(occ, 1)));
  k<<<grid, kFwdThreads, smem, st>>>(F);
  CNN_LAUNCHED("k_fwd");
  return GM_CNN_OK;
}

int run_fwd(FwdArgs& F, int BN, int KC, cudaStream_t st) {
  if (BN == 128) return KC == 64 ? launch_fwd<128, 64>(F, st) : launch_fwd<128, 32>(F, st);
  return KC == 64 ? launch_fwd<64, 64>(F, st) : launch_fwd<64, 32>(F, st);
}

// gm_cnn_test_starve_next: the poll limit of the next k_fwd launch made by this thread, 0 = none.
thread_local unsigned g_cnn_starve_polls = 0;

int fwd_common(FwdArgs& F, const float* b, int relu, int M, int N, void* y) {
  F.M = M;
  F.N = N;
  F.bias = b;
  F.relu = relu;
  F.polls = kFwdWaitSleep;
  if (g_cnn_starve_polls) {
    F.polls = g_cnn_starve_polls;
    F.starve = 1;
    g_cnn_starve_polls = 0;
  }
  int rc = err_flag(&F.err);
  if (rc) return rc;
  const int BN = N % 128 == 0 ? 128 : 64;
  F.n_ntiles = N / BN;
  F.n_tiles = ((M + kBM - 1) / kBM) * F.n_ntiles;
  const cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)M};
  const cuuint64_t strides[1] = {(cuuint64_t)N * 2};
  const cuuint32_t box[2] = {64, (cuuint32_t)kBM};
  const cuuint32_t estr[2] = {1, 1};
  return encode_bf16(&F.tc, 2, y, dims, strides, box, estr, CU_TENSOR_MAP_SWIZZLE_128B);
}

int conv_fwd_tma(const void* x, const void* w, const float* b, void* y, int nb, int H, int W, int ci, int co,
                 int relu, cudaStream_t st) {
  int TH = 0, TB = 0;
  conv_tile(H, W, ci, co, &TH, &TB);
  const int Ho = H / 2, Wo = W / 2, KC = ci % 64 == 0 ? 64 : 32;
  FwdArgs F;
  std::memset(&F, 0, sizeof(F));
  int rc = fwd_common(F, b, relu, nb * Ho * Wo, co, y);
  if (rc) return rc;
  const int BN = co / F.n_ntiles;
  const CUtensorMapSwizzle sw = KC == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  {
    const cuuint64_t dims[4] = {(cuuint64_t)ci, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)nb};
    const cuuint64_t strides[3] = {(cuuint64_t)ci * 2, (cuuint64_t)W * ci * 2, (cuuint64_t)H * W * ci * 2};
    const cuuint32_t box[4] = {(cuuint32_t)KC, (cuuint32_t)(2 * Wo), (cuuint32_t)(2 * TH), (cuuint32_t)TB};
    const cuuint32_t estr[4] = {1, 2, 2, 1};
    rc = encode_bf16(&F.ta, 4, x, dims, strides, box, estr, sw);
    if (rc) return rc;
  }
  {
    const cuuint64_t dims[2] = {(cuuint64_t)9 * ci, (cuuint64_t)co};
    const cuuint64_t strides[1] = {(cuuint64_t)9 * ci * 2};
    const cuuint32_t box[2] = {(cuuint32_t)KC, (cuuint32_t)BN};
    const cuuint32_t estr[2] = {1, 1};
    rc = encode_bf16(&F.tb, 2, w, dims, strides, box, estr, sw);
    if (rc) return rc;
  }
  F.conv = 1;
  F.cchunks = ci / KC;
  F.Ci = ci;
  F.P = Ho * Wo;
  F.Wo = Wo;
  F.nk = 9 * F.cchunks;
  return run_fwd(F, BN, KC, st);
}

int dense_fwd_tma(const void* x, const void* w, const float* b, void* y, int n, int fin, int fout, int relu,
                  cudaStream_t st) {
  FwdArgs F;
  std::memset(&F, 0, sizeof(F));
  int rc = fwd_common(F, b, relu, n, fout, y);
  if (rc) return rc;
  const int BN = fout / F.n_ntiles;
  {
    const cuuint64_t dims[4] = {(cuuint64_t)fin, (cuuint64_t)n, 1, 1};
    const cuuint64_t row = (cuuint64_t)fin * 2;
    const cuuint64_t strides[3] = {row, row * (cuuint64_t)n, row * (cuuint64_t)n};
    const cuuint32_t box[4] = {64, (cuuint32_t)kBM, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    rc = encode_bf16(&F.ta, 4, x, dims, strides, box, estr, CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return rc;
  }
  {
    const cuuint64_t dims[2] = {(cuuint64_t)fin, (cuuint64_t)fout};
    const cuuint64_t strides[1] = {(cuuint64_t)fin * 2};
    const cuuint32_t box[2] = {64, (cuuint32_t)BN};
    const cuuint32_t estr[2] = {1, 1};
    rc = encode_bf16(&F.tb, 2, w, dims, strides, box, estr, CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return rc;
  }
  F.conv = 0;
  F.nk = (fin + 63) / 64;
  return run_fwd(F, BN, 64, st);
}

int conv12(const void* x, const void* w1, const float* b1, const void* w2, const float* b2, void* y, int nb,
           cudaStream_t st) {
  Conv12Args C;
  std::memset(&C, 0, sizeof(C));
  int rc = err_flag(&C.err);
  if (rc) return rc;
  const cuuint32_t e2[2] = {1, 1}, e3[3] = {1, 1, 1};
  {
    const cuuint64_t dims[3] = {(cuuint64_t)kC12In, (cuuint64_t)kC12In, (cuuint64_t)nb};
    const cuuint64_t strides[2] = {(cuuint64_t)kC12In * 2, (cuuint64_t)kC12In * kC12In * 2};
    const cuuint32_t box[3] = {(cuuint32_t)kC12In, (cuuint32_t)kC12Rows, 1};
    rc = encode_bf16(&C.tx, 3, x, dims, strides, box, e3, CU_TENSOR_MAP_SWIZZLE_NONE);
    if (rc) return rc;
  }
  {
    const cuuint64_t dims[2] = {288, 64};
    const cuuint64_t strides[1] = {288 * 2};
    const cuuint32_t box[2] = {32, 64};
    rc = encode_bf16(&C.tw2, 2, w2, dims, strides, box, e2, CU_TENSOR_MAP_SWIZZLE_64B);
    if (rc) return rc;
  }
  {
    const cuuint64_t dims[2] = {64, (cuuint64_t)nb * 256};
    const cuuint64_t strides[1] = {64 * 2};
    const cuuint32_t box[2] = {64, (cuuint32_t)kBM};
    rc = encode_bf16(&C.ty, 2, y, dims, strides, box, e2, CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return rc;
  }
  C.w1 = (const bf16*)w1;
  C.b1 = b1;
  C.b2 = b2;
  C.n_tiles = 2 * nb;
  C.polls = kFwdWaitSleep;
  if (g_cnn_starve_polls) {
    C.polls = g_cnn_starve_polls;
    C.starve = 1;
    g_cnn_starve_polls = 0;
  }
  void (*k)(Conv12Args) = C.starve ? k_conv12<true> : k_conv12<false>;
  CNN_CUDA(cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, kC12Smem));
  k<<<std::min(C.n_tiles, sms()), kC12Threads, kC12Smem, st>>>(C);
  CNN_LAUNCHED("k_conv12");
  return GM_CNN_OK;
}

GemmArgs blank() {
  GemmArgs G;
  std::memset(&G, 0, sizeof(G));
  return G;
}

// ---------------------------------------------------------------------------
// small kernels
// ---------------------------------------------------------------------------
__global__ void k_reduce_splits(const float* __restrict__ part, int splits, long long n, float* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += part[z * n + i];
    out[i] = s;
  }
}

// db[c] = sum_r dy[r][c] (FP32 sums of BF16 rows); rows strided over the grid, one atomic per block and column
__global__ void k_colsum(const bf16* __restrict__ dy, int R, int C, float* db) {
  extern __shared__ float s_sum[];
  for (int c = threadIdx.x; c < C; c += blockDim.x) s_sum[c] = 0.f;
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)R * C;
       i += (long long)gridDim.x * blockDim.x)
    atomicAdd(&s_sum[i % C], __bfloat162float(dy[i]));
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) atomicAdd(&db[c], s_sum[c]);
}

// 2x2 block mean of an H x W stamp, then asinh(x * scale), as BF16 (one channel, NHWC)
__global__ void k_prep(const float* __restrict__ img, int G, int H, int W, float scale, bf16* out) {
  const int Ho = H / 2, Wo = W / 2;
  const long long n = (long long)G * Ho * Wo;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long g = i / (Ho * Wo);
    const int r = (int)(i - g * Ho * Wo), y = r / Wo, x = r - (r / Wo) * Wo;
    const float* p = img + (size_t)g * H * W + (size_t)(2 * y) * W + 2 * x;
    const float m = 0.25f * (p[0] + p[1] + p[W] + p[W + 1]);
    out[i] = __float2bfloat16(asinhf(m * scale));
  }
}

// The same values as k_prep, four outputs per thread: two float4 of each of the two input rows
// in, four BF16 out (8 bytes); needs w % 8 == 0 and fewer than 2^31 quads.
__global__ void k_prep4(const float* __restrict__ img, int G, int H, int W, float scale, bf16* out) {
  const int Ho = H / 2, Wq = W / 8;  // output quads per row
  const int per_img = Ho * Wq, n = G * per_img;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int g = i / per_img, r = i - g * per_img, y = r / Wq, xq = r - y * Wq;
    const float* p = img + (size_t)g * H * W + (size_t)(2 * y) * W + 8 * xq;
    const float4 a0 = *reinterpret_cast<const float4*>(p), a1 = *reinterpret_cast<const float4*>(p + 4);
    const float4 c0 = *reinterpret_cast<const float4*>(p + W), c1 = *reinterpret_cast<const float4*>(p + W + 4);
    const float m0 = 0.25f * (a0.x + a0.y + c0.x + c0.y), m1 = 0.25f * (a0.z + a0.w + c0.z + c0.w);
    const float m2 = 0.25f * (a1.x + a1.y + c1.x + c1.y), m3 = 0.25f * (a1.z + a1.w + c1.z + c1.w);
    bf16 o[4] = {__float2bfloat16(asinhf(m0 * scale)), __float2bfloat16(asinhf(m1 * scale)),
                 __float2bfloat16(asinhf(m2 * scale)), __float2bfloat16(asinhf(m3 * scale))};
    uint2 v;
    v.x = (unsigned)__bfloat16_as_ushort(o[0]) | ((unsigned)__bfloat16_as_ushort(o[1]) << 16);
    v.y = (unsigned)__bfloat16_as_ushort(o[2]) | ((unsigned)__bfloat16_as_ushort(o[3]) << 16);
    *reinterpret_cast<uint2*>(out + (size_t)g * Ho * (W / 2) + (size_t)y * (W / 2) + 4 * xq) = v;
  }
}

// loss = mean of (pred - t)^2 over the rows and the first dv of d columns; dpred = its gradient
// 2 (pred - t) / (n dv), zero in the other columns
__global__ void k_mse(const float* __restrict__ pred, const float* __restrict__ target, int n, int d, int dv,
                      float* loss, bf16* dpred) {
  __shared__ float s_part[32];
  float acc = 0.f;
  const float g = 2.f / ((float)n * dv);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)n * d;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / d;
    const int c = (int)(i - r * d);
    float e = 0.f;
    if (c < dv) e = pred[i] - target[r * dv + c];
    acc += e * e;
    dpred[i] = __float2bfloat16(g * e);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += s_part[w];
    atomicAdd(loss, s / ((float)n * dv));
  }
}

// Adam (Kingma & Ba 2015) with bias correction; the BF16 copy of every updated weight
__global__ void k_adam(float* p, const float* __restrict__ grad, float* m, float* v, bf16* p_bf, long long n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (p_bf) p_bf[i] = __float2bfloat16(pi);
  }
}

int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 8LL * sms())); }

bool bad_conv(int nb, int H, int W, int ci, int co) {
  return nb < 0 || H < 1 || W < 1 || ci < 1 || co < 1 || co % 8 != 0 || (ci != 1 && ci % 8 != 0);
}

}  // namespace

extern "C" {

const char* gm_cnn_last_error(void) { return g_cnn_err; }

int gm_cnn_fwd_path(int kind, int nb, int h, int w, int ci, int co, int fp32_out) {
  if (kind == 0) return bad_conv(nb, h, w, ci, co) ? GM_CNN_E_INVAL : fwd_path(0, h, w, ci, co, 0);
  if (kind == 1)
    return (nb < 0 || ci < 1 || co < 1 || ci % 8 != 0 || co % 8 != 0) ? GM_CNN_E_INVAL
                                                                          : fwd_path(1, 0, 0, ci, co, fp32_out);
  return GM_CNN_E_INVAL;
}

int gm_cnn_check_error(int* flag) {
  int* d = nullptr;
  int rc = err_flag(&d);
  if (rc) return rc;
  int h = 0;
  CNN_CUDA(cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) CNN_CUDA(cudaMemset(d, 0, sizeof(int)));
  if (flag) *flag = h;
  return GM_CNN_OK;
}

int gm_cnn_test_starve_next(unsigned polls) {
  g_cnn_starve_polls = polls;
  return GM_CNN_OK;
}

int gm_cnn_conv_fwd(const void* x, const void* w, const float* b, void* y, int nb, int H, int W, int ci, int co,
                    int relu, void* stream) {
  if (bad_conv(nb, H, W, ci, co) || !x || !w || !y)
    return fail(GM_CNN_E_INVAL, "conv_fwd: bad arguments (nb=%d %dx%d ci=%d co=%d)", nb, H, W, ci, co);
  CNN_ALIGNED("conv_fwd", x, w, y);
  if (nb == 0) return GM_CNN_OK;
  const int path = fwd_path(0, H, W, ci, co, 0);
  if (path == GM_CNN_PATH_TMA) return conv_fwd_tma(x, w, b, y, nb, H, W, ci, co, relu, (cudaStream_t)stream);
  GemmArgs G = blank();
  G.Ho = (H + 1) / 2;
  G.Wo = (W + 1) / 2;
  G.M = nb * G.Ho * G.Wo;
  G.N = co;
  G.K = 9 * ci;
  G.x = (const bf16*)x;
  G.w = (const bf16*)w;
  G.nb = nb, G.H = H, G.W = W, G.Ci = ci, G.Co = co;
  G.bias = b;
  G.relu = relu;
  G.out_bf = (bf16*)y;
  return run_gemm(CONV_FWD, G, 1, (cudaStream_t)stream);
}

int gm_cnn_conv12_fwd(const void* x, const void* w1, const float* b1, const void* w2, const float* b2, void* y,
                      int nb, void* stream) {
  if (nb < 0 || !x || !w1 || !w2 || !y) return fail(GM_CNN_E_INVAL, "conv12_fwd: bad arguments (nb=%d)", nb);
  CNN_ALIGNED("conv12_fwd", x, w1, w2, y);
  if (nb == 0) return GM_CNN_OK;
  return conv12(x, w1, b1, w2, b2, y, nb, (cudaStream_t)stream);
}

int gm_cnn_conv_bwd_data(const void* dy, const void* w, const void* mask, void* dx, int nb, int H, int W, int ci,
                         int co, void* stream) {
  if (bad_conv(nb, H, W, ci, co) || ci % 8 != 0 || !dy || !w || !dx)
    return fail(GM_CNN_E_INVAL, "conv_bwd_data: bad arguments (nb=%d %dx%d ci=%d co=%d)", nb, H, W, ci, co);
  CNN_ALIGNED("conv_bwd_data", dy, w, mask, dx);
  GemmArgs G = blank();
  G.Ho = (H + 1) / 2;
  G.Wo = (W + 1) / 2;
  G.M = nb * H * W;
  G.N = ci;
  G.K = 9 * co;
  G.dy = (const bf16*)dy;
  G.w = (const bf16*)w;
  G.nb = nb, G.H = H, G.W = W, G.Ci = ci, G.Co = co;
  G.mask = (const bf16*)mask;
  G.out_bf = (bf16*)dx;
  return run_gemm(CONV_BWD_DATA, G, 1, (cudaStream_t)stream);
}

size_t gm_cnn_conv_bwd_weight_workspace(int nb, int H, int W, int ci, int co) {
  if (bad_conv(nb, H, W, ci, co)) return 0;
  return (size_t)kMaxSplits * co * 9 * ci * sizeof(float);
}

int gm_cnn_conv_bwd_weight(const void* x, const void* dy, float* dw, float* db, int nb, int H, int W, int ci, int co,
                           void* workspace, size_t ws_bytes, void* stream) {
  if (bad_conv(nb, H, W, ci, co) || !x || !dy || !dw)
    return fail(GM_CNN_E_INVAL, "conv_bwd_weight: bad arguments (nb=%d %dx%d ci=%d co=%d)", nb, H, W, ci, co);
  CNN_ALIGNED("conv_bwd_weight", x, dy, workspace);
  if (!workspace || ws_bytes < gm_cnn_conv_bwd_weight_workspace(nb, H, W, ci, co))
    return fail(GM_CNN_E_NOMEM, "conv_bwd_weight: workspace too small");
  cudaStream_t st = (cudaStream_t)stream;
  GemmArgs G = blank();
  G.Ho = (H + 1) / 2;
  G.Wo = (W + 1) / 2;
  G.M = co;
  G.N = 9 * ci;
  G.K = nb * G.Ho * G.Wo;
  G.x = (const bf16*)x;
  G.dy = (const bf16*)dy;
  G.nb = nb, G.H = H, G.W = W, G.Ci = ci, G.Co = co;
  G.out_f = (float*)workspace;
  int used = 0;
  int rc = run_gemm(CONV_BWD_W, G, choose_splits(G.M, G.N, G.K, tile_n(G.N), kMaxSplits), st, &used);
  if (rc) return rc;
  const long long n = (long long)G.M * G.N;
  k_reduce_splits<<<grid_for(n), 256, 0, st>>>((const float*)workspace, used, n, dw);
  CNN_LAUNCHED("k_reduce_splits");
  if (db) {
    CNN_CUDA(cudaMemsetAsync(db, 0, co * sizeof(float), st));
    k_colsum<<<grid_for((long long)G.K * co), 256, co * sizeof(float), st>>>((const bf16*)dy, G.K, co, db);
    CNN_LAUNCHED("k_colsum");
  }
  return GM_CNN_OK;
}

int gm_cnn_dense_fwd(const void* x, const void* w, const float* b, void* y_bf16, float* y_f32, int n, int fin,
                     int fout, int relu, void* stream) {
  if (n < 0 || fin < 1 || fout < 1 || fin % 8 != 0 || fout % 8 != 0 || !x || !w || (!y_bf16 && !y_f32))
    return fail(GM_CNN_E_INVAL, "dense_fwd: bad arguments (n=%d fin=%d fout=%d)", n, fin, fout);
  CNN_ALIGNED("dense_fwd", x, w, y_bf16, y_f32);
  if (n == 0) return GM_CNN_OK;
  if (!y_f32 && fwd_path(1, 0, 0, fin, fout, 0) == GM_CNN_PATH_TMA)
    return dense_fwd_tma(x, w, b, y_bf16, n, fin, fout, relu, (cudaStream_t)stream);
  GemmArgs G = blank();
  G.M = n;
  G.N = fout;
  G.K = fin;
  G.x = (const bf16*)x;
  G.w = (const bf16*)w;
  G.fin = fin, G.fout = fout;
  G.bias = b;
  G.relu = relu;
  G.out_bf = (bf16*)y_bf16;
  G.out_f = y_f32;
  return run_gemm(DENSE_FWD, G, 1, (cudaStream_t)stream);
}

int gm_cnn_dense_bwd_data(const void* dy, const void* w, const void* mask, void* dx, int n, int fin, int fout,
                          void* stream) {
  if (n < 0 || fin < 1 || fout < 1 || fin % 8 != 0 || fout % 8 != 0 || !dy || !w || !dx)
    return fail(GM_CNN_E_INVAL, "dense_bwd_data: bad arguments (n=%d fin=%d fout=%d)", n, fin, fout);
  CNN_ALIGNED("dense_bwd_data", dy, w, mask, dx);
  GemmArgs G = blank();
  G.M = n;
  G.N = fin;
  G.K = fout;
  G.dy = (const bf16*)dy;
  G.w = (const bf16*)w;
  G.fin = fin, G.fout = fout;
  G.mask = (const bf16*)mask;
  G.out_bf = (bf16*)dx;
  return run_gemm(DENSE_BWD_DATA, G, 1, (cudaStream_t)stream);
}

size_t gm_cnn_dense_bwd_weight_workspace(int n, int fin, int fout) {
  if (n < 0 || fin < 1 || fout < 1) return 0;
  return (size_t)kMaxSplits * fin * fout * sizeof(float);
}

int gm_cnn_dense_bwd_weight(const void* x, const void* dy, float* dw, float* db, int n, int fin, int fout,
                            void* workspace, size_t ws_bytes, void* stream) {
  if (n < 0 || fin < 1 || fout < 1 || fin % 8 != 0 || fout % 8 != 0 || !x || !dy || !dw)
    return fail(GM_CNN_E_INVAL, "dense_bwd_weight: bad arguments (n=%d fin=%d fout=%d)", n, fin, fout);
  CNN_ALIGNED("dense_bwd_weight", x, dy, workspace);
  if (!workspace || ws_bytes < gm_cnn_dense_bwd_weight_workspace(n, fin, fout))
    return fail(GM_CNN_E_NOMEM, "dense_bwd_weight: workspace too small");
  cudaStream_t st = (cudaStream_t)stream;
  GemmArgs G = blank();
  G.M = fout;
  G.N = fin;
  G.K = n;
  G.x = (const bf16*)x;
  G.dy = (const bf16*)dy;
  G.fin = fin, G.fout = fout;
  G.out_f = (float*)workspace;
  int used = 0;
  int rc = run_gemm(DENSE_BWD_W, G, choose_splits(G.M, G.N, G.K, tile_n(G.N), kMaxSplits), st, &used);
  if (rc) return rc;
  const long long cnt = (long long)G.M * G.N;
  k_reduce_splits<<<grid_for(cnt), 256, 0, st>>>((const float*)workspace, used, cnt, dw);
  CNN_LAUNCHED("k_reduce_splits");
  if (db) {
    CNN_CUDA(cudaMemsetAsync(db, 0, fout * sizeof(float), st));
    k_colsum<<<grid_for((long long)n * fout), 256, fout * sizeof(float), st>>>((const bf16*)dy, n, fout, db);
    CNN_LAUNCHED("k_colsum");
  }
  return GM_CNN_OK;
}

int gm_cnn_prep(const float* image, int G, int H, int W, float scale, void* out, void* stream) {
  if (G < 0 || H < 2 || W < 2 || (H & 1) || (W & 1) || !image || !out)
    return fail(GM_CNN_E_INVAL, "prep: bad arguments (G=%d %dx%d)", G, H, W);
  const long long n = (long long)G * (H / 2) * (W / 2);
  if (n == 0) return GM_CNN_OK;
  if (W % 8 == 0 && (long long)G * (H / 2) * (W / 8) < (1LL << 31) && aligned16(image) && aligned16(out)) {
    k_prep4<<<grid_for(n / 4), 256, 0, (cudaStream_t)stream>>>(image, G, H, W, scale, (bf16*)out);
    CNN_LAUNCHED("k_prep4");
    return GM_CNN_OK;
  }
  k_prep<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(image, G, H, W, scale, (bf16*)out);
  CNN_LAUNCHED("k_prep");
  return GM_CNN_OK;
}

int gm_cnn_mse(const float* pred, const float* target, int n, int d, int dv, float* loss, void* dpred, void* stream) {
  if (n < 0 || d < 1 || dv < 1 || dv > d || !pred || !target || !loss || !dpred)
    return fail(GM_CNN_E_INVAL, "mse: bad arguments (n=%d d=%d dv=%d)", n, d, dv);
  cudaStream_t st = (cudaStream_t)stream;
  CNN_CUDA(cudaMemsetAsync(loss, 0, sizeof(float), st));
  if (n == 0) return GM_CNN_OK;
  k_mse<<<std::min(grid_for((long long)n * d), 1024), 256, 0, st>>>(pred, target, n, d, dv, loss, (bf16*)dpred);
  CNN_LAUNCHED("k_mse");
  return GM_CNN_OK;
}

int gm_cnn_adam(float* param, const float* grad, float* m, float* v, void* param_bf16, long long count, float lr,
                float beta1, float beta2, float eps, int step, void* stream) {
  if (count < 0 || step < 1 || !param || !grad || !m || !v)
    return fail(GM_CNN_E_INVAL, "adam: bad arguments (count=%lld step=%d)", count, step);
  if (count == 0) return GM_CNN_OK;
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  k_adam<<<grid_for(count), 256, 0, (cudaStream_t)stream>>>(param, grad, m, v, (bf16*)param_bf16, count, lr, beta1,
                                                            beta2, eps, c1, c2);
  CNN_LAUNCHED("k_adam");
  return GM_CNN_OK;
}

}  // extern "C"
