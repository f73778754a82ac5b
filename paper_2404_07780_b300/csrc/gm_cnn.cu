// gm_cnn.cu -- C ABI of the learned initialiser's layers (include/gm_cnn.h):
// BF16 tensor-core GEMMs for 3x3 stride-2 convolutions and dense layers,
// forward and backward, plus the input preparation, the loss, bias-gradient
// sums, split-K reduction and the Adam update.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/gm_cnn.h"
#include "gm_cnn.cuh"

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

int gm_cnn_check_error(int* flag) {
  int* d = nullptr;
  int rc = err_flag(&d);
  if (rc) return rc;
  int h = 0;
  CNN_CUDA(cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) *flag = h;
  return GM_CNN_OK;
}

int gm_cnn_conv_fwd(const void* x, const void* w, const float* b, void* y, int nb, int H, int W, int ci, int co,
                    int relu, void* stream) {
  if (bad_conv(nb, H, W, ci, co) || !x || !w || !y)
    return fail(GM_CNN_E_INVAL, "conv_fwd: bad arguments (nb=%d %dx%d ci=%d co=%d)", nb, H, W, ci, co);
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

int gm_cnn_conv_bwd_data(const void* dy, const void* w, const void* mask, void* dx, int nb, int H, int W, int ci,
                         int co, void* stream) {
  if (bad_conv(nb, H, W, ci, co) || ci % 8 != 0 || !dy || !w || !dx)
    return fail(GM_CNN_E_INVAL, "conv_bwd_data: bad arguments (nb=%d %dx%d ci=%d co=%d)", nb, H, W, ci, co);
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
