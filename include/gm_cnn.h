/*
 * gm_cnn.h -- C ABI of the learned initialiser's layers (libgm).
 *
 * The paper fits from starting values chosen by hand and lists that as a
 * limitation, pointing to convolutional networks that estimate the parameters
 * of galaxy images (arxiv 2404.07780, Sec. 1 and Sec. 6).  These calls are the
 * layers of such a network, run on the B300's tensor cores: 3x3 stride-2
 * convolutions with zero padding 1 and dense layers, BF16 weights and
 * activations with FP32 accumulation, forward and backward, the input
 * preparation (2x2 block mean, asinh scaling), a mean-squared-error loss and
 * the Adam update.  The network built from them, its training on stamps
 * rendered by gm_model and its use as the LM starting point live in
 * paper_2404_07780_b300/cnn.py.
 *
 * Conventions
 *   All array arguments are DEVICE pointers on the current device; the caller
 *   owns all memory.  BF16 arrays are IEEE bfloat16 (2 bytes per element).
 *   Activations are NHWC: [n][h][w][c].  Convolution weights are
 *   [co][3][3][ci], dense weights [out][in], biases FP32.  A convolution of an
 *   h x w input gives an ((h+1)/2) x ((w+1)/2) output:
 *     y[b][i][j][o] = b[o] + sum_{ky,kx,c} x[b][2i+ky-1][2j+kx-1][c] w[o][ky][kx][c]
 *   (x = 0 outside the image), followed by max(0, .) when relu is set.
 *   Channel counts and feature counts are multiples of 8 (a convolution's
 *   input may also have 1 channel).  Every device operand (activations,
 *   weights, gradients, masks, workspaces) starts on a 16-byte boundary;
 *   GM_CNN_E_INVAL otherwise.  `stream` is a cudaStream_t (NULL = legacy
 *   default stream); calls only enqueue work.
 *   Returns GM_CNN_OK or a negative code; gm_cnn_last_error() describes the
 *   calling thread's last failure.  A kernel whose internal wait gives up
 *   (it never should) sets a device flag that gm_cnn_check_error reads.
 */
#ifndef GM_CNN_H
#define GM_CNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GM_CNN_OK 0
#define GM_CNN_E_INVAL (-1)
#define GM_CNN_E_CUDA (-2)
#define GM_CNN_E_NOMEM (-3)

const char *gm_cnn_last_error(void);

/* *flag = 1 if any CNN kernel on this device gave up waiting for its copies or its
 * tensor-core work since the last call (the flag is cleared when read; synchronous;
 * host int).  The outputs of the call whose kernel gave up are undefined; later calls
 * are not affected. */
int gm_cnn_check_error(int *flag);

/* A test of the timeout path (not part of the paper's method): in the next launch made
 * by the calling thread of the TMA-fed GEMM (a GM_CNN_PATH_TMA forward layer) or of the
 * fused first two layers (gm_cnn_conv12_fwd), block 0 issues no copy for its first K
 * slice (its first input rows), so the wait for it runs out after `polls` tests (each
 * at most ~2 us) with nothing in flight; the kernel sets the flag gm_cnn_check_error
 * reads and every block leaves normally.  One launch only; polls = 0 cancels. */
int gm_cnn_test_starve_next(unsigned polls);

/* Kernels that compute a forward layer (the value gm_cnn_fwd_path returns). */
#define GM_CNN_PATH_GATHER 0 /* GEMM whose threads gather the operands into shared memory */
#define GM_CNN_PATH_TMA 1    /* persistent GEMM fed by tensor-map copies into swizzled tiles */

/* Which kernel gm_cnn_conv_fwd (kind 0: nb, h, w_, ci, co) or gm_cnn_dense_fwd
 * (kind 1: nb = n, ci = fin, co = fout, fp32_out = an FP32 output is asked for;
 * h, w_ ignored) runs for these sizes:
 *   GM_CNN_PATH_TMA: convolution with ci a multiple of 32, h and w even, co a
 *     multiple of 64 up to 256, (w/2) dividing 128 and (h/2)(w/2) a multiple or
 *     a divisor of 128 (a tile of 128 output pixels is whole rows of whole
 *     images); dense layer with a BF16 output only, fin >= 64 and fout a
 *     multiple of 64 up to 256;
 *   GM_CNN_PATH_GATHER: every other case.
 * All paths give the same sums up to FP32 accumulation order.  Host only; returns
 * GM_CNN_E_INVAL for sizes the layer calls refuse. */
int gm_cnn_fwd_path(int kind, int nb, int h, int w_, int ci, int co, int fp32_out);

/* Forward convolution: y = [relu](conv3x3_s2(x, w) + b).  b may be NULL. */
int gm_cnn_conv_fwd(const void *x, const void *w, const float *b, void *y, int nb, int h, int w_, int ci, int co,
                    int relu, void *stream);

/* The network's first two convolutions in one kernel (inference; nothing of the
 * first layer's output is stored): y = relu(conv3x3_s2(relu(conv3x3_s2(x, w1) + b1),
 * w2) + b2) for x [nb][64][64][1] BF16, w1 [32][3][3][1] BF16, b1 [32] FP32 (or
 * NULL), w2 [64][3][3][32] BF16, b2 [64] FP32 (or NULL), y [nb][16][16][64] BF16.
 * Equal bit for bit to gm_cnn_conv_fwd(x, w1, b1) followed by gm_cnn_conv_fwd(.,
 * w2, b2), both with relu. */
int gm_cnn_conv12_fwd(const void *x, const void *w1, const float *b1, const void *w2, const float *b2, void *y,
                      int nb, void *stream);

/* Gradient of the input: dx = conv3x3_s2^T(dy, w), times (mask > 0) element by
 * element when mask (the ReLU output of the layer below, shaped like dx) is
 * not NULL.  ci must be a multiple of 8. */
int gm_cnn_conv_bwd_data(const void *dy, const void *w, const void *mask, void *dx, int nb, int h, int w_, int ci,
                         int co, void *stream);

/* Gradients of the weights (FP32 [co][3][3][ci]) and, when db is not NULL, of the
 * bias (FP32 [co]) from the layer input x and dy (dy already includes the
 * derivative of this layer's ReLU).  workspace: gm_cnn_conv_bwd_weight_workspace bytes. */
size_t gm_cnn_conv_bwd_weight_workspace(int nb, int h, int w_, int ci, int co);
int gm_cnn_conv_bwd_weight(const void *x, const void *dy, float *dw, float *db, int nb, int h, int w_, int ci, int co,
                           void *workspace, size_t ws_bytes, void *stream);

/* Dense layer y[n][o] = [relu](sum_i x[n][i] w[o][i] + b[o]); output BF16 (y_bf16)
 * and/or FP32 (y_f32). */
int gm_cnn_dense_fwd(const void *x, const void *w, const float *b, void *y_bf16, float *y_f32, int n, int fin,
                     int fout, int relu, void *stream);

/* dx[n][i] = sum_o dy[n][o] w[o][i], times (mask > 0) when mask is not NULL. */
int gm_cnn_dense_bwd_data(const void *dy, const void *w, const void *mask, void *dx, int n, int fin, int fout,
                          void *stream);

/* dw[o][i] = sum_n dy[n][o] x[n][i] (FP32), db[o] = sum_n dy[n][o] when db is not NULL. */
size_t gm_cnn_dense_bwd_weight_workspace(int n, int fin, int fout);
int gm_cnn_dense_bwd_weight(const void *x, const void *dy, float *dw, float *db, int n, int fin, int fout,
                            void *workspace, size_t ws_bytes, void *stream);

/* Network input: out[g][i][j] = asinh(scale * mean of image[g][2i..2i+1][2j..2j+1]),
 * BF16 [G][h/2][w/2] (one channel); image FP32 [G][h][w], h and w even. */
int gm_cnn_prep(const float *image, int G, int h, int w_, float scale, void *out, void *stream);

/* *loss = mean over rows and the first dv of d columns of (pred - target)^2 (FP32,
 * device); dpred[n][d] BF16 = d loss / d pred = 2 (pred - target) / (n dv), zero in
 * the columns past dv.
 * pred [n][d] FP32, target [n][dv] FP32. */
int gm_cnn_mse(const float *pred, const float *target, int n, int d, int dv, float *loss, void *dpred, void *stream);

/* One Adam step (Kingma & Ba 2015, bias-corrected, step >= 1) on count FP32
 * parameters with their moments m, v; param_bf16 (NULL or count BF16) receives
 * the rounded weights the layers read. */
int gm_cnn_adam(float *param, const float *grad, float *m, float *v, void *param_bf16, long long count, float lr,
                float beta1, float beta2, float eps, int step, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GM_CNN_H */
