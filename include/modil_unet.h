/*
 * modil_unet.h -- C ABI of the learned warm start of libmodil.so.
 *
 * The paper has no counterpart to this part: it solves every problem from a
 * zero (or uniform-inflow) initial guess (Section 3.5).  This is a small 3-D
 * convolutional U-Net that maps masked sparse velocity measurements on a
 * cubic grid to a first guess of the fields (u, v, w, p, chihat) of the body
 * problem, written into one level of the multigrid decomposition before the
 * mODIL iterations start; zero-initialised mODIL stays the fallback and the
 * final mODIL loss judges the guess.
 *
 * Network (levels = 4, base channels c): encoder level l (grid S/2^l,
 * c*2^l channels) = two 3x3x3 convolutions with bias and ReLU, 2x2x2 average
 * pooling between levels; decoder level l = nearest-neighbour upsampling of
 * level l+1, concatenation with the encoder output of level l, two 3x3x3
 * convolutions with ReLU; a 1x1x1 convolution with bias maps level 0 to the
 * output channels.  Zero padding at the grid boundary.
 *
 * Arithmetic: activations and weights in BF16, every contraction accumulates
 * in FP32 on the tensor cores (tcgen05, kind::f16), activations are rounded to
 * BF16 after bias and ReLU, the output layer is FP32.  Training: loss = mean
 * over (samples, cells, output channels) of (out - target)^2, hand-written
 * backward pass with the same rounding points (gradients of activations in
 * BF16, of weights in FP32), Adam on FP32 master weights.
 *
 * Layouts: channels last.  input: [batch][S^3][in_ch] FP32, output and
 * target: [batch][S^3][out_ch] FP32, cells row-major (z, y, x).  Parameter
 * tensors, host view: conv weight [c_out][27][c_in] (taps (dz, dy, dx) in
 * {-1,0,1}^3 lexicographic) or [c_out][c_in] for the 1x1x1 head, bias [c_out].
 * All pointers to tensors are device pointers unless stated; all work is on
 * the stream given at creation; calls that return numbers to the host
 * synchronise it.  Status codes and modil_last_error() as in modil.h.
 */
#ifndef MODIL_UNET_H
#define MODIL_UNET_H

#include <stddef.h>

#include "modil.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct modil_unet modil_unet; /* opaque, library-owned */

typedef struct {
  int side;      /* S: cells per axis, a multiple of 2^(levels-1)            */
  int batch;     /* samples per forward / training call (>= 1)               */
  int in_ch;     /* input channels, 1..8                                     */
  int out_ch;    /* output channels, 1..16                                   */
  int base_ch;   /* channels of level 0 (a multiple of 8, <= 64)             */
  int levels;    /* encoder levels, 2..5                                     */
  double adam_lr, adam_beta1, adam_beta2, adam_eps;
} modil_unet_desc;

/* Create a network with every parameter zero (write them before use).  The
 * library allocates its weights, optimiser state and workspace on the device. */
modil_status modil_unet_create(const modil_unet_desc* desc, void* stream, modil_unet** out);
void modil_unet_destroy(modil_unet* net);

/* Number of parameter tensors, and the shape of tensor i: kind 0 = conv
 * weight (dims c_out, taps, c_in), kind 1 = bias (dims c_out, 1, 1). */
modil_status modil_unet_param_count(const modil_unet* net, int* n);
modil_status modil_unet_param_shape(const modil_unet* net, int i, int* kind, int dims[3]);
/* Host FP32 copies of parameter tensor i in the host view (count elements). */
modil_status modil_unet_write_param(modil_unet* net, int i, const float* host, size_t count);
modil_status modil_unet_read_param(modil_unet* net, int i, float* host, size_t count);
/* Gradient of the last modil_unet_eval_grad / modil_unet_train_step. */
modil_status modil_unet_read_grad(modil_unet* net, int i, float* host, size_t count);

/* output = f(input) for `batch` samples. */
modil_status modil_unet_forward(modil_unet* net, const float* input, float* output);
/* Loss and the gradient of every parameter (no update); loss to *loss (host,
 * synchronises) if not NULL. */
modil_status modil_unet_eval_grad(modil_unet* net, const float* input, const float* target,
                                  double* loss);
/* eval_grad followed by one Adam step on every parameter.  The first call
 * captures the step (launches and memsets, the input and target copied into
 * the network's own buffers first) as a CUDA graph that later calls replay;
 * Adam's step counter and bias corrections are kept on the device.  If the
 * capture fails the call falls back to direct launches. */
modil_status modil_unet_train_step(modil_unet* net, const float* input, const float* target,
                                   double* loss);
/* Per-launch device times of one training step (ms), launch by launch;
 * *n receives the number of launches timed (<= max). */
modil_status modil_unet_profile_step(modil_unet* net, const float* input, const float* target,
                                     float* ms, int max, int* n);

/* How the 3x3x3 convolutions and their input and weight gradients run on
 * grids of 8^3 and more: implicit = 1 (the default) as implicit GEMMs whose
 * operands TMA reads as shifted boxes of the activations; 0 through explicit
 * im2col / col2im buffers around the same GEMM.  Both give the same sums up to
 * the order of FP32 accumulation. */
modil_status modil_unet_set_implicit(modil_unet* net, int implicit);

/* Whether modil_unet_train_step replays a captured CUDA graph (1, the
 * default) or launches every kernel directly (0); the two give bit-identical
 * results. */
modil_status modil_unet_set_graph(modil_unet* net, int on);

/* D (+)= A B^T on the tensor cores: A [M][K] and B [N][K] BF16 row-major with
 * row pitches lda, ldb (elements, multiples of 8, 16-byte aligned bases);
 * FP32 accumulation.  mode 0: D BF16 = relu?(acc + bias); mode 1: D FP32 =
 * acc + bias; mode 2: D FP32 += acc (atomic; splits > 1 divides K).  bias:
 * device FP32 [N] or NULL.  Asynchronous on `stream`. */
modil_status modil_gemm_bf16(const void* A, long long lda, const void* B, long long ldb, void* D,
                             long long ldd, int M, int N, int K, int mode, int relu,
                             const float* bias, int splits, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MODIL_UNET_H */
