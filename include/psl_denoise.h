/*
 * psl_denoise.h -- C ABI of the dose denoiser that sits after the Monte
 * Carlo dose: a small BF16 3D convolutional encoder-decoder that maps a
 * low-history dose plus density to the high-history dose.  The paper has no
 * such step; it is trained on dose pairs the PSL method itself produces, and
 * the plain Monte Carlo run to 1 % uncertainty is its fallback and the reference
 * its accuracy is measured against.
 *
 * Conventions as in psl.h: return 0 (PSL_OK) or a negative PSL_E* code with
 * the text in psl_last_error(); device pointers are caller-owned; `stream` is
 * a cudaStream_t (NULL: the legacy default stream).  BF16 arrays are passed as
 * uint16_t (the raw bit pattern).  Volumes are channels-last: element
 * (z, y, x, c) of an nz x ny x nx volume with C channels is at
 * ((z*ny + y)*nx + x)*C + c.  BF16 arrays must be 16-byte aligned.
 */
#ifndef PSL_DENOISE_H
#define PSL_DENOISE_H

#include <stdint.h>

#include "psl.h"

#ifdef __cplusplus
extern "C" {
#endif

/* 3x3x3 convolution, zero padding 1.  Tap t = (dz+1)*9 + (dy+1)*3 + (dx+1)
 * for offsets dz, dy, dx in {-1, 0, 1}:
 *   out[v, o] = bias[o] + sum_t sum_i in[v + offset_t, i] w[t, i, o].
 * psl_conv3d_pack turns FP32 taps w[27][ci][co] (device) into the BF16 tile
 * layout the tensor-core kernel reads (psl_conv3d_packed_size(ci, co)
 * elements).  mirror = 1 packs the input-gradient form instead: the
 * convolution from co to ci channels with taps w'[t][o][i] = w[26-t][i][o],
 * so that psl_conv3d of an output gradient gives the input gradient. */
PSL_API int64_t psl_conv3d_packed_size(int32_t ci, int32_t co);
PSL_API int psl_conv3d_pack(const float *w, int32_t ci, int32_t co, int32_t mirror, uint16_t *wpk, void *stream);

/* The convolution on the tcgen05 tensor cores: BF16 operands, FP32
 * accumulation in tensor memory, then + bias (FP32, may be NULL), ReLU if
 * relu != 0, and the result written as BF16 to out and/or FP32 to out_f32
 * (either may be NULL, not both).  ci: a multiple of 8 up to 128; co: 16, 32,
 * 64 or 128; nx*ny*nz < 2^31.  Errors: PSL_EINVAL (shapes, alignment),
 * PSL_ETIMEOUT (a tensor-core completion wait gave up), PSL_ECUDA.
 * Synchronises stream. */
PSL_API int psl_conv3d(const uint16_t *in, int32_t ci, const uint16_t *wpk, const float *bias, int32_t co,
                       int32_t nx, int32_t ny, int32_t nz, int32_t relu, uint16_t *out, float *out_f32,
                       void *stream);

/* Which form psl_conv3d (and the network) uses: 0 (default) the halo form
 * where nx is a multiple of 128 and ci of 16 (a CTA's tiles are rows of 128
 * voxels; per 16-channel chunk and tap plane one input plane with its
 * one-voxel border is loaded by the tensor memory accelerator and the 9 taps
 * of the plane read shifted views of it), else the per-tap TMA form where
 * the volume allows (nx >= 128, or nx a power of two: the 128 voxels of a
 * CTA are one box of the volume, one shifted box per tap; warp-specialised
 * copy / MMA / epilogue roles, the copy engine's zero fill as the padding),
 * else the gather form; 1 the gather form everywhere (threads load the A
 * rows; two-stage ring); 2 as 0 without the halo form.  All give the same
 * result (the same products, summed in FP32 in the tensor core's order). */
PSL_API int psl_conv3d_form(int32_t form);

/* The tap gradient of that convolution, on the tensor cores:
 *   dw[t, i, o] += sum_v in[v + offset_t, i] gy[v, o]
 * (FP32 dw [27][ci][co], device, accumulated into: zero it first).  in BF16
 * [V][ci], gy BF16 [V][co]; shapes as psl_conv3d.  Synchronises stream. */
PSL_API int psl_conv3d_wgrad(const uint16_t *in, int32_t ci, const uint16_t *gy, int32_t co, int32_t nx, int32_t ny,
                             int32_t nz, float *dw, void *stream);

/* The denoiser network.  Input: dose / scale and density (two channels,
 * padded to 8); output: dose.  Layers (3x3x3 convolution + ReLU, channels):
 *   e0a 8->16, e0b 16->16  -> skip s0, 2x2x2 average pool
 *   e1 16->32              -> skip s1, pool
 *   e2 32->64              -> skip s2, pool
 *   b3a 64->128, b3b 128->64
 *   up x2 + s2, d2 64->32; up x2 + s1, d1 32->16; up x2 + s0, d0 16->16
 *   y = d0 . w_out + b_out + dose / scale;  out = y * scale.
 * Parameters (FP32, psl_denoiser_param_count() of them, in this order): for
 * each layer e0a..d0 its taps [27][ci][co] then its biases [co]; then w_out
 * [16], b_out [1].  psl_denoiser_create draws He-normal taps from `seed`,
 * zero biases and a zero output layer (the network starts as the identity
 * on the dose).  Volume sides must be multiples of 8.  All calls synchronise
 * stream. */
typedef struct psl_denoiser psl_denoiser_t;
PSL_API int64_t psl_denoiser_param_count(void);
PSL_API int psl_denoiser_create(uint64_t seed, psl_denoiser_t **out);
PSL_API void psl_denoiser_destroy(psl_denoiser_t *d);

/* Device arrays of psl_denoiser_param_count() floats, NULL to skip: `set`
 * replaces the parameters, `get` receives them, `grad` receives the
 * accumulated gradients (sums over the psl_denoiser_backward calls since the
 * last step). */
PSL_API int psl_denoiser_params(psl_denoiser_t *d, const float *set, float *get, float *grad, void *stream);

/* Denoise: dose and rho are FP32 device volumes [nz][ny][nx] (Gy, g/cm^3);
 * scale > 0 normalises the dose for the network (e.g. its maximum); out
 * (FP32, device, same shape) receives the denoised dose. */
PSL_API int psl_denoiser_forward(psl_denoiser_t *d, const float *dose, const float *rho, int32_t nx, int32_t ny,
                                 int32_t nz, float scale, float *out, void *stream);

/* One training sample: forward, the mean squared error against target / scale
 * over the voxels (written to *loss, host, may be NULL) and its gradient,
 * added to the accumulated gradients. */
PSL_API int psl_denoiser_backward(psl_denoiser_t *d, const float *dose, const float *rho, const float *target,
                                  int32_t nx, int32_t ny, int32_t nz, float scale, double *loss, void *stream);

/* Adam (beta1 0.9, beta2 0.999, eps 1e-8) with learning rate lr on the mean
 * of the accumulated gradients, which are then cleared. */
PSL_API int psl_denoiser_step(psl_denoiser_t *d, float lr, void *stream);

/* The k-th smallest (0-based, 0 <= k < n) of n FP32 values in device memory,
 * exactly, written to *out (host): radix selection on the values'
 * order-preserving bit patterns (three histogram passes over the values fix
 * 11, 11 and 10 bits of the answer).  The denoiser normalises a dose by its
 * 99.9th percentile: k = floor(0.999 n) - 1.  -0 orders below +0; NaNs with
 * the sign bit clear order above +inf, those with it set below -inf.  Uses
 * 8 KB of stream-ordered scratch; synchronises stream.  PSL_EINVAL for
 * n < 1, n >= 2^32, k out of range or null pointers. */
PSL_API int psl_kth_smallest(const float *x, int64_t n, int64_t k, float *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PSL_DENOISE_H */
