/*
 * psl_denoise.h -- C ABI of the dose denoiser that sits after the Monte
 * Carlo dose: a small BF16 3D convolutional encoder-decoder that maps a
 * low-history dose plus density to the high-history dose.  The paper has no
 * such step; it is trained on dose pairs the PSL method itself produces, and
 * the plain Monte Carlo run to 1 % uncertainty is its fallback and judge.
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

/* The tap gradient of that convolution, on the tensor cores:
 *   dw[t, i, o] += sum_v in[v + offset_t, i] gy[v, o]
 * (FP32 dw [27][ci][co], device, accumulated into: zero it first).  in BF16
 * [V][ci], gy BF16 [V][co]; shapes as psl_conv3d.  Synchronises stream. */
PSL_API int psl_conv3d_wgrad(const uint16_t *in, int32_t ci, const uint16_t *gy, int32_t co, int32_t nx, int32_t ny,
                             int32_t nz, float *dw, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PSL_DENOISE_H */
