// The dose denoiser's network on the GPU: a 4-level 3D encoder-decoder
// (16/32/64/128 channels, 3x3x3 convolutions with ReLU, 2x2x2 average
// pooling down, nearest 2x upsampling and additive skips up, a 1x1 output
// layer added to the input dose).  Activations are BF16, channels last; the
// convolutions and both of their gradients run on the tcgen05 tensor cores
// (conv.cu); pooling, skips, masks, the output layer, the loss and Adam are
// bandwidth-bound CUDA-core kernels.  Parameters, gradients and Adam moments
// are FP32 in one flat array each; after every update the taps are repacked
// into the BF16 tile layout (forward and mirrored).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <random>
#include <string>
#include <vector>

#include "../../include/psl_denoise.h"
#include "psl_internal.cuh"
#include "sort.cuh"

int psl_conv_ksteps(int ci);
int psl_conv3d_run(const __nv_bfloat16 *in, int ci, const __nv_bfloat16 *wpk, const float *bias, int co, int nx,
                   int ny, int nz, int relu, __nv_bfloat16 *out, float *out_f32, uint32_t *err, cudaStream_t st);
int psl_conv3d_pack_run(const float *w, int ci, int co, int mirror, __nv_bfloat16 *out, cudaStream_t st);
int psl_conv3d_wgrad_run(const __nv_bfloat16 *x, int ci, const __nv_bfloat16 *gy, int co, int nx, int ny, int nz,
                         float *dw, uint32_t *err, cudaStream_t st);

namespace {

typedef __nv_bfloat16 bf16;

struct LayerDef { int ci, co; };
enum { E0A, E0B, E1, E2, B3A, B3B, D2, D1, D0, NL };
constexpr LayerDef LAYERS[NL] = {{8, 16}, {16, 16}, {16, 32}, {32, 64}, {64, 128}, {128, 64}, {64, 32}, {32, 16}, {16, 16}};

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)psl_sm_count() * 16)); }

// ------------------------------------------------------------- kernels ---
__global__ void k_input(const float *dose, const float *rho, float inv_scale, int64_t V, bf16 *x8) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        __align__(16) bf16 h[8];
        h[0] = __float2bfloat16_rn(dose[v] * inv_scale);
        h[1] = __float2bfloat16_rn(rho[v]);
#pragma unroll
        for (int c = 2; c < 8; ++c) h[c] = __float2bfloat16_rn(0.0f);
        reinterpret_cast<uint4 *>(x8)[v] = *reinterpret_cast<uint4 *>(h);
    }
}

// out[Z][Y][X][c] = s * sum of in over the 2x2x2 block (in: 2Z x 2Y x 2X x C)
__global__ void k_pool(const bf16 *in, int C, int Z, int Y, int X, float s, bf16 *out) {
    const int64_t n = (int64_t)Z * Y * X * C;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(q % C);
        const int64_t v = q / C;
        const int x = (int)(v % X), y = (int)((v / X) % Y), z = (int)(v / ((int64_t)X * Y));
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int64_t iv = ((int64_t)(2 * z + (k >> 2)) * (2 * Y) + (2 * y + ((k >> 1) & 1))) * (2 * X) + (2 * x + (k & 1));
            acc += __bfloat162float(in[iv * C + c]);
        }
        out[q] = __float2bfloat16_rn(s * acc);
    }
}

// out[v][c] = skip[v][c] + s * low[v / 2][c]  (out: Z x Y x X x C; skip may be null)
__global__ void k_up_add(const bf16 *low, const bf16 *skip, int C, int Z, int Y, int X, float s, bf16 *out) {
    const int64_t n = (int64_t)Z * Y * X * C;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(q % C);
        const int64_t v = q / C;
        const int x = (int)(v % X), y = (int)((v / X) % Y), z = (int)(v / ((int64_t)X * Y));
        const int64_t lv = ((int64_t)(z >> 1) * (Y >> 1) + (y >> 1)) * (X >> 1) + (x >> 1);
        float r = s * __bfloat162float(low[lv * C + c]);
        if (skip) r += __bfloat162float(skip[q]);
        out[q] = __float2bfloat16_rn(r);
    }
}

// g = act > 0 ? g : 0 (the ReLU derivative from the layer's own output)
__global__ void k_mask(bf16 *g, const bf16 *act, int64_t n) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        if (!(__bfloat162float(act[q]) > 0.0f)) g[q] = __float2bfloat16_rn(0.0f);
}

// db[c] += sum_v g[v][c]  (C <= 128; blocks of 256 threads, C divides 256)
__global__ void k_colsum(const bf16 *g, int64_t V, int C, float *db) {
    __shared__ float acc[256];
    const int rows_per = 256 / C;
    const int c = threadIdx.x % C, r = threadIdx.x / C;
    float s = 0.0f;
    for (int64_t v = (int64_t)blockIdx.x * rows_per + r; v < V; v += (int64_t)gridDim.x * rows_per)
        s += __bfloat162float(g[v * C + c]);
    acc[threadIdx.x] = s;
    __syncthreads();
    if (r == 0) {
        for (int k = 1; k < rows_per; ++k) s += acc[k * C + c];
        atomicAdd(db + c, s);
    }
}

// y = sum_c d0[v][c] w[c] + b + x8[v][0]; with a target: r = y - t,
// gy = 2 r / V, loss += r^2
__global__ void k_out_fwd(const bf16 *d0, const float *w, const float *b, const bf16 *x8, const float *target,
                          float inv_scale, int64_t V, float *y, float *gy, double *loss) {
    double l = 0.0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        float acc = b[0] + __bfloat162float(x8[v * 8]);
#pragma unroll
        for (int c = 0; c < 16; ++c) acc += __bfloat162float(d0[v * 16 + c]) * w[c];
        y[v] = acc;
        if (target) {
            const float r = acc - target[v] * inv_scale;
            gy[v] = 2.0f * r / (float)V;
            l += (double)r * r;
        }
    }
    if (target) {
        for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xFFFFFFFFu, l, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(loss, l);
    }
}

// gz[v][c] = d0 > 0 ? gy[v] w[c] : 0; dw[c] += sum gy d0[v][c]; db += sum gy
__global__ void k_out_back(const bf16 *d0, const float *gy, const float *w, int64_t V, bf16 *gz, float *dw, float *db) {
    float sw[16], sb = 0.0f;
#pragma unroll
    for (int c = 0; c < 16; ++c) sw[c] = 0.0f;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        const float g = gy[v];
        sb += g;
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const float a = __bfloat162float(d0[v * 16 + c]);
            sw[c] += g * a;
            gz[v * 16 + c] = __float2bfloat16_rn(a > 0.0f ? g * w[c] : 0.0f);
        }
    }
#pragma unroll
    for (int c = 0; c < 16; ++c)
        for (int o = 16; o > 0; o >>= 1) sw[c] += __shfl_xor_sync(0xFFFFFFFFu, sw[c], o);
    for (int o = 16; o > 0; o >>= 1) sb += __shfl_xor_sync(0xFFFFFFFFu, sb, o);
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int c = 0; c < 16; ++c) atomicAdd(dw + c, sw[c]);
        atomicAdd(db, sb);
    }
}

__global__ void k_out_scale(const float *y, float scale, int64_t V, float *out) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x)
        out[v] = y[v] * scale;
}

// Adam (Kingma and Ba 2015) on the mean of the accumulated gradients
__global__ void k_adam(float *p, float *g, float *m, float *v, int64_t n, float lr, float b1, float b2, float eps,
                       float bc1, float bc2, float inv_count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i] * inv_count;
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        g[i] = 0.0f;
    }
}

}  // namespace

struct psl_denoiser {
    int device = 0;
    int64_t np = 0;
    int64_t off_w[NL], off_b[NL], off_ow = 0, off_ob = 0;
    float *P = nullptr, *G = nullptr, *M = nullptr, *Vv = nullptr;
    bf16 *wf[NL] = {}, *wm[NL] = {};
    int step = 0, accum = 0;
    uint32_t *err = nullptr;
    double *loss = nullptr;
    // activations and gradient scratch of the current volume
    int nx = 0, ny = 0, nz = 0;
    std::vector<void *> bufs;
    bf16 *x8, *e0a, *s0, *p0, *s1, *p1, *s2, *p2, *b3a, *b3b, *u2, *d2, *u1, *d1, *u0, *d0;
    bf16 *A[4], *B[4], *C[4];
    float *y, *gy;
};

namespace {

void free_volume(psl_denoiser *d) {
    for (void *p : d->bufs) cudaFree(p);
    d->bufs.clear();
    d->nx = d->ny = d->nz = 0;
}

int ensure_volume(psl_denoiser *d, int nx, int ny, int nz) {
    if (d->nx == nx && d->ny == ny && d->nz == nz) return PSL_OK;
    cudaDeviceSynchronize();
    free_volume(d);
    const int64_t V = (int64_t)nx * ny * nz;
    const int64_t lv[4] = {V, V / 8, V / 64, V / 512};
    auto get = [&](int64_t elems, size_t esz) -> void * {
        void *p = nullptr;
        if (cudaMalloc(&p, (size_t)std::max<int64_t>(elems, 8) * esz) != cudaSuccess) return nullptr;
        d->bufs.push_back(p);
        return p;
    };
    bool ok = true;
    auto gb = [&](int64_t e) { bf16 *p = (bf16 *)get(e, sizeof(bf16)); ok &= p != nullptr; return p; };
    d->x8 = gb(V * 8); d->e0a = gb(V * 16); d->s0 = gb(V * 16); d->u0 = gb(V * 16); d->d0 = gb(V * 16);
    d->p0 = gb(lv[1] * 16); d->s1 = gb(lv[1] * 32); d->u1 = gb(lv[1] * 32); d->d1 = gb(lv[1] * 16);
    d->p1 = gb(lv[2] * 32); d->s2 = gb(lv[2] * 64); d->u2 = gb(lv[2] * 64); d->d2 = gb(lv[2] * 32);
    d->p2 = gb(lv[3] * 64); d->b3a = gb(lv[3] * 128); d->b3b = gb(lv[3] * 64);
    const int wide[4] = {16, 32, 64, 128};
    for (int l = 0; l < 4; ++l) { d->A[l] = gb(lv[l] * wide[l]); d->B[l] = gb(lv[l] * wide[l]); d->C[l] = gb(lv[l] * wide[l]); }
    d->y = (float *)get(V, 4); d->gy = (float *)get(V, 4);
    ok &= d->y && d->gy;
    if (!ok) { free_volume(d); return psl_fail(PSL_ENOMEM, "denoiser: activation allocation"); }
    d->nx = nx; d->ny = ny; d->nz = nz;
    return PSL_OK;
}

int repack(psl_denoiser *d, cudaStream_t st) {
    int rc;
    for (int l = 0; l < NL; ++l) {
        if ((rc = psl_conv3d_pack_run(d->P + d->off_w[l], LAYERS[l].ci, LAYERS[l].co, 0, d->wf[l], st))) return rc;
        if (l != E0A && (rc = psl_conv3d_pack_run(d->P + d->off_w[l], LAYERS[l].ci, LAYERS[l].co, 1, d->wm[l], st)))
            return rc;
    }
    return PSL_OK;
}

int check_dims(int nx, int ny, int nz) {
    if (nx < 8 || ny < 8 || nz < 8 || nx % 8 || ny % 8 || nz % 8 || (int64_t)nx * ny * nz >= (1ll << 31))
        return psl_fail(PSL_EINVAL, "denoiser: volume sides must be multiples of 8 (>= 8)");
    return PSL_OK;
}

int conv(psl_denoiser *d, int l, const bf16 *in, int lev, bf16 *out, cudaStream_t st) {
    const int s = 1 << lev;
    return psl_conv3d_run(in, LAYERS[l].ci, d->wf[l], d->P + d->off_b[l], LAYERS[l].co, d->nx / s, d->ny / s,
                          d->nz / s, 1, out, nullptr, d->err, st);
}

int forward(psl_denoiser *d, const float *dose, const float *rho, float inv_scale, cudaStream_t st) {
    const int64_t V = (int64_t)d->nx * d->ny * d->nz;
    const int X = d->nx, Y = d->ny, Z = d->nz;
    int rc;
    k_input<<<grid_for(V), 256, 0, st>>>(dose, rho, inv_scale, V, d->x8); PSL_NOTE_LAUNCH();
    if ((rc = conv(d, E0A, d->x8, 0, d->e0a, st))) return rc;
    if ((rc = conv(d, E0B, d->e0a, 0, d->s0, st))) return rc;
    k_pool<<<grid_for(V / 8 * 16), 256, 0, st>>>(d->s0, 16, Z / 2, Y / 2, X / 2, 0.125f, d->p0); PSL_NOTE_LAUNCH();
    if ((rc = conv(d, E1, d->p0, 1, d->s1, st))) return rc;
    k_pool<<<grid_for(V / 64 * 32), 256, 0, st>>>(d->s1, 32, Z / 4, Y / 4, X / 4, 0.125f, d->p1); PSL_NOTE_LAUNCH();
    if ((rc = conv(d, E2, d->p1, 2, d->s2, st))) return rc;
    k_pool<<<grid_for(V / 512 * 64), 256, 0, st>>>(d->s2, 64, Z / 8, Y / 8, X / 8, 0.125f, d->p2); PSL_NOTE_LAUNCH();
    if ((rc = conv(d, B3A, d->p2, 3, d->b3a, st))) return rc;
    if ((rc = conv(d, B3B, d->b3a, 3, d->b3b, st))) return rc;
    k_up_add<<<grid_for(V / 64 * 64), 256, 0, st>>>(d->b3b, d->s2, 64, Z / 4, Y / 4, X / 4, 1.0f, d->u2); PSL_NOTE_LAUNCH();
    if ((rc = conv(d, D2, d->u2, 2, d->d2, st))) return rc;
    k_up_add<<<grid_for(V / 8 * 32), 256, 0, st>>>(d->d2, d->s1, 32, Z / 2, Y / 2, X / 2, 1.0f, d->u1); PSL_NOTE_LAUNCH();
    if ((rc = conv(d, D1, d->u1, 1, d->d1, st))) return rc;
    k_up_add<<<grid_for(V * 16), 256, 0, st>>>(d->d1, d->s0, 16, Z, Y, X, 1.0f, d->u0); PSL_NOTE_LAUNCH();
    return conv(d, D0, d->u0, 0, d->d0, st);
}

// Gradient of one convolution layer: g (BF16, the layer's output gradient,
// masked here by the ReLU) -> tap and bias gradients, and (if gin) the input
// gradient through the mirrored taps.
int layer_back(psl_denoiser *d, int l, const bf16 *in, const bf16 *act, bf16 *g, int lev, bf16 *gin, cudaStream_t st) {
    const int s = 1 << lev;
    const int nx = d->nx / s, ny = d->ny / s, nz = d->nz / s;
    const int64_t V = (int64_t)nx * ny * nz;
    const int ci = LAYERS[l].ci, co = LAYERS[l].co;
    int rc;
    k_mask<<<grid_for(V * co), 256, 0, st>>>(g, act, V * co); PSL_NOTE_LAUNCH();
    if ((rc = psl_conv3d_wgrad_run(in, ci, g, co, nx, ny, nz, d->G + d->off_w[l], d->err, st))) return rc;
    k_colsum<<<(int)std::min<int64_t>((V + 255) / 256 + 1, 1024), 256, 0, st>>>(g, V, co, d->G + d->off_b[l]); PSL_NOTE_LAUNCH();
    if (gin) return psl_conv3d_run(g, co, d->wm[l], nullptr, ci, nx, ny, nz, 0, gin, nullptr, d->err, st);
    return PSL_OK;
}

int backward(psl_denoiser *d, cudaStream_t st) {
    const int64_t V = (int64_t)d->nx * d->ny * d->nz;
    const int X = d->nx, Y = d->ny, Z = d->nz;
    bf16 **A = d->A, **B = d->B, **C = d->C;
    int rc;
    k_out_back<<<grid_for(V), 256, 0, st>>>(d->d0, d->gy, d->P + d->off_ow, V, A[0], d->G + d->off_ow, d->G + d->off_ob); PSL_NOTE_LAUNCH();
    // decoder
    if ((rc = layer_back(d, D0, d->u0, d->d0, A[0], 0, B[0], st))) return rc;                 // B0 = g u0
    k_pool<<<grid_for(V / 8 * 16), 256, 0, st>>>(B[0], 16, Z / 2, Y / 2, X / 2, 1.0f, A[1]); PSL_NOTE_LAUNCH();
    if ((rc = layer_back(d, D1, d->u1, d->d1, A[1], 1, B[1], st))) return rc;                 // B1 = g u1
    k_pool<<<grid_for(V / 64 * 32), 256, 0, st>>>(B[1], 32, Z / 4, Y / 4, X / 4, 1.0f, A[2]); PSL_NOTE_LAUNCH();
    if ((rc = layer_back(d, D2, d->u2, d->d2, A[2], 2, B[2], st))) return rc;                 // B2 = g u2
    k_pool<<<grid_for(V / 512 * 64), 256, 0, st>>>(B[2], 64, Z / 8, Y / 8, X / 8, 1.0f, A[3]); PSL_NOTE_LAUNCH();
    if ((rc = layer_back(d, B3B, d->b3a, d->b3b, A[3], 3, B[3], st))) return rc;              // B3 = g b3a
    if ((rc = layer_back(d, B3A, d->p2, d->b3a, B[3], 3, C[3], st))) return rc;              // C3 = g p2
    // encoder: skip gradient + pooled gradient
    k_up_add<<<grid_for(V / 64 * 64), 256, 0, st>>>(C[3], B[2], 64, Z / 4, Y / 4, X / 4, 0.125f, C[2]); PSL_NOTE_LAUNCH();
    if ((rc = layer_back(d, E2, d->p1, d->s2, C[2], 2, A[2], st))) return rc;                // A2 = g p1
    k_up_add<<<grid_for(V / 8 * 32), 256, 0, st>>>(A[2], B[1], 32, Z / 2, Y / 2, X / 2, 0.125f, C[1]); PSL_NOTE_LAUNCH();
    if ((rc = layer_back(d, E1, d->p0, d->s1, C[1], 1, A[1], st))) return rc;                // A1 = g p0
    k_up_add<<<grid_for(V * 16), 256, 0, st>>>(A[1], B[0], 16, Z, Y, X, 0.125f, C[0]); PSL_NOTE_LAUNCH();
    if ((rc = layer_back(d, E0B, d->e0a, d->s0, C[0], 0, A[0], st))) return rc;              // A0 = g e0a
    return layer_back(d, E0A, d->x8, d->e0a, A[0], 0, nullptr, st);
}

int finish(psl_denoiser *d, cudaStream_t st, const char *what) {
    uint32_t herr = 0;
    cudaMemcpyAsync(&herr, d->err, 4, cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return psl_fail(PSL_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    if (herr) { cudaMemsetAsync(d->err, 0, 4, st); return psl_fail(PSL_ETIMEOUT, std::string(what) + ": tensor-core wait gave up"); }
    return PSL_OK;
}

}  // namespace

extern "C" int64_t psl_denoiser_param_count(void) {
    int64_t n = 0;
    for (int l = 0; l < NL; ++l) n += 27ll * LAYERS[l].ci * LAYERS[l].co + LAYERS[l].co;
    return n + 16 + 1;
}

extern "C" void psl_denoiser_destroy(psl_denoiser_t *d) {
    if (!d) return;
    cudaDeviceSynchronize();
    free_volume(d);
    for (int l = 0; l < NL; ++l) { if (d->wf[l]) cudaFree(d->wf[l]); if (d->wm[l]) cudaFree(d->wm[l]); }
    for (void *p : {(void *)d->P, (void *)d->G, (void *)d->M, (void *)d->Vv, (void *)d->err, (void *)d->loss})
        if (p) cudaFree(p);
    delete d;
}

extern "C" int psl_denoiser_create(uint64_t seed, psl_denoiser_t **out) {
    if (!out) return psl_fail(PSL_EINVAL, "psl_denoiser_create: null output");
    *out = nullptr;
    psl_denoiser *d = new psl_denoiser();
    cudaGetDevice(&d->device);
    int64_t o = 0;
    for (int l = 0; l < NL; ++l) {
        d->off_w[l] = o; o += 27ll * LAYERS[l].ci * LAYERS[l].co;
        d->off_b[l] = o; o += LAYERS[l].co;
    }
    d->off_ow = o; o += 16;
    d->off_ob = o; o += 1;
    d->np = o;
    // He-normal taps, zero biases, zero output layer (starts as the identity on the dose)
    std::vector<float> h((size_t)o, 0.0f);
    std::mt19937_64 gen(seed);
    for (int l = 0; l < NL; ++l) {
        std::normal_distribution<float> nd(0.0f, std::sqrt(2.0f / (27.0f * LAYERS[l].ci)));
        for (int64_t k = 0; k < 27ll * LAYERS[l].ci * LAYERS[l].co; ++k) h[d->off_w[l] + k] = nd(gen);
    }
    bool ok = true;
    for (float **p : {&d->P, &d->G, &d->M, &d->Vv}) ok &= cudaMalloc((void **)p, o * sizeof(float)) == cudaSuccess;
    ok &= cudaMalloc((void **)&d->err, 16) == cudaSuccess;
    ok &= cudaMalloc((void **)&d->loss, 16) == cudaSuccess;
    for (int l = 0; l < NL && ok; ++l) {
        ok &= cudaMalloc((void **)&d->wf[l], psl_conv_ksteps(LAYERS[l].ci) * LAYERS[l].co * 16 * sizeof(bf16)) == cudaSuccess;
        ok &= cudaMalloc((void **)&d->wm[l], psl_conv_ksteps(LAYERS[l].co) * LAYERS[l].ci * 16 * sizeof(bf16)) == cudaSuccess;
    }
    if (!ok) { psl_denoiser_destroy(d); return psl_fail(PSL_ENOMEM, "psl_denoiser_create: allocation"); }
    cudaMemcpy(d->P, h.data(), o * sizeof(float), cudaMemcpyHostToDevice);
    cudaMemset(d->G, 0, o * sizeof(float));
    cudaMemset(d->M, 0, o * sizeof(float));
    cudaMemset(d->Vv, 0, o * sizeof(float));
    cudaMemset(d->err, 0, 16);
    int rc = repack(d, nullptr);
    cudaError_t e = cudaDeviceSynchronize();
    if (rc || e != cudaSuccess) { psl_denoiser_destroy(d); return rc ? rc : psl_fail(PSL_ECUDA, cudaGetErrorString(e)); }
    *out = d;
    return PSL_OK;
}

extern "C" int psl_denoiser_params(psl_denoiser_t *d, const float *set, float *get, float *grad, void *stream) {
    if (!d) return psl_fail(PSL_EINVAL, "psl_denoiser_params: null denoiser");
    cudaStream_t st = as_stream(stream);
    const size_t bytes = d->np * sizeof(float);
    if (set) {
        PSL_CUDA(cudaMemcpyAsync(d->P, set, bytes, cudaMemcpyDeviceToDevice, st));
        int rc = repack(d, st);
        if (rc) return rc;
    }
    if (get) PSL_CUDA(cudaMemcpyAsync(get, d->P, bytes, cudaMemcpyDeviceToDevice, st));
    if (grad) PSL_CUDA(cudaMemcpyAsync(grad, d->G, bytes, cudaMemcpyDeviceToDevice, st));
    PSL_CUDA(cudaStreamSynchronize(st));
    return PSL_OK;
}

extern "C" int psl_denoiser_forward(psl_denoiser_t *d, const float *dose, const float *rho, int32_t nx, int32_t ny,
                                    int32_t nz, float scale, float *out, void *stream) {
    if (!d || !dose || !rho || !out) return psl_fail(PSL_EINVAL, "psl_denoiser_forward: null argument");
    if (!(scale > 0)) return psl_fail(PSL_EINVAL, "psl_denoiser_forward: scale must be > 0");
    int rc = check_dims(nx, ny, nz);
    if (rc || (rc = ensure_volume(d, nx, ny, nz))) return rc;
    cudaStream_t st = as_stream(stream);
    if ((rc = forward(d, dose, rho, 1.0f / scale, st))) return rc;
    const int64_t V = (int64_t)nx * ny * nz;
    k_out_fwd<<<grid_for(V), 256, 0, st>>>(d->d0, d->P + d->off_ow, d->P + d->off_ob, d->x8, nullptr, 1.0f / scale, V,
                                          d->y, nullptr, nullptr); PSL_NOTE_LAUNCH();
    k_out_scale<<<grid_for(V), 256, 0, st>>>(d->y, scale, V, out); PSL_NOTE_LAUNCH();
    return finish(d, st, "psl_denoiser_forward");
}

extern "C" int psl_denoiser_backward(psl_denoiser_t *d, const float *dose, const float *rho, const float *target,
                                     int32_t nx, int32_t ny, int32_t nz, float scale, double *loss, void *stream) {
    if (!d || !dose || !rho || !target) return psl_fail(PSL_EINVAL, "psl_denoiser_backward: null argument");
    if (!(scale > 0)) return psl_fail(PSL_EINVAL, "psl_denoiser_backward: scale must be > 0");
    int rc = check_dims(nx, ny, nz);
    if (rc || (rc = ensure_volume(d, nx, ny, nz))) return rc;
    cudaStream_t st = as_stream(stream);
    if ((rc = forward(d, dose, rho, 1.0f / scale, st))) return rc;
    const int64_t V = (int64_t)nx * ny * nz;
    cudaMemsetAsync(d->loss, 0, 8, st);
    k_out_fwd<<<grid_for(V), 256, 0, st>>>(d->d0, d->P + d->off_ow, d->P + d->off_ob, d->x8, target, 1.0f / scale, V,
                                          d->y, d->gy, d->loss); PSL_NOTE_LAUNCH();
    if ((rc = backward(d, st))) return rc;
    d->accum++;
    double hl = 0.0;
    cudaMemcpyAsync(&hl, d->loss, 8, cudaMemcpyDeviceToHost, st);
    if ((rc = finish(d, st, "psl_denoiser_backward"))) return rc;
    if (loss) *loss = hl / (double)V;
    return PSL_OK;
}

extern "C" int psl_denoiser_step(psl_denoiser_t *d, float lr, void *stream) {
    if (!d || !(lr > 0)) return psl_fail(PSL_EINVAL, "psl_denoiser_step: bad argument");
    if (d->accum == 0) return psl_fail(PSL_EINVAL, "psl_denoiser_step: no gradients accumulated");
    cudaStream_t st = as_stream(stream);
    d->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = 1.0f - std::pow(b1, (float)d->step), bc2 = 1.0f - std::pow(b2, (float)d->step);
    k_adam<<<grid_for(d->np), 256, 0, st>>>(d->P, d->G, d->M, d->Vv, d->np, lr, b1, b2, 1e-8f, bc1, bc2,
                                           1.0f / (float)d->accum); PSL_NOTE_LAUNCH();
    d->accum = 0;
    int rc = repack(d, st);
    if (rc) return rc;
    return finish(d, st, "psl_denoiser_step");
}

// ------------------------------------------------------------ k-th value --
namespace {
// order-preserving map of a float's bits to an unsigned key (negatives below
// positives, larger magnitude negatives lower)
// k-th smallest by radix selection on the values' order-preserving bit
// patterns (sign flipped for non-negatives, all bits for negatives): three
// passes fix 11, 11 and 10 bits of the answer, each a histogram of the
// values that share the bits fixed so far, then a search for the bin that
// holds the k-th.  State: [0] the bits fixed so far, [1] k among the values
// that share them.
__device__ __forceinline__ uint32_t float_key(float v) {
    const uint32_t b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
constexpr int SEL_BINS = 2048;

__global__ void __launch_bounds__(256) k_select_hist(const float *x, uint32_t n, int shift, uint32_t field,
                                                     uint32_t prefix_mask, const uint32_t *state, uint32_t *hist) {
    __shared__ uint32_t h[SEL_BINS];
    for (int i = threadIdx.x; i < SEL_BINS; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const uint32_t prefix = state[0];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t key = float_key(__ldg(x + i));
        if ((key & prefix_mask) == prefix) atomicAdd(&h[(key >> shift) & field], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SEL_BINS; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// one block of 1024 threads: the bin holding the k-th value, by a block scan
// of the histogram (two bins per thread); the histogram is cleared for the
// next pass
__global__ void __launch_bounds__(1024) k_select_pick(uint32_t *hist, int shift, uint32_t *state) {
    __shared__ uint32_t warp_sum[32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const uint32_t a = hist[2 * t], b = hist[2 * t + 1];
    uint32_t x = a + b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t v = warp_sum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, v, o);
            if (lane >= o) v += y;
        }
        warp_sum[lane] = v;                          // inclusive sums of the warps
    }
    __syncthreads();
    const uint32_t below = x - (a + b) + (wid ? warp_sum[wid - 1] : 0u);   // values in bins < 2t
    const uint32_t k = state[1];
    __syncthreads();                                 // every thread has read state[1]
    if (k >= below && k < below + a) { state[0] |= (uint32_t)(2 * t) << shift; state[1] = k - below; }
    else if (k >= below + a && k < below + a + b) { state[0] |= (uint32_t)(2 * t + 1) << shift; state[1] = k - below - a; }
    hist[2 * t] = 0;
    hist[2 * t + 1] = 0;
}

__global__ void k_select_value(const uint32_t *state, float *out) {
    const uint32_t key = state[0];
    *out = __uint_as_float((key & 0x80000000u) ? (key & 0x7FFFFFFFu) : ~key);
}
}  // namespace

extern "C" int psl_kth_smallest(const float *x, int64_t n, int64_t k, float *out, void *stream_) {
    if (!x || !out || n < 1 || n >= ((int64_t)1 << 32) || k < 0 || k >= n)
        return psl_fail(PSL_EINVAL, "psl_kth_smallest: bad argument");
    cudaStream_t st = as_stream(stream_);
    const uint32_t m = (uint32_t)n;
    uint32_t *buf = nullptr;                         // [SEL_BINS] histogram, [2] state, value
    if (psl_malloc_async((void **)&buf, (SEL_BINS + 4) * sizeof(uint32_t), st) != cudaSuccess)
        return psl_fail(PSL_ENOMEM, "psl_kth_smallest: scratch");
    uint32_t *hist = buf, *state = buf + SEL_BINS;
    float *dv = reinterpret_cast<float *>(buf + SEL_BINS + 2);
    const uint32_t init[2] = {0u, (uint32_t)k};
    cudaMemsetAsync(hist, 0, SEL_BINS * sizeof(uint32_t), st);
    cudaMemcpyAsync(state, init, sizeof(init), cudaMemcpyHostToDevice, st);
    const int grid = (int)std::min<uint32_t>((m + 255) / 256, (uint32_t)psl_sm_count() * 4);
    const int shifts[3] = {21, 10, 0};
    const uint32_t fields[3] = {0x7FFu, 0x7FFu, 0x3FFu}, masks[3] = {0u, 0xFFE00000u, 0xFFFFFC00u};
    for (int p = 0; p < 3; ++p) {
        k_select_hist<<<grid, 256, 0, st>>>(x, m, shifts[p], fields[p], masks[p], state, hist); PSL_NOTE_LAUNCH();
        k_select_pick<<<1, 1024, 0, st>>>(hist, shifts[p], state); PSL_NOTE_LAUNCH();
    }
    k_select_value<<<1, 1, 0, st>>>(state, dv); PSL_NOTE_LAUNCH();
    cudaMemcpyAsync(out, dv, 4, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(buf, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return psl_fail(PSL_ECUDA, std::string("psl_kth_smallest: ") + cudaGetErrorString(e));
    return PSL_OK;
}
