// BF16 3D convolution (3x3x3 taps, zero padding 1, channels last) on the
// tcgen05 tensor cores: the forward pass and, with mirrored and transposed
// taps, the input gradient, as one implicit GEMM.
//
// GEMM view: D[voxel][o] = sum_k A[voxel][k] B[o][k], k = tap * C_in + i,
// A[v][k] = x[v + offset(tap)][i] (zero outside the volume), B[o][k] =
// w[tap][i][o].  A CTA owns 128 consecutive voxels (M = 128) and all C_out
// outputs (N = C_out, 16..128); the FP32 accumulator lives in tensor memory.
// K runs in steps of 16 (one MMA each), 8 steps per pipeline stage: the 128
// threads gather the stage's A rows (16-byte vectors: 8 channels of one tap)
// and copy its pre-packed B tile into shared memory, one thread issues the
// stage's MMAs and commits them to the stage buffer's mbarrier, and the
// threads go on to fill the other buffer.  The epilogue reads the
// accumulator back with tcgen05.ld, adds the bias, applies ReLU and stores
// BF16 (or FP32).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "../../include/psl_denoise.h"
#include "psl_internal.cuh"
#include "tc.cuh"

namespace {

constexpr int BM = 128;               // voxels per CTA
constexpr int SK = 8;                 // K steps (of 16) per stage
constexpr uint32_t WAIT_LIMIT = 1u << 24;

struct ConvArgs {
    const __nv_bfloat16 *in;          // [V][ci]
    const __nv_bfloat16 *wpk;         // packed taps, ksteps x N x 16
    const float *bias;                // [N] or null
    __nv_bfloat16 *out;               // [V][N] or null
    float *out_f32;                   // [V][N] or null
    int ci, D, H, W, relu, ksteps;
    uint32_t *err;
};

// one 16-byte chunk (8 channels of one tap) of voxel (z, y, x)'s A row
__device__ __forceinline__ uint4 gather_chunk(const ConvArgs &a, int z, int y, int x, bool row_ok, int kc) {
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    const int k0 = kc * 8;
    const int tap = k0 / a.ci, c0 = k0 - tap * a.ci;
    if (!row_ok || tap >= 27) return v;
    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    const int zz = z + dz, yy = y + dy, xx = x + dx;
    if (zz < 0 || zz >= a.D || yy < 0 || yy >= a.H || xx < 0 || xx >= a.W) return v;
    const int64_t nv = ((int64_t)zz * a.H + yy) * a.W + xx;
    return __ldg(reinterpret_cast<const uint4 *>(a.in + nv * a.ci + c0));
}

template <int N>
__global__ void __launch_bounds__(128, 1) k_conv3d(ConvArgs a) {
    extern __shared__ __align__(1024) uint8_t smem[];
    constexpr int A_STAGE = SK * BM * 32;          // bytes: 8 K steps x 128 rows x 16 BF16
    constexpr int B_STAGE = SK * N * 32;
    constexpr uint32_t TCOLS = N < 32 ? 32 : N;
    uint8_t *sA = smem;                             // [2][A_STAGE]
    uint8_t *sB = smem + 2 * A_STAGE;               // [2][B_STAGE]
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * A_STAGE + 2 * B_STAGE);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 2);

    const int t = threadIdx.x, warp = t >> 5;
    const int64_t V = (int64_t)a.D * a.H * a.W;
    const int64_t v = (int64_t)blockIdx.x * BM + t;
    const bool row_ok = v < V;
    int z = 0, y = 0, x = 0;
    if (row_ok) {
        x = (int)(v % a.W);
        y = (int)((v / a.W) % a.H);
        z = (int)(v / ((int64_t)a.W * a.H));
    }
    if (warp == 0) {
        tc::tmem_alloc(tslot, TCOLS);
        tc::tmem_relinquish();
    }
    if (t == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
        tc::mbar_fence_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = tc::idesc_bf16(BM, N);
    const int nst = (a.ksteps + SK - 1) / SK;
    bool ok = true;

    for (int st = 0; st < nst; ++st) {
        const int buf = st & 1;
        // the MMAs of stage st - 2 have finished reading this buffer
        if (st >= 2 && !tc::mbar_wait(&bar[buf], (uint32_t)((st - 2) >> 1) & 1u, WAIT_LIMIT)) ok = false;
        const int k0 = st * SK, nk = min(SK, a.ksteps - k0);
        uint8_t *A = sA + buf * A_STAGE, *B = sB + buf * B_STAGE;
        // A rows: this thread's voxel, core-matrix layout (LBO 128, SBO 256)
        for (int kk = 0; kk < nk; ++kk) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const uint4 c = gather_chunk(a, z, y, x, row_ok, 2 * (k0 + kk) + j);
                *reinterpret_cast<uint4 *>(A + kk * (BM * 32) + (t >> 3) * 256 + j * 128 + (t & 7) * 16) = c;
            }
        }
        // B tile: already packed in the same layout, copied as 16-byte chunks
        const uint4 *src = reinterpret_cast<const uint4 *>(a.wpk) + (size_t)k0 * N * 2;
        for (int i = t; i < nk * N * 2; i += BM) reinterpret_cast<uint4 *>(B)[i] = __ldg(src + i);
        tc::fence_async_smem();
        tc::fence_before_sync();
        if (!__syncthreads_and(ok)) { ok = false; break; }       // block-uniform
        if (t == 0) {
            tc::fence_after_sync();
            for (int kk = 0; kk < nk; ++kk) {
                const uint64_t ad = tc::desc_kmajor(tc::smem_u32(A + kk * (BM * 32)), 128, 256);
                const uint64_t bd = tc::desc_kmajor(tc::smem_u32(B + kk * (N * 32)), 128, 256);
                tc::mma_bf16(tmem, ad, bd, idesc, (st > 0 || kk > 0) ? 1u : 0u);
            }
            tc::mma_commit(&bar[buf]);
        }
    }
    if (ok && !tc::mbar_wait(&bar[(nst - 1) & 1], (uint32_t)((nst - 1) >> 1) & 1u, WAIT_LIMIT)) ok = false;
    ok = __syncthreads_and(ok) != 0;
    tc::fence_after_sync();
    if (!ok) {
        if (t == 0) atomicOr(a.err, PSL_DEV_ERR_TIMEOUT);
    } else {
        // epilogue: warp w holds accumulator rows 32w..32w+31
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
#pragma unroll
        for (int c0 = 0; c0 < N; c0 += 16) {
            float r[16];
            tc::tmem_ld16(tmem + lane_base + (uint32_t)c0, r);
            if (row_ok) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    float q = r[i] + (a.bias ? __ldg(a.bias + c0 + i) : 0.0f);
                    r[i] = a.relu ? fmaxf(q, 0.0f) : q;
                }
                if (a.out) {
                    __align__(16) __nv_bfloat16 h[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) h[i] = __float2bfloat16_rn(r[i]);
                    uint4 *dst = reinterpret_cast<uint4 *>(a.out + v * N + c0);
                    dst[0] = reinterpret_cast<uint4 *>(h)[0];
                    dst[1] = reinterpret_cast<uint4 *>(h)[1];
                }
                if (a.out_f32) {
                    float4 *dst = reinterpret_cast<float4 *>(a.out_f32 + v * N + c0);
#pragma unroll
                    for (int i = 0; i < 4; ++i) dst[i] = make_float4(r[4 * i], r[4 * i + 1], r[4 * i + 2], r[4 * i + 3]);
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, TCOLS);
}

// Weight gradient as a GEMM over voxels: dW[(t, i)][o] = sum_v A[(t,i)][v]
// B[o][v], A[(t,i)][v] = x[v + offset_t][i], B[o][v] = gy[v][o].  A CTA owns
// 128 rows (t, i) and one range of voxels (split K); per stage 128 voxels =
// 8 MMAs of 16.  Both operands are stored voxel-major in HBM, so each thread
// loads 8 voxels x 8 channels (eight 16-byte vectors) and transposes the 8x8
// BF16 block in registers into eight K-major rows.  The FP32 partial sums
// are added into dW with atomics.
__device__ __forceinline__ void transpose8(const uint4 (&in)[8], uint4 (&out)[8]) {
    const uint32_t *w[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) w[k] = reinterpret_cast<const uint32_t *>(&in[k]);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const uint32_t sel = (c & 1) ? 0x7632u : 0x5410u;
        uint32_t o[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) o[q] = __byte_perm(w[2 * q][c >> 1], w[2 * q + 1][c >> 1], sel);
        out[c] = make_uint4(o[0], o[1], o[2], o[3]);
    }
}

struct WgradArgs {
    const __nv_bfloat16 *x;           // [V][ci]
    const __nv_bfloat16 *gy;          // [V][N]
    float *dw;                        // [27 ci][N], added to
    int ci, D, H, W;
    int64_t vox_per_cta;
    uint32_t *err;
};

template <int N>
__global__ void __launch_bounds__(128, 1) k_conv3d_wgrad(WgradArgs a) {
    extern __shared__ __align__(1024) uint8_t smem[];
    constexpr int A_STAGE = SK * BM * 32, B_STAGE = SK * N * 32;
    constexpr uint32_t TCOLS = N < 32 ? 32 : N;
    uint8_t *sA = smem, *sB = smem + 2 * A_STAGE;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * A_STAGE + 2 * B_STAGE);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 2);
    const int t = threadIdx.x, warp = t >> 5;
    const int64_t V = (int64_t)a.D * a.H * a.W;
    const int rows = 27 * a.ci;
    const int m0 = blockIdx.x * BM;
    const int64_t vbeg = (int64_t)blockIdx.y * a.vox_per_cta, vend = min(V, vbeg + a.vox_per_cta);
    if (warp == 0) { tc::tmem_alloc(tslot, TCOLS); tc::tmem_relinquish(); }
    if (t == 0) { tc::mbar_init(&bar[0], 1); tc::mbar_init(&bar[1], 1); tc::mbar_fence_init(); }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = tc::idesc_bf16(BM, N);
    const int nst = vend > vbeg ? (int)((vend - vbeg + BM - 1) / BM) : 0;
    bool ok = true;
    for (int st = 0; st < nst; ++st) {
        const int buf = st & 1;
        if (st >= 2 && !tc::mbar_wait(&bar[buf], (uint32_t)((st - 2) >> 1) & 1u, WAIT_LIMIT)) ok = false;
        uint8_t *A = sA + buf * A_STAGE, *B = sB + buf * B_STAGE;
        const int64_t vs = vbeg + (int64_t)st * BM;
        // A: 16 row groups x 16 voxel groups, two 8x8 blocks per thread
        for (int blk = t; blk < 256; blk += BM) {
            const int g = blk >> 4, q = blk & 15;
            const int r0 = m0 + 8 * g;
            const int tap = r0 / a.ci, i0 = r0 - tap * a.ci;
            uint4 in[8], out[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                in[k] = make_uint4(0u, 0u, 0u, 0u);
                const int64_t vv = vs + 8 * q + k;
                if (r0 < rows && vv < vend) {
                    const int x = (int)(vv % a.W), y = (int)((vv / a.W) % a.H), z = (int)(vv / ((int64_t)a.W * a.H));
                    const int zz = z + tap / 9 - 1, yy = y + (tap / 3) % 3 - 1, xx = x + tap % 3 - 1;
                    if (zz >= 0 && zz < a.D && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W)
                        in[k] = __ldg(reinterpret_cast<const uint4 *>(a.x + (((int64_t)zz * a.H + yy) * a.W + xx) * a.ci + i0));
                }
            }
            transpose8(in, out);
            uint8_t *dst = A + (q >> 1) * (BM * 32) + g * 256 + (q & 1) * 128;
#pragma unroll
            for (int c = 0; c < 8; ++c) *reinterpret_cast<uint4 *>(dst + c * 16) = out[c];
        }
        // B: N/8 row groups x 16 voxel groups
        for (int blk = t; blk < (N / 8) * 16; blk += BM) {
            const int g = blk >> 4, q = blk & 15;
            uint4 in[8], out[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int64_t vv = vs + 8 * q + k;
                in[k] = vv < vend ? __ldg(reinterpret_cast<const uint4 *>(a.gy + vv * N + 8 * g)) : make_uint4(0u, 0u, 0u, 0u);
            }
            transpose8(in, out);
            uint8_t *dst = B + (q >> 1) * (N * 32) + g * 256 + (q & 1) * 128;
#pragma unroll
            for (int c = 0; c < 8; ++c) *reinterpret_cast<uint4 *>(dst + c * 16) = out[c];
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        if (!__syncthreads_and(ok)) { ok = false; break; }
        if (t == 0) {
            tc::fence_after_sync();
#pragma unroll 1
            for (int kk = 0; kk < SK; ++kk) {
                const uint64_t ad = tc::desc_kmajor(tc::smem_u32(A + kk * (BM * 32)), 128, 256);
                const uint64_t bd = tc::desc_kmajor(tc::smem_u32(B + kk * (N * 32)), 128, 256);
                tc::mma_bf16(tmem, ad, bd, idesc, (st > 0 || kk > 0) ? 1u : 0u);
            }
            tc::mma_commit(&bar[buf]);
        }
    }
    if (ok && nst > 0 && !tc::mbar_wait(&bar[(nst - 1) & 1], (uint32_t)((nst - 1) >> 1) & 1u, WAIT_LIMIT)) ok = false;
    ok = __syncthreads_and(ok) != 0;
    tc::fence_after_sync();
    if (!ok) {
        if (t == 0) atomicOr(a.err, PSL_DEV_ERR_TIMEOUT);
    } else if (nst > 0) {
        const int r = m0 + t;                         // this thread's TMEM lane = its row (t, i)
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
#pragma unroll
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + lane_base + (uint32_t)c0, v);
            if (r < rows) {
#pragma unroll
                for (int i = 0; i < 16; ++i) atomicAdd(a.dw + (int64_t)r * N + c0 + i, v[i]);
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, TCOLS);
}

// ------------------------------------------------------ TMA form ---
// The same implicit GEMM with its operands brought in by the tensor memory
// accelerator and the work split by warp role.  A CTA's 128 voxels are a
// box of BX x BY x BZ voxels of the volume; for one K chunk (8 channels of
// one tap) the A rows are one 4-D TMA box {8 channels, BX, BY, BZ} of the
// input at the tap's offset, its out-of-volume part filled with zeros by the
// copy engine (the convolution's padding), landing as 128 rows of 16 bytes
// (core matrices 128 bytes apart, the two chunks of a K step 2 KB apart).
// A CTA owns 2 x 128 voxels (two MMA tiles, two accumulators) so that each
// B stage serves both.  The B tile of a stage is one bulk copy of the packed
// taps.  Warp 0 issues
// the copies into a 2-stage ring (full / empty mbarriers), warp 1 issues the
// MMAs and frees each stage by committing to its empty barrier, warps 2-5
// read the accumulator back.  Two stages (96 KB for 128 output channels)
// let two CTAs share an SM (their accumulators fill its 512 tensor-memory
// columns), so one CTA's epilogue and set-up run under the other's MMAs:
// measured 637 -> 887 TFLOP/s on 128^3 x 128 -> 128 against 4 stages and
// one CTA per SM.
constexpr int TKS = 4;                // K steps per stage
constexpr int TST = 2;                // stages (two CTAs per SM overlap one's epilogue with the other's MMAs)
// 128-voxel MMA tiles per CTA, sharing every B stage: two for wide outputs
// (the B traffic dominates), one for narrow ones (more CTAs per SM)
__host__ __device__ constexpr int tiles_for(int n) { return n >= 64 ? 2 : 1; }

struct TmaConvArgs {
    const __nv_bfloat16 *wpk;
    const float *bias;
    __nv_bfloat16 *out;
    float *out_f32;
    int ci, D, H, W, relu, ksteps;
    int bx, by, bz;                   // the CTA's voxel box
    int wide;                         // 1: 16-channel boxes (C_in >= 16, 32-byte swizzle); 0: 8-channel boxes
    uint32_t *err;
};

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar) : "memory");
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
}

template <int N>
__global__ void __launch_bounds__(192, 1) k_conv3d_tma(const __grid_constant__ CUtensorMap map, TmaConvArgs a) {
    constexpr int TT = tiles_for(N);
    extern __shared__ __align__(1024) uint8_t smem[];
    constexpr int A_ST = TKS * TT * BM * 32, B_ST = TKS * N * 32;
    constexpr uint32_t TCOLS = TT * N < 32 ? 32 : TT * N;
    uint8_t *sA = smem, *sB = smem + TST * A_ST;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + TST * (A_ST + B_ST));
    uint64_t *empty = full + TST, *accum = empty + TST;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(accum + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int x0 = blockIdx.x * a.bx, y0 = blockIdx.y * a.by, z0 = blockIdx.z * a.bz;
    if (warp == 1) { tc::tmem_alloc(tslot, TCOLS); tc::tmem_relinquish(); }
    if (t == 0) {
        for (int s = 0; s < TST; ++s) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 1); }
        tc::mbar_init(accum, 1);
        *abort_flag = 0;
        tc::mbar_fence_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const int nkb = (a.ksteps + TKS - 1) / TKS;

    if (warp == 0 && lane == 0) {                           // producer
        for (int kb = 0; kb < nkb && !*abort_flag; ++kb) {
            const int s = kb % TST;
            const uint32_t ph = (uint32_t)(kb / TST) & 1u;
            if (!tc::mbar_wait(&empty[s], ph ^ 1u, WAIT_LIMIT)) { *abort_flag = 1; atomicOr(a.err, PSL_DEV_ERR_TIMEOUT); break; }
            const int nks = min(TKS, a.ksteps - kb * TKS);
            const uint32_t fb = tc::smem_u32(&full[s]);
            mbar_expect_tx(fb, (uint32_t)(nks * TT * BM * 32 + nks * N * 32));
            for (int kk = 0; kk < nks; ++kk) {
                if (a.wide) {                                // one 16-channel box per K step
                    const int k0 = (kb * TKS + kk) * 16;
                    const int tap = k0 / a.ci, c0 = k0 - tap * a.ci;
                    tma_load_4d(tc::smem_u32(sA + s * A_ST + kk * (TT * BM * 32)), &map, c0, x0 + tap % 3 - 1,
                                y0 + (tap / 3) % 3 - 1, z0 + tap / 9 - 1, fb);
                    continue;
                }
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int k0 = (2 * (kb * TKS + kk) + j) * 8;
                    const int tap = k0 / a.ci, c0 = k0 - tap * a.ci;
                    const uint32_t dst = tc::smem_u32(sA + s * A_ST + kk * (TT * BM * 32) + j * (TT * BM * 16));
                    if (tap < 27)
                        tma_load_4d(dst, &map, c0, x0 + tap % 3 - 1, y0 + (tap / 3) % 3 - 1, z0 + tap / 9 - 1, fb);
                    else                                             // K padding: a box wholly outside, all zeros
                        tma_load_4d(dst, &map, 0, x0, y0, -4 * a.bz - 8, fb);
                }
            }
            bulk_load(tc::smem_u32(sB + s * B_ST), a.wpk + (size_t)kb * TKS * N * 16, (uint32_t)(nks * N * 32), fb);
        }
    } else if (warp == 1 && lane == 0) {                    // MMA issuer
        const uint32_t idesc = tc::idesc_bf16(BM, N);
        for (int kb = 0; kb < nkb && !*abort_flag; ++kb) {
            const int s = kb % TST;
            if (!tc::mbar_wait(&full[s], (uint32_t)(kb / TST) & 1u, WAIT_LIMIT)) { *abort_flag = 1; atomicOr(a.err, PSL_DEV_ERR_TIMEOUT); break; }
            tc::fence_after_sync();
            const int nks = min(TKS, a.ksteps - kb * TKS);
            for (int kk = 0; kk < nks; ++kk) {
                const uint64_t bd = tc::desc_kmajor(tc::smem_u32(sB + s * B_ST + kk * (N * 32)), 128, 256);
#pragma unroll
                for (int tt = 0; tt < TT; ++tt) {
                    // tile tt: rows 128 tt .. 128 tt + 127 of the stage's boxes
                    const uint32_t base = tc::smem_u32(sA + s * A_ST + kk * (TT * BM * 32));
                    const uint64_t ad = a.wide ? tc::desc_kmajor_sw32(base + tt * (BM * 32), 256)
                                               : tc::desc_kmajor(base + tt * (BM * 16), TT * BM * 16, 128);
                    tc::mma_bf16(tmem + (uint32_t)(tt * N), ad, bd, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
                }
            }
            tc::mma_commit(&empty[s]);
        }
        tc::mma_commit(accum);
    } else if (warp >= 2) {                                  // epilogue
        const bool ok = tc::mbar_wait(accum, 0u, WAIT_LIMIT) && !*abort_flag;
        if (!ok && t == 64) { *abort_flag = 1; atomicOr(a.err, PSL_DEV_ERR_TIMEOUT); }
        tc::fence_after_sync();
        const int q = warp & 3;                              // TMEM lanes 32q..32q+31
        for (int tt = 0; tt < TT && __any_sync(0xFFFFFFFFu, ok); ++tt) {
            const int m = tt * BM + 32 * q + lane;
            const int xx = x0 + m % a.bx, yy = y0 + (m / a.bx) % a.by, zz = z0 + m / (a.bx * a.by);
            const bool row_ok = ok && xx < a.W && yy < a.H && zz < a.D;
            const int64_t v = ((int64_t)zz * a.H + yy) * a.W + xx;
#pragma unroll
            for (int c0 = 0; c0 < N; c0 += 16) {
                float r[16];
                tc::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(tt * N + c0), r);
                if (row_ok) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const float qv = r[i] + (a.bias ? __ldg(a.bias + c0 + i) : 0.0f);
                        r[i] = a.relu ? fmaxf(qv, 0.0f) : qv;
                    }
                    if (a.out) {
                        __align__(16) __nv_bfloat16 h[16];
#pragma unroll
                        for (int i = 0; i < 16; ++i) h[i] = __float2bfloat16_rn(r[i]);
                        uint4 *dst = reinterpret_cast<uint4 *>(a.out + v * N + c0);
                        dst[0] = reinterpret_cast<uint4 *>(h)[0];
                        dst[1] = reinterpret_cast<uint4 *>(h)[1];
                    }
                    if (a.out_f32) {
                        float4 *dst = reinterpret_cast<float4 *>(a.out_f32 + v * N + c0);
#pragma unroll
                        for (int i = 0; i < 4; ++i) dst[i] = make_float4(r[4 * i], r[4 * i + 1], r[4 * i + 2], r[4 * i + 3]);
                    }
                }
            }
        }
    }
    __syncwarp();
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tmem, TCOLS);
}

// ------------------------------------------------------ halo form ---
// For volumes whose rows hold whole 128-voxel tiles (W a multiple of 128)
// and C_in a multiple of 16: a CTA's TT tiles are TT consecutive rows
// (y0 .. y0 + TT - 1) of 128 voxels at one z.  For each 16-channel chunk c
// of the input and each plane dz of the taps, one pipeline stage brings in
// the input plane z0 + dz over the rows y0 - 1 .. y0 + TT and the columns
// x0 - 1 .. x0 + 128 (two TMA boxes of 8 channels; the copy engine's zero
// fill is the padding) and the 9 taps of that plane and chunk (9 packed K
// steps, bulk copies).  The plane lands as rows of 16 bytes, so the A
// operand of tap (dy, dx) for tile tt is a view of it: 128 rows starting at
// row (tt + dy + 1) * 130 + dx + 1 (the no-swizzle K-major layout, 8-row
// groups 128 bytes apart, the two 8-channel halves HALF bytes apart).  One
// plane serves 9 x TT MMAs, where the per-tap form loads a shifted box for
// every tap: a third of the input traffic from L2.  Warp roles and the
// completion handshakes are those of the TMA form.
#ifndef PSL_HALO_TILES_WIDE
#define PSL_HALO_TILES_WIDE 4                    // 128-voxel rows per CTA for C_out = 128 (all 512 TMEM columns)
#endif
#ifndef PSL_HALO_TILES_64
#define PSL_HALO_TILES_64 2                      // the same for C_out = 64
#endif
#ifndef PSL_HALO_STAGES
#define PSL_HALO_STAGES 2
#endif
constexpr int HX = BM + 2;                       // plane row: x0 - 1 .. x0 + 128
constexpr int HST = PSL_HALO_STAGES;             // stages

__host__ __device__ constexpr int round128(int b) { return (b + 127) / 128 * 128; }
template <int N> struct Halo {
    static constexpr int TT = N == 128 ? PSL_HALO_TILES_WIDE : (N == 64 ? PSL_HALO_TILES_64 : tiles_for(N));
    static constexpr int HY = TT + 2;            // plane rows: y0 - 1 .. y0 + TT
    static constexpr int HALF = round128(HY * HX * 16);      // one 8-channel half of a plane
    static constexpr int A_ST = 2 * HALF;
    static constexpr int B_ST = 9 * N * 32;      // 9 packed K steps
    static constexpr int ST = round128(A_ST + B_ST);
    static constexpr size_t SMEM = (size_t)HST * ST + 128;
};

struct HaloConvArgs {
    const __nv_bfloat16 *wpk;
    const float *bias;
    __nv_bfloat16 *out;
    float *out_f32;
    int ci, D, H, W, relu;
    uint32_t *err;
};

template <int N>
__global__ void __launch_bounds__(192, 1) k_conv3d_halo(const __grid_constant__ CUtensorMap map, HaloConvArgs a) {
    using G = Halo<N>;
    constexpr int TT = G::TT;
    extern __shared__ __align__(1024) uint8_t smem[];
    constexpr uint32_t TCOLS = TT * N < 32 ? 32 : TT * N;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + HST * G::ST);
    uint64_t *empty = full + HST, *accum = empty + HST;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(accum + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int x0 = blockIdx.x * BM, y0 = blockIdx.y * TT, z0 = blockIdx.z;
    if (warp == 1) { tc::tmem_alloc(tslot, TCOLS); tc::tmem_relinquish(); }
    if (t == 0) {
        for (int s = 0; s < HST; ++s) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 1); }
        tc::mbar_init(accum, 1);
        *abort_flag = 0;
        tc::mbar_fence_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const int nch = a.ci / 16;                       // 16-channel chunks
    const int nit = 3 * nch;                         // stages: (chunk, plane)

    if (warp == 0 && lane == 0) {                           // producer
        for (int it = 0; it < nit && !*abort_flag; ++it) {
            const int s = it % HST, c = it / 3, dz = it % 3;
            const uint32_t ph = (uint32_t)(it / HST) & 1u;
            if (!tc::mbar_wait(&empty[s], ph ^ 1u, WAIT_LIMIT)) { *abort_flag = 1; atomicOr(a.err, PSL_DEV_ERR_TIMEOUT); break; }
            uint8_t *st = smem + s * G::ST;
            const uint32_t fb = tc::smem_u32(&full[s]);
            mbar_expect_tx(fb, (uint32_t)(2 * G::HY * HX * 16 + G::B_ST));       // the bytes the copies bring
            tma_load_4d(tc::smem_u32(st), &map, 16 * c, x0 - 1, y0 - 1, z0 + dz - 1, fb);
            tma_load_4d(tc::smem_u32(st + G::HALF), &map, 16 * c + 8, x0 - 1, y0 - 1, z0 + dz - 1, fb);
            // tap (dz, j): packed K step tap * nch + c
            for (int j = 0; j < 9; ++j)
                bulk_load(tc::smem_u32(st + G::A_ST + j * N * 32), a.wpk + (size_t)((dz * 9 + j) * nch + c) * N * 16,
                          (uint32_t)(N * 32), fb);
        }
    } else if (warp == 1 && lane == 0) {                    // MMA issuer
        const uint32_t idesc = tc::idesc_bf16(BM, N);
        for (int it = 0; it < nit && !*abort_flag; ++it) {
            const int s = it % HST;
            if (!tc::mbar_wait(&full[s], (uint32_t)(it / HST) & 1u, WAIT_LIMIT)) { *abort_flag = 1; atomicOr(a.err, PSL_DEV_ERR_TIMEOUT); break; }
            tc::fence_after_sync();
            const uint32_t base = tc::smem_u32(smem + s * G::ST);
            for (int j = 0; j < 9; ++j) {
                const int dy = j / 3 - 1, dx = j % 3 - 1;
                const uint64_t bd = tc::desc_kmajor(base + G::A_ST + j * (N * 32), 128, 256);
#pragma unroll
                for (int tt = 0; tt < TT; ++tt) {
                    const int row = (tt + dy + 1) * HX + dx + 1;
                    const uint64_t ad = tc::desc_kmajor(base + row * 16, G::HALF, 128);
                    tc::mma_bf16(tmem + (uint32_t)(tt * N), ad, bd, idesc, (it > 0 || j > 0) ? 1u : 0u);
                }
            }
            tc::mma_commit(&empty[s]);
        }
        tc::mma_commit(accum);
    } else if (warp >= 2) {                                  // epilogue
        const bool ok = tc::mbar_wait(accum, 0u, WAIT_LIMIT) && !*abort_flag;
        if (!ok && t == 64) { *abort_flag = 1; atomicOr(a.err, PSL_DEV_ERR_TIMEOUT); }
        tc::fence_after_sync();
        const int q = warp & 3;                              // TMEM lanes 32q..32q+31
        for (int tt = 0; tt < TT && __any_sync(0xFFFFFFFFu, ok); ++tt) {
            const int xx = x0 + 32 * q + lane, yy = y0 + tt;
            const bool row_ok = ok && xx < a.W && yy < a.H;
            const int64_t v = ((int64_t)z0 * a.H + yy) * a.W + xx;
#pragma unroll
            for (int c0 = 0; c0 < N; c0 += 16) {
                float r[16];
                tc::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(tt * N + c0), r);
                if (row_ok) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const float qv = r[i] + (a.bias ? __ldg(a.bias + c0 + i) : 0.0f);
                        r[i] = a.relu ? fmaxf(qv, 0.0f) : qv;
                    }
                    if (a.out) {
                        __align__(16) __nv_bfloat16 h[16];
#pragma unroll
                        for (int i = 0; i < 16; ++i) h[i] = __float2bfloat16_rn(r[i]);
                        uint4 *dst = reinterpret_cast<uint4 *>(a.out + v * N + c0);
                        dst[0] = reinterpret_cast<uint4 *>(h)[0];
                        dst[1] = reinterpret_cast<uint4 *>(h)[1];
                    }
                    if (a.out_f32) {
                        float4 *dst = reinterpret_cast<float4 *>(a.out_f32 + v * N + c0);
#pragma unroll
                        for (int i = 0; i < 4; ++i) dst[i] = make_float4(r[4 * i], r[4 * i + 1], r[4 * i + 2], r[4 * i + 3]);
                    }
                }
            }
        }
    }
    __syncwarp();
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tmem, TCOLS);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// the CTA box of the TMA form, or false when the volume needs the gather form
bool tma_box(int W, int H, int D, int tt, int &bx, int &by, int &bz) {
    auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
    const int vox = tt * BM;                      // voxels of one CTA
    int rest;
    if (W >= BM) { bx = BM; rest = vox / BM; }
    else if (pow2(W)) { bx = W; rest = vox / bx; }
    else return false;
    int h = 1;
    while (h * 2 <= H && h * 2 <= rest) h *= 2;
    by = h;
    bz = rest / by;
    return bz <= 256 && by <= 256 && bx <= 256 && D >= 1;
}

template <int N>
int launch_tma(const ConvArgs &c, int bx, int by, int bz, cudaStream_t st) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return psl_fail(PSL_ECUDA, "conv3d: cuTensorMapEncodeTiled unavailable");
    CUtensorMap map;
    // 16-channel boxes fill whole 32-byte L2 sectors (8-channel ones fetch
    // half of every sector for nothing); they land 32-byte swizzled
    const int wide = c.ci >= 16 ? 1 : 0;
    const cuuint64_t dims[4] = {(cuuint64_t)c.ci, (cuuint64_t)c.W, (cuuint64_t)c.H, (cuuint64_t)c.D};
    const cuuint64_t strides[3] = {(cuuint64_t)c.ci * 2, (cuuint64_t)c.ci * 2 * c.W, (cuuint64_t)c.ci * 2 * c.W * c.H};
    const cuuint32_t box[4] = {wide ? 16u : 8u, (cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16 *>(c.in), dims, strides, box,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, wide ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return psl_fail(PSL_ECUDA, "conv3d: tensor map encoding failed");
    constexpr int TT = tiles_for(N);
    const size_t smem = (size_t)TST * (TKS * TT * BM * 32 + TKS * N * 32) + 128;
    static bool attr = false;
    if (!attr) {
        PSL_CUDA(cudaFuncSetAttribute(k_conv3d_tma<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    TmaConvArgs a{c.wpk, c.bias, c.out, c.out_f32, c.ci, c.D, c.H, c.W, c.relu, c.ksteps, bx, by, bz, wide, c.err};
    const dim3 grid((c.W + bx - 1) / bx, (c.H + by - 1) / by, (c.D + bz - 1) / bz);
    k_conv3d_tma<N><<<grid, 192, smem, st>>>(map, a); PSL_NOTE_LAUNCH();
    PSL_CUDA(cudaGetLastError());
    return PSL_OK;
}

template <int N>
int launch_halo(const ConvArgs &c, cudaStream_t st) {
    using G = Halo<N>;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return psl_fail(PSL_ECUDA, "conv3d: cuTensorMapEncodeTiled unavailable");
    CUtensorMap map;
    const cuuint64_t dims[4] = {(cuuint64_t)c.ci, (cuuint64_t)c.W, (cuuint64_t)c.H, (cuuint64_t)c.D};
    const cuuint64_t strides[3] = {(cuuint64_t)c.ci * 2, (cuuint64_t)c.ci * 2 * c.W, (cuuint64_t)c.ci * 2 * c.W * c.H};
    const cuuint32_t box[4] = {8u, (cuuint32_t)HX, (cuuint32_t)G::HY, 1u};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16 *>(c.in), dims, strides, box,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return psl_fail(PSL_ECUDA, "conv3d: tensor map encoding failed");
    static bool attr = false;
    if (!attr) {
        PSL_CUDA(cudaFuncSetAttribute(k_conv3d_halo<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM));
        attr = true;
    }
    HaloConvArgs a{c.wpk, c.bias, c.out, c.out_f32, c.ci, c.D, c.H, c.W, c.relu, c.err};
    const dim3 grid((c.W + BM - 1) / BM, (c.H + G::TT - 1) / G::TT, c.D);
    k_conv3d_halo<N><<<grid, 192, G::SMEM, st>>>(map, a); PSL_NOTE_LAUNCH();
    PSL_CUDA(cudaGetLastError());
    return PSL_OK;
}

// Taps W[27][ci][co] (FP32) -> BF16 B tiles: K step s, 8-row group g of the
// outputs, K chunk j, row n % 8, element e: k = 16 s + 8 j + e, tap = k / ci.
// mirror: the input-gradient form, W'[t][o][i] = W[26 - t][i][o] (a
// convolution from co channels to ci).
__global__ void k_pack(const float *w, int ci, int co, int mirror, __nv_bfloat16 *out, int ksteps) {
    const int cin = mirror ? co : ci, cout = mirror ? ci : co;
    const int64_t total = (int64_t)ksteps * cout * 16;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(q / (cout * 16));
        const int r = (int)(q % (cout * 16));
        const int g = r / 128, j = (r % 128) / 64, n8 = (r % 64) / 8, e = r % 8;
        const int n = g * 8 + n8;
        const int k = 16 * s + 8 * j + e;
        const int tap = k / cin, c = k % cin;
        float val = 0.0f;
        if (tap < 27) val = mirror ? w[((int64_t)(26 - tap) * ci + n) * co + c] : w[((int64_t)tap * ci + c) * co + n];
        out[q] = __float2bfloat16_rn(val);
    }
}

template <int N>
int launch(const ConvArgs &a, int64_t V, cudaStream_t st) {
    const size_t smem = 2 * (size_t)(SK * BM * 32) + 2 * (size_t)(SK * N * 32) + 64;
    static bool attr = false;
    if (!attr) {
        PSL_CUDA(cudaFuncSetAttribute(k_conv3d<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    const int grid = (int)((V + BM - 1) / BM);
    k_conv3d<N><<<grid, 128, smem, st>>>(a); PSL_NOTE_LAUNCH();
    PSL_CUDA(cudaGetLastError());
    return PSL_OK;
}

template <int N>
int launch_wgrad(const WgradArgs &a0, int64_t V, cudaStream_t st) {
    const size_t smem = 2 * (size_t)(SK * BM * 32) + 2 * (size_t)(SK * N * 32) + 64;
    static bool attr = false;
    if (!attr) {
        PSL_CUDA(cudaFuncSetAttribute(k_conv3d_wgrad<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    WgradArgs a = a0;
    const int mt = (27 * a.ci + BM - 1) / BM;
    // enough voxel splits to fill the GPU about twice, each a whole number of stages
    const int64_t want = std::max<int64_t>(1, (int64_t)psl_sm_count() * 2 / mt);
    int64_t per = (V + want - 1) / want;
    per = std::max<int64_t>(BM, (per + BM - 1) / BM * BM);
    a.vox_per_cta = per;
    const dim3 grid(mt, (unsigned)((V + per - 1) / per));
    k_conv3d_wgrad<N><<<grid, 128, smem, st>>>(a); PSL_NOTE_LAUNCH();
    PSL_CUDA(cudaGetLastError());
    return PSL_OK;
}

}  // namespace

int psl_conv_ksteps(int ci) { return (27 * ci + 15) / 16; }

int psl_conv3d_wgrad_run(const __nv_bfloat16 *x, int ci, const __nv_bfloat16 *gy, int co, int nx, int ny, int nz,
                         float *dw, uint32_t *err, cudaStream_t st) {
    WgradArgs a{x, gy, dw, ci, nz, ny, nx, 0, err};
    const int64_t V = (int64_t)nx * ny * nz;
    if (V == 0) return PSL_OK;
    switch (co) {
        case 16: return launch_wgrad<16>(a, V, st);
        case 32: return launch_wgrad<32>(a, V, st);
        case 64: return launch_wgrad<64>(a, V, st);
        case 128: return launch_wgrad<128>(a, V, st);
        default: return psl_fail(PSL_EINVAL, "conv3d wgrad: C_out must be 16, 32, 64 or 128");
    }
}

static int g_conv_form = 0;             // 0: halo, else per-tap TMA, else gather; 1: gather only; 2: no halo

static int conv3d_dispatch(const __nv_bfloat16 *in, int ci, const __nv_bfloat16 *wpk, const float *bias, int co,
                           int nx, int ny, int nz, int relu, __nv_bfloat16 *out, float *out_f32, uint32_t *err,
                           cudaStream_t st);

// the convolution, timed (device time, CUDA events on its stream) while the
// library's profiler is on
int psl_conv3d_run(const __nv_bfloat16 *in, int ci, const __nv_bfloat16 *wpk, const float *bias, int co, int nx,
                   int ny, int nz, int relu, __nv_bfloat16 *out, float *out_f32, uint32_t *err, cudaStream_t st) {
    void *tk = nullptr;
    if (psl_timer_on()) psl_timer_begin(PK_CONV, st, &tk);
    const int rc = conv3d_dispatch(in, ci, wpk, bias, co, nx, ny, nz, relu, out, out_f32, err, st);
    if (tk) psl_timer_end(PK_CONV, st, tk);
    return rc;
}

static int conv3d_dispatch(const __nv_bfloat16 *in, int ci, const __nv_bfloat16 *wpk, const float *bias, int co,
                           int nx, int ny, int nz, int relu, __nv_bfloat16 *out, float *out_f32, uint32_t *err,
                           cudaStream_t st) {
    ConvArgs a{in, wpk, bias, out, out_f32, ci, nz, ny, nx, relu, psl_conv_ksteps(ci), err};
    const int64_t V = (int64_t)nx * ny * nz;
    if (V == 0) return PSL_OK;
    int bx, by, bz;
    if (g_conv_form == 0 && nx % BM == 0 && ci % 16 == 0 && nz <= 65535 && ny <= 65535) {
        switch (co) {
            case 16: return launch_halo<16>(a, st);
            case 32: return launch_halo<32>(a, st);
            case 64: return launch_halo<64>(a, st);
            case 128: return launch_halo<128>(a, st);
            default: break;
        }
    }
    if (g_conv_form != 1 && (co == 16 || co == 32 || co == 64 || co == 128) && tma_box(nx, ny, nz, tiles_for(co), bx, by, bz)) {
        switch (co) {
            case 16: return launch_tma<16>(a, bx, by, bz, st);
            case 32: return launch_tma<32>(a, bx, by, bz, st);
            case 64: return launch_tma<64>(a, bx, by, bz, st);
            case 128: return launch_tma<128>(a, bx, by, bz, st);
            default: break;
        }
    }
    switch (co) {
        case 16: return launch<16>(a, V, st);
        case 32: return launch<32>(a, V, st);
        case 64: return launch<64>(a, V, st);
        case 128: return launch<128>(a, V, st);
        default: return psl_fail(PSL_EINVAL, "conv3d: C_out must be 16, 32, 64 or 128");
    }
}

int psl_conv3d_pack_run(const float *w, int ci, int co, int mirror, __nv_bfloat16 *out, cudaStream_t st) {
    const int cin = mirror ? co : ci, cout = mirror ? ci : co;
    const int ks = psl_conv_ksteps(cin);
    const int64_t total = (int64_t)ks * cout * 16;
    k_pack<<<(int)std::min<int64_t>((total + 255) / 256, 4096), 256, 0, st>>>(w, ci, co, mirror, out, ks); PSL_NOTE_LAUNCH();
    PSL_CUDA(cudaGetLastError());
    return PSL_OK;
}

static bool conv_shape_ok(int ci, int co) {
    return ci >= 8 && ci <= 128 && ci % 8 == 0 && (co == 16 || co == 32 || co == 64 || co == 128);
}

extern "C" int psl_conv3d_pack(const float *w, int32_t ci, int32_t co, int32_t mirror, uint16_t *wpk, void *stream) {
    if (!w || !wpk) return psl_fail(PSL_EINVAL, "psl_conv3d_pack: null pointer");
    if (!conv_shape_ok(mirror ? co : ci, mirror ? ci : co))
        return psl_fail(PSL_EINVAL, "psl_conv3d_pack: channels (C_in multiple of 8 up to 128; C_out 16/32/64/128)");
    return psl_conv3d_pack_run(w, ci, co, mirror, reinterpret_cast<__nv_bfloat16 *>(wpk), as_stream(stream));
}

extern "C" int64_t psl_conv3d_packed_size(int32_t ci, int32_t co) { return (int64_t)psl_conv_ksteps(ci) * co * 16; }

extern "C" int psl_conv3d(const uint16_t *in, int32_t ci, const uint16_t *wpk, const float *bias, int32_t co,
                          int32_t nx, int32_t ny, int32_t nz, int32_t relu, uint16_t *out, float *out_f32,
                          void *stream) {
    if (!in || !wpk || (!out && !out_f32)) return psl_fail(PSL_EINVAL, "psl_conv3d: null pointer");
    if (!conv_shape_ok(ci, co)) return psl_fail(PSL_EINVAL, "psl_conv3d: channels (C_in multiple of 8 up to 128; C_out 16/32/64/128)");
    if (nx <= 0 || ny <= 0 || nz <= 0 || (int64_t)nx * ny * nz >= (1ll << 31))
        return psl_fail(PSL_EINVAL, "psl_conv3d: volume size");
    if (((uintptr_t)in | (uintptr_t)wpk | (uintptr_t)out | (uintptr_t)out_f32) & 15)
        return psl_fail(PSL_EINVAL, "psl_conv3d: arrays must be 16-byte aligned");
    cudaStream_t st = as_stream(stream);
    uint32_t *err = nullptr;
    PSL_CUDA(psl_malloc_async((void **)&err, 4, st));
    cudaMemsetAsync(err, 0, 4, st);
    int rc = psl_conv3d_run(reinterpret_cast<const __nv_bfloat16 *>(in), ci, reinterpret_cast<const __nv_bfloat16 *>(wpk),
                            bias, co, nx, ny, nz, relu, reinterpret_cast<__nv_bfloat16 *>(out), out_f32, err, st);
    uint32_t herr = 0;
    cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(err, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (rc) return rc;
    if (e != cudaSuccess) return psl_fail(PSL_ECUDA, cudaGetErrorString(e));
    if (herr) return psl_fail(PSL_ETIMEOUT, "psl_conv3d: tensor-core completion wait gave up");
    return PSL_OK;
}

extern "C" int psl_conv3d_wgrad(const uint16_t *x, int32_t ci, const uint16_t *gy, int32_t co, int32_t nx,
                                int32_t ny, int32_t nz, float *dw, void *stream) {
    if (!x || !gy || !dw) return psl_fail(PSL_EINVAL, "psl_conv3d_wgrad: null pointer");
    if (!conv_shape_ok(ci, co)) return psl_fail(PSL_EINVAL, "psl_conv3d_wgrad: channels (C_in multiple of 8 up to 128; C_out 16/32/64/128)");
    if (nx <= 0 || ny <= 0 || nz <= 0 || (int64_t)nx * ny * nz >= (1ll << 31))
        return psl_fail(PSL_EINVAL, "psl_conv3d_wgrad: volume size");
    if (((uintptr_t)x | (uintptr_t)gy) & 15) return psl_fail(PSL_EINVAL, "psl_conv3d_wgrad: arrays must be 16-byte aligned");
    cudaStream_t st = as_stream(stream);
    uint32_t *err = nullptr;
    PSL_CUDA(psl_malloc_async((void **)&err, 4, st));
    cudaMemsetAsync(err, 0, 4, st);
    int rc = psl_conv3d_wgrad_run(reinterpret_cast<const __nv_bfloat16 *>(x), ci, reinterpret_cast<const __nv_bfloat16 *>(gy),
                                  co, nx, ny, nz, dw, err, st);
    uint32_t herr = 0;
    cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(err, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (rc) return rc;
    if (e != cudaSuccess) return psl_fail(PSL_ECUDA, cudaGetErrorString(e));
    if (herr) return psl_fail(PSL_ETIMEOUT, "psl_conv3d_wgrad: tensor-core completion wait gave up");
    return PSL_OK;
}

extern "C" int psl_conv3d_form(int32_t form) {
    if (form < 0 || form > 2)
        return psl_fail(PSL_EINVAL, "psl_conv3d_form: 0 (halo or TMA where possible), 1 (gather) or 2 (per-tap TMA)");
    g_conv_form = form;
    return PSL_OK;
}
