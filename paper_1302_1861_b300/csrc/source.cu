// Source stage (Sec. 2.2, 2.3.3, 2.4): history -> (entry, read number) ->
// sorted record -> jaw model, fluence map, MU weight -> rotation and
// projection to the phantom surface -> photon / electron primaries.
//
// Acceptance and weights are taken in float32 with explicit round-to-nearest
// intrinsics (no fused multiply-add) in the documented operation order, so
// they are reproducible bit for bit on any IEEE float32 implementation.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "psl_internal.cuh"

namespace {

struct PlanDev {
    const int64_t *group_start, *group_seg, *seg_h, *seg_r0;
    const int32_t *seg_w;
    const uint32_t *sorted;
    const int64_t *e_start, *e_nrec, *e_offset;
    const int32_t *e_beam;
    const BeamDev *beams;
    const PslRecord *rec;
    int n_groups;
    float z_psl;
    float L[3], origin[3];
};

struct SrcOut {
    int64_t entry, use, rec;
    int beam;
    int status;
    int ptype;
    float s[8];                    // x y z u v w e wt (phantom-local)
};

__device__ __forceinline__ int64_t upper_bound_i64(const int64_t *a, int64_t lo, int64_t hi, int64_t v) {
    // first index in [lo, hi) with a[i] > v
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] <= v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ void source_one(const PlanDev &P, const int64_t *gs_sh, int64_t h, SrcOut &o) {
    // group, segment, round, position
    int lo = 0, hi = P.n_groups;            // last g with group_start[g] <= h
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (gs_sh[mid] <= h) lo = mid; else hi = mid;
    }
    const int g = lo;
    const int64_t hl = h - gs_sh[g];
    const int64_t q = upper_bound_i64(P.seg_h, P.group_seg[g], P.group_seg[g + 1], hl) - 1;
    const int64_t off = hl - P.seg_h[q];
    const int64_t w = P.seg_w[q];
    const int64_t r = P.seg_r0[q] + off / w;
    const int64_t pidx = off % w;
    const int64_t entry = P.sorted[P.group_seg[g] + pidx];
    const int64_t nrec = P.e_nrec[entry];
    const int64_t rec = P.e_start[entry] + (P.e_offset[entry] + r) % nrec;
    o.entry = entry; o.use = r; o.rec = rec;
    const int b = P.e_beam[entry];
    o.beam = b;
    const PslRecord R = P.rec[rec];
    const BeamDev &B = P.beams[b];
    o.ptype = R.q == 0 ? 0 : (R.q < 0 ? 1 : 2);
    // jaw model (Sec. 2.2)
    float w2 = __fsub_rn(__fsub_rn(1.0f, __fmul_rn(R.u, R.u)), __fmul_rn(R.v, R.v));
    if (!(w2 > 0.0f)) { o.status = PSL_SRC_JAW; return; }
    const float wz = __fsqrt_rn(w2);
    const float xj = __fadd_rn(R.x, __fmul_rn(R.u, __fdiv_rn(B.dzx, wz)));
    const float yj = __fadd_rn(R.y, __fmul_rn(R.v, __fdiv_rn(B.dzy, wz)));
    if (!(xj >= B.xlo && xj <= B.xhi && yj >= B.ylo && yj <= B.yhi)) { o.status = PSL_SRC_JAW; return; }
    // fluence map at the isocentre plane (Sec. 2.2, 2.4)
    float wt = R.wt;
    if (B.fluence) {
        const float ti = __fdiv_rn(B.diso, wz);
        const float fx = __fdiv_rn(__fsub_rn(__fadd_rn(R.x, __fmul_rn(R.u, ti)), B.fx0), B.fdx);
        const float fy = __fdiv_rn(__fsub_rn(__fadd_rn(R.y, __fmul_rn(R.v, ti)), B.fy0), B.fdy);
        const float ix = floorf(fx), iy = floorf(fy);
        if (!(ix >= 0.0f && ix < (float)B.fnx && iy >= 0.0f && iy < (float)B.fny)) { o.status = PSL_SRC_FLUENCE; return; }
        wt = __fmul_rn(wt, __ldg(B.fluence + (int)iy * B.fnx + (int)ix));
    }
    wt = __fmul_rn(wt, B.mu_ratio);        // MU weight (Sec. 2.3.3)
    if (wt == 0.0f) { o.status = PSL_SRC_ZERO_WEIGHT; return; }
    // rotate about the isocentre into the patient frame, then phantom-local
    const float pb[3] = {R.x, R.y, P.z_psl - B.sad};
    const float db[3] = {R.u, R.v, wz};
    float p[3], d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        p[k] = B.r[3 * k] * pb[0] + B.r[3 * k + 1] * pb[1] + B.r[3 * k + 2] * pb[2] + B.iso[k] - P.origin[k];
        d[k] = B.r[3 * k] * db[0] + B.r[3 * k + 1] * db[1] + B.r[3 * k + 2] * db[2];
    }
    // entry of the full line into the phantom box [0, L]
    float tin = -INFINITY, tout = INFINITY;
    bool miss = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (d[k] != 0.0f) {
            float t0 = (0.0f - p[k]) / d[k], t1 = (P.L[k] - p[k]) / d[k];
            tin = fmaxf(tin, fminf(t0, t1));
            tout = fminf(tout, fmaxf(t0, t1));
        } else if (p[k] < 0.0f || p[k] > P.L[k]) {
            miss = true;
        }
    }
    o.s[6] = R.e; o.s[7] = wt;
    if (miss || !(tin < tout)) { o.status = PSL_SRC_MISS; return; }
#pragma unroll
    for (int k = 0; k < 3; ++k) { o.s[k] = p[k] + tin * d[k]; o.s[3 + k] = d[k]; }
    o.status = PSL_SRC_TRANSPORT;
}

__device__ __forceinline__ unsigned long long fixed_point(float e, float wt) {
    return (unsigned long long)__float2ll_rn(__fmul_rn(e, wt) * 4294967296.0f);
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// production: write the primaries of histories [first, first+n) to the batch
__global__ void __launch_bounds__(256) k_source(PlanDev P, int64_t first, int64_t n, int64_t stride, Particle *out,
                                                int64_t cap, uint32_t *counts, unsigned long long *ledger) {
    __shared__ int64_t gs[1025];
    for (int i = threadIdx.x; i <= P.n_groups; i += blockDim.x) gs[i] = P.group_start[i];
    __syncthreads();
    unsigned long long emitted = 0, missed = 0;
    const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n_round = (n + gstride - 1) / gstride * gstride;   // whole warps iterate together
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += gstride) {
        SrcOut o;
        o.status = -1;
        if (i < n) source_one(P, gs, first + i * stride, o);
        if (o.status == PSL_SRC_TRANSPORT || o.status == PSL_SRC_MISS) {
            unsigned long long q = fixed_point(o.s[6], o.s[7]);
            emitted += q;
            if (o.status == PSL_SRC_MISS) missed += q;
        }
        if (o.status == PSL_SRC_TRANSPORT) {
            Particle pt;
            pt.x = o.s[0]; pt.y = o.s[1]; pt.z = o.s[2]; pt.e = o.s[6];
            pt.u = o.s[3]; pt.v = o.s[4]; pt.w = o.s[5]; pt.wt = o.s[7];
            const uint64_t pid = (uint64_t)(first + i * stride);
            pt.pid_lo = (uint32_t)pid; pt.pid_hi = (uint32_t)(pid >> 32);
            pt.type = o.ptype; pt.root = (uint32_t)i;
            const bool is_ph = o.ptype == 0;
            // warp-aggregated slot: photons grow from the front, charged from the back
            unsigned mask = __activemask();
            unsigned same = __match_any_sync(mask, is_ph ? 0 : 1);
            int lane = threadIdx.x & 31, leader = __ffs(same) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(&counts[is_ph ? 0 : 1], (uint32_t)__popc(same));
            base = __shfl_sync(same, base, leader);
            uint32_t idx = base + __popc(same & ((1u << lane) - 1u));
            Particle *dst = is_ph ? out + idx : out + (cap - 1 - idx);
            store_particle(dst, pt);
        }
    }
    emitted = warp_sum_u64(emitted);
    missed = warp_sum_u64(missed);
    if ((threadIdx.x & 31) == 0) {
        if (emitted) atomicAdd(&ledger[0], emitted);
        if (missed) atomicAdd(&ledger[1], missed);
    }
}

__global__ void __launch_bounds__(256) k_source_trace(PlanDev P, int64_t first, int64_t n, int64_t stride, int64_t *entry, int64_t *use,
                                                      int64_t *rec, int32_t *beam, int8_t *status, float *state,
                                                      int32_t *ptype) {
    __shared__ int64_t gs[1025];
    for (int i = threadIdx.x; i <= P.n_groups; i += blockDim.x) gs[i] = P.group_start[i];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        SrcOut o;
        for (int k = 0; k < 8; ++k) o.s[k] = 0.f;
        source_one(P, gs, first + i * stride, o);
        if (entry) entry[i] = o.entry;
        if (use) use[i] = o.use;
        if (rec) rec[i] = o.rec;
        if (beam) beam[i] = o.beam;
        if (status) status[i] = (int8_t)o.status;
        if (ptype) ptype[i] = o.ptype;
        if (state)
            for (int k = 0; k < 8; ++k) state[8 * i + k] = o.s[k];
    }
}

PlanDev make_plan_dev(const psl_plan *p, const psl_phantom_t *ph) {
    PlanDev P;
    P.group_start = p->group_start; P.group_seg = p->group_seg; P.seg_h = p->seg_h; P.seg_r0 = p->seg_r0;
    P.seg_w = p->seg_w; P.sorted = p->sorted; P.e_start = p->e_start; P.e_nrec = p->e_nrec;
    P.e_offset = p->e_offset; P.e_beam = p->e_beam; P.beams = p->beams; P.rec = p->store->rec;
    P.n_groups = p->n_groups; P.z_psl = p->store->z_psl;
    P.L[0] = ph->nx * ph->vx; P.L[1] = ph->ny * ph->vy; P.L[2] = ph->nz * ph->vz;
    for (int k = 0; k < 3; ++k) P.origin[k] = ph->origin[k];
    return P;
}

int check_phantom(const psl_phantom_t *ph) {
    if (!ph || ph->nx <= 0 || ph->ny <= 0 || ph->nz <= 0 || !(ph->vx > 0) || !(ph->vy > 0) || !(ph->vz > 0))
        return psl_fail(PSL_EINVAL, "bad phantom");
    return PSL_OK;
}

__global__ void k_from_particles(const float *state, const int32_t *ptype, const uint64_t *pid, int64_t n, Particle *out,
                                 int64_t cap, uint32_t *counts) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        Particle pt;
        pt.x = state[8 * i]; pt.y = state[8 * i + 1]; pt.z = state[8 * i + 2];
        pt.u = state[8 * i + 3]; pt.v = state[8 * i + 4]; pt.w = state[8 * i + 5];
        pt.e = state[8 * i + 6]; pt.wt = state[8 * i + 7];
        pt.pid_lo = (uint32_t)pid[i]; pt.pid_hi = (uint32_t)(pid[i] >> 32);
        pt.type = (uint32_t)ptype[i]; pt.root = (uint32_t)i;
        uint32_t idx;
        if (pt.type == 0) { idx = atomicAdd(&counts[0], 1u); store_particle(out + idx, pt); }
        else { idx = atomicAdd(&counts[1], 1u); store_particle(out + (cap - 1 - idx), pt); }
    }
}

}  // namespace

static int alloc_batch(int64_t n, int64_t first, cudaStream_t st, psl_batch **out) {
    psl_batch *b = new psl_batch();
    b->n_histories = n; b->first_history = first; b->cap = std::max<int64_t>(n, 1);
    b->stream = st;
    cudaError_t e1 = cudaMallocAsync((void **)&b->p, b->cap * sizeof(Particle), st);
    cudaError_t e2 = cudaMallocAsync((void **)&b->counts, 32, st);
    if (e1 != cudaSuccess || e2 != cudaSuccess) { psl_batch_destroy(b); return psl_fail(PSL_ENOMEM, "batch allocation"); }
    cudaMemsetAsync(b->counts, 0, 32, st);
    *out = b;
    return PSL_OK;
}

static int finish_batch(psl_batch *b, cudaStream_t st) {
    uint32_t c[2] = {0, 0};
    cudaMemcpyAsync(c, b->counts, 8, cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return psl_fail(PSL_ECUDA, cudaGetErrorString(e));
    b->n_photons = c[0]; b->n_electrons = c[1];
    return PSL_OK;
}

static bool range_ok(const psl_plan_t *plan, int64_t first, int64_t n, int64_t stride) {
    if (n < 0 || first < 0 || stride < 1) return false;
    if (n == 0) return true;
    return first < plan->n_histories && (n - 1) <= (plan->n_histories - 1 - first) / stride;
}

extern "C" int psl_source_batch(const psl_plan_t *plan, const psl_phantom_t *phantom, int64_t first, int64_t n,
                                int64_t stride, psl_batch_t **out, void *stream_) {
    if (!plan || !out || !range_ok(plan, first, n, stride))
        return psl_fail(PSL_EINVAL, "psl_source_batch: bad argument or history range");
    if (n >= (1ll << 32)) return psl_fail(PSL_EINVAL, "psl_source_batch: batch too large");
    int rc = check_phantom(phantom);
    if (rc) return rc;
    if (plan->n_groups > 1024) return psl_fail(PSL_EINVAL, "psl_source_batch: too many energy divisions");
    cudaStream_t st = as_stream(stream_);
    psl_batch *b = nullptr;
    if ((rc = alloc_batch(n, first, st, &b))) return rc;
    b->seed = plan->seed;
    PlanDev P = make_plan_dev(plan, phantom);
    if (n > 0) {
        int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)psl_sm_count() * 16));
        { void *tk_ = nullptr; if (psl_timer_on()) psl_timer_begin(PK_SOURCE, st, &tk_); k_source<<<grid, 256, 0, st>>>(P, first, n, stride, b->p, b->cap, b->counts, (unsigned long long *)(b->counts + 2)); PSL_NOTE_LAUNCH(); if (tk_) psl_timer_end(PK_SOURCE, st, tk_); }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { psl_batch_destroy(b); return psl_fail(PSL_ECUDA, cudaGetErrorString(e)); }
    if ((rc = finish_batch(b, st))) { psl_batch_destroy(b); return rc; }
    *out = b;
    return PSL_OK;
}

extern "C" int psl_source_trace(const psl_plan_t *plan, const psl_phantom_t *phantom, int64_t first, int64_t n,
                                int64_t stride, int64_t *entry, int64_t *use, int64_t *rec, int32_t *beam,
                                int8_t *status, float *state, int32_t *ptype, void *stream_) {
    if (!plan || !range_ok(plan, first, n, stride))
        return psl_fail(PSL_EINVAL, "psl_source_trace: bad argument or history range");
    int rc = check_phantom(phantom);
    if (rc) return rc;
    if (plan->n_groups > 1024) return psl_fail(PSL_EINVAL, "psl_source_trace: too many energy divisions");
    if (n == 0) return PSL_OK;
    PlanDev P = make_plan_dev(plan, phantom);
    int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)psl_sm_count() * 16));
    k_source_trace<<<grid, 256, 0, as_stream(stream_)>>>(P, first, n, stride, entry, use, rec, beam, status, state, ptype); PSL_NOTE_LAUNCH();
    PSL_CUDA(cudaGetLastError());
    return PSL_OK;
}

extern "C" int psl_batch_from_particles(const float *state, const int32_t *ptype, const uint64_t *pid, int64_t n,
                                        uint64_t seed, psl_batch_t **out, void *stream_) {
    if (!out || n < 0 || n >= (1ll << 32) || (n > 0 && (!state || !ptype || !pid)))
        return psl_fail(PSL_EINVAL, "psl_batch_from_particles: bad argument");
    cudaStream_t st = as_stream(stream_);
    psl_batch *b = nullptr;
    int rc = alloc_batch(n, 0, st, &b);
    if (rc) return rc;
    b->seed = seed;
    if (n > 0) {
        int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096));
        k_from_particles<<<grid, 256, 0, st>>>(state, ptype, pid, n, b->p, b->cap, b->counts); PSL_NOTE_LAUNCH();
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { psl_batch_destroy(b); return psl_fail(PSL_ECUDA, cudaGetErrorString(e)); }
    if ((rc = finish_batch(b, st))) { psl_batch_destroy(b); return rc; }
    *out = b;
    return PSL_OK;
}

extern "C" int psl_batch_info(const psl_batch_t *b, int64_t *n_histories, int64_t *n_photons, int64_t *n_electrons) {
    if (!b) return psl_fail(PSL_EINVAL, "psl_batch_info: null batch");
    if (n_histories) *n_histories = b->n_histories;
    if (n_photons) *n_photons = b->n_photons;
    if (n_electrons) *n_electrons = b->n_electrons;
    return PSL_OK;
}

extern "C" void psl_batch_destroy(psl_batch_t *b) {
    if (!b) return;
    if (b->p) cudaFreeAsync(b->p, b->stream);
    if (b->counts) cudaFreeAsync(b->counts, b->stream);
    delete b;
}
