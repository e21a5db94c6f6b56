// The per-history source stage (Sec. 2.2, 2.3.3, 2.4) shared by the source
// kernels and the fused first transport pass: history -> (entry, read number)
// -> sorted record -> jaw model, fluence map, MU weight -> rotation and entry
// into the phantom.  Acceptance and weights are taken in float32 with
// round-to-nearest intrinsics (no fused multiply-add) in a fixed order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "psl_internal.cuh"

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

// group g and segment q of history h (the last segment whose first history
// is <= h's group-local index)
__device__ __forceinline__ void locate(const PlanDev &P, const int64_t *gs_sh, int64_t h, int &g, int64_t &q) {
    int lo = 0, hi = P.n_groups;            // last g with group_start[g] <= h
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (gs_sh[mid] <= h) lo = mid; else hi = mid;
    }
    g = lo;
    q = upper_bound_i64(P.seg_h, P.group_seg[g], P.group_seg[g + 1], h - gs_sh[g]) - 1;
}

// locate with a guess (g, q), e.g. a neighbouring history's: kept if it is
// exactly what locate() would return, otherwise searched
__device__ __forceinline__ void locate_hinted(const PlanDev &P, const int64_t *gs_sh, int64_t h, int &g, int64_t &q) {
    if (g >= 0 && gs_sh[g] <= h && h < gs_sh[g + 1]) {
        const int64_t hl = h - gs_sh[g];
        if (P.seg_h[q] <= hl && (q + 1 == P.group_seg[g + 1] || P.seg_h[q + 1] > hl)) return;
    }
    locate(P, gs_sh, h, g, q);
}

// a / b and a % b for non-negative a and 0 < b; 32-bit arithmetic when both fit
__device__ __forceinline__ void divmod_u64(uint64_t a, uint64_t b, uint64_t &q, uint64_t &r) {
    if ((a >> 32) == 0 && (b >> 32) == 0) {
        const uint32_t q32 = (uint32_t)a / (uint32_t)b;
        q = q32;
        r = (uint32_t)a - q32 * (uint32_t)b;
    } else {
        q = a / b;
        r = a - q * b;
    }
}

// Sec. 2.2, 2.3.3, 2.4 for one record and field: jaw model and fluence map
// (when `collimate`), MU weight, rotation into the patient and entry into the
// phantom box [0, L].  Sets o.ptype, o.status and o.s.
__device__ __forceinline__ void record_to_phantom(const PslRecord &R, const BeamDev &B, float z_psl, const float L[3],
                                                  const float origin[3], bool collimate, SrcOut &o) {
    o.ptype = R.q == 0 ? 0 : (R.q < 0 ? 1 : 2);
    // jaw model (Sec. 2.2)
    float w2 = __fsub_rn(__fsub_rn(1.0f, __fmul_rn(R.u, R.u)), __fmul_rn(R.v, R.v));
    if (!(w2 > 0.0f)) { o.status = PSL_SRC_JAW; return; }
    const float wz = __fsqrt_rn(w2);
    const float xj = __fadd_rn(R.x, __fmul_rn(R.u, __fdiv_rn(B.dzx, wz)));
    const float yj = __fadd_rn(R.y, __fmul_rn(R.v, __fdiv_rn(B.dzy, wz)));
    if (collimate && !(xj >= B.xlo && xj <= B.xhi && yj >= B.ylo && yj <= B.yhi)) { o.status = PSL_SRC_JAW; return; }
    // fluence map at the isocentre plane (Sec. 2.2, 2.4)
    float wt = R.wt;
    if (collimate && B.fluence) {
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
    const float pb[3] = {R.x, R.y, z_psl - B.sad};
    const float db[3] = {R.u, R.v, wz};
    float p[3], d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        p[k] = B.r[3 * k] * pb[0] + B.r[3 * k + 1] * pb[1] + B.r[3 * k + 2] * pb[2] + B.iso[k] - origin[k];
        d[k] = B.r[3 * k] * db[0] + B.r[3 * k + 1] * db[1] + B.r[3 * k + 2] * db[2];
    }
    // entry of the full line into the phantom box [0, L]
    float tin = -INFINITY, tout = INFINITY;
    bool miss = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (d[k] != 0.0f) {
            float t0 = (0.0f - p[k]) / d[k], t1 = (L[k] - p[k]) / d[k];
            tin = fmaxf(tin, fminf(t0, t1));
            tout = fminf(tout, fmaxf(t0, t1));
        } else if (p[k] < 0.0f || p[k] > L[k]) {
            miss = true;
        }
    }
    o.s[6] = R.e; o.s[7] = wt;
    if (miss || !(tin < tout)) { o.status = PSL_SRC_MISS; return; }
#pragma unroll
    for (int k = 0; k < 3; ++k) { o.s[k] = p[k] + tin * d[k]; o.s[3 + k] = d[k]; }
    o.status = PSL_SRC_TRANSPORT;
}

__device__ __forceinline__ void source_at(const PlanDev &P, const int64_t *gs_sh, int64_t h, int g, int64_t q,
                                          SrcOut &o) {
    const int64_t hl = h - gs_sh[g];
    uint64_t rq, pidx, rr, rw;
    divmod_u64((uint64_t)(hl - P.seg_h[q]), (uint64_t)P.seg_w[q], rq, pidx);
    const int64_t r = P.seg_r0[q] + (int64_t)rq;
    const int64_t entry = P.sorted[P.group_seg[g] + pidx];
    const int64_t nrec = P.e_nrec[entry];
    divmod_u64((uint64_t)(P.e_offset[entry] + r), (uint64_t)nrec, rw, rr);
    const int64_t rec = P.e_start[entry] + (int64_t)rr;
    o.entry = entry; o.use = r; o.rec = rec;
    const int b = P.e_beam[entry];
    o.beam = b;
    record_to_phantom(P.rec[rec], P.beams[b], P.z_psl, P.L, P.origin, true, o);
}

__device__ __forceinline__ void source_one(const PlanDev &P, const int64_t *gs_sh, int64_t h, SrcOut &o) {
    int g;
    int64_t q;
    locate(P, gs_sh, h, g, q);
    source_at(P, gs_sh, h, g, q, o);
}

inline PlanDev make_plan_dev(const psl_plan *p, const psl_phantom_t *ph) {
    PlanDev P;
    P.group_start = p->group_start; P.group_seg = p->group_seg; P.seg_h = p->seg_h; P.seg_r0 = p->seg_r0;
    P.seg_w = p->seg_w; P.sorted = p->sorted; P.e_start = p->e_start; P.e_nrec = p->e_nrec;
    P.e_offset = p->e_offset; P.e_beam = p->e_beam; P.beams = p->beams; P.rec = p->store->rec;
    P.n_groups = p->n_groups; P.z_psl = p->store->z_psl;
    P.L[0] = ph->nx * ph->vx; P.L[1] = ph->ny * ph->vy; P.L[2] = ph->nz * ph->vz;
    for (int k = 0; k < 3; ++k) P.origin[k] = ph->origin[k];
    return P;
}

