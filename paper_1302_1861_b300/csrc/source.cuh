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
    const int64_t *group_start, *group_seg;
    const SegDev *seg;               // segments, packed
    const EntryDev *ent;             // entries in visiting order, packed
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

// A block's copy of the group bounds (at most 1024 groups: energy
// divisions x types): first history and first segment of each group.
struct PlanShared {
    int64_t gs[1025], gseg[1025];
};

__device__ __forceinline__ void plan_shared_load(const PlanDev &P, PlanShared &S) {
    for (int i = threadIdx.x; i <= P.n_groups; i += blockDim.x) {
        S.gs[i] = P.group_start[i];
        S.gseg[i] = P.group_seg[i];
    }
}

// group g and segment q of history h (the last segment whose first history
// is <= h's group-local index)
__device__ __forceinline__ void locate(const PlanDev &P, const PlanShared &S, int64_t h, int &g, int64_t &q) {
    int lo = 0, hi = P.n_groups;            // last g with group_start[g] <= h
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (S.gs[mid] <= h) lo = mid; else hi = mid;
    }
    g = lo;
    const int64_t hl = h - S.gs[g];
    int64_t a = S.gseg[g], b = S.gseg[g + 1];  // first segment in [a, b) whose first history is > hl
    while (a < b) {
        const int64_t mid = (a + b) >> 1;
        if (P.seg[mid].h <= hl) a = mid + 1; else b = mid;
    }
    q = a - 1;
}

// locate with a guess (g, q), e.g. a neighbouring history's: kept if it is
// exactly what locate() would return, moved to the next segment if that one
// holds h, otherwise searched
__device__ __forceinline__ void locate_hinted(const PlanDev &P, const PlanShared &S, int64_t h, int &g, int64_t &q) {
    if (g >= 0 && S.gs[g] <= h && h < S.gs[g + 1]) {
        const int64_t hl = h - S.gs[g], end = S.gseg[g + 1];
        if (P.seg[q].h <= hl) {
            if (q + 1 == end || P.seg[q + 1].h > hl) return;
            if (q + 2 == end || P.seg[q + 2].h > hl) { ++q; return; }
        }
    }
    locate(P, S, h, g, q);
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
            const float id = 1.0f / d[k];             // (one division per axis)
            float t0 = (0.0f - p[k]) * id, t1 = (L[k] - p[k]) * id;
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

__device__ __forceinline__ void source_at(const PlanDev &P, const PlanShared &S, int64_t h, int g, int64_t q,
                                          SrcOut &o) {
    const int64_t hl = h - S.gs[g];
    const SegDev sg = P.seg[q];
    uint64_t rq, pidx, rr, rw;
    divmod_u64((uint64_t)(hl - sg.h), (uint64_t)sg.w, rq, pidx);
    const int64_t r = sg.r0 + (int64_t)rq;
    const EntryDev E = P.ent[S.gseg[g] + (int64_t)pidx];
    divmod_u64((uint64_t)(E.offset + r), (uint64_t)E.nrec, rw, rr);
    const int64_t rec = E.start + (int64_t)rr;
    o.entry = E.entry; o.use = r; o.rec = rec;
    o.beam = E.beam;
    record_to_phantom(P.rec[rec], P.beams[E.beam], P.z_psl, P.L, P.origin, true, o);
}

__device__ __forceinline__ void source_one(const PlanDev &P, const PlanShared &S, int64_t h, SrcOut &o) {
    int g;
    int64_t q;
    locate(P, S, h, g, q);
    source_at(P, S, h, g, q, o);
}

inline PlanDev make_plan_dev(const psl_plan *p, const psl_phantom_t *ph) {
    PlanDev P;
    P.group_start = p->group_start; P.group_seg = p->group_seg; P.seg = p->seg; P.ent = p->ent;
    P.beams = p->beams; P.rec = p->store->rec;
    P.n_groups = p->n_groups; P.z_psl = p->store->z_psl;
    P.L[0] = ph->nx * ph->vx; P.L[1] = ph->ny * ph->vy; P.L[2] = ph->nz * ph->vz;
    for (int k = 0; k < 3; ++k) P.origin[k] = ph->origin[k];
    return P;
}

