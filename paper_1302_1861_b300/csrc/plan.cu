// psl_plan_create (Sec. 2.3.3): PSL selection per field, histories per PSL
// and the tables that map a history number to the PSL record it reads.
//
//   entries   for every beam, every (type, energy division, position) PSL
//             whose position bin overlaps the beam's ROI, in PSL-id order
//   counts    floor(N C_{k+1} / N_total) - floor(N C_k / N_total), exact in
//             integers (C_k = records in the entries before k)
//   order     groups (energy division major, photons before electrons);
//             inside a group, rounds of one read per entry still owed
//             histories, entries in order of decreasing count.  Sorting the
//             group's entries by count makes every round's active set a
//             prefix, so the rounds fall into segments of equal width and a
//             history is located by two binary searches.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "psl_internal.cuh"
#include "sort.cuh"

namespace {

__global__ void k_beams(const psl_beam_t *b, int n, float sad, float z_psl, BeamDev *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double tot = 0.0;
    for (int i = 0; i < n; ++i) tot += (double)b[i].mu;
    for (int i = 0; i < n; ++i) {
        const psl_beam_t &s = b[i];
        BeamDev d;
        // jaw bounds at the jaw planes, float32 in a fixed order
        d.xlo = __fdiv_rn(__fmul_rn(s.x1, s.z_jaw_x), sad);
        d.xhi = __fdiv_rn(__fmul_rn(s.x2, s.z_jaw_x), sad);
        d.ylo = __fdiv_rn(__fmul_rn(s.y1, s.z_jaw_y), sad);
        d.yhi = __fdiv_rn(__fmul_rn(s.y2, s.z_jaw_y), sad);
        d.dzx = __fsub_rn(s.z_jaw_x, z_psl);
        d.dzy = __fsub_rn(s.z_jaw_y, z_psl);
        d.diso = __fsub_rn(sad, z_psl);
        d.mu_ratio = (float)((double)s.mu / tot);
        d.fx0 = s.fx0; d.fy0 = s.fy0; d.fdx = s.fdx; d.fdy = s.fdy;
        d.fnx = s.fluence ? s.fnx : 0; d.fny = s.fluence ? s.fny : 0;
        d.fluence = s.fluence;
        // rotation beam -> patient: couch(z) * gantry(y) * collimator(z)
        double sc, cc, sg, cg, st, ct;
        sincospi((double)s.collimator / 180.0, &sc, &cc);
        sincospi((double)s.gantry / 180.0, &sg, &cg);
        sincospi((double)s.couch / 180.0, &st, &ct);
        double Rc[9] = {cc, -sc, 0, sc, cc, 0, 0, 0, 1};
        double Rg[9] = {cg, 0, sg, 0, 1, 0, -sg, 0, cg};
        double Rt[9] = {ct, -st, 0, st, ct, 0, 0, 0, 1};
        double A[9], R[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                A[3 * r + c] = 0;
                for (int k = 0; k < 3; ++k) A[3 * r + c] += Rg[3 * r + k] * Rc[3 * k + c];
            }
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                R[3 * r + c] = 0;
                for (int k = 0; k < 3; ++k) R[3 * r + c] += Rt[3 * r + k] * A[3 * k + c];
            }
        for (int k = 0; k < 9; ++k) d.r[k] = (float)R[k];
        d.iso[0] = s.iso[0]; d.iso[1] = s.iso[1]; d.iso[2] = s.iso[2];
        d.sad = sad;
        out[i] = d;
    }
}

// flag of (beam, position): the position bin overlaps the beam's ROI
__global__ void k_roi(const psl_beam_t *b, int n_beams, const float *xe, const float *ye, int nx, int ny, float z_psl,
                      float sad, int64_t *flags) {
    int64_t npos = (int64_t)nx * ny;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_beams * npos; t += (int64_t)gridDim.x * blockDim.x) {
        int i = (int)(t / npos);
        int pos = (int)(t % npos), bx = pos % nx, by = pos / nx;
        float s = __fdiv_rn(z_psl, sad), m = b[i].roi_margin;
        float xlo = __fmul_rn(__fsub_rn(b[i].x1, m), s), xhi = __fmul_rn(__fadd_rn(b[i].x2, m), s);
        float ylo = __fmul_rn(__fsub_rn(b[i].y1, m), s), yhi = __fmul_rn(__fadd_rn(b[i].y2, m), s);
        bool sel = xe[bx] < xhi && xe[bx + 1] > xlo && ye[by] < yhi && ye[by + 1] > ylo;
        flags[t] = sel ? 1 : 0;
    }
}

__global__ void k_beam_entries(const int64_t *X, int n_beams, int64_t npos, int n_te, int64_t *cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_beams) cnt[i] = (X[(i + 1) * npos] - X[i * npos]) * n_te;
}

__global__ void k_selpos(const int64_t *flags, const int64_t *X, int64_t total, int64_t npos, int32_t *selpos) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
        if (flags[t]) selpos[X[t]] = (int32_t)(t % npos);
}

__global__ void k_entries(const int64_t *ebase, int n_beams, const int64_t *X, const int32_t *selpos, int64_t npos,
                          int ne, const int64_t *offsets, int64_t n_entries, int32_t *e_beam, int32_t *e_psl,
                          int64_t *e_start, int64_t *e_nrec, int32_t *e_group) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_entries; k += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = n_beams;   // last beam with ebase <= k
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (ebase[mid] <= k) lo = mid; else hi = mid;
        }
        int i = lo;
        int64_t local = k - ebase[i];
        int64_t s0 = X[(int64_t)i * npos], nsel = X[(int64_t)(i + 1) * npos] - s0;
        int64_t te = local / nsel, j = local % nsel;
        int64_t psl = te * npos + selpos[s0 + j];
        e_beam[k] = i;
        e_psl[k] = (int32_t)psl;
        e_start[k] = offsets[psl];
        e_nrec[k] = offsets[psl + 1] - offsets[psl];
        int t = (int)(te / ne), e = (int)(te % ne);
        e_group[k] = e * 2 + t;
    }
}

// floor(a * b / c) for a, b, c < 2^63, c > 0, a*b < 2^126: double estimate
// corrected against the exact 128-bit product
__device__ __forceinline__ uint64_t muldiv_floor(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t ph = __umul64hi(a, b), pl = a * b;
    double est = (double)a * (double)b / (double)c;
    uint64_t q = est < 1.8e19 ? (uint64_t)est : 0;
    // q*c <= a*b < (q+1)*c
    for (int it = 0; it < 64; ++it) {
        uint64_t qh = __umul64hi(q, c), ql = q * c;
        if (qh > ph || (qh == ph && ql > pl)) { --q; continue; }
        uint64_t q1 = q + 1;
        uint64_t rh = __umul64hi(q1, c), rl = q1 * c;
        if (rh < ph || (rh == ph && rl <= pl)) { ++q; continue; }
        break;
    }
    return q;
}

__global__ void k_counts(const int64_t *C, int64_t n_entries, uint64_t n_sim, const int32_t *e_beam, const int32_t *e_psl,
                         const int64_t *e_nrec, uint64_t seed, int64_t *e_count, int64_t *e_offset, int64_t *act) {
    const uint64_t T = (uint64_t)C[n_entries];
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_entries; k += (int64_t)gridDim.x * blockDim.x) {
        uint64_t a = muldiv_floor(n_sim, (uint64_t)C[k], T), b = muldiv_floor(n_sim, (uint64_t)C[k + 1], T);
        int64_t cnt = (int64_t)(b - a);
        e_count[k] = cnt;
        act[k] = cnt > 0 ? 1 : 0;
        uint64_t nrec = (uint64_t)e_nrec[k];
        u32x4 r = philox10((uint32_t)e_beam[k], TAG_OFFSET, (uint32_t)e_psl[k], 0u, (uint32_t)seed, (uint32_t)(seed >> 32));
        uint64_t r64 = (uint64_t)r.a | ((uint64_t)r.b << 32);
        e_offset[k] = nrec ? (int64_t)__umul64hi(r64, nrec) : 0;
    }
}

__global__ void k_max_count(const int64_t *e_count, int64_t n, unsigned long long *mx) {
    unsigned long long m = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)e_count[k]);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(mx, m);
}

__global__ void k_compact(const int64_t *act, const int64_t *A, const int64_t *e_count, int64_t n_entries,
                          uint32_t *keys, uint32_t *vals) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_entries; k += (int64_t)gridDim.x * blockDim.x)
        if (act[k]) {
            keys[A[k]] = ~(uint32_t)e_count[k];     // ascending ~count = descending count
            vals[A[k]] = (uint32_t)k;
        }
}

__global__ void k_group_keys(const uint32_t *vals, int64_t n, const int32_t *e_group, uint32_t *keys, int64_t *ghist) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        int g = e_group[vals[t]];
        keys[t] = (uint32_t)g;
        atomicAdd((unsigned long long *)&ghist[g], 1ull);
    }
}

__global__ void k_segments(const uint32_t *sorted, int64_t n, const int32_t *e_group, const int64_t *e_count,
                           const int64_t *ges, int64_t *lens, int64_t *seg_r0, int32_t *seg_w, int32_t *seg_g) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        uint32_t k = sorted[t];
        int g = e_group[k];
        int64_t s = t - ges[g], m = ges[g + 1] - ges[g];
        int64_t c = e_count[k], cn = (s + 1 < m) ? e_count[sorted[t + 1]] : 0;
        int64_t q = ges[g] + m - 1 - s;
        lens[q] = (s + 1) * (c - cn);
        seg_r0[q] = cn;
        seg_w[q] = (int32_t)(s + 1);
        seg_g[q] = g;
    }
}

__global__ void k_seg_h(const int64_t *X2, const int64_t *ges, const int32_t *seg_g, int64_t n, int64_t *seg_h) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        seg_h[q] = X2[q] - X2[ges[seg_g[q]]];
}

__global__ void k_group_start(const int64_t *X2, const int64_t *ges, int n_groups, int64_t *gs) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g <= n_groups) gs[g] = X2[ges[g]];
}

__global__ void k_plan_read(int64_t n, const int32_t *b, const int32_t *p, const int64_t *c, const int64_t *o,
                            int64_t *ob, int64_t *op, int64_t *oc, int64_t *oo) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        if (ob) ob[k] = b[k];
        if (op) op[k] = p[k];
        if (oc) oc[k] = c[k];
        if (oo) oo[k] = o[k];
    }
}

inline int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)psl_sm_count() * 16)); }

struct Pool {   // frees temporaries at scope exit (stream ordered)
    cudaStream_t st;
    std::vector<void *> ptrs;
    bool ok = true;
    template <class T> T *get(int64_t n) {
        void *p = nullptr;
        if (psl_malloc_async(&p, (size_t)std::max<int64_t>(n, 1) * sizeof(T), st) != cudaSuccess) { ok = false; return nullptr; }
        ptrs.push_back(p);
        return (T *)p;
    }
    void *raw(size_t bytes) {
        void *p = nullptr;
        if (psl_malloc_async(&p, std::max<size_t>(bytes, 16), st) != cudaSuccess) { ok = false; return nullptr; }
        ptrs.push_back(p);
        return p;
    }
    ~Pool() { for (void *p : ptrs) cudaFreeAsync(p, st); }
};

// the source stage's packed copies of the visiting order and its segments
__global__ void k_pack_order(const uint32_t *sorted, int64_t n, const int64_t *e_start, const int64_t *e_nrec,
                             const int64_t *e_offset, const int32_t *e_beam, const int64_t *seg_h,
                             const int64_t *seg_r0, const int32_t *seg_w, EntryDev *ent, SegDev *seg) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = sorted[t];
        EntryDev e;
        e.start = e_start[k]; e.nrec = e_nrec[k]; e.offset = e_offset[k]; e.beam = e_beam[k]; e.entry = k;
        ent[t] = e;
        SegDev g;
        g.h = seg_h[t]; g.r0 = seg_r0[t]; g.w = seg_w[t]; g.pad = 0;
        seg[t] = g;
    }
}

}  // namespace

extern "C" void psl_plan_destroy(psl_plan_t *p) {
    if (!p) return;
    void *ptrs[] = {p->beams, p->e_beam, p->e_psl, p->e_start, p->e_nrec, p->e_count, p->e_offset,
                    p->group_start, p->group_seg, p->sorted, p->seg_h, p->seg_r0, p->seg_w, p->ent, p->seg};
    for (void *q : ptrs)
        if (q) cudaFreeAsync(q, p->stream);
    delete p;
}

int psl_beams_dev(const psl_beam_t *beams, int n, float sad, float z_psl, BeamDev **out, cudaStream_t st) {
    *out = nullptr;
    psl_beam_t *bd = nullptr;
    if (psl_malloc_async((void **)&bd, n * sizeof(psl_beam_t), st) != cudaSuccess ||
        psl_malloc_async((void **)out, n * sizeof(BeamDev), st) != cudaSuccess) {
        if (bd) cudaFreeAsync(bd, st);
        if (*out) { cudaFreeAsync(*out, st); *out = nullptr; }
        return psl_fail(PSL_ENOMEM, "beam table allocation");
    }
    cudaMemcpyAsync(bd, beams, n * sizeof(psl_beam_t), cudaMemcpyHostToDevice, st);
    k_beams<<<1, 32, 0, st>>>(bd, n, sad, z_psl, *out); PSL_NOTE_LAUNCH();
    cudaFreeAsync(bd, st);
    PSL_CUDA(cudaGetLastError());
    return PSL_OK;
}

extern "C" int psl_plan_create(const psl_store_t *store, const psl_beam_t *beams, int32_t n_beams, float sad,
                               int64_t n_histories, uint64_t seed, psl_plan_t **out, void *stream_) {
    if (!store || !beams || !out || n_beams <= 0) return psl_fail(PSL_EINVAL, "psl_plan_create: bad argument");
    *out = nullptr;
    if (n_histories <= 0 || n_histories >= (1ll << 62)) return psl_fail(PSL_EINVAL, "psl_plan_create: n_histories out of range");
    if (!(sad > 0.f)) return psl_fail(PSL_EINVAL, "psl_plan_create: sad must be > 0");
    double mu_tot = 0;
    for (int i = 0; i < n_beams; ++i) {
        const psl_beam_t &b = beams[i];
        if (!(b.mu > 0.f) || !(b.x1 < b.x2) || !(b.y1 < b.y2)) return psl_fail(PSL_EINVAL, "psl_plan_create: bad beam");
        if (b.fluence && (b.fnx <= 0 || b.fny <= 0 || !(b.fdx > 0.f) || !(b.fdy > 0.f)))
            return psl_fail(PSL_EINVAL, "psl_plan_create: bad fluence map");
        mu_tot += b.mu;
    }
    cudaStream_t st = as_stream(stream_);
    psl_plan *p = new psl_plan();
    p->store = store; p->n_beams = n_beams; p->sad = sad; p->n_histories = n_histories; p->seed = seed;
    p->n_incident = store->n_records;
    p->stream = st;
    const int nx = store->nx, ny = store->ny, ne = store->n_ebins;
    const int64_t npos = (int64_t)nx * ny;
    const int n_te = 2 * ne;
    p->n_groups = n_te;
    const float *xe = store->edges, *ye = store->edges + nx + 1;
    int rc = PSL_OK;
    {
        Pool tmp{st};
        psl_beam_t *bd = tmp.get<psl_beam_t>(n_beams);
        int64_t nflag = n_beams * npos;
        int64_t *flags = tmp.get<int64_t>(nflag), *X = tmp.get<int64_t>(nflag + 1);
        int64_t *cnt = tmp.get<int64_t>(n_beams), *ebase = tmp.get<int64_t>(n_beams + 1);
        int32_t *selpos = tmp.get<int32_t>(nflag);
        void *sscr = tmp.raw(scan_i64_scratch_bytes(std::max<int64_t>(nflag, 1 << 20)));
        cudaError_t e = psl_malloc_async((void **)&p->beams, n_beams * sizeof(BeamDev), st);
        if (!tmp.ok || e != cudaSuccess) { psl_plan_destroy(p); return psl_fail(PSL_ENOMEM, "psl_plan_create: allocation"); }
        cudaMemcpyAsync(bd, beams, n_beams * sizeof(psl_beam_t), cudaMemcpyHostToDevice, st);
        k_beams<<<1, 32, 0, st>>>(bd, n_beams, sad, store->z_psl, p->beams); PSL_NOTE_LAUNCH();
        k_roi<<<grid_for(nflag), 256, 0, st>>>(bd, n_beams, xe, ye, nx, ny, store->z_psl, sad, flags); PSL_NOTE_LAUNCH();
        scan_i64(flags, X, nflag, sscr, st);
        k_beam_entries<<<(n_beams + 255) / 256, 256, 0, st>>>(X, n_beams, npos, n_te, cnt); PSL_NOTE_LAUNCH();
        scan_i64(cnt, ebase, n_beams, sscr, st);
        k_selpos<<<grid_for(nflag), 256, 0, st>>>(flags, X, nflag, npos, selpos); PSL_NOTE_LAUNCH();
        int64_t n_entries = 0;
        cudaMemcpyAsync(&n_entries, ebase + n_beams, 8, cudaMemcpyDeviceToHost, st);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { psl_plan_destroy(p); return psl_fail(PSL_ECUDA, cudaGetErrorString(e)); }
        if (n_entries <= 0 || n_entries >= (1ll << 32)) { psl_plan_destroy(p); return psl_fail(PSL_EINVAL, "psl_plan_create: no PSL selected (or too many)"); }
        p->n_entries = n_entries;
        bool ok = true;
        ok &= psl_malloc_async((void **)&p->e_beam, n_entries * 4, st) == cudaSuccess;
        ok &= psl_malloc_async((void **)&p->e_psl, n_entries * 4, st) == cudaSuccess;
        ok &= psl_malloc_async((void **)&p->e_start, n_entries * 8, st) == cudaSuccess;
        ok &= psl_malloc_async((void **)&p->e_nrec, n_entries * 8, st) == cudaSuccess;
        ok &= psl_malloc_async((void **)&p->e_count, n_entries * 8, st) == cudaSuccess;
        ok &= psl_malloc_async((void **)&p->e_offset, n_entries * 8, st) == cudaSuccess;
        int32_t *e_group = tmp.get<int32_t>(n_entries);
        int64_t *C = tmp.get<int64_t>(n_entries + 1), *act = tmp.get<int64_t>(n_entries), *A = tmp.get<int64_t>(n_entries + 1);
        void *sscr2 = tmp.raw(scan_i64_scratch_bytes(n_entries + 1));
        if (!ok || !tmp.ok) { psl_plan_destroy(p); return psl_fail(PSL_ENOMEM, "psl_plan_create: entry arrays"); }
        k_entries<<<grid_for(n_entries), 256, 0, st>>>(ebase, n_beams, X, selpos, npos, ne, store->offsets, n_entries,
                                                       p->e_beam, p->e_psl, p->e_start, p->e_nrec, e_group); PSL_NOTE_LAUNCH();
        scan_i64(p->e_nrec, C, n_entries, sscr2, st);
        cudaMemcpyAsync(&p->n_total_psl, C + n_entries, 8, cudaMemcpyDeviceToHost, st);
        k_counts<<<grid_for(n_entries), 256, 0, st>>>(C, n_entries, (uint64_t)n_histories, p->e_beam, p->e_psl, p->e_nrec,
                                                      seed, p->e_count, p->e_offset, act); PSL_NOTE_LAUNCH();
        scan_i64(act, A, n_entries, sscr2, st);
        int64_t n_active = 0;
        unsigned long long *mx = tmp.get<unsigned long long>(1), max_count = 0;
        if (!tmp.ok) { psl_plan_destroy(p); return psl_fail(PSL_ENOMEM, "psl_plan_create: entry arrays"); }
        cudaMemsetAsync(mx, 0, 8, st);
        k_max_count<<<grid_for(n_entries), 256, 0, st>>>(p->e_count, n_entries, mx); PSL_NOTE_LAUNCH();
        cudaMemcpyAsync(&n_active, A + n_entries, 8, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(&max_count, mx, 8, cudaMemcpyDeviceToHost, st);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { psl_plan_destroy(p); return psl_fail(PSL_ECUDA, cudaGetErrorString(e)); }
        if (p->n_total_psl <= 0) { psl_plan_destroy(p); return psl_fail(PSL_EINVAL, "psl_plan_create: selected PSLs hold no records"); }
        // a PSL's history count keys the entry order sort (32 bits)
        if (max_count >= 0xFFFFFFFFull) { psl_plan_destroy(p); return psl_fail(PSL_EINVAL, "psl_plan_create: a PSL would get 2^32 or more histories"); }
        p->n_active = n_active;
        // order entries: (group, count descending, entry) via two stable sorts
        uint32_t *k0 = tmp.get<uint32_t>(n_active), *v0 = tmp.get<uint32_t>(n_active);
        uint32_t *k1 = tmp.get<uint32_t>(n_active), *v1 = tmp.get<uint32_t>(n_active);
        void *sort_scr = tmp.raw(sort_pairs_scratch_bytes((uint32_t)n_active));
        int64_t *ghist = tmp.get<int64_t>(n_te), *lens = tmp.get<int64_t>(n_active), *X2 = tmp.get<int64_t>(n_active + 1);
        int32_t *seg_g = tmp.get<int32_t>(n_active);
        ok = tmp.ok;
        ok &= psl_malloc_async((void **)&p->sorted, n_active * 4, st) == cudaSuccess;
        ok &= psl_malloc_async((void **)&p->seg_h, n_active * 8, st) == cudaSuccess;
        ok &= psl_malloc_async((void **)&p->seg_r0, n_active * 8, st) == cudaSuccess;
        ok &= psl_malloc_async((void **)&p->seg_w, n_active * 4, st) == cudaSuccess;
        ok &= psl_malloc_async((void **)&p->ent, n_active * sizeof(EntryDev), st) == cudaSuccess;
        ok &= psl_malloc_async((void **)&p->seg, n_active * sizeof(SegDev), st) == cudaSuccess;
        ok &= psl_malloc_async((void **)&p->group_seg, (n_te + 1) * 8, st) == cudaSuccess;
        ok &= psl_malloc_async((void **)&p->group_start, (n_te + 1) * 8, st) == cudaSuccess;
        void *sscr3 = tmp.raw(scan_i64_scratch_bytes(n_active + 1));
        if (!ok || !tmp.ok) { psl_plan_destroy(p); return psl_fail(PSL_ENOMEM, "psl_plan_create: order arrays"); }
        k_compact<<<grid_for(n_entries), 256, 0, st>>>(act, A, p->e_count, n_entries, k0, v0); PSL_NOTE_LAUNCH();
        int alt = 0;
        sort_pairs_u32(k0, v0, k1, v1, (uint32_t)n_active, 32, nullptr, false, sort_scr, &alt, st);
        uint32_t *kk = alt ? k1 : k0, *vv = alt ? v1 : v0, *ka = alt ? k0 : k1, *va = alt ? v0 : v1;
        cudaMemsetAsync(ghist, 0, n_te * 8, st);
        k_group_keys<<<grid_for(n_active), 256, 0, st>>>(vv, n_active, e_group, kk, ghist); PSL_NOTE_LAUNCH();
        int gbits = 1;
        while ((1 << gbits) < n_te) ++gbits;
        int alt2 = 0;
        sort_pairs_u32(kk, vv, ka, va, (uint32_t)n_active, gbits, nullptr, false, sort_scr, &alt2, st);
        uint32_t *sorted_vals = alt2 ? va : vv;
        cudaMemcpyAsync(p->sorted, sorted_vals, n_active * 4, cudaMemcpyDeviceToDevice, st);
        scan_i64(ghist, p->group_seg, n_te, sscr3, st);
        k_segments<<<grid_for(n_active), 256, 0, st>>>(p->sorted, n_active, e_group, p->e_count, p->group_seg, lens,
                                                       p->seg_r0, p->seg_w, seg_g); PSL_NOTE_LAUNCH();
        scan_i64(lens, X2, n_active, sscr3, st);
        k_seg_h<<<grid_for(n_active), 256, 0, st>>>(X2, p->group_seg, seg_g, n_active, p->seg_h); PSL_NOTE_LAUNCH();
        k_group_start<<<(n_te + 256) / 256, 256, 0, st>>>(X2, p->group_seg, n_te, p->group_start); PSL_NOTE_LAUNCH();
        k_pack_order<<<grid_for(n_active), 256, 0, st>>>(p->sorted, n_active, p->e_start, p->e_nrec, p->e_offset,
                                                         p->e_beam, p->seg_h, p->seg_r0, p->seg_w, p->ent, p->seg);
        PSL_NOTE_LAUNCH();
        uint32_t herr = 0;
        cudaMemcpyAsync(&herr, sort_err_word(sort_scr), 4, cudaMemcpyDeviceToHost, st);
        if ((e = cudaGetLastError()) != cudaSuccess) rc = psl_fail(PSL_ECUDA, cudaGetErrorString(e));
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess && rc == PSL_OK) rc = psl_fail(PSL_ECUDA, cudaGetErrorString(e));
        if (rc == PSL_OK && (herr & PSL_DEV_ERR_TIMEOUT)) rc = psl_fail(PSL_ETIMEOUT, "psl_plan_create: sort wait gave up");
    }
    cudaStreamSynchronize(st);
    if (rc != PSL_OK) { psl_plan_destroy(p); return rc; }
    *out = p;
    return PSL_OK;
}

extern "C" int psl_plan_info(const psl_plan_t *p, int64_t *n_entries, int64_t *n_total_psl, int64_t *n_histories) {
    if (!p) return psl_fail(PSL_EINVAL, "psl_plan_info: null plan");
    if (n_entries) *n_entries = p->n_entries;
    if (n_total_psl) *n_total_psl = p->n_total_psl;
    if (n_histories) *n_histories = p->n_histories;
    return PSL_OK;
}

extern "C" int psl_plan_read(const psl_plan_t *p, int64_t *beam, int64_t *psl, int64_t *count, int64_t *offset,
                             void *stream_) {
    if (!p) return psl_fail(PSL_EINVAL, "psl_plan_read: null plan");
    k_plan_read<<<grid_for(p->n_entries), 256, 0, as_stream(stream_)>>>(p->n_entries, p->e_beam, p->e_psl, p->e_count,
                                                                         p->e_offset, beam, psl, count, offset); PSL_NOTE_LAUNCH();
    PSL_CUDA(cudaGetLastError());
    return PSL_OK;
}
