// Methods 1 and 2 (Sec. 2.1, 2.2): an unsorted phase-space stream binned on
// the fly by particle type and energy, then transported group by group.
//
// The paper fills 2 x N_E bins of a fixed capacity sequentially on the CPU
// and sends a bin to the GPU when it is full.  That sequence is a function of
// the stream: bin b's j-th group holds the particles of bin b ranked
// [j C, (j+1) C) in stream order, and a full group is sent when its last
// particle arrives.  So the B300 form computes it in parallel: the source
// stage per history, a stable radix sort by bin (the PSL build's onesweep
// sort), groups cut from each bin's run, the groups sorted by the stream
// position at which they filled (partial groups last, in bin order), and a
// gather of the particles into that order.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "psl_internal.cuh"
#include "sort.cuh"
#include "source.cuh"

namespace {

constexpr unsigned FULLMASK = 0xFFFFFFFFu;

struct StreamArgs {
    psl_records_t r;
    int64_t first, n_rec;
    uint32_t n;
    int method;
    const float *ee;             // interior energy edges [ne - 1]
    int ne;
    float z_psl;
    float L[3], origin[3];
    const BeamDev *beam;
};

// number of entries of a[0..n) that are <= v (a ascending)
__device__ __forceinline__ int count_le_f(const float *a, int n, float v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (__ldg(a + mid) <= v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Source stage of every history of the stream: acceptance, weight, entry
// into the phantom; the bin of each binned particle (sentinel 2 ne for the
// rest); the emitted and missed energy in fixed point.
__global__ void __launch_bounds__(256) k_stream_source(StreamArgs S, uint32_t *keys, uint32_t *vals, Particle *stage,
                                                       uint8_t *status, unsigned long long *energy) {
    unsigned long long em = 0, mi = 0;
    const uint32_t sentinel = 2u * (uint32_t)S.ne;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < S.n; i += gridDim.x * blockDim.x) {
        const int64_t h = S.first + (int64_t)i;
        uint64_t q_, rr;
        divmod_u64((uint64_t)h, (uint64_t)S.n_rec, q_, rr);
        PslRecord R;
        R.x = __ldg(S.r.x + rr); R.y = __ldg(S.r.y + rr); R.u = __ldg(S.r.u + rr); R.v = __ldg(S.r.v + rr);
        R.e = __ldg(S.r.e + rr); R.wt = __ldg(S.r.wt + rr); R.src = (uint32_t)rr; R.q = (int32_t)__ldg(S.r.q + rr);
        SrcOut o;
        for (int k = 0; k < 8; ++k) o.s[k] = 0.f;
        record_to_phantom(R, *S.beam, S.z_psl, S.L, S.origin, S.method == PSL_METHOD_JAW_MODEL, o);
        uint32_t key = sentinel;
        if ((o.status == PSL_SRC_TRANSPORT || o.status == PSL_SRC_MISS) && R.e > 0.0f) {
            const int eb = count_le_f(S.ee, S.ne - 1, R.e);
            key = (uint32_t)((R.q != 0) * S.ne + eb);
            const unsigned long long f = (unsigned long long)__float2ll_rn(__fmul_rn(o.s[6], o.s[7]) * 4294967296.0f);
            em += f;
            if (o.status == PSL_SRC_MISS) mi += f;
        }
        keys[i] = key;
        vals[i] = i;
        status[i] = (uint8_t)o.status;
        Particle p;
        p.x = o.s[0]; p.y = o.s[1]; p.z = o.s[2]; p.e = o.s[6];
        p.u = o.s[3]; p.v = o.s[4]; p.w = o.s[5]; p.wt = o.s[7];
        p.pid_lo = (uint32_t)h; p.pid_hi = (uint32_t)((uint64_t)h >> 32);
        p.type = (uint32_t)o.ptype; p.root = i;
        store_particle(stage + i, p);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        em += __shfl_xor_sync(FULLMASK, em, o);
        mi += __shfl_xor_sync(FULLMASK, mi, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (em) atomicAdd(energy, em);
        if (mi) atomicAdd(energy + 1, mi);
    }
}

// offs[b] = first sorted position with bin >= b, b = 0..nbins
__global__ void k_bin_offsets(const uint32_t *skeys, uint32_t n, uint32_t nbins, int64_t *offs) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t prev = i == 0 ? -1 : (int64_t)skeys[i - 1];
        int64_t cur = i == n ? nbins : (int64_t)skeys[i];
        if (cur > nbins) cur = nbins;
        for (int64_t k = prev + 1; k <= cur; ++k) offs[k] = i;
    }
}

__device__ __forceinline__ int bin_of_group(const int64_t *gbase, int nbins, int64_t g) {
    int lo = 0, hi = nbins;                 // last b with gbase[b] <= g
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (gbase[mid] <= g) lo = mid; else hi = mid;
    }
    return lo;
}

// Each group's emission time: the stream position of its last particle for
// a full group, n + bin for the partial group of a bin (sent at the end).
__global__ void k_groups(const int64_t *offs, const int64_t *gbase, int nbins, uint32_t G, uint32_t cap,
                         const uint32_t *svals, uint32_t n, uint32_t *gkey, uint32_t *gval) {
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
        const int b = bin_of_group(gbase, nbins, g);
        const int64_t j = g - gbase[b];
        const int64_t start = offs[b] + j * cap, cnt = offs[b + 1] - start;
        gkey[g] = cnt >= cap ? svals[start + cap - 1] : n + (uint32_t)b;
        gval[g] = g;
    }
}

// Bin, size and sorted start of the groups in emission order.
__global__ void k_group_table(const uint32_t *order, const int64_t *offs, const int64_t *gbase, int nbins,
                              uint32_t G, uint32_t cap, int64_t *gbin, int64_t *gcount, int64_t *gstart) {
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < G; k += gridDim.x * blockDim.x) {
        const uint32_t g = order[k];
        const int b = bin_of_group(gbase, nbins, g);
        const int64_t j = g - gbase[b];
        const int64_t start = offs[b] + j * cap;
        gbin[k] = b;
        const int64_t left = offs[b + 1] - start;
        gcount[k] = left < (int64_t)cap ? left : (int64_t)cap;
        gstart[k] = start;
    }
}

__device__ __forceinline__ int64_t group_of(const int64_t *gofs, int64_t G, int64_t t) {
    int64_t lo = 0, hi = G;                 // last k with gofs[k] <= t
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (gofs[mid] <= t) lo = mid; else hi = mid;
    }
    return lo;
}

// Particle t of the group order: its history, and its slot flags (kept
// photon in the low half, kept charged particle in the high half).
__global__ void k_stream_order(const int64_t *gofs, const int64_t *gstart, int64_t G, int64_t nb,
                               const uint32_t *svals, const uint8_t *status, const Particle *stage, int64_t first,
                               int64_t *hist, int64_t *flags, uint32_t *src) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nb; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = group_of(gofs, G, t);
        const uint32_t i = svals[gstart[k] + (t - gofs[k])];
        hist[t] = first + i;
        src[t] = i;
        int64_t f = 0;
        if (status[i] == PSL_SRC_TRANSPORT) f = stage[i].type == 0 ? 1 : (1ll << 32);
        flags[t] = f;
    }
}

__global__ void k_stream_emit(const int64_t *flags, const int64_t *pos, const uint32_t *src, int64_t nb,
                              const Particle *stage, Particle *out, int64_t cap) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nb; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = flags[t];
        if (!f) continue;
        const Particle p = load_particle(stage + src[t]);
        if (f == 1) store_particle(out + (pos[t] & 0xFFFFFFFFll), p);
        else store_particle(out + (cap - 1 - (pos[t] >> 32)), p);
    }
}

__global__ void k_stream_counts(const int64_t *pos, int64_t nb, uint32_t *counts) {
    const int64_t tot = pos[nb];
    counts[0] = (uint32_t)(tot & 0xFFFFFFFFll);
    counts[1] = (uint32_t)(tot >> 32);
}

int grid_of(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)psl_sm_count() * 8)); }

int bit_length(uint64_t v) {
    int b = 1;
    while (b < 64 && (1ull << b) <= v) ++b;
    return b;
}

}  // namespace

extern "C" int psl_stream_bin(const psl_records_t *rec, const float *e_edges, int32_t n_ebins, const psl_beam_t *beam,
                              int32_t method, float z_psl, float sad, const psl_phantom_t *ph, int64_t first,
                              int64_t n, uint64_t seed, int64_t capacity, psl_batch_t **out, void *stream_) {
    if (!out) return psl_fail(PSL_EINVAL, "psl_stream_bin: null output");
    *out = nullptr;
    if (!rec || !beam || !ph || !e_edges) return psl_fail(PSL_EINVAL, "psl_stream_bin: null argument");
    if (method != PSL_METHOD_PATIENT_DEPENDENT && method != PSL_METHOD_JAW_MODEL)
        return psl_fail(PSL_EINVAL, "psl_stream_bin: method must be 1 or 2");
    if (n_ebins < 1 || n_ebins > 4096) return psl_fail(PSL_EINVAL, "psl_stream_bin: n_ebins out of range");
    for (int i = 0; i < n_ebins; ++i)
        if (!(e_edges[i] < e_edges[i + 1])) return psl_fail(PSL_EINVAL, "psl_stream_bin: energy edges not ascending");
    if (n < 0 || n >= (1ll << 31) || first < 0 || capacity < 1)
        return psl_fail(PSL_EINVAL, "psl_stream_bin: bad history range or capacity");
    if (n > 0 && (rec->n <= 0 || !rec->x || !rec->y || !rec->u || !rec->v || !rec->e || !rec->wt || !rec->q))
        return psl_fail(PSL_EINVAL, "psl_stream_bin: empty or null phase space");
    if (ph->nx <= 0 || ph->ny <= 0 || ph->nz <= 0 || !(ph->vx > 0) || !(ph->vy > 0) || !(ph->vz > 0))
        return psl_fail(PSL_EINVAL, "psl_stream_bin: bad phantom");
    if (!(beam->mu > 0)) return psl_fail(PSL_EINVAL, "psl_stream_bin: beam MU must be > 0");
    cudaStream_t st = as_stream(stream_);
    const uint32_t nn = (uint32_t)n, nbins = 2u * (uint32_t)n_ebins;
    const uint32_t cap = (uint32_t)std::min<int64_t>(capacity, 0x7FFFFFFF);

    psl_batch *B = new psl_batch();
    B->n_histories = n; B->first_history = first; B->seed = seed; B->stream = st;
    B->cap = std::max<int64_t>(n, 1);
    int rc = PSL_OK;
    auto fail = [&](int code, const std::string &m) { rc = psl_fail(code, m); };
    // scratch
    BeamDev *bdev = nullptr;
    float *ee = nullptr;
    uint32_t *keys[2] = {nullptr, nullptr}, *vals[2] = {nullptr, nullptr}, *src = nullptr;
    Particle *stage = nullptr;
    uint8_t *status = nullptr;
    int64_t *offs = nullptr, *gbase_d = nullptr, *gstart = nullptr, *gsize = nullptr, *gofs = nullptr;
    int64_t *flags = nullptr, *pos = nullptr;
    uint32_t *gk[2] = {nullptr, nullptr}, *gv[2] = {nullptr, nullptr};
    void *scratch = nullptr, *sscr = nullptr;
    do {
        const size_t m = std::max<int64_t>(n, 1);
        bool ok = psl_malloc_async((void **)&B->p, B->cap * sizeof(Particle), st) == cudaSuccess;
        ok &= psl_malloc_async((void **)&B->counts, 32, st) == cudaSuccess;
        ok &= psl_malloc_async((void **)&ee, (n_ebins + 1) * sizeof(float), st) == cudaSuccess;
        for (int k = 0; k < 2; ++k) {
            ok &= psl_malloc_async((void **)&keys[k], m * 4, st) == cudaSuccess;
            ok &= psl_malloc_async((void **)&vals[k], m * 4, st) == cudaSuccess;
        }
        ok &= psl_malloc_async((void **)&stage, m * sizeof(Particle), st) == cudaSuccess;
        ok &= psl_malloc_async((void **)&status, m, st) == cudaSuccess;
        ok &= psl_malloc_async((void **)&offs, (nbins + 1) * 8, st) == cudaSuccess;
        ok &= psl_malloc_async((void **)&gbase_d, (nbins + 1) * 8, st) == cudaSuccess;
        ok &= psl_malloc_async(&scratch, sort_pairs_scratch_bytes((uint32_t)m), st) == cudaSuccess;
        if (!ok) { fail(PSL_ENOMEM, "psl_stream_bin: allocation"); break; }
        cudaMemsetAsync(B->counts, 0, 32, st);
        if ((rc = psl_beams_dev(beam, 1, sad, z_psl, &bdev, st))) break;
        cudaMemcpyAsync(ee, e_edges + 1, std::max(n_ebins - 1, 0) * sizeof(float), cudaMemcpyHostToDevice, st);
        if (n == 0) {
            B->n_photons = B->n_electrons = 0;
            break;
        }
        StreamArgs S;
        S.r = *rec; S.first = first; S.n_rec = rec->n; S.n = nn; S.method = method; S.ee = ee; S.ne = n_ebins;
        S.z_psl = z_psl;
        S.L[0] = ph->nx * ph->vx; S.L[1] = ph->ny * ph->vy; S.L[2] = ph->nz * ph->vz;
        for (int k = 0; k < 3; ++k) S.origin[k] = ph->origin[k];
        S.beam = bdev;
        unsigned long long *energy = reinterpret_cast<unsigned long long *>(B->counts + 2);
        k_stream_source<<<grid_of(n), 256, 0, st>>>(S, keys[0], vals[0], stage, status, energy); PSL_NOTE_LAUNCH();
        int alt = 0;
        if (sort_pairs_u32(keys[0], vals[0], keys[1], vals[1], nn, bit_length(nbins), nullptr, true, scratch, &alt, st)) {
            fail(PSL_EINVAL, "psl_stream_bin: sort");
            break;
        }
        const uint32_t *skeys = alt ? keys[1] : keys[0], *svals = alt ? vals[1] : vals[0];
        k_bin_offsets<<<grid_of(n + 1), 256, 0, st>>>(skeys, nn, nbins, offs); PSL_NOTE_LAUNCH();
        std::vector<int64_t> ho(nbins + 1);
        uint32_t herr = 0;
        cudaMemcpyAsync(ho.data(), offs, (nbins + 1) * 8, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(&herr, sort_err_word(scratch), 4, cudaMemcpyDeviceToHost, st);
        unsigned long long hen[2] = {0, 0};
        cudaMemcpyAsync(hen, energy, 16, cudaMemcpyDeviceToHost, st);
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { fail(PSL_ECUDA, cudaGetErrorString(e)); break; }
        B->s_emitted = hen[0]; B->s_missed = hen[1];
        if (herr & PSL_DEV_ERR_TIMEOUT) { fail(PSL_ETIMEOUT, "psl_stream_bin: look-back wait gave up"); break; }
        // groups per bin: ceil(count / capacity)
        std::vector<int64_t> gb(nbins + 1, 0);
        for (uint32_t b = 0; b < nbins; ++b) {
            const int64_t c = ho[b + 1] - ho[b];
            gb[b + 1] = gb[b] + (c + cap - 1) / cap;
        }
        const int64_t G = gb[nbins], nb = ho[nbins];
        B->s_groups = G; B->s_binned = nb;
        ok = psl_malloc_async((void **)&B->s_gbin, std::max<int64_t>(G, 1) * 8, st) == cudaSuccess;
        ok &= psl_malloc_async((void **)&B->s_gcount, std::max<int64_t>(G, 1) * 8, st) == cudaSuccess;
        ok &= psl_malloc_async((void **)&B->s_hist, std::max<int64_t>(nb, 1) * 8, st) == cudaSuccess;
        if (!ok) { fail(PSL_ENOMEM, "psl_stream_bin: group allocation"); break; }
        if (G == 0) { B->n_photons = B->n_electrons = 0; break; }
        const size_t gm = (size_t)G;
        for (int k = 0; k < 2; ++k) {
            ok &= psl_malloc_async((void **)&gk[k], gm * 4, st) == cudaSuccess;
            ok &= psl_malloc_async((void **)&gv[k], gm * 4, st) == cudaSuccess;
        }
        ok &= psl_malloc_async((void **)&gstart, gm * 8, st) == cudaSuccess;
        ok &= psl_malloc_async((void **)&gsize, gm * 8, st) == cudaSuccess;
        ok &= psl_malloc_async((void **)&gofs, (gm + 1) * 8, st) == cudaSuccess;
        ok &= psl_malloc_async((void **)&flags, nb * 8, st) == cudaSuccess;
        ok &= psl_malloc_async((void **)&pos, (nb + 1) * 8, st) == cudaSuccess;
        ok &= psl_malloc_async((void **)&src, nb * 4, st) == cudaSuccess;
        ok &= psl_malloc_async(&sscr, scan_i64_scratch_bytes(std::max<int64_t>(nb, G)), st) == cudaSuccess;
        if (!ok) { fail(PSL_ENOMEM, "psl_stream_bin: group allocation"); break; }
        cudaMemcpyAsync(gbase_d, gb.data(), (nbins + 1) * 8, cudaMemcpyHostToDevice, st);
        // the groups in emission order (stable sort of their emission times)
        k_groups<<<grid_of(G), 256, 0, st>>>(offs, gbase_d, (int)nbins, (uint32_t)G, cap, svals, nn, gk[0], gv[0]); PSL_NOTE_LAUNCH();
        int galt = 0;
        if (sort_pairs_u32(gk[0], gv[0], gk[1], gv[1], (uint32_t)G, bit_length((uint64_t)nn + nbins), nullptr, true,
                           scratch, &galt, st)) { fail(PSL_EINVAL, "psl_stream_bin: group sort"); break; }
        const uint32_t *order = galt ? gv[1] : gv[0];
        k_group_table<<<grid_of(G), 256, 0, st>>>(order, offs, gbase_d, (int)nbins, (uint32_t)G, cap, B->s_gbin, gsize,
                                                   gstart); PSL_NOTE_LAUNCH();
        cudaMemcpyAsync(B->s_gcount, gsize, gm * 8, cudaMemcpyDeviceToDevice, st);
        scan_i64(gsize, gofs, G, sscr, st);
        // particles in group order; kept ones go photons-front / charged-back
        k_stream_order<<<grid_of(nb), 256, 0, st>>>(gofs, gstart, G, nb, svals, status, stage, first, B->s_hist, flags,
                                                     src); PSL_NOTE_LAUNCH();
        scan_i64(flags, pos, nb, sscr, st);
        k_stream_emit<<<grid_of(nb), 256, 0, st>>>(flags, pos, src, nb, stage, B->p, B->cap); PSL_NOTE_LAUNCH();
        k_stream_counts<<<1, 1, 0, st>>>(pos, nb, B->counts); PSL_NOTE_LAUNCH();
        uint32_t c[2] = {0, 0}, herr2 = 0;
        cudaMemcpyAsync(c, B->counts, 8, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(&herr2, sort_err_word(scratch), 4, cudaMemcpyDeviceToHost, st);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { fail(PSL_ECUDA, cudaGetErrorString(e)); break; }
        if (herr2 & PSL_DEV_ERR_TIMEOUT) { fail(PSL_ETIMEOUT, "psl_stream_bin: look-back wait gave up"); break; }
        B->n_photons = c[0]; B->n_electrons = c[1];
        if ((e = cudaGetLastError()) != cudaSuccess) { fail(PSL_ECUDA, cudaGetErrorString(e)); break; }
    } while (0);
    if (bdev) cudaFreeAsync(bdev, st);
    if (ee) cudaFreeAsync(ee, st);
    for (int k = 0; k < 2; ++k) {
        if (keys[k]) cudaFreeAsync(keys[k], st);
        if (vals[k]) cudaFreeAsync(vals[k], st);
        if (gk[k]) cudaFreeAsync(gk[k], st);
        if (gv[k]) cudaFreeAsync(gv[k], st);
    }
    for (void *q : {(void *)stage, (void *)status, (void *)offs, (void *)gbase_d, (void *)gstart, (void *)gsize,
                    (void *)gofs, (void *)flags, (void *)pos, (void *)src, scratch, sscr})
        if (q) cudaFreeAsync(q, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (rc == PSL_OK && e2 != cudaSuccess) rc = psl_fail(PSL_ECUDA, cudaGetErrorString(e2));
    if (rc != PSL_OK) { psl_batch_destroy(B); return rc; }
    *out = B;
    return PSL_OK;
}

extern "C" int psl_stream_info(const psl_batch_t *b, int64_t *n_groups, int64_t *n_kept, int64_t *emitted_fp,
                               int64_t *missed_fp) {
    if (!b) return psl_fail(PSL_EINVAL, "psl_stream_info: null batch");
    if (n_groups) *n_groups = b->s_groups;
    if (n_kept) *n_kept = b->n_photons + b->n_electrons;
    if (emitted_fp) *emitted_fp = (int64_t)b->s_emitted;
    if (missed_fp) *missed_fp = (int64_t)b->s_missed;
    return PSL_OK;
}

extern "C" int psl_stream_read(const psl_batch_t *b, int64_t *group_bin, int64_t *group_count, int64_t *history,
                               void *stream_) {
    if (!b) return psl_fail(PSL_EINVAL, "psl_stream_read: null batch");
    cudaStream_t st = as_stream(stream_);
    if (group_bin && b->s_groups) PSL_CUDA(cudaMemcpyAsync(group_bin, b->s_gbin, b->s_groups * 8, cudaMemcpyDeviceToDevice, st));
    if (group_count && b->s_groups) PSL_CUDA(cudaMemcpyAsync(group_count, b->s_gcount, b->s_groups * 8, cudaMemcpyDeviceToDevice, st));
    if (history && b->s_binned) PSL_CUDA(cudaMemcpyAsync(history, b->s_hist, b->s_binned * 8, cudaMemcpyDeviceToDevice, st));
    return PSL_OK;
}
