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
#include "source.cuh"

namespace {

__global__ void __launch_bounds__(256) k_source_trace(PlanDev P, int64_t first, int64_t n, int64_t stride, int64_t *entry, int64_t *use,
                                                      int64_t *rec, int32_t *beam, int8_t *status, float *state,
                                                      int32_t *ptype) {
    __shared__ PlanShared S;
    plan_shared_load(P, S);
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        SrcOut o;
        for (int k = 0; k < 8; ++k) o.s[k] = 0.f;
        source_one(P, S, first + i * stride, o);
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

__global__ void k_batch_read(const Particle *p, int64_t cap, int64_t nph, int64_t nel, float *state, int32_t *ptype,
                             uint64_t *pid) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nph + nel; t += (int64_t)gridDim.x * blockDim.x) {
        const Particle q = load_particle(p + (t < nph ? t : cap - 1 - (t - nph)));
        if (state) {
            state[8 * t] = q.x; state[8 * t + 1] = q.y; state[8 * t + 2] = q.z;
            state[8 * t + 3] = q.u; state[8 * t + 4] = q.v; state[8 * t + 5] = q.w;
            state[8 * t + 6] = q.e; state[8 * t + 7] = q.wt;
        }
        if (ptype) ptype[t] = (int32_t)q.type;
        if (pid) pid[t] = ((uint64_t)q.pid_hi << 32) | q.pid_lo;
    }
}

}  // namespace

static int alloc_batch(int64_t n, int64_t first, cudaStream_t st, psl_batch **out) {
    psl_batch *b = new psl_batch();
    b->n_histories = n; b->first_history = first; b->cap = std::max<int64_t>(n, 1);
    b->stream = st;
    cudaError_t e1 = psl_malloc_async((void **)&b->p, b->cap * sizeof(Particle), st);
    cudaError_t e2 = psl_malloc_async((void **)&b->counts, 32, st);
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
    // the source stage runs inside transport_run (fused with the first photon pass)
    psl_batch *b = new psl_batch();
    b->n_histories = n; b->first_history = first; b->stride = stride; b->lazy = 1;
    b->plan = plan; b->phantom = *phantom; b->seed = plan->seed;
    b->stream = as_stream(stream_);
    b->n_photons = -1; b->n_electrons = -1;
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

extern "C" int psl_batch_read(const psl_batch_t *b, float *state, int32_t *ptype, uint64_t *pid, void *stream_) {
    if (!b || b->lazy) return psl_fail(PSL_EINVAL, "psl_batch_read: null or lazy batch");
    const int64_t n = b->n_photons + b->n_electrons;
    if (n <= 0) return PSL_OK;
    int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096));
    k_batch_read<<<grid, 256, 0, as_stream(stream_)>>>(b->p, b->cap, b->n_photons, b->n_electrons, state, ptype, pid); PSL_NOTE_LAUNCH();
    PSL_CUDA(cudaGetLastError());
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
    if (b->s_gbin) cudaFreeAsync(b->s_gbin, b->stream);
    if (b->s_gcount) cudaFreeAsync(b->s_gcount, b->stream);
    if (b->s_hist) cudaFreeAsync(b->s_hist, b->stream);
    delete b;
}
