// Tallies and dose readout (Sec. 2.3.3 batches and uncertainty, Sec. 2.5
// normalisation).  The int64 fixed-point counters are the only place where
// FP64 is used on the device: the final conversion to dose and its batch
// standard error, and the energy-ledger sums.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "psl_internal.cuh"

void workspace_release(Workspace *w);
int64_t workspace_bytes_of(const Workspace *w);

namespace {

__global__ void __launch_bounds__(256) k_readout(const unsigned long long *t, int64_t nvox, int nb, const float *rho,
                                                 double scale, double *dose, double *sigma, unsigned long long *dep) {
    unsigned long long local = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += (int64_t)gridDim.x * blockDim.x) {
        long long sum = 0;
        for (int b = 0; b < nb; ++b) sum += (long long)t[(size_t)b * nvox + v];
        local += (unsigned long long)sum;
        const double r = (double)rho[v];
        const double c = r > 0.0 ? scale / r : 0.0;     // Gy per fixed-point unit
        const double tot = (double)sum;
        if (dose) dose[v] = tot * c;
        if (sigma) {
            double s = 0.0;
            if (nb > 1) {
                const double mean = tot / nb;
                double var = 0.0;
                for (int b = 0; b < nb; ++b) {
                    const double d = (double)(long long)t[(size_t)b * nvox + v] - mean;
                    var += d * d;
                }
                s = c * sqrt((double)nb / (nb - 1.0) * var);
            }
            sigma[v] = s;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xFFFFFFFFu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(dep, local);
}

// ledger slot 2 (deposited) is the sum of the tally: set from the sum the
// readout took (the transport kernels do not count it separately)
__global__ void k_ledger_out(unsigned long long *ledger, const unsigned long long *dep, double *out) {
    ledger[2] = dep[0];
    if (!out) return;
    const double s = 1.0 / 4294967296.0;
    out[0] = (double)(long long)ledger[0] * s;
    out[1] = (double)(long long)ledger[1] * s;
    out[2] = (double)(long long)dep[0] * s;
}

// sum of every counter of the tally (two's complement, as the ledger keeps it)
__global__ void __launch_bounds__(256) k_tally_sum(const unsigned long long *t, int64_t n, unsigned long long *out) {
    unsigned long long local = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        local += t[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xFFFFFFFFu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(out, local);
}

}  // namespace

extern "C" int psl_tally_create(const psl_phantom_t *ph, int32_t n_batches, psl_tally_t **out) {
    if (!ph || !out || n_batches <= 0 || n_batches > PSL_MAX_BATCHES || ph->nx <= 0 || ph->ny <= 0 || ph->nz <= 0)
        return psl_fail(PSL_EINVAL, "psl_tally_create: bad argument");
    if ((int64_t)ph->nx * ph->ny * ph->nz >= (int64_t)1 << 31)
        return psl_fail(PSL_EINVAL, "psl_tally_create: the phantom must have fewer than 2^31 voxels");
    *out = nullptr;
    psl_tally *t = new psl_tally();
    t->nx = ph->nx; t->ny = ph->ny; t->nz = ph->nz; t->n_batches = n_batches;
    t->nvox = (int64_t)ph->nx * ph->ny * ph->nz;
    cudaError_t e1 = cudaMalloc((void **)&t->t, (size_t)n_batches * t->nvox * 8);
    cudaError_t e2 = cudaMalloc((void **)&t->ledger, 16 * 8);
    if (e1 != cudaSuccess || e2 != cudaSuccess) { psl_tally_destroy(t); return psl_fail(PSL_ENOMEM, "psl_tally_create: allocation"); }
    cudaMemset(t->t, 0, (size_t)n_batches * t->nvox * 8);
    cudaMemset(t->ledger, 0, 16 * 8);
    PSL_CUDA(cudaDeviceSynchronize());
    *out = t;
    return PSL_OK;
}

extern "C" int psl_tally_set_order(psl_tally_t *t, int32_t order) {
    if (!t || order < PSL_ORDER_AUTO || order > PSL_ORDER_BATCH) return psl_fail(PSL_EINVAL, "psl_tally_set_order: bad argument");
    t->order = order;
    return PSL_OK;
}

extern "C" int psl_tally_reset(psl_tally_t *t, void *stream_) {
    if (!t) return psl_fail(PSL_EINVAL, "psl_tally_reset: null tally");
    cudaStream_t st = as_stream(stream_);
    PSL_CUDA(cudaMemsetAsync(t->t, 0, (size_t)t->n_batches * t->nvox * 8, st));
    PSL_CUDA(cudaMemsetAsync(t->ledger, 0, 16 * 8, st));
    return PSL_OK;
}

extern "C" int psl_tally_read(const psl_tally_t *t, int64_t *tallies, int64_t *ledger, void *stream_) {
    if (!t) return psl_fail(PSL_EINVAL, "psl_tally_read: null tally");
    cudaStream_t st = as_stream(stream_);
    if (tallies) PSL_CUDA(cudaMemcpyAsync(tallies, t->t, (size_t)t->n_batches * t->nvox * 8, cudaMemcpyDeviceToDevice, st));
    if (ledger) {
        // slot 2 (deposited) is the sum of the tally
        PSL_CUDA(cudaMemsetAsync(t->ledger + 2, 0, 8, st));
        const int64_t n = (int64_t)t->n_batches * t->nvox;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)psl_sm_count() * 8));
        k_tally_sum<<<grid, 256, 0, st>>>(t->t, n, t->ledger + 2); PSL_NOTE_LAUNCH();
        PSL_CUDA(cudaMemcpyAsync(ledger, t->ledger, 12 * 8, cudaMemcpyDeviceToDevice, st));
    }
    return PSL_OK;
}

extern "C" int psl_tally_buffers(psl_tally_t *t, int64_t **tallies, int64_t **ledger) {
    if (!t) return psl_fail(PSL_EINVAL, "psl_tally_buffers: null tally");
    if (tallies) *tallies = reinterpret_cast<int64_t *>(t->t);
    if (ledger) *ledger = reinterpret_cast<int64_t *>(t->ledger);
    return PSL_OK;
}

extern "C" int psl_tally_trace_source(psl_tally_t *t, int64_t first, int64_t n, int64_t *entry, int64_t *use,
                                      int64_t *rec, int8_t *status, float *state, int32_t *ptype) {
    if (!t || first < 0 || n < 0) return psl_fail(PSL_EINVAL, "psl_tally_trace_source: bad argument");
    SrcTraceDev T;
    if (n > 0) {
        T.first = first; T.n = n;
        T.entry = entry; T.use = use; T.rec = rec; T.status = status; T.state = state; T.ptype = ptype;
    }
    t->trace = T;
    return PSL_OK;
}

extern "C" int psl_tally_set_queue_depth(psl_tally_t *t, int64_t depth) {
    if (!t || depth < ((int64_t)1 << 12) || depth > ((int64_t)1 << 26))
        return psl_fail(PSL_EINVAL, "psl_tally_set_queue_depth: depth outside [2^12, 2^26]");
    t->chunk_cap = depth;
    return PSL_OK;
}

extern "C" int psl_tally_info(const psl_tally_t *t, int64_t *n_counters, int64_t *workspace_bytes,
                              int64_t *queue_depth, int32_t *blocks_per_sm) {
    if (!t) return psl_fail(PSL_EINVAL, "psl_tally_info: null tally");
    if (n_counters) *n_counters = (int64_t)t->n_batches * t->nvox;
    if (workspace_bytes) *workspace_bytes = workspace_bytes_of(t->ws);
    if (queue_depth) *queue_depth = t->chunk_cap;
    if (blocks_per_sm) *blocks_per_sm = t->grid_mult;
    return PSL_OK;
}

// Sec. 2.5: D = D_o N_total^phsp / (N_simulated N_incident).  With PSL
// selection the simulated histories stand for the N_total^psl records of the
// selected PSLs, so N_total^psl takes the place of the phase space's total.
extern "C" int psl_dose_normalisation(const psl_plan_t *plan, int64_t n_histories, int64_t n_incident,
                                      double calibration, double *norm) {
    if (!plan || !norm || n_histories <= 0 || n_incident < 0 || !(calibration > 0.0))
        return psl_fail(PSL_EINVAL, "psl_dose_normalisation: bad argument");
    const int64_t inc = n_incident > 0 ? n_incident : plan->n_incident;
    if (inc <= 0) return psl_fail(PSL_EINVAL, "psl_dose_normalisation: no incident particle count");
    *norm = calibration * (double)plan->n_total_psl / ((double)n_histories * (double)inc);
    return PSL_OK;
}

extern "C" int dose_readout(const psl_tally_t *t, const psl_phantom_t *ph, double norm, double *dose, double *sigma,
                            double *ledger, void *stream_) {
    if (!t || !ph || !ph->rho) return psl_fail(PSL_EINVAL, "dose_readout: null argument");
    if (ph->nx != t->nx || ph->ny != t->ny || ph->nz != t->nz) return psl_fail(PSL_EINVAL, "dose_readout: phantom mismatch");
    cudaStream_t st = as_stream(stream_);
    // Gy per fixed-point unit at unit density: 2^-32 MeV * J/MeV / (V cm^3 * 1e-3 kg/g)
    const double vol = (double)ph->vx * (double)ph->vy * (double)ph->vz;
    const double scale = norm * (1.0 / 4294967296.0) * 1.602176634e-13 / (vol * 1e-3);
    unsigned long long *dep = t->ledger + 12;         // scratch slot for the deposited sum
    PSL_CUDA(cudaMemsetAsync(dep, 0, 8, st));
    int grid = (int)std::max<int64_t>(1, std::min<int64_t>((t->nvox + 255) / 256, (int64_t)psl_sm_count() * 8));
    // (no timer events inside a stream capture: psl_plan_replay records this call into its graph)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cap);
    const bool timed = psl_timer_on() && cap == cudaStreamCaptureStatusNone;
    { void *tk_ = nullptr; if (timed) psl_timer_begin(PK_READOUT, st, &tk_); k_readout<<<grid, 256, 0, st>>>(t->t, t->nvox, t->n_batches, ph->rho, scale, dose, sigma, dep); PSL_NOTE_LAUNCH(); if (tk_) psl_timer_end(PK_READOUT, st, tk_); }
    k_ledger_out<<<1, 1, 0, st>>>(t->ledger, dep, ledger); PSL_NOTE_LAUNCH();
    PSL_CUDA(cudaGetLastError());
    return PSL_OK;
}

extern "C" void psl_tally_destroy(psl_tally_t *t) {
    if (!t) return;
    if (t->t) cudaFree(t->t);
    if (t->ledger) cudaFree(t->ledger);
    if (t->ws) workspace_release(t->ws);            // kept for the next tally
    delete t;
}

// --------------------------------------------------------------------------
// Diagnostic: throughput of int64 atomic adds into an L2-resident array, the
// operation every dose deposit performs.  Each thread adds 1 to pseudo-random
// cells (a multiplicative hash of its update index), return values unused.
namespace {
__global__ void __launch_bounds__(256) k_atomic_peak(unsigned long long *cells, uint64_t n_cells, uint64_t n_updates) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_updates; i += stride) {
        uint64_t h = (i + 1) * 0x9E3779B97F4A7C15ull;
        atomicAdd(cells + (h >> 32) % n_cells, 1ull);
    }
}
}  // namespace

extern "C" int psl_atomic_peak(int64_t n_cells, int64_t n_updates, double *updates_per_s, void *stream_) {
    if (n_cells <= 0 || n_updates <= 0 || !updates_per_s) return psl_fail(PSL_EINVAL, "psl_atomic_peak: bad argument");
    cudaStream_t st = as_stream(stream_);
    unsigned long long *cells = nullptr;
    PSL_CUDA(psl_malloc_async((void **)&cells, n_cells * 8, st));
    PSL_CUDA(cudaMemsetAsync(cells, 0, n_cells * 8, st));
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int grid = psl_sm_count() * 8;
    k_atomic_peak<<<grid, 256, 0, st>>>(cells, n_cells, n_updates / 8 + 1); PSL_NOTE_LAUNCH();   // warm-up
    cudaEventRecord(a, st);
    k_atomic_peak<<<grid, 256, 0, st>>>(cells, n_cells, n_updates); PSL_NOTE_LAUNCH();
    cudaEventRecord(b, st);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFreeAsync(cells, st);
    if (e != cudaSuccess) return psl_fail(PSL_ECUDA, cudaGetErrorString(e));
    *updates_per_s = (double)n_updates / (ms * 1e-3);
    return PSL_OK;
}

// ------------------------------------------------------------------ gamma --
// Global gamma index (Sec. 3 comparisons; 2 % / 2 mm in the paper's tables):
// at every reference voxel with D_ref >= threshold * max(ref), the minimum
// over evaluated points r within the search radius of sqrt(|r - r_ref|^2 /
// dta^2 + (D_ev(r) - D_ref)^2 / (dose_crit max ref)^2), with D_ev trilinear
// between voxel centres on a grid of voxel / upsample; points outside the
// volume are skipped.  FP64 throughout.
namespace {
__global__ void k_max(const double *a, int64_t n, unsigned long long *mx) {
    double m = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, a[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
    // non-negative doubles order as their bit patterns
    if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(mx, (unsigned long long)__double_as_longlong(m));
}

__device__ __forceinline__ bool trilinear(const double *a, int nx, int ny, int nz, double fz, double fy, double fx,
                                          double &out) {
    if (!(fz >= 0.0 && fz <= nz - 1 && fy >= 0.0 && fy <= ny - 1 && fx >= 0.0 && fx <= nx - 1)) return false;
    int z0 = (int)floor(fz), y0 = (int)floor(fy), x0 = (int)floor(fx);
    z0 = min(z0, nz - 2 < 0 ? 0 : nz - 2); y0 = min(y0, ny - 2 < 0 ? 0 : ny - 2); x0 = min(x0, nx - 2 < 0 ? 0 : nx - 2);
    const int z1 = min(z0 + 1, nz - 1), y1 = min(y0 + 1, ny - 1), x1 = min(x0 + 1, nx - 1);
    const double tz = fz - z0, ty = fy - y0, tx = fx - x0;
    auto at = [&](int z, int y, int x) { return a[((int64_t)z * ny + y) * nx + x]; };
    const double c00 = at(z0, y0, x0) * (1 - tx) + at(z0, y0, x1) * tx;
    const double c01 = at(z0, y1, x0) * (1 - tx) + at(z0, y1, x1) * tx;
    const double c10 = at(z1, y0, x0) * (1 - tx) + at(z1, y0, x1) * tx;
    const double c11 = at(z1, y1, x0) * (1 - tx) + at(z1, y1, x1) * tx;
    out = (c00 * (1 - ty) + c01 * ty) * (1 - tz) + (c10 * (1 - ty) + c11 * ty) * tz;
    return true;
}

__global__ void k_gamma(const double *ref, const double *ev, int nx, int ny, int nz, double vx, double vy, double vz,
                        const unsigned long long *mx, double dose_crit, double dta, double threshold, int upsample,
                        double rad, unsigned long long *counts) {
    const double dmax = __longlong_as_double((long long)*mx);
    const double dd = dose_crit * dmax, thr = threshold * dmax;
    const int64_t n = (int64_t)nx * ny * nz;
    const double hz = vz / upsample, hy = vy / upsample, hx = vx / upsample;
    const int mz = (int)ceil(rad / hz), my = (int)ceil(rad / hy), mxx = (int)ceil(rad / hx);
    unsigned long long pass = 0, eval = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const double dr = ref[v];
        if (!(dr >= thr) || dmax <= 0.0) continue;
        const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((int64_t)nx * ny));
        double best = (ev[v] - dr) / dd;
        best *= best;
        for (int iz = -mz; iz <= mz && best > 0.0; ++iz)
            for (int iy = -my; iy <= my; ++iy)
                for (int ix = -mxx; ix <= mxx; ++ix) {
                    const double oz = iz * hz, oy = iy * hy, ox = ix * hx;
                    const double r2 = oz * oz + oy * oy + ox * ox;
                    if (r2 == 0.0 || r2 > rad * rad || r2 / (dta * dta) >= best) continue;
                    double val;
                    if (!trilinear(ev, nx, ny, nz, z + oz / vz, y + oy / vy, x + ox / vx, val)) continue;
                    const double t = (val - dr) / dd;
                    best = fmin(best, r2 / (dta * dta) + t * t);
                }
        eval++;
        if (best <= 1.0) pass++;
    }
    for (int o = 16; o > 0; o >>= 1) {
        pass += __shfl_xor_sync(0xFFFFFFFFu, pass, o);
        eval += __shfl_xor_sync(0xFFFFFFFFu, eval, o);
    }
    if ((threadIdx.x & 31) == 0) { atomicAdd(counts, pass); atomicAdd(counts + 1, eval); }
}
}  // namespace

extern "C" int psl_gamma(const double *ref, const double *ev, int32_t nx, int32_t ny, int32_t nz, float vx, float vy,
                         float vz, double dose_crit, double dta_cm, double threshold, int32_t upsample,
                         double max_radius_cm, double *pass_rate, int64_t *n_evaluated, void *stream_) {
    if (!ref || !ev || nx <= 0 || ny <= 0 || nz <= 0 || !(vx > 0) || !(vy > 0) || !(vz > 0) || !(dose_crit > 0) ||
        !(dta_cm > 0) || upsample < 1 || upsample > 16)
        return psl_fail(PSL_EINVAL, "psl_gamma: bad argument");
    cudaStream_t st = as_stream(stream_);
    const int64_t n = (int64_t)nx * ny * nz;
    unsigned long long *buf = nullptr;
    PSL_CUDA(psl_malloc_async((void **)&buf, 24, st));
    cudaMemsetAsync(buf, 0, 24, st);
    const int g = (int)std::min<int64_t>((n + 255) / 256, (int64_t)psl_sm_count() * 8);
    k_max<<<g, 256, 0, st>>>(ref, n, buf); PSL_NOTE_LAUNCH();
    const double rad = max_radius_cm > 0 ? max_radius_cm : 1.5 * dta_cm;
    k_gamma<<<g, 256, 0, st>>>(ref, ev, nx, ny, nz, vx, vy, vz, buf, dose_crit, dta_cm, threshold, upsample, rad,
                               buf + 1); PSL_NOTE_LAUNCH();
    unsigned long long h[2] = {0, 0};
    cudaMemcpyAsync(h, buf + 1, 16, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(buf, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return psl_fail(PSL_ECUDA, cudaGetErrorString(e));
    if (pass_rate) *pass_rate = h[1] ? (double)h[0] / (double)h[1] : 0.0;
    if (n_evaluated) *n_evaluated = (int64_t)h[1];
    return PSL_OK;
}
