// psl_build (Sec. 2.3.2): PSL id per record, stable LSD onesweep radix sort of
// (id, input index), gather of the records into 32-byte sorted records and
// the bin-offset table.
//
// Sort design (B300): 8-bit digits.  One upsweep pass computes the ids and
// the digit histograms of every pass at once; each digit pass is a single
// onesweep kernel: tiles of 4096 keys are ranked inside the block with warp
// match/ballot multisplit, the block's per-digit counts are published to a
// decoupled look-back table (one 32-bit word per tile and digit holding a
// 2-bit state and a 30-bit count), and the keys are scattered through shared
// memory so that each digit run is written contiguously.  Tiles are taken in
// order from an atomic counter so a tile only ever waits on tiles already
// running; every wait has an iteration limit after which the kernel records
// a timeout and proceeds.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "psl_internal.cuh"
#include "sort.cuh"

namespace {

constexpr int RADIX = 256;
constexpr int MAX_PASSES = SORT_MAX_PASSES;

struct Edges {
    int nx, ny, ne;
    const float *xe, *ye, *ee;
};

// number of entries of a[0..n) that are <= v (a ascending)
__device__ __forceinline__ int count_le(const float *a, int n, float v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] <= v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Azimuthal redistribution (Sec. 2.3.1): cos and sin of copy c's angle for
// record i.  A uniform point of the unit disc by rejection from Philox pairs;
// its doubled angle is uniform.  Each step is one float32 operation rounded
// to nearest, so the result is the same on any IEEE machine.
struct Apr {
    int32_t k;                 // copies per record
    uint32_t s0, s1;           // Philox key
};

__device__ __forceinline__ float apr_coord(uint32_t w) {
    // 2 U - 1 with U = ((w >> 9) + 0.5) 2^-23: both steps exact in float
    const float u = __fmul_rn(__fadd_rn((float)(w >> 9), 0.5f), 1.0f / 8388608.0f);
    return __fsub_rn(__fmul_rn(2.0f, u), 1.0f);
}

__device__ __forceinline__ void apr_angle(const Apr &A, uint32_t i, uint32_t c, float &cs, float &sn) {
    cs = 1.0f; sn = 0.0f;
    for (uint32_t b = 0; b < PSL_APR_MAX_BLOCKS; ++b) {
        const u32x4 o = philox10(b, PSL_TAG_APR, i, c, A.s0, A.s1);
        const uint32_t w[4] = {o.a, o.b, o.c, o.d};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float a = apr_coord(w[2 * h]), d = apr_coord(w[2 * h + 1]);
            const float aa = __fmul_rn(a, a), dd = __fmul_rn(d, d);
            const float r2 = __fadd_rn(aa, dd);
            if (r2 <= 1.0f) {
                cs = __fdiv_rn(__fsub_rn(aa, dd), r2);
                sn = __fdiv_rn(__fmul_rn(2.0f, __fmul_rn(a, d)), r2);
                return;
            }
        }
    }
}

// record and copy of redistributed index j (< 2^30)
__device__ __forceinline__ void apr_split(const Apr &A, int64_t j, uint32_t &i, uint32_t &c) {
    if (A.k == 1) { i = (uint32_t)j; c = 0; return; }
    i = (uint32_t)j / (uint32_t)A.k;
    c = (uint32_t)j - i * (uint32_t)A.k;
}

__device__ __forceinline__ void apr_rotate(float cs, float sn, float &x, float &y) {
    const float nx = __fsub_rn(__fmul_rn(x, cs), __fmul_rn(y, sn));
    const float ny = __fadd_rn(__fmul_rn(x, sn), __fmul_rn(y, cs));
    x = nx; y = ny;
}

// PSL id of every (copy of a) record + digit histograms of all passes (upsweep)
__global__ void __launch_bounds__(256) k_key(psl_records_t r, Edges ed, Apr apr, int64_t n, uint32_t n_bins,
                                             uint32_t *keys, int passes, uint32_t *hist) {
    extern __shared__ float sh[];
    float *xe = sh, *ye = xe + ed.nx + 1, *ee = ye + ed.ny + 1;
    __shared__ uint32_t h[MAX_PASSES * RADIX];
    for (int i = threadIdx.x; i <= ed.nx; i += blockDim.x) xe[i] = ed.xe[i];
    for (int i = threadIdx.x; i <= ed.ny; i += blockDim.x) ye[i] = ed.ye[i];
    for (int i = threadIdx.x; i <= ed.ne; i += blockDim.x) ee[i] = ed.ee[i];
    for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        uint32_t i, c;
        apr_split(apr, j, i, c);
        float x = __ldg(r.x + i), y = __ldg(r.y + i), e = __ldg(r.e + i);
        int q = __ldg(r.q + i);
        if (c) {
            float cs, sn;
            apr_angle(apr, i, c, cs, sn);
            apr_rotate(cs, sn, x, y);
        }
        int bx = count_le(xe, ed.nx + 1, x) - 1;
        int by = count_le(ye, ed.ny + 1, y) - 1;
        uint32_t key = n_bins;
        if (bx >= 0 && bx < ed.nx && by >= 0 && by < ed.ny && e > 0.f) {
            int eb = count_le(ee + 1, ed.ne - 1, e);
            int t = q != 0;
            key = (uint32_t)((t * ed.ne + eb) * (ed.nx * ed.ny) + by * ed.nx + bx);
        }
        keys[j] = key;
        for (int p = 0; p < passes; ++p) atomicAdd(&h[p * RADIX + ((key >> (8 * p)) & 0xFF)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// records packed as 32-byte AoS in input order (coalesced reads and writes),
// so that the gather below reads one 32-byte record per sorted position
// instead of seven scattered SoA elements
__global__ void __launch_bounds__(256) k_pack(psl_records_t r, Apr apr, int64_t n, PslRecord *__restrict__ out) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        uint32_t i, c;
        apr_split(apr, j, i, c);
        PslRecord o;
        o.x = __ldg(r.x + i); o.y = __ldg(r.y + i); o.u = __ldg(r.u + i); o.v = __ldg(r.v + i);
        o.e = __ldg(r.e + i); o.wt = __ldg(r.wt + i); o.src = (uint32_t)j; o.q = (int32_t)__ldg(r.q + i);
        if (c) {
            float cs, sn;
            apr_angle(apr, i, c, cs, sn);
            apr_rotate(cs, sn, o.x, o.y);
            apr_rotate(cs, sn, o.u, o.v);
        }
        float4 *d = reinterpret_cast<float4 *>(out + j);
        const float4 *sp = reinterpret_cast<const float4 *>(&o);
        d[0] = sp[0]; d[1] = sp[1];
    }
}

// sorted records straight from the caller's SoA arrays (no staging copy)
__global__ void __launch_bounds__(256) k_gather_soa(psl_records_t r, const uint32_t *__restrict__ perm, int64_t n_valid,
                                                    PslRecord *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_valid; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t s = perm[i];
        PslRecord o;
        o.x = __ldg(r.x + s); o.y = __ldg(r.y + s); o.u = __ldg(r.u + s); o.v = __ldg(r.v + s);
        o.e = __ldg(r.e + s); o.wt = __ldg(r.wt + s); o.src = s; o.q = (int32_t)__ldg(r.q + s);
        float4 *d = reinterpret_cast<float4 *>(out + i);
        const float4 *sp = reinterpret_cast<const float4 *>(&o);
        d[0] = sp[0]; d[1] = sp[1];
    }
}

// sorted records (AoS, 32 B) from the permutation
__global__ void __launch_bounds__(256) k_gather(const PslRecord *__restrict__ packed, const uint32_t *__restrict__ perm,
                                                int64_t n_valid, PslRecord *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_valid; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 *sp = reinterpret_cast<const float4 *>(packed + perm[i]);
        float4 *d = reinterpret_cast<float4 *>(out + i);
        const float4 a = __ldg(sp), b = __ldg(sp + 1);
        d[0] = a; d[1] = b;
    }
}

// offsets[k] = first sorted position with key >= k, from the boundaries of the sorted keys
__global__ void __launch_bounds__(256) k_offsets(const uint32_t *__restrict__ keys, int64_t n, int64_t n_bins,
                                                 int64_t *__restrict__ offsets) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t prev = i == 0 ? -1 : (int64_t)keys[i - 1];
        int64_t cur = i == n ? n_bins : (int64_t)keys[i];
        if (cur > n_bins) cur = n_bins;
        for (int64_t k = prev + 1; k <= cur; ++k) offsets[k] = i;
    }
}

__global__ void k_count_valid(const int64_t *offsets, int64_t n_bins, int64_t *out) { *out = offsets[n_bins]; }

}  // namespace

int psl_sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    return sms;
}

extern "C" int psl_build(const psl_params_t *prm, const psl_records_t *rec, psl_store_t **out, void *stream_) {
    if (!prm || !rec || !out) return psl_fail(PSL_EINVAL, "psl_build: null argument");
    *out = nullptr;
    if (prm->apr_copies < 1) return psl_fail(PSL_EINVAL, "psl_build: apr_copies must be >= 1");
    if (prm->nx <= 0 || prm->ny <= 0 || prm->n_ebins <= 0) return psl_fail(PSL_EINVAL, "psl_build: bad bin counts");
    const int64_t n_bins = 2ll * prm->n_ebins * prm->nx * prm->ny;
    if (n_bins >= (1ll << 31) - 1) return psl_fail(PSL_EINVAL, "psl_build: too many bins");
    if (rec->n < 0 || rec->n >= (1ll << 30) || rec->n * (int64_t)prm->apr_copies >= (1ll << 30))
        return psl_fail(PSL_EINVAL, "psl_build: record count (times apr_copies) out of range");
    if (!prm->x_edges || !prm->y_edges || !prm->e_edges) return psl_fail(PSL_EINVAL, "psl_build: null edges");
    for (int i = 0; i < prm->nx; ++i)
        if (!(prm->x_edges[i] < prm->x_edges[i + 1])) return psl_fail(PSL_EINVAL, "psl_build: x edges not ascending");
    for (int i = 0; i < prm->ny; ++i)
        if (!(prm->y_edges[i] < prm->y_edges[i + 1])) return psl_fail(PSL_EINVAL, "psl_build: y edges not ascending");
    for (int i = 0; i < prm->n_ebins; ++i)
        if (!(prm->e_edges[i] < prm->e_edges[i + 1])) return psl_fail(PSL_EINVAL, "psl_build: e edges not ascending");
    if (rec->n > 0 && (!rec->x || !rec->y || !rec->u || !rec->v || !rec->e || !rec->wt || !rec->q))
        return psl_fail(PSL_EINVAL, "psl_build: null record array");

    cudaStream_t st = as_stream(stream_);
    const uint32_t n = (uint32_t)(rec->n * prm->apr_copies);     // records after redistribution
    const Apr apr{prm->apr_copies, (uint32_t)prm->apr_seed, (uint32_t)(prm->apr_seed >> 32)};
    psl_store *s = new psl_store();
    s->n_records = n; s->n_bins = n_bins; s->nx = prm->nx; s->ny = prm->ny; s->n_ebins = prm->n_ebins;
    s->z_psl = prm->z_psl;
    s->stream = st;
    cudaGetDevice(&s->device);
    std::vector<float> edges;
    edges.insert(edges.end(), prm->x_edges, prm->x_edges + prm->nx + 1);
    edges.insert(edges.end(), prm->y_edges, prm->y_edges + prm->ny + 1);
    edges.insert(edges.end(), prm->e_edges, prm->e_edges + prm->n_ebins + 1);

    int bits = 1;
    while ((1ll << bits) <= n_bins) ++bits;              // ids 0..n_bins inclusive
    const int passes = (bits + 7) / 8;

    uint32_t *keys[2] = {nullptr, nullptr}, *vals[2] = {nullptr, nullptr}, *hist = nullptr;
    void *scratch = nullptr;
    PslRecord *packed = nullptr;
    int64_t *nvalid_d = nullptr;
    int rc = PSL_OK;
    auto fail = [&](int code, const std::string &m) { rc = psl_fail(code, m); };
    do {
        cudaError_t e;
        if ((e = psl_malloc_async((void **)&s->edges, edges.size() * sizeof(float), st)) != cudaSuccess) { fail(PSL_ENOMEM, cudaGetErrorString(e)); break; }
        if ((e = cudaMemcpyAsync(s->edges, edges.data(), edges.size() * sizeof(float), cudaMemcpyHostToDevice, st)) != cudaSuccess) { fail(PSL_ECUDA, cudaGetErrorString(e)); break; }
        if ((e = psl_malloc_async((void **)&s->offsets, (n_bins + 1) * sizeof(int64_t), st)) != cudaSuccess) { fail(PSL_ENOMEM, cudaGetErrorString(e)); break; }
        size_t nn = std::max<uint32_t>(n, 1);
        bool ok = true;
        for (int b = 0; b < 2 && ok; ++b) {
            ok &= psl_malloc_async((void **)&keys[b], nn * 4, st) == cudaSuccess;
            ok &= psl_malloc_async((void **)&vals[b], nn * 4, st) == cudaSuccess;
        }
        ok &= psl_malloc_async(&scratch, sort_pairs_scratch_bytes(n), st) == cudaSuccess;
        ok &= psl_malloc_async((void **)&hist, MAX_PASSES * RADIX * 4 + 16, st) == cudaSuccess;
        if (!ok) { fail(PSL_ENOMEM, "psl_build: sort buffers"); break; }
        nvalid_d = reinterpret_cast<int64_t *>(hist + MAX_PASSES * RADIX);
        cudaMemsetAsync(hist, 0, MAX_PASSES * RADIX * 4, st);
        Edges ed{prm->nx, prm->ny, prm->n_ebins, s->edges, s->edges + prm->nx + 1, s->edges + prm->nx + prm->ny + 2};
        const int sms = psl_sm_count();
        if (n == 0) {
            cudaMemsetAsync(s->offsets, 0, (n_bins + 1) * sizeof(int64_t), st);
            psl_malloc_async((void **)&s->rec, sizeof(PslRecord), st);
            break;
        }
        int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
        { void *tk_ = nullptr; if (psl_timer_on()) psl_timer_begin(PK_KEY, st, &tk_); k_key<<<grid, 256, edges.size() * sizeof(float), st>>>(*rec, ed, apr, (int64_t)n, (uint32_t)n_bins, keys[0], passes, hist); PSL_NOTE_LAUNCH(); if (tk_) psl_timer_end(PK_KEY, st, tk_); }
        int alt = 0;
        sort_pairs_u32(keys[0], vals[0], keys[1], vals[1], n, bits, hist, true, scratch, &alt, st);
        // after an odd number of passes the result is in the alternate buffers
        uint32_t *skeys = alt ? keys[1] : keys[0], *svals = alt ? vals[1] : vals[0];
        int g2 = (int)std::min<int64_t>((int64_t)n / 256 + 1, (int64_t)sms * 8);
        k_offsets<<<g2, 256, 0, st>>>(skeys, n, n_bins, s->offsets); PSL_NOTE_LAUNCH();
        k_count_valid<<<1, 1, 0, st>>>(s->offsets, n_bins, nvalid_d); PSL_NOTE_LAUNCH();
        if ((e = psl_malloc_async((void **)&packed, (size_t)n * sizeof(PslRecord), st)) != cudaSuccess) { fail(PSL_ENOMEM, cudaGetErrorString(e)); break; }
        {
            void *tk_ = nullptr;
            if (psl_timer_on()) psl_timer_begin(PK_GATHER, st, &tk_);
            k_pack<<<(int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 16), 256, 0, st>>>(*rec, apr, n, packed); PSL_NOTE_LAUNCH();
            if (tk_) psl_timer_end(PK_GATHER, st, tk_);
        }
        int64_t nvalid = 0;
        uint32_t herr = 0;
        cudaMemcpyAsync(&nvalid, nvalid_d, 8, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(&herr, sort_err_word(scratch), 4, cudaMemcpyDeviceToHost, st);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { fail(PSL_ECUDA, cudaGetErrorString(e)); break; }
        if (herr & PSL_DEV_ERR_TIMEOUT) { fail(PSL_ETIMEOUT, "psl_build: look-back wait gave up"); break; }
        s->n_valid = nvalid;
        if ((e = psl_malloc_async((void **)&s->rec, std::max<int64_t>(nvalid, 1) * sizeof(PslRecord), st)) != cudaSuccess) { fail(PSL_ENOMEM, cudaGetErrorString(e)); break; }
        if (nvalid > 0) {
            int g3 = (int)std::min<int64_t>((nvalid + 255) / 256, (int64_t)sms * 16);
            { void *tk_ = nullptr; if (psl_timer_on()) psl_timer_begin(PK_GATHER, st, &tk_); k_gather<<<g3, 256, 0, st>>>(packed, svals, nvalid, s->rec); PSL_NOTE_LAUNCH(); if (tk_) psl_timer_end(PK_GATHER, st, tk_); }
        }
        if ((e = cudaGetLastError()) != cudaSuccess) { fail(PSL_ECUDA, cudaGetErrorString(e)); break; }
    } while (0);
    for (int b = 0; b < 2; ++b) { if (keys[b]) cudaFreeAsync(keys[b], st); if (vals[b]) cudaFreeAsync(vals[b], st); }
    if (scratch) cudaFreeAsync(scratch, st);
    if (hist) cudaFreeAsync(hist, st);
    if (packed) cudaFreeAsync(packed, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (rc == PSL_OK && e2 != cudaSuccess) rc = psl_fail(PSL_ECUDA, cudaGetErrorString(e2));
    if (rc != PSL_OK) { psl_store_destroy(s); return rc; }
    *out = s;
    return PSL_OK;
}

extern "C" int psl_store_info(const psl_store_t *s, int64_t *n_records, int64_t *n_valid, int64_t *n_bins) {
    if (!s) return psl_fail(PSL_EINVAL, "psl_store_info: null store");
    if (n_records) *n_records = s->n_records;
    if (n_valid) *n_valid = s->n_valid;
    if (n_bins) *n_bins = s->n_bins;
    return PSL_OK;
}

namespace {
__global__ void k_store_read(const PslRecord *rec, int64_t n, int64_t *perm, float *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        PslRecord r = rec[i];
        if (perm) perm[i] = r.src;
        if (out) {
            const float *f = reinterpret_cast<const float *>(&r);
            for (int k = 0; k < 8; ++k) out[8 * i + k] = f[k];
        }
    }
}
}  // namespace

extern "C" int psl_store_read(const psl_store_t *s, int64_t *offsets, int64_t *perm, float *records, void *stream_) {
    if (!s) return psl_fail(PSL_EINVAL, "psl_store_read: null store");
    cudaStream_t st = as_stream(stream_);
    if (offsets) PSL_CUDA(cudaMemcpyAsync(offsets, s->offsets, (s->n_bins + 1) * 8, cudaMemcpyDeviceToDevice, st));
    if ((perm || records) && s->n_valid > 0) {
        int g = (int)std::min<int64_t>((s->n_valid + 255) / 256, 4096);
        k_store_read<<<g, 256, 0, st>>>(s->rec, s->n_valid, perm, records); PSL_NOTE_LAUNCH();
        PSL_CUDA(cudaGetLastError());
    }
    return PSL_OK;
}

extern "C" void psl_store_destroy(psl_store_t *s) {
    if (!s) return;
    if (s->rec) cudaFreeAsync(s->rec, s->stream);
    if (s->offsets) cudaFreeAsync(s->offsets, s->stream);
    if (s->edges) cudaFreeAsync(s->edges, s->stream);
    delete s;
}

// --------------------------------------------------------------------------
// psl_build_static: the same PSL build for callers that cannot allocate
// device memory.  All scratch (ids, values, digit histograms, look-back
// table, edges, the kept-record count) lives in one file-scope device array
// of fixed size; the caller passes the inputs and the output arrays.
// --------------------------------------------------------------------------
namespace {

constexpr size_t ST_MAX_N = PSL_STATIC_MAX_RECORDS;
constexpr size_t ST_ROUND = 64;                                   // 256 bytes in 4-byte words
constexpr size_t st_round(size_t w) { return (w + ST_ROUND - 1) / ST_ROUND * ST_ROUND; }
constexpr size_t ST_TILES = (ST_MAX_N + SORT_TILE - 1) / SORT_TILE;
// word offsets of the regions
constexpr size_t ST_KEYS0 = 0;
constexpr size_t ST_KEYS1 = ST_KEYS0 + ST_MAX_N;
constexpr size_t ST_VALS0 = ST_KEYS1 + ST_MAX_N;
constexpr size_t ST_VALS1 = ST_VALS0 + ST_MAX_N;
constexpr size_t ST_HIST = ST_VALS1 + ST_MAX_N;                  // digit histograms + kept count (int64)
constexpr size_t ST_EDGES = ST_HIST + st_round(MAX_PASSES * RADIX + 4);
constexpr size_t ST_SORT = ST_EDGES + st_round(PSL_STATIC_MAX_EDGES);
constexpr size_t ST_SORT_WORDS = st_round(SORT_HEAD_WORDS + ST_TILES * 256);
constexpr size_t ST_WORDS = ST_SORT + ST_SORT_WORDS;
// sort_pairs_u32 writes SORT_HEAD_WORDS words, then a look-back table of 256
// words per tile of SORT_TILE keys: the region must hold both at the limit
static_assert(ST_SORT_WORDS >= SORT_HEAD_WORDS + ((ST_MAX_N + SORT_TILE - 1) / SORT_TILE) * 256,
              "static sort scratch too small for sort_pairs_u32");

// Held by every device that loads the library, until the process exits.
static __device__ __align__(256) uint32_t g_build_scratch[ST_WORDS];

// Device address of g_build_scratch in the current CUDA context.  Host code
// cannot use the symbol itself as an address: it is looked up with
// cudaGetSymbolAddress once per context (keyed by the driver's unique
// context id, so a context torn down and created again - cudaDeviceReset -
// gets its own lookup instead of a stale address).
typedef int (*ctx_get_current_fn)(void **);                     // cuCtxGetCurrent
typedef int (*ctx_get_id_fn)(void *, unsigned long long *);       // cuCtxGetId (driver API 12.0)

struct StaticSlot {
    unsigned long long ctx_id = 0;
    uint32_t *addr = nullptr;
};
std::mutex g_static_mu;
StaticSlot g_static_slots[64];

int current_context_id(unsigned long long *id) {
    static ctx_get_current_fn get_current = nullptr;
    static ctx_get_id_fn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess)
            get_current = (ctx_get_current_fn)f1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess)
            get_id = (ctx_get_id_fn)f2;
        looked_up = true;
    }
    if (!get_current || !get_id) return psl_fail(PSL_ECUDA, "psl_build_static: driver context queries unavailable");
    void *ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx) return psl_fail(PSL_ECUDA, "psl_build_static: no current CUDA context");
    if (get_id(ctx, id) != 0) return psl_fail(PSL_ECUDA, "psl_build_static: cuCtxGetId failed");
    return PSL_OK;
}

int static_scratch(uint32_t **out) {
    int dev = 0;
    PSL_CUDA(cudaGetDevice(&dev));
    PSL_CUDA(cudaFree(nullptr));                 // make the device's primary context current
    unsigned long long id = 0;
    int rc = current_context_id(&id);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_static_mu);
    StaticSlot *free_slot = nullptr;
    for (auto &s : g_static_slots) {
        if (s.addr && s.ctx_id == id) { *out = s.addr; return PSL_OK; }
        if (!s.addr && !free_slot) free_slot = &s;
    }
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_build_scratch);
    if (e != cudaSuccess)
        return psl_fail(PSL_ECUDA, std::string("psl_build_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    if (!free_slot) free_slot = &g_static_slots[id % 64];      // more contexts than slots: reuse one
    free_slot->ctx_id = id;
    free_slot->addr = (uint32_t *)p;
    *out = free_slot->addr;
    return PSL_OK;
}

}  // namespace

extern "C" int psl_build_static(const psl_params_t *prm, const psl_records_t *rec, int64_t *offsets, float *sorted,
                                int64_t *n_valid, void *stream_) {
    if (!prm || !rec || !offsets || !sorted || !n_valid) return psl_fail(PSL_EINVAL, "psl_build_static: null argument");
    if (prm->apr_copies != 1) return psl_fail(PSL_EINVAL, "psl_build_static: apr_copies must be 1");
    if (prm->nx <= 0 || prm->ny <= 0 || prm->n_ebins <= 0) return psl_fail(PSL_EINVAL, "psl_build_static: bad bin counts");
    const int64_t n_bins = 2ll * prm->n_ebins * prm->nx * prm->ny;
    if (n_bins >= (1ll << 31) - 1) return psl_fail(PSL_EINVAL, "psl_build_static: too many bins");
    if (rec->n < 0) return psl_fail(PSL_EINVAL, "psl_build_static: negative record count");
    if (rec->n > (int64_t)PSL_STATIC_MAX_RECORDS)
        return psl_fail(PSL_EINVAL, "psl_build_static: " + std::to_string(rec->n) + " records exceed the static limit of " +
                                        std::to_string((long long)PSL_STATIC_MAX_RECORDS) + "; use psl_build");
    const int64_t n_edges = (int64_t)prm->nx + prm->ny + prm->n_ebins + 3;
    if (n_edges > PSL_STATIC_MAX_EDGES)
        return psl_fail(PSL_EINVAL, "psl_build_static: " + std::to_string(n_edges) + " bin edges exceed the static limit of " +
                                        std::to_string(PSL_STATIC_MAX_EDGES));
    if (!prm->x_edges || !prm->y_edges || !prm->e_edges) return psl_fail(PSL_EINVAL, "psl_build_static: null edges");
    for (int i = 0; i < prm->nx; ++i)
        if (!(prm->x_edges[i] < prm->x_edges[i + 1])) return psl_fail(PSL_EINVAL, "psl_build_static: x edges not ascending");
    for (int i = 0; i < prm->ny; ++i)
        if (!(prm->y_edges[i] < prm->y_edges[i + 1])) return psl_fail(PSL_EINVAL, "psl_build_static: y edges not ascending");
    for (int i = 0; i < prm->n_ebins; ++i)
        if (!(prm->e_edges[i] < prm->e_edges[i + 1])) return psl_fail(PSL_EINVAL, "psl_build_static: e edges not ascending");
    if (rec->n > 0 && (!rec->x || !rec->y || !rec->u || !rec->v || !rec->e || !rec->wt || !rec->q))
        return psl_fail(PSL_EINVAL, "psl_build_static: null record array");

    uint32_t *base = nullptr;
    int rc = static_scratch(&base);
    if (rc) return rc;
    cudaStream_t st = as_stream(stream_);
    const uint32_t n = (uint32_t)rec->n;
    uint32_t *keys0 = base + ST_KEYS0, *keys1 = base + ST_KEYS1, *vals0 = base + ST_VALS0, *vals1 = base + ST_VALS1;
    uint32_t *hist = base + ST_HIST;
    int64_t *nvalid_d = reinterpret_cast<int64_t *>(hist + MAX_PASSES * RADIX);
    float *edges = reinterpret_cast<float *>(base + ST_EDGES);
    void *sort_scratch = base + ST_SORT;

    // edges: x | y | e, copied from the host arrays (pageable copies, no allocation)
    PSL_CUDA(cudaMemcpyAsync(edges, prm->x_edges, (prm->nx + 1) * sizeof(float), cudaMemcpyHostToDevice, st));
    PSL_CUDA(cudaMemcpyAsync(edges + prm->nx + 1, prm->y_edges, (prm->ny + 1) * sizeof(float), cudaMemcpyHostToDevice, st));
    PSL_CUDA(cudaMemcpyAsync(edges + prm->nx + prm->ny + 2, prm->e_edges, (prm->n_ebins + 1) * sizeof(float),
                             cudaMemcpyHostToDevice, st));
    // the array keeps the previous call's contents: clear what must start at zero
    PSL_CUDA(cudaMemsetAsync(hist, 0, (MAX_PASSES * RADIX + 4) * sizeof(uint32_t), st));
    if (n == 0) {
        PSL_CUDA(cudaMemsetAsync(offsets, 0, (n_bins + 1) * sizeof(int64_t), st));
        PSL_CUDA(cudaStreamSynchronize(st));
        *n_valid = 0;
        return PSL_OK;
    }
    int bits = 1;
    while ((1ll << bits) <= n_bins) ++bits;
    const int passes = (bits + 7) / 8;
    Edges ed{prm->nx, prm->ny, prm->n_ebins, edges, edges + prm->nx + 1, edges + prm->nx + prm->ny + 2};
    const int sms = psl_sm_count();
    int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
    k_key<<<grid, 256, n_edges * sizeof(float), st>>>(*rec, ed, Apr{1, 0u, 0u}, rec->n, (uint32_t)n_bins, keys0, passes, hist); PSL_NOTE_LAUNCH();
    int alt = 0;
    sort_pairs_u32(keys0, vals0, keys1, vals1, n, bits, hist, true, sort_scratch, &alt, st);
    uint32_t *skeys = alt ? keys1 : keys0, *svals = alt ? vals1 : vals0;
    int g2 = (int)std::min<int64_t>((int64_t)n / 256 + 1, (int64_t)sms * 8);
    k_offsets<<<g2, 256, 0, st>>>(skeys, n, n_bins, offsets); PSL_NOTE_LAUNCH();
    k_count_valid<<<1, 1, 0, st>>>(offsets, n_bins, nvalid_d); PSL_NOTE_LAUNCH();
    int64_t nvalid = 0;
    uint32_t herr = 0;
    PSL_CUDA(cudaMemcpyAsync(&nvalid, nvalid_d, 8, cudaMemcpyDeviceToHost, st));
    PSL_CUDA(cudaMemcpyAsync(&herr, sort_err_word(sort_scratch), 4, cudaMemcpyDeviceToHost, st));
    PSL_CUDA(cudaStreamSynchronize(st));
    if (herr & PSL_DEV_ERR_TIMEOUT) return psl_fail(PSL_ETIMEOUT, "psl_build_static: look-back wait gave up");
    if (nvalid > 0) {
        int g3 = (int)std::min<int64_t>((nvalid + 255) / 256, (int64_t)sms * 16);
        k_gather_soa<<<g3, 256, 0, st>>>(*rec, svals, nvalid, reinterpret_cast<PslRecord *>(sorted)); PSL_NOTE_LAUNCH();
    }
    PSL_CUDA(cudaGetLastError());
    PSL_CUDA(cudaStreamSynchronize(st));
    *n_valid = nvalid;
    return PSL_OK;
}
