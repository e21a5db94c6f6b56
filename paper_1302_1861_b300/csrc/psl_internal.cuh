// Internal declarations of the B300 PSL library: handles, particle layout,
// device helpers (Philox, warp-aggregated queue pushes), error reporting.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "../../include/psl.h"

// ------------------------------------------------------------------ errors --
void psl_set_error(const std::string &msg);
int psl_fail(int code, const std::string &msg);

#define PSL_CUDA(call)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return psl_fail(e_ == cudaErrorMemoryAllocation ? PSL_ENOMEM : PSL_ECUDA,       \
                            std::string(#call) + ": " + cudaGetErrorString(e_));            \
    } while (0)

#define PSL_CHECK_LAUNCH(name) PSL_CUDA(cudaGetLastError())

// opt-in event timing of the main kernels (psl_profile)
enum { PK_KEY = 0, PK_ONESWEEP, PK_GATHER, PK_SOURCE, PK_PHOTON, PK_ELECTRON, PK_BAND, PK_READOUT, PK_CONV };
bool psl_timer_on();

// failure-detection hooks (psl_debug_waits): polls of a bounded wait (dflt
// unless a test set a limit), the stall flags and a cap on queue capacity
long long psl_wait_polls(long long dflt);
unsigned psl_debug_flags();
long long psl_debug_queue_cap();
void psl_timer_begin(int k, cudaStream_t st, void **tok);
void psl_timer_end(int k, cudaStream_t st, void *tok);

// host-side count of kernel launches (psl_kernel_launches)
void psl_note_launch();
#define PSL_NOTE_LAUNCH() psl_note_launch()

static inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// device error word bits
#define PSL_DEV_ERR_TIMEOUT 1u
#define PSL_DEV_ERR_QUEUE 2u
#define PSL_DEV_ERR_STEPS 4u

// ------------------------------------------------------------- particles --
// 48-byte particle: three 16-byte words, loaded and stored as float4.
struct __align__(16) Particle {
    float x, y, z, e;        // phantom-local position (cm), kinetic energy (MeV)
    float u, v, w, wt;       // direction cosines, statistical weight
    uint32_t pid_lo, pid_hi; // Philox stream id
    uint32_t type;           // 0 photon, 1 electron, 2 positron
    uint32_t root;           // history index inside its batch (per-history traces)
};
static_assert(sizeof(Particle) == 48, "particle layout");

// ----------------------------------------------------------------- store --
struct PslRecord {           // 32-byte sorted record
    float x, y, u, v, e, wt;
    uint32_t src;            // input index
    int32_t q;
};
static_assert(sizeof(PslRecord) == 32, "record layout");

struct psl_store {
    int64_t n_records = 0, n_valid = 0, n_bins = 0;
    int32_t nx = 0, ny = 0, n_ebins = 0;
    float z_psl = 0.f;
    PslRecord *rec = nullptr;        // [n_valid]
    int64_t *offsets = nullptr;      // [n_bins + 1]
    float *edges = nullptr;          // device: x_edges | y_edges | e_edges
    int device = 0;
    cudaStream_t stream = nullptr;   // allocations are stream ordered on it
};

// Per-beam constants precomputed on the device (float32, fixed op order).
struct BeamDev {
    float xlo, xhi, ylo, yhi;        // jaw bounds at the jaw planes
    float dzx, dzy, diso;            // z_jaw_x - z_psl, z_jaw_y - z_psl, sad - z_psl
    float mu_ratio;                  // mu_i / mu_total
    float fx0, fy0, fdx, fdy;
    int32_t fnx, fny;
    const float *fluence;
    float r[9];                      // beam-to-patient rotation (row major)
    float iso[3];
    float sad;
};

// One entry of a plan's reading order in visiting position, packed so that
// the source stage reads it with one 32-byte load: the PSL's first sorted
// record, its record count, the entry's random start offset (Sec. 2.3.3),
// its beam and the entry's index in the entry list.
struct __align__(16) EntryDev {
    int64_t start, nrec, offset;
    int32_t beam;
    uint32_t entry;
};

// One segment of a group's reading order (rounds of constant width): its
// group-local first history, first round and active entries.
struct __align__(16) SegDev {
    int64_t h, r0;
    int32_t w, pad;
};

struct psl_plan {
    const psl_store *store = nullptr;
    int32_t n_beams = 0;
    float sad = 100.f;
    int64_t n_histories = 0, n_entries = 0, n_total_psl = 0;
    int64_t n_incident = 0;          // the store's records (input records x redistribution copies)
    uint64_t seed = 0;
    int32_t n_groups = 0;
    BeamDev *beams = nullptr;        // [n_beams]
    // per entry (entry-list order)
    int32_t *e_beam = nullptr;
    int32_t *e_psl = nullptr;
    int64_t *e_start = nullptr, *e_nrec = nullptr, *e_count = nullptr, *e_offset = nullptr;
    // reading order
    int64_t *group_start = nullptr;  // [n_groups + 1] first history of each group
    int64_t *group_seg = nullptr;    // [n_groups + 1] first segment of each group
    uint32_t *sorted = nullptr;      // [n_active] entries in visiting order, grouped
    int64_t *seg_h = nullptr;        // [n_active] group-local first history of segment
    int64_t *seg_r0 = nullptr;       // first round of segment
    int32_t *seg_w = nullptr;        // active entries in the segment's rounds
    EntryDev *ent = nullptr;         // [n_active] entry data in visiting order (sorted[])
    SegDev *seg = nullptr;           // [n_active] seg_h, seg_r0, seg_w packed
    int64_t n_active = 0;
    cudaStream_t stream = nullptr;
};

struct psl_batch {
    int64_t n_histories = 0;         // histories (or caller particles) covered
    int64_t first_history = 0;
    int64_t stride = 1;              // histories first + i * stride
    int lazy = 0;                    // 1: source stage runs inside transport_run
    const psl_plan *plan = nullptr;  // lazy batches: the plan to read
    psl_phantom_t phantom{};         // lazy batches: the phantom box
    uint64_t seed = 0;               // keys the particles' random streams
    Particle *p = nullptr;           // photons from the front, electrons from the back
    int64_t cap = 0;
    uint32_t *counts = nullptr;      // device [2]: photons, electrons
    int64_t n_photons = 0, n_electrons = 0;
    int consumed = 0;
    cudaStream_t stream = nullptr;
    // batches from psl_stream_bin: the on-the-fly groups (device arrays)
    int64_t s_groups = 0, s_binned = 0;
    int64_t *s_gbin = nullptr, *s_gcount = nullptr, *s_hist = nullptr;
    unsigned long long s_emitted = 0, s_missed = 0;
};

struct Workspace;
// Per-history record of what the production source stage decided, for the
// histories [first, first + n) of later transport calls on a tally.
struct SrcTraceDev {
    int64_t first = 0, n = 0;        // n = 0: off
    int64_t *entry = nullptr, *use = nullptr, *rec = nullptr;
    int8_t *status = nullptr;
    float *state = nullptr;          // n x 8 (transported histories only)
    int32_t *ptype = nullptr;
};

struct psl_tally {
    int32_t nx = 0, ny = 0, nz = 0, n_batches = 0;
    int64_t nvox = 0;
    int32_t grid_mult = 4;            // persistent transport grid: blocks per SM
    int64_t chunk_cap = 1 << 24;      // primaries per transport pass (queue depth)
    int32_t order = 0;                // psl_run history order: 0 auto, 1 reading order, 2 batch by batch
    unsigned long long *t = nullptr;  // [n_batches][nvox] (a batch's slice contiguous)
    unsigned long long *ledger = nullptr;  // [16]: 12 reported slots, then scratch
    Workspace *ws = nullptr;
    SrcTraceDev trace;                // psl_tally_trace_source
};

// ----------------------------------------------------------------- Philox --
#define TAG_PARTICLE 0u
#define TAG_OFFSET 1u
#define TAG_CHILD 2u
#define TAG_BATCH 4u

// A particle's `root` word: bits 22-31 hold the tally slice (batch) of its
// history, bits 0-21 the history's index in a traced transport call.
#define ROOT_SLICE_SHIFT 22
#define ROOT_INDEX_MASK ((1u << ROOT_SLICE_SHIFT) - 1u)

struct u32x4 { uint32_t a, b, c, d; };

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64 products
// with the key bumped by the Weyl constants between rounds.
__host__ __device__ __forceinline__ u32x4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                   uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        uint32_t hi0 = mulhi32(m0, c0), lo0 = m0 * c0;
        uint32_t hi1 = mulhi32(m1, c2), lo1 = m1 * c2;
        uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    return {c0, c1, c2, c3};
}

// Philox4x32-10 with a precomputed key schedule rk[2r], rk[2r+1] = the key
// of round r (the seed's words plus r times the Weyl constants).
__device__ __forceinline__ u32x4 philox10_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, const uint32_t *rk) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
        uint32_t hi0 = __umulhi(m0, c0), lo0 = m0 * c0;
        uint32_t hi1 = __umulhi(m1, c2), lo1 = m1 * c2;
        uint32_t n0 = hi1 ^ c1 ^ rk[2 * r], n2 = hi0 ^ c3 ^ rk[2 * r + 1];
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    return {c0, c1, c2, c3};
}

// Per-particle random stream: draw d uses word d%4 of block d/4 of
// Philox(key = seed; counter = (d/4, TAG_PARTICLE, pid (p0, p1))).
// Only the draw counter and the current block live in registers; the key
// schedule and the particle id are passed in.
struct Rng {
    uint32_t draw;
    u32x4 blk;
    // start the next draw at a fresh block: every event begins on a block
    // boundary, so the lanes of a warp compute their blocks together
    __device__ __forceinline__ void align() { draw = (draw + 3u) & ~3u; }
    // ((r >> 9) + 0.5) * 2^-23: 24 significant bits, exact in float
    __device__ __forceinline__ float next(const uint32_t *rk, uint32_t p0, uint32_t p1) {
        uint32_t w = draw & 3u;
        if (w == 0) blk = philox10_rk(draw >> 2, TAG_PARTICLE, p0, p1, rk);
        uint32_t r = w == 0 ? blk.a : (w == 1 ? blk.b : (w == 2 ? blk.c : blk.d));
        ++draw;
        return ((float)(r >> 9) + 0.5f) * (1.0f / 8388608.0f);
    }
    // compute the block of an aligned draw index ahead of its draws, at one
    // program point for every lane; take() then reads words of that block
    // (at most 4 takes per fill; next() continues correctly afterwards)
    __device__ __forceinline__ void fill(const uint32_t *rk, uint32_t p0, uint32_t p1) {
        blk = philox10_rk(draw >> 2, TAG_PARTICLE, p0, p1, rk);
    }
    __device__ __forceinline__ float take() {
        uint32_t w = draw & 3u;
        uint32_t r = w == 0 ? blk.a : (w == 1 ? blk.b : (w == 2 ? blk.c : blk.d));
        ++draw;
        return ((float)(r >> 9) + 0.5f) * (1.0f / 8388608.0f);
    }
};

// Tally slice of history (p0, p1) among nb (Sec. 2.3.3 batches): the first
// word of Philox(key seed; counter (0, TAG_BATCH, history id)) scaled to
// [0, nb).  Every batch is an independent pseudo-random subset of the
// histories, whatever the reading order.
// Batches are drawn per block of BATCH_BLOCK consecutive history ids: block
// B = h >> BATCH_BLOCK_SHIFT goes to batch floor(r N_b / 2^32), r the first
// word of Philox(key = seed; counter = (0, TAG_BATCH, B)).
#define BATCH_BLOCK_SHIFT 8
#define BATCH_BLOCK (1 << BATCH_BLOCK_SHIFT)
static_assert(BATCH_BLOCK == PSL_BATCH_BLOCK, "psl.h states the batch block");

__device__ __forceinline__ uint32_t block_slice(uint64_t blk, const uint32_t *rk, uint32_t nb) {
    const u32x4 r = philox10_rk(0u, TAG_BATCH, (uint32_t)blk, (uint32_t)(blk >> 32), rk);
    return __umulhi(r.a, nb);
}

// the batch of history (or caller particle) id p1:p0
__device__ __forceinline__ uint32_t history_slice(uint32_t p0, uint32_t p1, const uint32_t *rk, uint32_t nb) {
    return block_slice((((uint64_t)p1 << 32) | p0) >> BATCH_BLOCK_SHIFT, rk, nb);
}

__device__ __forceinline__ void child_id(uint64_t seed, uint32_t p0, uint32_t p1, uint32_t ordinal,
                                         uint32_t &c0, uint32_t &c1) {
    u32x4 o = philox10(ordinal, TAG_CHILD, p0, p1, (uint32_t)seed, (uint32_t)(seed >> 32));
    c0 = o.a;
    c1 = o.b | 0x80000000u;
}

// ------------------------------------------------------------ queue push --
struct Queue {
    Particle *data;
    uint32_t *count;
    uint32_t cap;
};

__device__ __forceinline__ void store_particle(Particle *dst, const Particle &p) {
    const float4 *s = reinterpret_cast<const float4 *>(&p);
    float4 *d = reinterpret_cast<float4 *>(dst);
    d[0] = s[0]; d[1] = s[1]; d[2] = s[2];
}

__device__ __forceinline__ Particle load_particle(const Particle *src) {
    Particle p;
    const float4 *s = reinterpret_cast<const float4 *>(src);
    float4 *d = reinterpret_cast<float4 *>(&p);
    d[0] = __ldg(s); d[1] = __ldg(s + 1); d[2] = __ldg(s + 2);
    return p;
}

// Append with one atomic per group of converged lanes.
__device__ __forceinline__ void queue_push(const Queue &q, const Particle &p, uint32_t *err) {
    unsigned mask = __activemask();
    int lane = threadIdx.x & 31;
    int leader = __ffs(mask) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(q.count, (uint32_t)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    uint32_t idx = base + __popc(mask & ((1u << lane) - 1u));
    if (idx < q.cap) store_particle(q.data + idx, p);
    else atomicOr(err, PSL_DEV_ERR_QUEUE);
}

// grid size for a memory-bound kernel: multiple of the SM count
int psl_sm_count();

// Stream-ordered allocation from the library's device memory pool (freed
// blocks stay in the pool for the next call; see psl_memory_trim).
cudaError_t psl_malloc_async(void **ptr, size_t bytes, cudaStream_t st);

// Device copies of beams (host array) with their float32 jaw bounds, MU
// ratios and rotation matrices; *out is stream-ordered device memory the
// caller frees with cudaFreeAsync.
int psl_beams_dev(const psl_beam_t *beams, int n, float sad, float z_psl, BeamDev **out, cudaStream_t st);
