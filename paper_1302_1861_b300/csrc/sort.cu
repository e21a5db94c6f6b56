// Generic stable LSD radix sort of (u32 key, u32 value) pairs: 8-bit digit
// onesweep passes with decoupled look-back, plus device scans of int64
// arrays.  Used by the PSL build (Sec. 2.3.2) and by the plan builder to order
// entries (Sec. 2.3.3).
//
// Onesweep pass: a block ranks a tile of 4096 keys with warp match/ballot
// multisplit (stable: warps own consecutive key ranges, lanes keep input
// order), publishes its per-digit counts to a look-back table (one 32-bit
// word per tile and digit: 2-bit state + 30-bit count), adds the counts of
// the preceding tiles and scatters through shared memory so that each digit
// run is written contiguously.  Tiles are taken in order from an atomic
// counter, so a tile only waits on tiles that are already running, and every
// wait is bounded (on timeout the error word is set and the kernel goes on).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "psl_internal.cuh"
#include "sort.cuh"

namespace {

constexpr int RADIX = 256;
constexpr int SORT_THREADS = 256;     // 8 warps
constexpr int SORT_ITEMS = 16;        // keys per thread
constexpr int TILE = SORT_THREADS * SORT_ITEMS;
static_assert(TILE == SORT_TILE, "sort.cuh states the onesweep tile size");
static_assert(RADIX == 256, "sort.cuh sizes the look-back table with 256 digits");
constexpr uint32_t LB_AGG = 1u << 30;
constexpr uint32_t LB_INC = 2u << 30;
constexpr uint32_t LB_MASK = (1u << 30) - 1u;
constexpr long long SPIN_LIMIT = 1ll << 22;   // ~1 s of polling

// exclusive scan of each pass's 256-bucket histogram (one block of 256)
__global__ void k_digit_offsets(const uint32_t *hist, uint32_t *offs, int passes) {
    __shared__ uint32_t s[RADIX];
    for (int p = 0; p < passes; ++p) {
        uint32_t v = hist[p * RADIX + threadIdx.x];
        s[threadIdx.x] = v;
        __syncthreads();
        for (int d = 1; d < RADIX; d <<= 1) {
            uint32_t t = threadIdx.x >= d ? s[threadIdx.x - d] : 0;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        offs[p * RADIX + threadIdx.x] = s[threadIdx.x] - v;
        __syncthreads();
    }
}

// One onesweep digit pass.  vals_in == nullptr means the identity.
__global__ void __launch_bounds__(SORT_THREADS) k_onesweep(const uint32_t *__restrict__ keys_in,
                                                          const uint32_t *__restrict__ vals_in,
                                                          uint32_t *__restrict__ keys_out,
                                                          uint32_t *__restrict__ vals_out, uint32_t n, int shift,
                                                          const uint32_t *__restrict__ digit_offs,
                                                          uint32_t *lookback, uint32_t *tile_counter, uint32_t *err,
                                                          long long spin_limit, bool stall) {
    __shared__ uint32_t s_keys[TILE];
    __shared__ uint32_t s_vals[TILE];
    __shared__ uint32_t whist[SORT_THREADS / 32][RADIX];   // per-warp digit counts, then warp prefixes
    __shared__ uint32_t blk_excl[RADIX];                    // block-local exclusive digit offsets
    __shared__ uint32_t glob_base[RADIX];                   // global position of the block's first key of digit d
    __shared__ uint32_t s_tile;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
    for (int i = tid; i < (SORT_THREADS / 32) * RADIX; i += SORT_THREADS) (&whist[0][0])[i] = 0;
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint32_t tile_base = tile * TILE;
    const uint32_t warp_base = tile_base + warp * (32 * SORT_ITEMS);

    uint32_t key[SORT_ITEMS], val[SORT_ITEMS], rank[SORT_ITEMS];
#pragma unroll
    for (int j = 0; j < SORT_ITEMS; ++j) {
        uint32_t idx = warp_base + j * 32 + lane;
        bool ok = idx < n;
        key[j] = ok ? keys_in[idx] : 0xFFFFFFFFu;
        val[j] = ok ? (vals_in ? vals_in[idx] : idx) : 0u;
    }
    const unsigned lt = (1u << lane) - 1u;
    // warp multisplit: rank of each key among equal digits of this warp, in input order
#pragma unroll
    for (int j = 0; j < SORT_ITEMS; ++j) {
        uint32_t idx = warp_base + j * 32 + lane;
        bool ok = idx < n;
        uint32_t d = ok ? ((key[j] >> shift) & 0xFF) : RADIX;   // padding gets its own class
        unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
        uint32_t prior = ok ? whist[warp][d] : 0;
        __syncwarp();
        if (ok && (peers & lt) == 0) whist[warp][d] = prior + __popc(peers);
        __syncwarp();
        rank[j] = prior + __popc(peers & lt);
    }
    __syncthreads();
    // per digit (thread = digit): counts over warps -> warp prefixes, block total
    uint32_t total = 0;
    {
        const int d = tid;
#pragma unroll
        for (int w = 0; w < SORT_THREADS / 32; ++w) {
            uint32_t c = whist[w][d];
            whist[w][d] = total;
            total += c;
        }
    }
    // publish the aggregate, then look back for the exclusive prefix
    {
        const int d = tid;
        volatile uint32_t *lb = lookback;
        if (tile == 0) {
            lb[d] = LB_INC | total;
            glob_base[d] = digit_offs[d];
        } else {
            lb[(size_t)tile * RADIX + d] = LB_AGG | total;
            uint32_t excl = 0;
            int64_t t = (int64_t)tile - 1;
            long long spins = 0;
            while (t >= 0) {
                uint32_t v = lb[(size_t)t * RADIX + d];
                uint32_t st = stall ? 0u : (v & ~LB_MASK);      // (stall: a test's flag nothing sets)
                if (st == 0) {
                    if (++spins > spin_limit) { atomicOr(err, PSL_DEV_ERR_TIMEOUT); break; }
                    continue;
                }
                excl += v & LB_MASK;
                if (st == LB_INC) break;
                --t;
            }
            lb[(size_t)tile * RADIX + d] = LB_INC | (excl + total);
            glob_base[d] = digit_offs[d] + excl;
        }
    }
    // block-local exclusive offsets of each digit (scan of `total` over digits)
    blk_excl[tid] = total;
    __syncthreads();
    for (int off = 1; off < RADIX; off <<= 1) {
        uint32_t t = tid >= off ? blk_excl[tid - off] : 0;
        __syncthreads();
        blk_excl[tid] += t;
        __syncthreads();
    }
    uint32_t incl = blk_excl[tid];
    __syncthreads();
    blk_excl[tid] = incl - total;
    __syncthreads();
    // scatter into shared memory in block-sorted order
#pragma unroll
    for (int j = 0; j < SORT_ITEMS; ++j) {
        uint32_t idx = warp_base + j * 32 + lane;
        if (idx < n) {
            uint32_t d = (key[j] >> shift) & 0xFF;
            uint32_t pos = blk_excl[d] + whist[warp][d] + rank[j];
            s_keys[pos] = key[j];
            s_vals[pos] = val[j];
        }
    }
    __syncthreads();
    // write out: consecutive threads write consecutive positions of one digit run
    const uint32_t tile_n = (n - tile_base) < (uint32_t)TILE ? (n - tile_base) : (uint32_t)TILE;
    for (uint32_t i = tid; i < tile_n; i += SORT_THREADS) {
        uint32_t k = s_keys[i];
        uint32_t d = (k >> shift) & 0xFF;
        uint32_t dst = glob_base[d] + (i - blk_excl[d]);
        keys_out[dst] = k;
        vals_out[dst] = s_vals[i];
    }
}


__global__ void __launch_bounds__(256) k_digit_hist(const uint32_t *__restrict__ keys, uint32_t n, int passes,
                                                    uint32_t *hist) {
    __shared__ uint32_t h[SORT_MAX_PASSES * RADIX];
    for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint32_t k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&h[p * RADIX + ((k >> (8 * p)) & 0xFF)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

}  // namespace

size_t sort_pairs_scratch_bytes(uint32_t n) {
    uint32_t n_tiles = std::max<uint32_t>((n + TILE - 1) / TILE, 1);
    return (size_t)(SORT_HEAD_WORDS + (size_t)n_tiles * RADIX) * 4 + (size_t)std::max<uint32_t>(n, 1) * 16;
}

int sort_pairs_u32(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt, uint32_t n, int bits,
                   const uint32_t *hist_in, bool vals_identity, void *scratch_v, int *result_in_alt, cudaStream_t st) {
    *result_in_alt = 0;
    if (n == 0) return 0;
    int passes = std::max(1, (bits + 7) / 8);
    if (passes > SORT_MAX_PASSES) return -1;
    uint32_t n_tiles = (n + TILE - 1) / TILE;
    uint32_t *scratch = (uint32_t *)scratch_v;
    uint32_t *hist = scratch, *doffs = scratch + SORT_MAX_PASSES * RADIX, *err = doffs + SORT_MAX_PASSES * RADIX;
    uint32_t *tile_ctr = err + 1, *lookback = err + 4;
    static_assert(2 * SORT_MAX_PASSES * RADIX + 4 == SORT_HEAD_WORDS, "look-back table offset");
    cudaMemsetAsync(scratch, 0, SORT_HEAD_WORDS * 4, st);
    if (hist_in) cudaMemcpyAsync(hist, hist_in, passes * RADIX * 4, cudaMemcpyDeviceToDevice, st);
    else { k_digit_hist<<<std::min<uint32_t>((n + 255) / 256, 1184), 256, 0, st>>>(keys, n, passes, hist); PSL_NOTE_LAUNCH(); }
    k_digit_offsets<<<1, RADIX, 0, st>>>(hist, doffs, passes); PSL_NOTE_LAUNCH();
    uint32_t *kb[2] = {keys, keys_alt}, *vb[2] = {vals, vals_alt};
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        cudaMemsetAsync(tile_ctr, 0, 4, st);
        cudaMemsetAsync(lookback, 0, (size_t)n_tiles * RADIX * 4, st);
        { void *tk_ = nullptr; if (psl_timer_on()) psl_timer_begin(PK_ONESWEEP, st, &tk_); k_onesweep<<<n_tiles, SORT_THREADS, 0, st>>>(kb[cur], (p == 0 && vals_identity) ? nullptr : vb[cur], kb[cur ^ 1],
                                                     vb[cur ^ 1], n, 8 * p, doffs + p * RADIX, lookback, tile_ctr, err,
                                                     psl_wait_polls(SPIN_LIMIT), (psl_debug_flags() & PSL_DEBUG_LOOKBACK_STALL) != 0); PSL_NOTE_LAUNCH(); if (tk_) psl_timer_end(PK_ONESWEEP, st, tk_); }
        cur ^= 1;
    }
    *result_in_alt = cur;
    return 0;
}

uint32_t *sort_err_word(void *scratch_v) {
    return (uint32_t *)scratch_v + 2 * SORT_MAX_PASSES * RADIX;
}

// ------------------------------------------------------------------ scan --
namespace {
constexpr int SCAN_THREADS = 256, SCAN_ITEMS = 8, SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t *sh, int64_t *total) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= o) w += y;
        }
        sh[lane] = w;
    }
    __syncthreads();
    int64_t before = warp ? sh[warp - 1] : 0;
    *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_tile_sums(const int64_t *in, int64_t n, int64_t *sums) {
    __shared__ int64_t sh[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE, s = 0;
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        int64_t i = base + (int64_t)j * SCAN_THREADS + threadIdx.x;
        if (i < n) s += in[i];
    }
    int64_t tot;
    block_excl_scan(s, sh, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_sums(int64_t *sums, int64_t m) {
    __shared__ int64_t sh[32];
    int64_t carry = 0;
    for (int64_t c = 0; c < m; c += blockDim.x) {
        int64_t i = c + threadIdx.x;
        int64_t v = i < m ? sums[i] : 0, tot;
        int64_t e = block_excl_scan(v, sh, &tot);
        if (i < m) sums[i] = carry + e;
        carry += tot;
    }
}

__global__ void __launch_bounds__(SCAN_THREADS) k_tile_scan(const int64_t *in, int64_t n, const int64_t *sums,
                                                            int64_t *out) {
    __shared__ int64_t sh[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t v[SCAN_ITEMS], s = 0;
    // blocked arrangement: thread t owns items base + t*ITEMS .. +ITEMS-1
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + j;
        v[j] = i < n ? in[i] : 0;
        s += v[j];
    }
    int64_t tot;
    int64_t run = sums[blockIdx.x] + block_excl_scan(s, sh, &tot);
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        int64_t i = base + (int64_t)threadIdx.x * SCAN_ITEMS + j;
        if (i < n) out[i] = run;
        run += v[j];
        if (i == n - 1) out[n] = run;
    }
}
__global__ void k_zero1(int64_t *p) { *p = 0; }
}  // namespace

size_t scan_i64_scratch_bytes(int64_t n) { return (size_t)(std::max<int64_t>((n + SCAN_TILE - 1) / SCAN_TILE, 1)) * 8; }

void scan_i64(const int64_t *in, int64_t *out, int64_t n, void *scratch, cudaStream_t st) {
    if (n <= 0) { k_zero1<<<1, 1, 0, st>>>(out); PSL_NOTE_LAUNCH(); return; }
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    int64_t *sums = (int64_t *)scratch;
    k_tile_sums<<<(unsigned)tiles, SCAN_THREADS, 0, st>>>(in, n, sums); PSL_NOTE_LAUNCH();
    k_scan_sums<<<1, 1024, 0, st>>>(sums, tiles); PSL_NOTE_LAUNCH();
    k_tile_scan<<<(unsigned)tiles, SCAN_THREADS, 0, st>>>(in, n, sums, out); PSL_NOTE_LAUNCH();
}
