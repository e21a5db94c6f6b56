// Device sort and scan primitives shared by the PSL build and the plan builder.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define SORT_MAX_PASSES 4
// Keys one onesweep block ranks (its tile): 256 threads x 16 keys.  The
// look-back table of sort_pairs_u32 holds 256 words per tile.
#define SORT_TILE 4096
// 32-bit words of sort_pairs_u32's scratch before the look-back table:
// digit histograms and offsets, the error word, the tile counter.
#define SORT_HEAD_WORDS (2 * SORT_MAX_PASSES * 256 + 4)

// Scratch needed by sort_pairs_u32 for n keys (bytes).
size_t sort_pairs_scratch_bytes(uint32_t n);

// Stable LSD radix sort of (keys, vals) on the low `bits` bits of the keys,
// ping-ponging with (keys_alt, vals_alt).  vals_identity: the input values
// are the indices 0..n-1 and `vals` is only storage.  hist_in: optional
// precomputed digit histograms
// (passes x 256).  *result_in_alt tells which buffer pair holds the result.
// The error word (sort_err_word) gets PSL_DEV_ERR_TIMEOUT if a look-back
// wait gave up.  Returns -1 if bits > 32.
int sort_pairs_u32(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt, uint32_t n, int bits,
                   const uint32_t *hist_in, bool vals_identity, void *scratch, int *result_in_alt, cudaStream_t st);
uint32_t *sort_err_word(void *scratch);

// Exclusive scan of int64 in[0..n) into out[0..n], out[n] = total.
size_t scan_i64_scratch_bytes(int64_t n);
void scan_i64(const int64_t *in, int64_t *out, int64_t n, void *scratch, cudaStream_t st);
