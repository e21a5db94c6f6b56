/*
 * Oracle of the on-the-fly particle binning of Methods 1 and 2 (Sec. 2.1,
 * Sec. 2.2) -- TEST INFRASTRUCTURE, loaded only by the tests, the package
 * smoke check and the benchmark's CPU-baseline leg.  Shares no code with the
 * CUDA library.
 *
 * The paper's steps, in its order: particles arrive one after another from
 * the phase-space stream; each goes into the bin of its type and energy; a
 * bin holds at most `capacity` particles and, once full, its particles are
 * sent to the GPU as one group and the bin is emptied; when the stream ends,
 * the bins that still hold particles are sent as well.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* key[i]: bin of stream particle i in [0, nbins), or -1 if it is not binned
 * (rejected by the collimator model).  Outputs: group_bin[g] and
 * group_count[g] for every group in the order the groups are sent, and
 * order[] the stream indices of the particles in that order.  The bins left
 * at the end of the stream are sent in bin order.  Returns the number of
 * groups, or -1 on bad arguments or memory exhaustion. */
int64_t ora_stream_bin(int64_t n, const int32_t *key, int32_t nbins, int64_t capacity, int64_t *group_bin,
                       int64_t *group_count, int64_t *order) {
    if (n < 0 || nbins <= 0 || capacity < 1) return -1;
    int64_t *total = calloc((size_t)nbins, sizeof(int64_t));
    int64_t *fill = calloc((size_t)nbins, sizeof(int64_t));
    int64_t **bin = calloc((size_t)nbins, sizeof(int64_t *));
    if (!total || !fill || !bin) { free(total); free(fill); free(bin); return -1; }
    for (int64_t i = 0; i < n; ++i)
        if (key[i] >= 0 && key[i] < nbins) total[key[i]]++;
    int ok = 1;
    for (int32_t b = 0; b < nbins && ok; ++b) {
        int64_t size = total[b] < capacity ? total[b] : capacity;
        if (size > 0) ok = (bin[b] = malloc((size_t)size * sizeof(int64_t))) != NULL;
    }
    int64_t groups = 0, sent = 0;
    if (ok) {
        for (int64_t i = 0; i < n; ++i) {              /* the stream, in order */
            int32_t b = key[i];
            if (b < 0 || b >= nbins) continue;
            bin[b][fill[b]++] = i;
            if (fill[b] == capacity) {                 /* a full bin goes to transport */
                group_bin[groups] = b;
                group_count[groups] = capacity;
                memcpy(order + sent, bin[b], (size_t)capacity * sizeof(int64_t));
                sent += capacity;
                groups++;
                fill[b] = 0;
            }
        }
        for (int32_t b = 0; b < nbins; ++b) {         /* end of the stream */
            if (fill[b] == 0) continue;
            group_bin[groups] = b;
            group_count[groups] = fill[b];
            memcpy(order + sent, bin[b], (size_t)fill[b] * sizeof(int64_t));
            sent += fill[b];
            groups++;
        }
    }
    for (int32_t b = 0; b < nbins; ++b) free(bin[b]);
    free(bin); free(fill); free(total);
    return ok ? groups : -1;
}
