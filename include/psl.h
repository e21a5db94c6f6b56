/*
 * psl.h -- C ABI of the B300 phase-space-let (PSL) Monte Carlo dose path.
 *
 * The calls follow the paper's statement of the problem (Townson et al.,
 * "GPU-based Monte Carlo radiotherapy dose calculation using phase-space
 * sources"):
 *
 *   psl_build          Sec. 2.3.2  commission a phase space once: sort its
 *                                  records into PSLs by particle type, energy
 *                                  bin and position bin.
 *   psl_plan_create    Sec. 2.3.3  per treatment plan: select the PSLs inside
 *                                  each field's region of interest (Fig. 1)
 *                                  and give each selected PSL its share of the
 *                                  histories (the N_total^psl and P_ij
 *                                  equations).
 *   psl_source_batch   Sec. 2.2, 2.3.3, 2.4  read the particles of a range of
 *                                  histories in the paper's order (energy
 *                                  division by division, PSLs interleaved,
 *                                  random start and wrap), apply the jaw
 *                                  model, fluence map and MU weight, rotate
 *                                  and project them to the phantom surface.
 *   transport_run      Sec. 2.3.3  photon/electron transport with dose tallied
 *                                  by atomic counters, one tally per batch.
 *   dose_readout       Sec. 2.3.3, 2.5  dose, batch uncertainty and the
 *                                  normalisation factor.
 *
 * Conventions common to every call:
 *   - Return PSL_OK (0) on success or a negative PSL_E* code; the text of the
 *     last error of the calling thread is in psl_last_error().
 *   - Arrays in the structs below are DEVICE pointers owned by the caller
 *     unless a field says "host".  They must stay valid until the call that
 *     uses them has completed on its stream.
 *   - Handles (psl_store_t, psl_plan_t, psl_batch_t, psl_tally_t) are owned
 *     by the library and freed with the matching *_destroy call.  Store, plan
 *     and batch memory is allocated and freed stream-ordered on the stream of
 *     the call that created the handle: destroy them before that stream.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous on it unless stated otherwise; calls
 *     that size an allocation from device data synchronise that stream.
 *   - Determinism: the same inputs and seed give bitwise-identical integer
 *     tallies whatever the launch shape, the number of batches a history
 *     range is split into, or the order the ranges are run in.
 *   - Units: cm, MeV, g/cm^3, Gy, degrees.  The beam frame has the source at
 *     the origin and the beam travelling along +z; the isocentre is at
 *     (0, 0, SAD).
 */
#ifndef PSL_H
#define PSL_H

#include <stdint.h>

#if defined(__GNUC__)
#define PSL_API __attribute__((visibility("default")))
#else
#define PSL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define PSL_OK 0
#define PSL_EINVAL (-1)     /* bad argument or handle */
#define PSL_ENOMEM (-2)     /* device allocation failed */
#define PSL_ECUDA (-3)      /* a CUDA call failed (text in psl_last_error) */
#define PSL_ETIMEOUT (-4)   /* a bounded device-side wait gave up */
#define PSL_EOVERFLOW (-5)  /* a particle queue or tally headroom overflowed */

/* physics switches used by the tests; 0 in production */
#define PSL_PHYS_LOCAL_SECONDARIES 1u  /* secondaries deposit their energy in place */
#define PSL_PHYS_FIRST_INTERACTION 2u  /* photons deposit all at the first real interaction */
#define PSL_PHYS_NO_MSC 4u             /* electrons are not deflected by multiple scattering */
#define PSL_PHYS_NO_HARD 8u            /* electrons make no hard delta rays or bremsstrahlung */

/* source status of one history (psl_source_trace) */
#define PSL_SRC_TRANSPORT 0   /* accepted and entering the phantom */
#define PSL_SRC_JAW 1         /* stopped by a jaw (Sec. 2.2) */
#define PSL_SRC_FLUENCE 2     /* outside the fluence map (weight 0) */
#define PSL_SRC_ZERO_WEIGHT 3 /* fluence or weight zero */
#define PSL_SRC_MISS 4        /* accepted but its line misses the phantom */

/* Phase-space records at the PSL plane, structure of arrays (device, n each).
 * q: 0 photon, -1 electron, +1 positron.  w = +sqrt(1 - u^2 - v^2). */
typedef struct psl_records {
    const float *x, *y, *u, *v, *e, *wt;
    const int8_t *q;
    int64_t n;                 /* 0 <= n < 2^30 */
} psl_records_t;

/* PSL binning (Sec. 2.3.2).  Bins are half-open [edge_k, edge_k+1).  Records
 * outside [x_edges[0], x_edges[nx]) x [y_edges[0], y_edges[ny]) or with
 * e <= 0 belong to no PSL and are dropped.  Energies are binned by the
 * interior edges only (below e_edges[1]: bin 0; at or above
 * e_edges[n_ebins-1]: the last bin).  PSL id =
 * (type * n_ebins + energy bin) * nx * ny + y bin * nx + x bin, type 0 for
 * photons and 1 for electrons and positrons. */
typedef struct psl_params {
    int32_t nx, ny;            /* position bins, nx*ny*n_ebins*2 < 2^31 */
    int32_t n_ebins;           /* energy bins per type, >= 1 */
    int32_t apr_copies;        /* K >= 1: copies per record (azimuthal redistribution) */
    const float *x_edges;      /* host, nx+1 ascending */
    const float *y_edges;      /* host, ny+1 ascending */
    const float *e_edges;      /* host, n_ebins+1 ascending */
    float z_psl;               /* PSL plane, cm from the source */
    uint64_t apr_seed;         /* Philox key of the redistribution angles */
} psl_params_t;

/* Azimuthal particle redistribution (Sec. 2.3.1), applied by psl_build
 * before the PSL sort when apr_copies = K > 1.  Record i of the caller's
 * phase space becomes the K records j = i*K + c, c = 0..K-1: copy 0 is the
 * record as given, copy c > 0 is the record rotated about the beam axis
 * (x = y = 0) by its own uniform azimuth phi, position (x, y) and direction
 * cosines (u, v) alike, energy, weight and charge unchanged.  The angle:
 * Philox4x32-10 with key apr_seed and counter (b, PSL_TAG_APR, i, c) gives,
 * for b = 0, 1, ..., two candidate points per block, (a, b) = (2 U0 - 1,
 * 2 U1 - 1) and (2 U2 - 1, 2 U3 - 1) with U = ((word >> 9) + 0.5) 2^-23; the
 * first with a*a + b*b <= 1 gives cos phi = (a*a - b*b) / (a*a + b*b) and
 * sin phi = 2 a b / (a*a + b*b) (the doubled angle of a uniform point of the
 * disc is uniform); after 64 blocks without one, phi = 0.  Every operation
 * is one IEEE float32 operation rounded to nearest (no fused multiply-add),
 * so the rotated records are reproducible bit for bit on any IEEE machine:
 *   x' = x cos - y sin,  y' = x sin + y cos  (the same for u, v).
 * The store's input index of a copy is j, and a phase space of N records
 * with K copies stands for K*N incident particles in the dose normalisation
 * (Sec. 2.5).  K = 1 leaves the records as given. */
#define PSL_TAG_APR 3u
#define PSL_APR_MAX_BLOCKS 64

/* One treatment field (Sec. 2.2, 2.3.3, 2.4). */
typedef struct psl_beam {
    float x1, x2, y1, y2;      /* jaw edges projected to SAD, cm; x1 < x2, y1 < y2 */
    float z_jaw_x, z_jaw_y;    /* planes of the X and Y jaws, cm from the source */
    float gantry, collimator, couch;   /* degrees */
    float mu;                  /* monitor units, > 0 */
    float roi_margin;          /* cm added around the jaw opening at SAD for PSL selection */
    float iso[3];              /* isocentre in patient coordinates, cm */
    int32_t fnx, fny;          /* fluence map cells; 0 = no map */
    float fx0, fy0, fdx, fdy;  /* map corner and cell size at SAD, cm */
    const float *fluence;      /* device, fny*fnx row-major, or NULL */
} psl_beam_t;

/* Voxel phantom.  Voxel (ix, iy, iz) is element (iz*ny + iy)*nx + ix and
 * spans origin + [i, i+1) * voxel size. */
typedef struct psl_phantom {
    int32_t nx, ny, nz;
    float vx, vy, vz;          /* voxel size, cm */
    float origin[3];           /* patient coordinates of the (0,0,0) corner */
    const uint8_t *mat;        /* device, 0 water-like medium, 1 bone */
    const float *rho;          /* device, mass density g/cm^3, > 0 */
} psl_phantom_t;

/* Transport cut-offs (Sec. 2.6) and class-II thresholds.  psl_physics_default
 * fills photon_cut 0.010 MeV, electron_cut 0.700 MeV total energy (0.18900105
 * MeV kinetic), wcc = wcb = 0.200 MeV, flags 0. */
typedef struct psl_physics {
    float photon_cut, electron_cut, wcc, wcb;
    uint32_t flags;            /* PSL_PHYS_* */
} psl_physics_t;

typedef struct psl_store psl_store_t;
typedef struct psl_plan psl_plan_t;
typedef struct psl_batch psl_batch_t;
typedef struct psl_tally psl_tally_t;

PSL_API void psl_physics_default(psl_physics_t *out);

/* Sec. 2.3.2.  Compute every record's PSL id, sort the records stably by it
 * (LSD onesweep radix sort) and gather them into the store as 32-byte records
 * (x, y, u, v, e, wt, input index, q), with the bin offsets
 * offsets[0..n_bins] (offsets[n_bins] = records kept).  The store is
 * independent of the caller's arrays once the call has completed.
 * With apr_copies K > 1 the sorted records are the K redistributed copies
 * of every record (see PSL_TAG_APR above); records->n * K < 2^30.
 * Errors: PSL_EINVAL (sizes, edges, apr_copies < 1), PSL_ENOMEM, PSL_ECUDA,
 * PSL_ETIMEOUT (a look-back wait of the sort gave up). Synchronises stream. */
PSL_API int psl_build(const psl_params_t *params, const psl_records_t *records, psl_store_t **out, void *stream);

/* psl_build for callers that cannot allocate device memory: code running
 * inside another runtime's memory pool, under a fixed device-memory budget, or
 * in a process that must not call cudaMalloc after start-up.  The paper has
 * no counterpart; it is the same PSL sort written into caller arrays.
 * Scratch lives in one fixed device array of about 17 MB, part of the
 * library's device code: a CUDA context commits it when it loads that code
 * (with lazy module loading, at the first psl_build_static call in the
 * context) and holds it until the context ends, so a caller under a fixed
 * device-memory budget should make its first call at start-up.  Limits: at most
 * PSL_STATIC_MAX_RECORDS records, apr_copies = 1 (no redistribution) and
 * PSL_STATIC_MAX_EDGES bin edges
 * (nx+1 + ny+1 + n_ebins+1); larger inputs return PSL_EINVAL with the limit
 * in psl_last_error.  Outputs (device, caller-owned): offsets [n_bins+1]
 * int64 and sorted [n x 8] float32 (16-byte aligned) in the psl_store_read
 * record layout (the
 * first *n_valid rows are written); *n_valid (host) receives the records
 * kept.  The first call in each CUDA context looks up the array's device
 * address there (cudaGetSymbolAddress; a context created again after
 * cudaDeviceReset gets a lookup of its own), so make that first call before
 * any stream capture.
 * All calls share the array: calls that overlap on the GPU (other streams,
 * other threads) race and must be serialised by the caller.  Calls no
 * cudaMalloc, cudaFree or allocating library routine.  Synchronises stream. */
#define PSL_STATIC_MAX_RECORDS (1 << 20)
#define PSL_STATIC_MAX_EDGES 4096
PSL_API int psl_build_static(const psl_params_t *params, const psl_records_t *records, int64_t *offsets,
                             float *sorted, int64_t *n_valid, void *stream);

/* Sizes of a store (host outputs): records after redistribution (input
 * records x apr_copies), records kept in some PSL, PSL bins. */
PSL_API int psl_store_info(const psl_store_t *store, int64_t *n_records, int64_t *n_valid, int64_t *n_bins);

/* Copy the store out (device outputs, NULL to skip): offsets (n_bins+1
 * int64), perm (n_valid int64: input index of each sorted record), records
 * (n_valid x 8 float32: x y u v e wt, then the input index and q as int32
 * bit patterns). */
PSL_API int psl_store_read(const psl_store_t *store, int64_t *offsets, int64_t *perm, float *records, void *stream);

/* Sec. 2.3.3.  Select, for every beam, the PSLs whose position bin overlaps
 * the ROI: the jaw opening at SAD widened by roi_margin and scaled by
 * z_psl / sad (strict overlap: touching edges do not count).  Entry list =
 * beams in order, each beam's selected PSLs in PSL-id order.  With N_j the
 * records of the entry's PSL and C_k the sum of N_j over the entries before
 * entry k, entry k gets floor(N C_{k+1} / N_total) - floor(N C_k / N_total)
 * histories (N = n_histories, N_total = sum of N_j over all entries), so the
 * counts sum to N exactly.  Each entry reads its PSL from a random record
 * offset drawn from Philox(seed; beam, PSL id).  `beams` is a host array.
 * Requires 0 < n_histories < 2^62 and fewer than 2^32 - 1 histories for
 * every selected PSL (PSL_EINVAL otherwise).  Synchronises stream. */
PSL_API int psl_plan_create(const psl_store_t *store, const psl_beam_t *beams, int32_t n_beams, float sad,
                    int64_t n_histories, uint64_t seed, psl_plan_t **out, void *stream);

/* Plan sizes: entries, N_total^psl and the histories of the plan (host). */
PSL_API int psl_plan_info(const psl_plan_t *plan, int64_t *n_entries, int64_t *n_total_psl, int64_t *n_histories);

/* Copy per-entry arrays out (device int64 [n_entries] each, NULL to skip):
 * beam, PSL id, histories assigned, random start offset. */
PSL_API int psl_plan_read(const psl_plan_t *plan, int64_t *beam, int64_t *psl, int64_t *count, int64_t *offset,
                  void *stream);

/* Sec. 2.2, 2.3.3, 2.4.  Source stage for histories h = first + i * stride,
 * 0 <= i < n, of the plan (stride >= 1; the last must be < the plan's
 * histories).  Independent batches for the uncertainty estimate of Sec. 2.3.3
 * take first = b, stride = N_b, so that every batch samples every energy
 * division.  History h is mapped to (entry, read number k): energy divisions in
 * order, photons before electrons inside one; within that group, round r
 * reads one particle from every entry still owed more than r histories,
 * entries visited in order of decreasing count (ties: entry order).  The
 * record read is start + (offset + k) mod N_j.  Jaw test, fluence map and MU
 * weight are decided in float32 (round-to-nearest, no fused multiply-add):
 *   w   = sqrt((1 - u*u) - v*v)
 *   xj  = x + u * ((z_jaw_x - z_psl) / w), accepted if (x1*z_jaw_x)/sad <= xj <= (x2*z_jaw_x)/sad
 *   (same for y), fluence cell floor((x + u*((sad - z_psl)/w) - fx0) / fdx),
 *   weight = (wt * F) * mu_i/mu_total.
 * Survivors are rotated (collimator about z, gantry about y, couch about z,
 * about the isocentre) and moved along their line to its entry into the
 * phantom box.  The call only records the range: the source stage runs inside
 * transport_run, fused with the first photon pass (each lane that needs work
 * sources the next history), so the plan must stay alive until the batch has
 * been transported.  The phantom is read for its box only.  No device work,
 * no synchronisation. */
PSL_API int psl_source_batch(const psl_plan_t *plan, const psl_phantom_t *phantom, int64_t first_history,
                     int64_t n_histories, int64_t stride, psl_batch_t **out, void *stream);

/* The source stage of histories first + i * stride, 0 <= i < n, written out per history
 * (device outputs, NULL to skip): entry, read number k, sorted record
 * index, beam, status (PSL_SRC_*), state (n x 8 float32: x y z u v w e wt,
 * phantom-local entry point, only for PSL_SRC_TRANSPORT), particle type
 * (0 photon, 1 electron, 2 positron). */
PSL_API int psl_source_trace(const psl_plan_t *plan, const psl_phantom_t *phantom, int64_t first_history,
                     int64_t n_histories, int64_t stride, int64_t *entry, int64_t *use, int64_t *rec,
                     int32_t *beam, int8_t *status, float *state, int32_t *ptype, void *stream);

/* A batch made from caller particles (device arrays, n each): state n x 8
 * float32 (x y z u v w e wt, phantom-local), type (0/1/2) and particle id;
 * `seed` keys their random streams.  Used to transport given particles
 * (tests, other sources). */
PSL_API int psl_batch_from_particles(const float *state, const int32_t *ptype, const uint64_t *pid, int64_t n,
                             uint64_t seed, psl_batch_t **out, void *stream);

/* Methods 1 and 2 (Sec. 2.1, 2.2): the phase space read as an unsorted
 * stream and binned on the fly by particle type and energy, without the PSL
 * position bins.  History h = first + i, 0 <= i < n, reads record h mod N of
 * the caller's phase space (N = records->n; the stream recycled).
 *   method 2: a phase space above the collimators; the field's jaw model and
 *     fluence map decide acceptance and weight (Sec. 2.2, 2.4), as in the PSL
 *     path.
 *   method 1: a patient-dependent phase space that already holds the
 *     collimation: every record is accepted with its own weight.
 * Accepted particles are rotated into the patient and entered into the
 * phantom box as in the PSL path (a single field: MU weight 1).  Then the
 * paper's binning: 2 x n_ebins bins (photons; electrons and positrons; the
 * energy bin by the interior edges of e_edges, as psl_build), each holding
 * at most `capacity` particles; a bin that fills is sent to transport as one
 * group and emptied, and at the end of the stream the partly filled bins are
 * sent in bin order.  The groups come out in exactly that order: full groups
 * in the order of the stream position at which they filled, then the partial
 * ones.  The returned batch holds the accepted particles in group order
 * (photons from the front, electrons and positrons from the back), particle
 * id = history id, keyed by `seed`; transport_run transports it and adds the
 * emitted and missed energy of the stream to the ledger.  Particles that
 * miss the phantom are counted as emitted and escaped and not kept.
 * records: device SoA, caller-owned; e_edges: host, n_ebins+1 ascending;
 * beam: host, its fluence device.  0 <= n < 2^31, capacity >= 1.
 * Errors: PSL_EINVAL, PSL_ENOMEM, PSL_ECUDA, PSL_ETIMEOUT (sort look-back).
 * Synchronises stream. */
#define PSL_METHOD_PATIENT_DEPENDENT 1
#define PSL_METHOD_JAW_MODEL 2
PSL_API int psl_stream_bin(const psl_records_t *records, const float *e_edges, int32_t n_ebins,
                           const psl_beam_t *beam, int32_t method, float z_psl, float sad,
                           const psl_phantom_t *phantom, int64_t first_history, int64_t n_histories,
                           uint64_t seed, int64_t capacity, psl_batch_t **out, void *stream);

/* Groups of a batch from psl_stream_bin and the particles it kept (host
 * outputs); the stream's emitted and missed energy in fixed point (2^-32
 * MeV per unit weight). */
PSL_API int psl_stream_info(const psl_batch_t *batch, int64_t *n_groups, int64_t *n_kept,
                            int64_t *emitted_fp, int64_t *missed_fp);

/* The groups in transport order (device int64 outputs, NULL to skip): bin
 * (type * n_ebins + energy bin), particle count, and for each kept particle
 * in group order its history id.  Particles that missed the phantom are not
 * in any group. */
PSL_API int psl_stream_read(const psl_batch_t *batch, int64_t *group_bin, int64_t *group_count,
                            int64_t *history, void *stream);

/* The particles of a batch from psl_batch_from_particles or psl_stream_bin
 * (device outputs, NULL to skip): photons first, then electrons and
 * positrons, each in the batch's transport order: state n x 8 float32
 * (x y z u v w e wt, phantom-local), type, particle id.  n = photons +
 * charged particles of psl_batch_info.  PSL_EINVAL for a batch from
 * psl_source_batch (its particles exist only inside transport_run). */
PSL_API int psl_batch_read(const psl_batch_t *batch, float *state, int32_t *ptype, uint64_t *pid, void *stream);

/* Histories (or caller particles) in a batch, and its photon and charged
 * particle counts (-1 for a batch from psl_source_batch: known only once
 * transported). */
PSL_API int psl_batch_info(const psl_batch_t *batch, int64_t *n_histories, int64_t *n_photons, int64_t *n_electrons);

/* Tally slices (batches, Sec. 2.3.3).  A history's deposits all go to one
 * slice; with PSL_SLICE_BY_HISTORY the history ids are cut into blocks of
 * PSL_BATCH_BLOCK consecutive ids and block B = id / PSL_BATCH_BLOCK goes to
 * slice floor(r n_batches / 2^32), r the first word of Philox(key = seed;
 * counter = (0, 4, B)), so every slice is an independent pseudo-random
 * subset of blocks of the reading order, whatever order they are read in,
 * and the batch standard deviation is a valid uncertainty.
 * 1 <= n_batches <= PSL_MAX_BATCHES. */
#define PSL_BATCH_BLOCK 256
#define PSL_SLICE_BY_HISTORY (-1)
#define PSL_MAX_BATCHES 1024

/* One int64 tally of nz*ny*nx voxels per batch, plus a 12-slot ledger:
 * 0 emitted, 1 escaped, 2 deposited (fixed point, 2^-32 MeV per unit
 * weight), 3 Compton, 4 photoelectric and 5 pair events, 6 electron steps,
 * 7 errors, 8 tally atomics issued by photon passes, 9 by electron passes,
 * 10 Woodcock (photon) steps, 11 hard Moller (e-) and Bhabha (e+) collisions.
 * Slot 2 is the sum of the tally's counters: psl_tally_read and dose_readout
 * take it from them (in the array of psl_tally_buffers it holds the value
 * the last of those calls took).  The phantom must have fewer
 * than 2^31 voxels (PSL_EINVAL otherwise): transport indexes voxels in
 * 32 bits. */
PSL_API int psl_tally_create(const psl_phantom_t *phantom, int32_t n_batches, psl_tally_t **out);
PSL_API int psl_tally_reset(psl_tally_t *tally, void *stream);

/* Order in which psl_run visits its history range (the dose is the same
 * bit for bit in every order: integer counters, per-history streams).
 * PSL_ORDER_READING: the range in reading order, every pass depositing into
 * all n_batches slices.  PSL_ORDER_BATCH: windows of the range's batch
 * blocks are partitioned by batch (a stable sort of the blocks' batch
 * indices) and run batch by batch, so a pass deposits into one slice; this keeps the
 * hot part of a tally larger than about half the L2 cache resident (the
 * 30x30 CT and IMRT tallies of 128^3 and 128x128x100 voxels x 10 batches are
 * 168 and 131 MB).  PSL_ORDER_AUTO (the default): batch by batch when the
 * tally (voxels x n_batches x 8 bytes) exceeds half the device's L2 and
 * n_batches > 1.  The batch order holds, per tally, 16 bytes per batch
 * block of a window (at most 2^24 blocks: ~n_batches x the queue depth /
 * PSL_BATCH_BLOCK) and the sort's scratch, allocated by the first psl_run
 * that uses it.  Returns PSL_EINVAL for other values. */
#define PSL_ORDER_AUTO 0
#define PSL_ORDER_READING 1
#define PSL_ORDER_BATCH 2
PSL_API int psl_tally_set_order(psl_tally_t *tally, int32_t order);

/* Device addresses of the tally's own counters (outputs, NULL to skip):
 * int64 [n_batches][nvox] (the psl_tally_read layout) and the int64 [12]
 * ledger.  Owned by the tally, valid until psl_tally_destroy.  They are for
 * combining tallies of one plan run in pieces by several processes (Sec.
 * 2.3.3: a job split over GPUs): after every rank's transport has completed,
 * an element-wise integer SUM of both arrays across the ranks (for example
 * an NCCL all-reduce in place) leaves on every rank the tally of the whole
 * history range, bit for bit, since the counters are integers and each
 * history is run on one rank only; dose_readout then reads it as usual.  The
 * caller orders its own work on these arrays with the library's streams. */
PSL_API int psl_tally_buffers(psl_tally_t *tally, int64_t **tallies, int64_t **ledger);

/* Sizes of a tally (host outputs, NULL to skip): its int64 counters
 * (n_batches x voxels, the array of psl_tally_buffers); the device bytes of its transport workspace (0 until the first
 * transport call sizes it: particle queues of 33 x 48 bytes per primary of
 * a pass, i.e. 1584 bytes x the queue depth when a call runs at least that
 * many histories, else x the call's histories; plus 4 bytes per voxel and
 * the batch-order buffers); the queue depth (primaries per transport pass)
 * and the persistent grid (256-thread blocks per SM) later calls use. */
PSL_API int psl_tally_info(const psl_tally_t *tally, int64_t *n_counters, int64_t *workspace_bytes,
                           int64_t *queue_depth, int32_t *blocks_per_sm);

/* Set the queue depth (primaries per transport pass, 2^12 <= depth <= 2^26;
 * default 2^24) of later transport calls on the tally: the bound on its
 * transport workspace (1584 bytes per primary of a pass), for callers that
 * share the device.  A workspace sized for a larger depth is kept until the
 * tally is destroyed.  PSL_EINVAL outside the range. */
PSL_API int psl_tally_set_queue_depth(psl_tally_t *tally, int64_t depth);

/* Sec. 2.2, 2.3.3, 2.4: a record of the production source stage.  Later
 * psl_run and transport_run calls on the tally write, for every history h
 * in [first, first + n) that they source, at index h - first (device
 * arrays, caller-owned, NULL to skip): the plan entry, its read number k,
 * the sorted record index, the status (PSL_SRC_*), the particle type (0
 * photon, 1 electron, 2 positron) and, for PSL_SRC_TRANSPORT only, the state
 * (8 float32: x y z u v w e wt, phantom-local) - the same quantities
 * psl_source_trace computes, here from the source kernel that feeds
 * transport (reading order or batch by batch).  n = 0 turns the record
 * off.  The arrays must stay valid while it is on.  A CUDA graph of
 * psl_run is captured again when the record changes.  For tests and
 * diagnostics; it costs nothing when off.  PSL_EINVAL for first < 0 or
 * n < 0. */
PSL_API int psl_tally_trace_source(psl_tally_t *tally, int64_t first, int64_t n, int64_t *entry, int64_t *use,
                                   int64_t *rec, int8_t *status, float *state, int32_t *ptype);

/* Copy raw tallies (device int64 [n_batches][nvox]: batch b's voxels at
 * b * nvox, the layout the tally keeps, so that one batch's slice is
 * contiguous for the batch-by-batch order) and ledger (device int64 [12])
 * out; NULL to skip. */
PSL_API int psl_tally_read(const psl_tally_t *tally, int64_t *tallies, int64_t *ledger, void *stream);

/* Sec. 2.3.3.  Transport every particle of the batch and its secondaries
 * through the phantom and add the deposits to tally slice `batch_index`, or,
 * with PSL_SLICE_BY_HISTORY, to the slice of each particle's history (for
 * caller particles: of its particle id).
 * Photons: Woodcock tracking, Klein-Nishina Compton (Kahn), photoelectric,
 * pair.  Electrons/positrons: class-II condensed history, restricted Bethe
 * stopping (Moller form for electrons, Bhabha form for positrons), hard
 * Moller (e-) or Bhabha (e+) collisions and bremsstrahlung, Highland
 * multiple scattering; a positron that stops annihilates into two 0.511 MeV
 * photons.
 * Electrons are grouped by energy band before each transport pass so that a
 * warp steps one band.  Deposits are rounded to int64 in units of 2^-32
 * MeV and added atomically.  The batch is consumed (transport it once).
 * Errors: PSL_EOVERFLOW if a secondary queue overflowed (tally incomplete).
 * Synchronises stream. */
PSL_API int transport_run(const psl_phantom_t *phantom, const psl_physics_t *physics, psl_batch_t *batch,
                  psl_tally_t *tally, int32_t batch_index, void *stream);

/* transport_run that also adds, per history (or caller particle) i of the
 * batch, its deposited and escaped fixed-point energy and its event count
 * (device arrays of the batch's n_histories, added to).  At most 2^22
 * histories (or particles) per traced batch. */
PSL_API int transport_trace(const psl_phantom_t *phantom, const psl_physics_t *physics, psl_batch_t *batch,
                    psl_tally_t *tally, int32_t batch_index, int64_t *hist_dep, int64_t *hist_esc,
                    int32_t *hist_events, void *stream);

/* Sec. 2.3.3, all fields of a plan in one call (the batched IMRT launch).
 * Runs histories [first, first+n) of the plan in reading order (or window by
 * window, batch by batch: see psl_tally_set_order), each
 * history's deposits into its tally slice (PSL_SLICE_BY_HISTORY): source
 * stage and transport of every beam/segment, in chunks of the queue depth,
 * each chunk's secondaries joining the next chunk's passes, with no host
 * synchronisation until the last chunk; its secondaries are then drained
 * generation by generation: 3 generations launched unchecked, after which
 * the host reads the queue counts once per further generation.  use_graph = 1
 * records the whole sequence once as a CUDA graph with a fixed budget of 10
 * drain generations (kernels of an empty generation exit at once), keeps it
 * in the tally for this plan, range, phantom and settings, and replays it
 * with a single launch on `stream`; the first such call sets up outside the
 * capture.  Synchronises stream at the end; PSL_EOVERFLOW if a queue
 * overflowed or secondaries were left after the budget. */
PSL_API int psl_run(const psl_plan_t *plan, const psl_phantom_t *phantom, const psl_physics_t *physics,
                    psl_tally_t *tally, int64_t first, int64_t n, int32_t use_graph, void *stream);

/* Autotuner for psl_run: times the plan's first histories with each
 * candidate persistent-grid size (2, 3, 4, 6 blocks of 256 threads per SM)
 * and queue depth (2^21 ... 2^26 primaries per transport pass; depths above
 * the plan's histories, or whose workspace would take more than 80 % of the
 * free device memory, are skipped), each on max(n_probe, 2 x depth)
 * histories (capped at the plan's), keeps the fastest in histories per
 * second in the tally (used by later transport calls on it), clears the
 * tally, and returns the choice (host outputs, may be NULL). */
PSL_API int psl_autotune(const psl_plan_t *plan, const psl_phantom_t *phantom, const psl_physics_t *physics,
                         psl_tally_t *tally, int64_t n_probe, int32_t *blocks_per_sm, int64_t *queue_depth,
                         void *stream);

/* Sec. 2.3.3 and 2.5: the whole dose computation of a plan that is run
 * again and again (a service recomputing one plan, a denoiser's training
 * runs) as one CUDA graph launch: the tally is cleared, histories
 * [first, first+n) of the plan are run as psl_run runs them, and the dose is
 * read out with dose_readout's arguments (norm, dose, sigma, ledger: device,
 * NULL to skip).  The graph is recorded by the first call for this plan,
 * range, phantom, settings and outputs (outside any other capture) and kept
 * in the tally; later calls replay it in one launch.  Synchronises stream;
 * errors as psl_run. */
PSL_API int psl_plan_replay(const psl_plan_t *plan, const psl_phantom_t *phantom, const psl_physics_t *physics,
                            psl_tally_t *tally, int64_t first, int64_t n, double norm, double *dose, double *sigma,
                            double *ledger, void *stream);

/* Sec. 2.3.2, 2.3.3 ("the size of the PSL bins ... benchmarking"): autotune
 * the PSL position-bin size for a plan.  For every candidate cell size
 * cell_cm[k] (> 0, cm) the store is built from the records with square
 * cells over the extent of params' x and y edges (rounded to a whole number
 * of cells; energy bins as given), the plan of n_histories created, and
 * n_probe of its histories run on a tally of n_batches (once to warm up,
 * once timed).  plan_seconds[k] (host, may be NULL) receives the estimate
 * plan creation + probe time x n_histories / n_probe; *best_cell (host, may
 * be NULL) the fastest size.  The dose does not depend on the cell size
 * (every selected PSL's records are sampled in proportion), only the time
 * does.  Synchronises stream. */
PSL_API int psl_autotune_bins(const psl_params_t *params, const psl_records_t *records, const psl_beam_t *beams,
                              int32_t n_beams, float sad, const psl_phantom_t *phantom, const psl_physics_t *physics,
                              int64_t n_histories, uint64_t seed, int32_t n_batches, const float *cell_cm,
                              int32_t n_cells, int64_t n_probe, float *best_cell, double *plan_seconds, void *stream);

/* Sec. 2.3.3 and 2.5.  dose[v] = norm * sum_b T_bv * 2^-32 MeV * 1.602176634e-13
 * J/MeV / (rho_v * voxel volume * 1e-3 kg), sigma[v] = the standard error of
 * the mean of the N_b batch estimates, ledger[0..2] = emitted, escaped,
 * deposited energy in MeV (FP64).  dose, sigma: device float64 [nvox];
 * ledger: device float64 [3]; any may be NULL. */
PSL_API int dose_readout(const psl_tally_t *tally, const psl_phantom_t *phantom, double norm, double *dose,
                 double *sigma, double *ledger, void *stream);

/* Sec. 2.5: the normalisation factor of dose_readout,
 *   norm = calibration * N_total^psl / (n_histories * N_incident),
 * the paper's D = D_o N_total^phsp / (N_simulated N_incident) with the
 * records of the PSLs the plan selected (N_total^psl, psl_plan_info) in place
 * of the whole phase space, since the simulated histories are drawn from
 * them only.  n_histories: the histories whose deposits the tally holds (all
 * ranks of a split job together).  n_incident: the particles incident on the
 * accelerator that the phase space stands for; 0 takes the plan's store
 * records (input records x redistribution copies), the reading for a
 * synthetic phase space that is its own incident set.  calibration: the
 * absolute dose calibration factor (> 0; 1 for none).  Host output *norm.
 * PSL_EINVAL for a null plan or output, n_histories <= 0, n_incident < 0 or
 * calibration <= 0.  No device work. */
PSL_API int psl_dose_normalisation(const psl_plan_t *plan, int64_t n_histories, int64_t n_incident,
                                   double calibration, double *norm);

/* Destroy functions free what the handle owns (NULL is ignored).  A tally's
 * transport workspace (its particle queues, ~30 x 48 B per primary of a
 * pass: 26 GB at the default 2^24 primaries per pass) is not freed but kept
 * for the next tally created on the same device (at most one is kept), since
 * mapping it again costs ~14 ms; psl_tally_destroy first waits for the
 * device.  psl_memory_trim frees it. */
PSL_API void psl_store_destroy(psl_store_t *store);
PSL_API void psl_plan_destroy(psl_plan_t *plan);
PSL_API void psl_batch_destroy(psl_batch_t *batch);
PSL_API void psl_tally_destroy(psl_tally_t *tally);

/* Opt-in timing of the main kernels with CUDA events recorded on the stream
 * each kernel is launched on.  psl_profile(1) clears the totals and starts
 * recording, psl_profile(0) stops; psl_profile_read returns, for kernel
 * index 0 <= k < PSL_NK (key, onesweep, gather, source, photon, electron,
 * band_sort, readout, conv3d: the denoiser's convolutions), the summed
 * device time in ms, the launches timed and the kernel's name (static
 * string).  Reading waits for the recorded events. */
#define PSL_NK 9
PSL_API int psl_profile(int enable);
PSL_API int psl_profile_read(int32_t kernel, double *total_ms, int64_t *launches, const char **name);

/* Diagnostic: measured throughput (updates/s) of int64 atomic adds into an
 * array of n_cells int64 counters (pseudo-random cells, as dose deposits
 * land), used as the peak of the transport kernels' tally roofline.
 * Allocates and frees the cells on `stream`; synchronises it. */
PSL_API int psl_atomic_peak(int64_t n_cells, int64_t n_updates, double *updates_per_s, void *stream);

/* Failure-detection hooks for tests (process-wide; psl_debug_waits(0, 0, 0)
 * restores the defaults).  Every device-side wait of the library is bounded
 * and gives up with an error status instead of hanging: the onesweep sort's
 * look-back (psl_build, psl_build_static, psl_stream_bin, psl_plan_create)
 * returns PSL_ETIMEOUT, the photon pass's staged queue feed (an mbarrier
 * wait) makes transport_run / psl_run return PSL_ETIMEOUT with the tally
 * incomplete.  polls > 0 sets how many times such a wait polls before it
 * gives up (default: about a second's worth).  flags make a wait wait on
 * something that never comes, so that the limit runs out:
 *   PSL_DEBUG_LOOKBACK_STALL  a sort tile never sees its predecessors'
 *                             counts (every tile but the first gives up; the
 *                             sort's output is then wrong but in bounds);
 *   PSL_DEBUG_FEED_STALL      no chunk a photon warp claims into its second
 *                             buffer is ever copied, so that buffer's
 *                             mbarrier never completes (no copy is left in
 *                             flight when the warp stops; a pass needs more
 *                             photons than one chunk per warp for it).
 * queue_cap > 0 caps every particle queue of later transport calls at that
 * many particles, so that secondaries overflow it (PSL_EOVERFLOW, tally
 * incomplete).  Nothing here faults or hangs the device.  PSL_EINVAL for
 * negative values or unknown flags. */
#define PSL_DEBUG_LOOKBACK_STALL 1u
#define PSL_DEBUG_FEED_STALL 2u
PSL_API int psl_debug_waits(int64_t polls, uint32_t flags, int64_t queue_cap);

/* Number of kernels this library has launched in this process (all threads);
 * a diagnostic for counting the launches of a timed region. */
PSL_API int64_t psl_kernel_launches(void);

/* Dose comparison by the global gamma index (the paper's Sec. 3 criteria,
 * e.g. 2 % / 2 mm): the fraction of reference voxels with D_ref >= threshold
 * * max(ref) whose gamma <= 1.  Gamma at a reference voxel is the minimum
 * over evaluated points r within max_radius_cm (<= 0: 1.5 dta) of
 * sqrt(|r - r_ref|^2 / dta^2 + (D_ev(r) - D_ref)^2 / (dose_crit max ref)^2),
 * D_ev trilinear between voxel centres, on a grid of voxel / upsample
 * (1..16); points outside the volume are skipped.  ref, ev: device float64
 * [nz][ny][nx]; voxel sizes in cm; outputs on the host.  FP64 throughout.
 * Synchronises stream. */
PSL_API int psl_gamma(const double *ref, const double *ev, int32_t nx, int32_t ny, int32_t nz, float vx, float vy,
                      float vz, double dose_crit, double dta_cm, double threshold, int32_t upsample,
                      double max_radius_cm, double *pass_rate, int64_t *n_evaluated, void *stream);

/* The library takes its stream-ordered scratch (psl_build, psl_plan_create,
 * psl_stream_bin, batches) from its own device memory pool, one per device,
 * which keeps freed blocks for the next call.  psl_memory_trim frees the
 * transport workspace kept from a destroyed tally on the current device,
 * waits for the device (cudaDeviceSynchronize), then returns pool memory
 * beyond keep_bytes to the driver; *held_bytes (may be NULL) receives what
 * the pool still reserves.  Errors: PSL_ECUDA. */
PSL_API int psl_memory_trim(uint64_t keep_bytes, uint64_t *held_bytes);

/* Text of the calling thread's last error ("" if none). */
PSL_API const char *psl_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PSL_H */
