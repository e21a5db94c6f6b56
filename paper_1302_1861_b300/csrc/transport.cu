// transport_run (Sec. 2.3.3): photon and electron transport through the voxel
// phantom with 64-bit fixed-point dose counters.
//
// Work is organised as generations of typed queues.  A photon pass moves
// every photon of its queue to the end of its life (Woodcock tracking) and
// appends the charged secondaries to the electron queue; the electron queue
// is then regrouped by energy band (counting sort on 32 log bands) so that
// consecutive particles - and therefore warps - step one type and one band;
// an electron pass moves each electron to its cut-off, appending delta rays
// to the next electron queue and bremsstrahlung / annihilation photons to
// the next photon queue.  Passes repeat until the queues are empty.
//
// Inside a pass each lane owns one particle and runs one event per loop
// iteration; a lane whose particle ends takes the next queue entry
// (warp-aggregated atomic), so warps stay full until the queue drains.
// Every particle draws from its own Philox stream keyed by its id, and
// secondaries get ids derived from (parent id, ordinal), so the integer tally
// does not depend on how particles are scheduled.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "physics.cuh"
#include "psl_internal.cuh"
#include "source.cuh"
#include "sort.cuh"

namespace {

constexpr int NT = 2048;                  // table nodes
constexpr double T_LO = 1.0e-3, T_HI = 30.0;
constexpr int NBANDS = 32;
constexpr float F_ME = 0.51099895f;
constexpr int MAX_E_STEPS = 100000;
constexpr int MAX_GEN = 64;
constexpr unsigned FULL = 0xFFFFFFFFu;
#ifndef PSL_BAND_DESC
#define PSL_BAND_DESC 1
#endif
#ifndef SRC_RUN
#define SRC_RUN 256u                   // consecutive histories a warp of the source stage takes at a time
#endif
#ifndef SRC_ILP
#define SRC_ILP 1                      // histories a lane of the source stage looks up at once (2-4 need
#endif                                 // 80-126 registers; the lost occupancy cost more than they gained)
#ifndef SRC_MIN_BLOCKS
#define SRC_MIN_BLOCKS 4               // resident 256-thread source blocks per SM (register cap 64)
#endif
#ifndef PSL_G_DEFER
#define PSL_G_DEFER 28                 // lanes with a pending real photon interaction before a warp runs them
#endif
#ifndef PSL_G_INNER
#define PSL_G_INNER 3                  // Woodcock steps a photon may take in one pass of the photon loop
#endif
#ifndef PSL_E_CLAIM
#define PSL_E_CLAIM 32                 // electron queue entries a warp claims with one atomic (the refills of
#endif                                 // ~17 loop passes: one atomic's latency per claim, not per refill)
#ifndef PSL_E_DEFER
#define PSL_E_DEFER 2                  // lanes with a pending hard event before a warp runs them
#endif
#ifndef PSL_DEP_COMBINE
#define PSL_DEP_COMBINE 0              // 1: an electron sums its consecutive deposits into one voxel in
#endif                                 //    registers and adds them with one atomic when it leaves the voxel
#ifndef PSL_PHOTON_MIN_BLOCKS
#define PSL_PHOTON_MIN_BLOCKS 3        // resident 256-thread photon blocks per SM (register cap 80)
#endif
#ifndef PSL_TRANSPORT_MIN_BLOCKS
#define PSL_TRANSPORT_MIN_BLOCKS 4     // resident 256-thread blocks per SM (register cap 64)
#endif

// Charged-particle tables hold the electron's NT nodes, then the positron's
// (species offset NT): the species of a particle selects its rows.
struct Tables {
    const float4 *ph0, *ph1;   // material 0/1: mu_c, mu_pe, mu_pp, mu_total (cm^2/g)
    const float4 *el;          // [2][NT] S_restricted (MeV cm^2/g), sigma_moller or sigma_bhabha, sigma_brem (cm^2/g), 0
    const float4 *rng;         // [2][NT] CSDA range on node interval i: R = c0 + g (c1 + g (c2 + g c3)), g in [0, 1]
    const float *irng;         // [2][NT] ln T at uniform steps of ln R (inverse range)
    float lnE0, inv_dln;
    float dln;                 // 1 / inv_dln, rounded to float (the node spacing in ln E)
    float lnR0[2], inv_dlnR[2];  // grid of each species' inverse range table
};

// A thread's ledger counts, in few registers: steps and tally atomics, the
// escaped energy, and the event counts packed 21 bits each into one word
// (photon kernel: Compton, photoelectric, pair; electron kernel: hard
// collisions in the first field); a thread handles far fewer than 2^21
// events of a kind in one launch.  The deposited total is not counted: it is
// the sum of the tally, taken when the tally is read.
struct Acc {
    uint32_t steps, atomics;
    unsigned long long esc, ev;
};
constexpr int NLEDGER = 12;
constexpr unsigned long long EV_COMPTON = 1ull, EV_PHOTO = 1ull << 21, EV_PAIR = 1ull << 42, EV_HARD = 1ull;

struct Args {
    int nx, ny, nz;
    float vx, vy, vz, ivx, ivy, ivz;
    const uint8_t *mat;
    const float *rho;
    const float *mrho;        // rho, negated for bone (one load per lookup)
    const int *rmax;          // largest density of each material (float bits), phantom dependent
    float pcut, ecut, wcc, wcb;
    uint32_t flags;
    uint64_t seed;
    uint32_t k0, k1;          // the seed's two words (Philox key)
    uint32_t rk[20];          // Philox key schedule of the seed
    Tables tab;
    unsigned long long *tally;  // [slice][voxel] (a history's slice is in its root word)
    int64_t nvox;
    uint32_t n_slices;
    unsigned long long *ledger;
    unsigned long long *hist_dep, *hist_esc;
    int32_t *hist_events;
    uint32_t *err;
    Queue e_out, p_out;
    float band_ln0, band_scale;
    uint32_t *band_hist;      // band counts of the electrons queued for the next regrouping
    uint32_t wait_polls;      // polls of a bounded wait before it gives up
    uint32_t dbg;             // failure-detection stalls (PSL_DEBUG_*)
};

// The transport kernels' arguments with a compile-time switch for the
// per-history record of transport_trace (tests): the production instances
// (TR = false) compile without its checks and atomics.
template <bool TR> struct ArgsT : Args {
    static constexpr bool trace = TR;
};

// ----------------------------------------------------------- tables ------
__global__ void k_tables(float4 *ph0, float4 *ph1, float4 *el, double wcc, double wcb) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NT) return;
    const double lnE = log(T_LO) + (log(T_HI) - log(T_LO)) * i / (NT - 1);
    const double E = exp(lnE);
    double mc, mpe, mpp;
    ph_mu_rho(E, 0, mc, mpe, mpp);
    ph0[i] = make_float4((float)mc, (float)mpe, (float)mpp, (float)(mc + mpe + mpp));
    ph_mu_rho(E, 1, mc, mpe, mpp);
    ph1[i] = make_float4((float)mc, (float)mpe, (float)mpp, (float)(mc + mpe + mpp));
    el[i] = make_float4((float)el_stop_restricted(E, wcc, wcb), (float)el_moller_sigma(E, wcc),
                        (float)el_brem_sigma(E, wcb), 0.f);
    el[NT + i] = make_float4((float)pos_stop_restricted(E, wcc, wcb), (float)pos_bhabha_sigma(E, wcc),
                             (float)el_brem_sigma(E, wcb), 0.f);
}

// CSDA range with the restricted stopping power: R_i = integral from T_0 to
// T_i of dT/S, each interval by 8-point Gauss-Legendre in double (one thread
// per interval), then a running sum
__global__ void k_range_intervals(double *iv, double wcc, double wcb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, sp = blockIdx.y;   // species: 0 e-, 1 e+
    if (i >= NT) return;
    iv += sp * NT;
    const double x8[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
    const double w8[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};
    const double l0 = log(T_LO), dl = (log(T_HI) - log(T_LO)) / (NT - 1);
    if (i == 0) { iv[0] = 0.0; return; }
    const double T = exp(l0 + dl * i), Tp = exp(l0 + dl * (i - 1));
    const double m = 0.5 * (T + Tp), h = 0.5 * (T - Tp);
    double acc = 0.0;
    for (int k = 0; k < 4; ++k)
        acc += w8[k] * (1.0 / stop_restricted(sp, m - h * x8[k], wcc, wcb) + 1.0 / stop_restricted(sp, m + h * x8[k], wcc, wcb));
    iv[i] = h * acc;
}

// One block: the running sum of the interval ranges in order (one thread),
// then the node values, the forward table and the inverse table (all
// threads).  The forward table holds, for each pair of neighbouring nodes,
// the cubic Hermite interpolant of R in g = (ln T - ln T_i) / dlnT through
// the node values and the exact node slopes dR/dg = T dlnT / S, as the
// coefficients of its powers of g (one 16-byte load and three FMAs per
// evaluation).  The inverse node j takes the same pair of forward nodes as a
// walk along the nodes would (ln R is increasing), found by binary search.
__global__ void __launch_bounds__(1024) k_range_table(double *iv, float4 *rt, float *irt, float *igrid, double wcc,
                                                      double wcb) {
    __shared__ double liv[NT];
    __shared__ double slope[NT];
    const int sp = blockIdx.x;                       // one block per species
    iv += sp * NT; rt += sp * NT; irt += sp * NT; igrid += 2 * sp;
    const double l0 = log(T_LO), dl = (log(T_HI) - log(T_LO)) / (NT - 1);
    if (threadIdx.x == 0) {
        double R = 0.0;
        for (int i = 0; i < NT; ++i) {
            R += iv[i];
            iv[i] = R;                               // keep the cumulative range for the inverse
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NT; i += blockDim.x) {
        const double R = iv[i], T = exp(l0 + dl * i);
        slope[i] = T * dl / stop_restricted(sp, T, wcc, wcb);
        liv[i] = i > 0 ? log(R) : 0.0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NT; i += blockDim.x) {
        // the last node starts no interval (lookups stop below it): its row
        // continues the range linearly
        const double a0 = iv[i], d0 = slope[i];
        const double a1 = i + 1 < NT ? iv[i + 1] : a0 + d0, d1 = i + 1 < NT ? slope[i + 1] : d0;
        rt[i] = make_float4((float)a0, (float)d0, (float)(3.0 * (a1 - a0) - 2.0 * d0 - d1),
                            (float)(2.0 * (a0 - a1) + d0 + d1));
    }
    // inverse: ln T at NT uniform points of ln R over [R_1, R_{NT-1}], by
    // interpolating ln T linearly in ln R between the forward nodes
    const double a = liv[1], b = liv[NT - 1], dr = (b - a) / (NT - 1);
    for (int j = threadIdx.x; j < NT; j += blockDim.x) {
        const double lr = a + dr * j;
        int lo = 2, hi = NT;                         // first k >= 2 with ln R_k >= lr
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (liv[mid] < lr) lo = mid + 1; else hi = mid;
        }
        const int i = min(max(lo - 1, 1), NT - 2);
        const double r0 = liv[i], r1 = liv[i + 1];
        const double f = (lr - r0) / (r1 - r0);
        irt[j] = (float)(l0 + dl * (i + f));
    }
    if (threadIdx.x == 0) {
        igrid[0] = (float)a;
        igrid[1] = (float)(1.0 / dr);
    }
}

__global__ void k_rho_max(const uint8_t *mat, const float *rho, int64_t n, int *out, float *mrho) {
    __shared__ int m[2];
    if (threadIdx.x < 2) m[threadIdx.x] = 0;
    __syncthreads();
    int l0 = 0, l1 = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float ri = fmaxf(rho[i], 0.f);
        int r = __float_as_int(ri);                     // non-negative floats order as ints
        const bool bone = mat[i] != 0;
        if (bone) l1 = max(l1, r); else l0 = max(l0, r);
        mrho[i] = bone ? -ri : ri;
    }
    atomicMax(&m[0], l0);
    atomicMax(&m[1], l1);
    __syncthreads();
    if (threadIdx.x < 2) atomicMax(&out[threadIdx.x], m[threadIdx.x]);
}

__device__ __forceinline__ void tab_pos(const Tables &T, float E, int &i, float &f) {
    float x = (__logf(E) - T.lnE0) * T.inv_dln;
    x = fminf(fmaxf(x, 0.0f), (float)(NT - 1) - 1e-3f);
    i = (int)x;
    f = x - (float)i;
}

__device__ __forceinline__ float4 lerp4(const float4 *a, int i, float f) {
    float4 p = __ldg(a + i), q = __ldg(a + i + 1);
    return make_float4(p.x + f * (q.x - p.x), p.y + f * (q.y - p.y), p.z + f * (q.z - p.z), p.w + f * (q.w - p.w));
}

// R(E): cubic Hermite in ln E with the exact node derivatives dR/dlnE = E/S
// (i: node index including the species offset)
__device__ __forceinline__ float range_at(const Tables &T, int i, float f) {
    const float4 c = __ldg(T.rng + i);
    return fmaf(f, fmaf(f, fmaf(f, c.w, c.z), c.y), c.x);
}

// sp: the species offset (0 electron, NT positron)
__device__ __forceinline__ float range_of(const Tables &T, float E, int sp) {
    int i; float f;
    tab_pos(T, E, i, f);
    return range_at(T, i + sp, f);
}

// ------------------------------------------------------------- helpers ---
__device__ __forceinline__ unsigned long long fixed_point(float e, float wt) {
    return (unsigned long long)__float2ll_rn(__fmul_rn(e, wt) * 4294967296.0f);
}

template <class AT>
__device__ __forceinline__ void deposit(const AT &A, Acc &acc, uint32_t iv, float e, float wt, uint32_t root) {
    unsigned long long q = fixed_point(e, wt);
    if (!q) return;
    atomicAdd(&A.tally[(uint64_t)(root >> ROOT_SLICE_SHIFT) * (uint64_t)A.nvox + iv], q);
    acc.atomics++;
    if (AT::trace && A.hist_dep) atomicAdd(&A.hist_dep[root & ROOT_INDEX_MASK], q);
}

template <class AT>
__device__ __forceinline__ void escape(const AT &A, Acc &acc, float e, float wt, uint32_t root) {
    unsigned long long q = fixed_point(e, wt);
    acc.esc += q;
    if (AT::trace && A.hist_esc) atomicAdd(&A.hist_esc[root & ROOT_INDEX_MASK], q);
}

template <class AT>
__device__ __forceinline__ void count_event(const AT &A, uint32_t root) {
    if (AT::trace && A.hist_events) atomicAdd(&A.hist_events[root & ROOT_INDEX_MASK], 1);
}

// An event's random draws: the particle's draw counter is loaded at the
// start of the event and stored back at its end; the Philox block lives only
// inside the event (every event starts its draws on a fresh block), so no
// register holds it between events.
struct EventRng {
    uint32_t &saved;
    Rng r;
    __device__ __forceinline__ explicit EventRng(uint32_t &d) : saved(d) { r.draw = d; }
    __device__ __forceinline__ ~EventRng() { saved = r.draw; }
};

// Angles and logarithms keep the accuracy FP32 offers where it decides
// something: the sine of a polar angle comes from a form without
// cancellation (never sqrt(1 - c^2) near c = 1), 1 - w^2 of a direction is
// u^2 + v^2, and the logarithms of uniforms behind a multiple-scattering
// angle or an electron's mean free path count go through logf (a uniform
// near 1 has a small logarithm that the fast intrinsic only gets to an
// absolute error, or rounds to zero).  Sines and cosines that only turn a
// direction take the hardware approximations on [-pi, pi] (absolute error
// below 2^-21.4): the azimuth 2 pi xi as 2 pi (xi - 1/2) + pi, the
// multiple-scattering polar angle after its reduction by 2 pi; so does the
// Woodcock step length (photon_step).  Measured against sincospif and logf
// on the 30x30 CT plan: the electron pass 3.5 % and the photon pass 7 %
// faster, per-history event parity with the oracle unchanged.
__device__ __forceinline__ float ln_uniform(float xi) { return logf(xi); }
__device__ __forceinline__ void sincos_2pi(float xi, float *s, float *c) {
    float sn, cs;
    __sincosf(6.28318531f * (xi - 0.5f), &sn, &cs);         // xi - 1/2 is exact
    *s = -sn;
    *c = -cs;
}
__device__ __forceinline__ void sincos_polar(float th, float *s, float *c) {
    // th - 2 pi k in two parts (Cody and Waite): 6.28125 has 8 significant
    // bits, so k * 6.28125 is exact for any angle drawn, and the rest of 2 pi
    // follows; the result lies in [-pi, pi]
    const float k = rintf(th * 0.159154943f);
    __sincosf(fmaf(-k, 1.93530718e-3f, fmaf(-k, 6.28125f, th)), s, c);
}

// rotate unit direction by the polar angle (cosine c, sine st >= 0) and the
// azimuth (sine sp, cosine cp), the azimuth measured from the plane through
// the direction and the z axis (exact for every direction off the axis;
// only one on the axis itself takes the x-y pair); renormalised
__device__ __forceinline__ void rotate_dir(float &u, float &v, float &w, float c, float st, float sp, float cp) {
    float nu, nv, nw;
    const float s2 = u * u + v * v;                               // 1 - w^2 without cancellation
    if (s2 <= 1e-30f) {
        nu = st * cp; nv = st * sp; nw = w > 0.0f ? c : -c;
    } else {
        const float it = rsqrtf(s2), t = s2 * it;
        nu = u * c + st * (u * w * cp - v * sp) * it;
        nv = v * c + st * (v * w * cp + u * sp) * it;
        nw = w * c - st * cp * t;
    }
    float n = rsqrtf(nu * nu + nv * nv + nw * nw);
    u = nu * n; v = nv * n; w = nw * n;
}

__device__ __forceinline__ void push_particle(const Queue &q, const Args &A, uint32_t type, float x, float y, float z,
                                              float u, float v, float w, float e, float wt, uint32_t p0, uint32_t p1,
                                              uint32_t &nchild, uint32_t root) {
    Particle c;
    c.x = x; c.y = y; c.z = z; c.e = e; c.u = u; c.v = v; c.w = w; c.wt = wt;
    child_id(A.seed, p0, p1, nchild++, c.pid_lo, c.pid_hi);
    c.type = type; c.root = root;
    queue_push(q, c, A.err);
}

__device__ __forceinline__ void annihilate(const Args &A, Rng &rng, float x, float y, float z, float wt, uint32_t p0, uint32_t p1,
                           uint32_t &nchild, uint32_t root) {
    rng.align();
    const float xi = rng.next(A.rk, p0, p1);
    float cth = 2.0f * xi - 1.0f, sp, cp;
    float sth = 2.0f * sqrtf(fmaxf(0.0f, xi * (1.0f - xi)));     // sqrt(1 - cth^2)
    sincos_2pi(rng.next(A.rk, p0, p1), &sp, &cp);
    float a0 = sth * cp, a1 = sth * sp, a2 = cth;
    push_particle(A.p_out, A, 0, x, y, z, a0, a1, a2, F_ME, wt, p0, p1, nchild, root);
    push_particle(A.p_out, A, 0, x, y, z, -a0, -a1, -a2, F_ME, wt, p0, p1, nchild, root);
}

// energy band of an electron (32 log bands above the cut-off)
__device__ __forceinline__ int band_of(const Args &A, float e) {
    int b = (int)((__logf(e) - A.band_ln0) * A.band_scale);
    return min(max(b, 0), NBANDS - 1);
}

// Every kernel that queues electrons counts them by band in a block-shared
// histogram (bh) and adds it to the queue's band histogram when it ends, so
// the regrouping before the electron pass needs no counting pass of its own.
__device__ __forceinline__ void band_hist_init(uint32_t *bh) {
    if (threadIdx.x < NBANDS) bh[threadIdx.x] = 0;
}
__device__ __forceinline__ void band_hist_flush(const Args &A, const uint32_t *bh) {
    __syncthreads();
    if (threadIdx.x < NBANDS && bh[threadIdx.x]) atomicAdd(&A.band_hist[threadIdx.x], bh[threadIdx.x]);
}

// a charged secondary: queued for transport, or deposited in place
template <class AT>
__device__ __forceinline__ void emit_charged(const AT &A, Acc &acc, Rng &rng, uint32_t *bh, uint32_t type, float T,
                             float x, float y, float z, float u, float v, float w, float wt, uint32_t iv, uint32_t p0,
                             uint32_t p1, uint32_t &nchild, uint32_t root) {
    if (T > A.ecut && !(A.flags & PSL_PHYS_LOCAL_SECONDARIES)) {
        if (type == 1) atomicAdd(&bh[band_of(A, T)], 1u);     // (positrons leave the band sort)
        push_particle(A.e_out, A, type, x, y, z, u, v, w, T, wt, p0, p1, nchild, root);
        return;
    }
    deposit(A, acc, iv, T, wt, root);
    if (type == 2) {
        if (A.flags & PSL_PHYS_LOCAL_SECONDARIES) deposit(A, acc, iv, 2.0f * F_ME, wt, root);
        else annihilate(A, rng, x, y, z, wt, p0, p1, nchild, root);
    }
}

// ledger slots: 0 emitted, 1 escaped, 2 deposited (fixed point; taken from
// the tally when it is read), 3 Compton, 4 photoelectric, 5 pair, 6 electron
// steps, 7 errors, 8 tally atomics of photon passes, 9 tally atomics of
// electron passes, 10 Woodcock steps, 11 hard Moller / Bhabha collisions
__device__ __forceinline__ void acc_init(unsigned long long *s) {
    if (threadIdx.x < NLEDGER) s[threadIdx.x] = 0ull;
}

// End of a kernel: every thread's counts into the block's ledger s (shared
// memory; steps, tally atomics and the packed events into their slots: ev_slot
// holds the first packed field's slot, or -1), then the block's ledger into
// the tally's.
__device__ __forceinline__ void flush_acc(const Args &A, const Acc &a, unsigned long long *s, int steps_slot,
                                          int atomics_slot, int ev_slot) {
    unsigned long long v[6] = {a.steps, a.atomics, a.esc, a.ev & 0x1FFFFFull, (a.ev >> 21) & 0x1FFFFFull, a.ev >> 42};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(FULL, v[k], o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (v[0]) atomicAdd(&s[steps_slot], v[0]);
        if (v[1]) atomicAdd(&s[atomics_slot], v[1]);
        if (v[2]) atomicAdd(&s[1], v[2]);
        if (ev_slot >= 0) {
#pragma unroll
            for (int k = 0; k < 3; ++k)
                if (v[3 + k] && ev_slot + k < NLEDGER) atomicAdd(&s[ev_slot + k], v[3 + k]);
        }
    }
    __syncthreads();
    if (threadIdx.x < NLEDGER && s[threadIdx.x]) atomicAdd(&A.ledger[threadIdx.x], s[threadIdx.x]);
}

// ------------------------------------------------------------ warp feed ---
// A warp claims queue entries FEED_CHUNK at a time and stages each chunk in
// shared memory with one bulk asynchronous copy (cp.async.bulk completing on
// an mbarrier), one chunk ahead of use.  A lane that needs a new particle
// then reads it from shared memory instead of waiting on HBM.  The current
// chunk is always resident; its successor is in flight or resident.  (The
// packed feed state holds counts below 64; a photon warp takes ~12 new
// photons per loop pass, so a chunk of 48 lasts about four passes.)
#define FEED_CHUNK 48
#define FEED_WARPS 8                     // 256-thread blocks
#define FEED_SPIN (1u << 22)

// The particles a feed hands out: queue 1's n1 particles, then queue 2's n2,
// as one index space in which queue 2 starts at n1 rounded up to a chunk
// (claims are whole chunks, so none straddles the two queues)
struct FeedSrc {
    const Particle *p1, *p2;
    uint32_t n1, n1p, n2;
};

struct FeedSmem {
    Particle buf[FEED_WARPS][2][FEED_CHUNK];
    unsigned long long bar[FEED_WARPS][2];
};

// Per-warp state, packed in one register: bits 0-5 and 6-11 the particle
// counts of buffers 0 and 1, 12-17 the read position in the current buffer,
// 18 the current buffer, 19-20 the mbarrier phase of each buffer.
struct Feed {
    uint32_t st;

    __device__ __forceinline__ uint32_t cnt(uint32_t b) const { return (st >> (6u * b)) & 63u; }
    __device__ __forceinline__ void set_cnt(uint32_t b, uint32_t c) { st = (st & ~(63u << (6u * b))) | (c << (6u * b)); }
    __device__ __forceinline__ uint32_t pos() const { return (st >> 12) & 63u; }
    __device__ __forceinline__ uint32_t cur() const { return (st >> 18) & 1u; }
    __device__ __forceinline__ static uint32_t bar_addr(FeedSmem &sm, uint32_t b) {
        return (uint32_t)__cvta_generic_to_shared(&sm.bar[threadIdx.x >> 5][b]);
    }
    __device__ __forceinline__ static Particle *slot(FeedSmem &sm, uint32_t b, uint32_t i) {
        return &sm.buf[threadIdx.x >> 5][b][i];
    }

    __device__ __forceinline__ void init(FeedSmem &sm, const FeedSrc &src, uint32_t *head, uint32_t *err,
                                         uint32_t polls, bool stall) {
        st = 0;
        if ((threadIdx.x & 31) == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar_addr(sm, 0)) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar_addr(sm, 1)) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncwarp();
        set_cnt(0, claim(sm, 0, src, head));
        // (stall: a failure-detection test; no copy into buffer 1 is ever
        // issued, so its mbarrier never completes and the wait runs out)
        set_cnt(1, claim(sm, 1, src, head, stall));
        if (cnt(0)) wait(sm, 0, err, polls);
    }
    // claim the next chunk into buffer b; returns its particle count
    __device__ __forceinline__ static uint32_t claim(FeedSmem &sm, uint32_t b, const FeedSrc &fs,
                                                     uint32_t *head, bool no_copy = false) {
        uint32_t base = 0;
        if ((threadIdx.x & 31) == 0) base = atomicAdd(head, (uint32_t)FEED_CHUNK);
        base = __shfl_sync(FULL, base, 0);
        // (base is a multiple of the chunk, so base < n1p means base < n1)
        const bool first = base < fs.n1p;
        const uint32_t j = first ? base : base - fs.n1p, n = first ? fs.n1 : fs.n2;
        const Particle *src = first ? fs.p1 : fs.p2;
        const uint32_t c = j < n ? min(n - j, (uint32_t)FEED_CHUNK) : 0u;
        if (c && !no_copy && (threadIdx.x & 31) == 0) {
            const uint32_t bytes = c * (uint32_t)sizeof(Particle);
            const uint32_t mb = bar_addr(sm, b);
            const uint32_t dst = (uint32_t)__cvta_generic_to_shared(slot(sm, b, 0));
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mb), "r"(bytes) : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         :: "r"(dst), "l"(src + j), "r"(bytes), "r"(mb) : "memory");
        }
        return c;
    }
    // wait (bounded: `polls` tries) until buffer b's copy has landed
    __device__ __forceinline__ void wait(FeedSmem &sm, uint32_t b, uint32_t *err, uint32_t polls) {
        const uint32_t mb = bar_addr(sm, b), par = (st >> (19u + b)) & 1u;
        uint32_t ok = 0;
        for (uint32_t it = 0; it < polls && !ok; ++it)
            asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                         : "=r"(ok) : "r"(mb), "r"(par) : "memory");
        st ^= 1u << (19u + b);
        if (!ok) {
            atomicOr(err, PSL_DEV_ERR_TIMEOUT);
            st &= ~4095u;                     // nothing more is read from this warp's buffers
        }
    }
    // Hand particles to the lanes in `need` (ranked by lane order).  Returns
    // true and fills p for a lane in `need` that got one; a lane in `need`
    // that got none finds the queue exhausted.
    __device__ __forceinline__ bool take(FeedSmem &sm, unsigned need, unsigned lt, bool mine, Particle &p,
                                         const FeedSrc &src, uint32_t *head, uint32_t *err,
                                         uint32_t polls, bool stall) {
        const uint32_t k = __popc(need), rank = __popc(need & lt);
        const uint32_t c = cur(), nx = c ^ 1u, avail = cnt(c) - pos();
        if (k >= avail && cnt(nx)) wait(sm, nx, err, polls);
        const uint32_t cn = cnt(nx);                    // after a failed wait this is 0
        bool got = false;
        if (mine) {
            const Particle *q = nullptr;
            if (rank < avail) q = slot(sm, c, pos() + rank);
            else if (rank - avail < cn) q = slot(sm, nx, rank - avail);
            if (q) {
                const float4 *s4 = reinterpret_cast<const float4 *>(q);
                float4 *d4 = reinterpret_cast<float4 *>(&p);
                d4[0] = s4[0]; d4[1] = s4[1]; d4[2] = s4[2];
                got = true;
            }
        }
        if (k >= avail) {                               // the current chunk is used up
            __syncwarp();                               // every lane has read it
            const uint32_t np = min(k - avail, cn);
            st = (st & ~((63u << 12) | (1u << 18))) | (np << 12) | (nx << 18);
            set_cnt(c, cn ? claim(sm, c, src, head, stall && c == 1u) : 0u);   // a short chunk: queue exhausted
        } else {
            st += k << 12;
        }
        return got;
    }
};

// ------------------------------------------------------------- photons ---
struct Photon {
    float x, y, z, u, v, w, e, wt;
    uint32_t p0, p1, root, nchild;
    uint32_t draw;             // draws taken from the particle's Philox stream
    float mumax, inv_mumax;
    int ti;
    float tf;
    uint32_t chan;             // channel of a drawn real interaction: 0 Compton, 1 photoelectric, 2 pair
};

// Table position and Woodcock majorant at the photon's energy: the largest
// attenuation coefficient any voxel can have, max over the materials of
// (largest density of the material) x (its coefficients), summed without
// contraction in the order photon_step sums a voxel's, so that no voxel's
// coefficient exceeds it (rounding is monotone) and none is given headroom.
__device__ __forceinline__ float mu_of(float rho, const float4 &c) {
    return __fadd_rn(__fadd_rn(__fmul_rn(rho, c.x), __fmul_rn(rho, c.y)), __fmul_rn(rho, c.z));
}

__device__ __forceinline__ void photon_energy(const Args &A, Photon &g) {
    tab_pos(A.tab, g.e, g.ti, g.tf);
    const float r0 = __int_as_float(__ldg(A.rmax)), r1 = __int_as_float(__ldg(A.rmax + 1));
    g.mumax = fmaxf(mu_of(r0, lerp4(A.tab.ph0, g.ti, g.tf)), mu_of(r1, lerp4(A.tab.ph1, g.ti, g.tf)));
    g.inv_mumax = __frcp_rn(g.mumax);
}

// One Woodcock step.  Returns G_END when the photon leaves the phantom,
// G_ON after a virtual interaction, G_REAL when a real interaction was drawn
// (its channel in g.chan; photon_interact() runs it and the caller may
// defer it).
enum { G_END = 0, G_ON = 1, G_REAL = 2 };

__device__ __forceinline__ uint32_t photon_voxel(const Args &A, const Photon &g) {
    const float fx = floorf(g.x * A.ivx), fy = floorf(g.y * A.ivy), fz = floorf(g.z * A.ivz);
    return ((uint32_t)fz * (uint32_t)A.ny + (uint32_t)fy) * (uint32_t)A.nx + (uint32_t)fx;
}

template <class AT>
__device__ __forceinline__ int photon_step(const AT &A, Acc &acc, Photon &g) {
    acc.steps++;
    EventRng ev(g.draw);
    Rng &rng = ev.r;
    rng.align();                                                // Woodcock step: step, virtual, channel
    // (the fast logarithm: a virtual step's length needs no more than its
    // relative accuracy away from u = 1, and one near 1 is short either way)
    const float s = fmaxf(-__logf(rng.next(A.rk, g.p0, g.p1)), 0.0f) * g.inv_mumax;
    g.x += s * g.u; g.y += s * g.v; g.z += s * g.w;
    const float fx = floorf(g.x * A.ivx), fy = floorf(g.y * A.ivy), fz = floorf(g.z * A.ivz);
    if (!(fx >= 0.0f && fy >= 0.0f && fz >= 0.0f && fx < (float)A.nx && fy < (float)A.ny && fz < (float)A.nz)) {
        escape(A, acc, g.e, g.wt, g.root);
        return G_END;
    }
    const uint32_t iv = ((uint32_t)fz * (uint32_t)A.ny + (uint32_t)fy) * (uint32_t)A.nx + (uint32_t)fx;
    const float mr = __ldg(A.mrho + iv);
    const float rho = fabsf(mr);
    // both materials' rows are loaded with the density, not after it
    const float4 c0 = lerp4(A.tab.ph0, g.ti, g.tf), c1 = lerp4(A.tab.ph1, g.ti, g.tf);
    const float4 c = mr < 0.0f ? c1 : c0;
    const float mc = __fmul_rn(rho, c.x), mpe = __fmul_rn(rho, c.y), mpp = __fmul_rn(rho, c.z);
    const float mu = __fadd_rn(__fadd_rn(mc, mpe), mpp);          // = mu_of(rho, c)
    if (mu > g.mumax) atomicOr(A.err, 8u);
    if (rng.next(A.rk, g.p0, g.p1) * g.mumax >= mu) return G_ON;          // virtual interaction
    count_event(A, g.root);
    const float r = rng.next(A.rk, g.p0, g.p1) * mu;
    g.chan = r < mc ? 0u : (r < mc + mpe ? 1u : 2u);
    return G_REAL;
}

// the real interaction drawn by the last step; returns false when the photon ends
template <class AT>
__device__ __forceinline__ bool photon_interact(const AT &A, Acc &acc, Photon &g, uint32_t *bh) {
    const uint32_t iv = photon_voxel(A, g);
    EventRng ev(g.draw);
    Rng &rng = ev.r;
    rng.align();                                                // the interaction's draws
    const bool first = A.flags & PSL_PHYS_FIRST_INTERACTION;
    if (g.chan == 0u) {                                           // Compton (Kahn's method)
        acc.ev += EV_COMPTON;
        if (first) { deposit(A, acc, iv, g.e, g.wt, g.root); return false; }
        const float k = g.e * (1.0f / F_ME), ik = __fdividef(1.0f, k);     // (reciprocals: the hardware approximation)
        const float p_first = __fdividef(1.0f + 2.0f * k, 9.0f + 2.0f * k);
        float x = 1.0f, ix = 1.0f;
        for (int it = 0; it < 1000; ++it) {
            const float r1 = rng.next(A.rk, g.p0, g.p1), r2 = rng.next(A.rk, g.p0, g.p1), r3 = rng.next(A.rk, g.p0, g.p1);
            if (r1 <= p_first) {
                x = 1.0f + 2.0f * k * r2;
                ix = __fdividef(1.0f, x);
                if (r3 <= 4.0f * (ix - ix * ix)) break;
            } else {
                ix = __fdividef(1.0f + 2.0f * k * r2, 1.0f + 2.0f * k);
                x = __fdividef(1.0f, ix);
                const float cc = 1.0f - (x - 1.0f) * ik;
                if (r3 <= 0.5f * (cc * cc + ix)) break;
            }
        }
        const float dc = fminf(2.0f, fmaxf(0.0f, (x - 1.0f) * ik));   // 1 - cos(theta)
        const float cth = 1.0f - dc, sth = sqrtf(dc * (2.0f - dc));
        const float ep = g.e * ix;
        float sp, cp;
        sincos_2pi(rng.next(A.rk, g.p0, g.p1), &sp, &cp);
        float nu = g.u, nv = g.v, nw = g.w;
        rotate_dir(nu, nv, nw, cth, sth, sp, cp);
        const float te = g.e - ep;
        float du = g.e * g.u - ep * nu, dv = g.e * g.v - ep * nv, dw = g.e * g.w - ep * nw;
        const float nn2 = du * du + dv * dv + dw * dw;
        if (nn2 > 0.0f) { const float in = rsqrtf(nn2); du *= in; dv *= in; dw *= in; } else { du = g.u; dv = g.v; dw = g.w; }
        emit_charged(A, acc, rng, bh, 1, te, g.x, g.y, g.z, du, dv, dw, g.wt, iv, g.p0, g.p1, g.nchild, g.root);
        g.e = ep; g.u = nu; g.v = nv; g.w = nw;
        if (g.e < A.pcut) { deposit(A, acc, iv, g.e, g.wt, g.root); return false; }
        photon_energy(A, g);
        return true;
    } else if (g.chan == 1u) {                                    // photoelectric
        acc.ev += EV_PHOTO;
        if (first) { deposit(A, acc, iv, g.e, g.wt, g.root); return false; }
        emit_charged(A, acc, rng, bh, 1, g.e, g.x, g.y, g.z, g.u, g.v, g.w, g.wt, iv, g.p0, g.p1, g.nchild, g.root);
        return false;
    }
    acc.ev += EV_PAIR;                                             // pair production
    if (first) { deposit(A, acc, iv, g.e, g.wt, g.root); return false; }
    const float avail = g.e - 2.0f * F_ME, eps = rng.next(A.rk, g.p0, g.p1);
    const float t1 = eps * avail, t2 = avail - t1;
    emit_charged(A, acc, rng, bh, 1, t1, g.x, g.y, g.z, g.u, g.v, g.w, g.wt, iv, g.p0, g.p1, g.nchild, g.root);
    emit_charged(A, acc, rng, bh, 2, t2, g.x, g.y, g.z, g.u, g.v, g.w, g.wt, iv, g.p0, g.p1, g.nchild, g.root);
    return false;
}

// Parking slots (PSL_PHOTON_SLOTS): one per lane in shared memory, holding
// a photon whose Woodcock step drew a real interaction (PENDING) or one set
// aside to make room for such a photon (READY).  A lane whose photon draws a
// real interaction parks it and steps another photon (from its slot or the
// feed) instead of idling; a lane whose own slot is taken parks it in the
// empty slot of another lane of the warp (the k-th such lane in the k-th
// empty slot); the parked interactions run together once enough lanes have
// one (or every live lane is blocked), so that the interaction code runs
// with most lanes active while stepping keeps the lanes busy.  Every photon
// keeps its own random stream, so the order changes nothing.
// A slot is 20 words (the 18 of Photon and a pad), moved as four 16-byte
// and one 8-byte shared-memory access: at an 80-byte stride the eight lanes
// of each quarter-warp phase of a 16-byte access hit disjoint banks.
#ifndef PSL_PHOTON_SLOTS
#define PSL_PHOTON_SLOTS 1
#endif
enum { SLOT_EMPTY = 0, SLOT_READY = 1, SLOT_PENDING = 2 };
constexpr int SLOT_WORDS = 20;

__device__ __forceinline__ void slot_store(uint32_t *s, const Photon &g) {
    uint4 *q = reinterpret_cast<uint4 *>(s);
    q[0] = make_uint4(__float_as_uint(g.x), __float_as_uint(g.y), __float_as_uint(g.z), __float_as_uint(g.u));
    q[1] = make_uint4(__float_as_uint(g.v), __float_as_uint(g.w), __float_as_uint(g.e), __float_as_uint(g.wt));
    q[2] = make_uint4(g.p0, g.p1, g.root, g.nchild);
    q[3] = make_uint4(g.draw, __float_as_uint(g.mumax), __float_as_uint(g.inv_mumax), (uint32_t)g.ti);
    reinterpret_cast<uint2 *>(s)[8] = make_uint2(__float_as_uint(g.tf), g.chan);
}

__device__ __forceinline__ void slot_load(const uint32_t *s, Photon &g) {
    const uint4 *q = reinterpret_cast<const uint4 *>(s);
    const uint4 a = q[0], b = q[1], c = q[2], d = q[3];
    const uint2 e = reinterpret_cast<const uint2 *>(s)[8];
    g.x = __uint_as_float(a.x); g.y = __uint_as_float(a.y); g.z = __uint_as_float(a.z); g.u = __uint_as_float(a.w);
    g.v = __uint_as_float(b.x); g.w = __uint_as_float(b.y); g.e = __uint_as_float(b.z); g.wt = __uint_as_float(b.w);
    g.p0 = c.x; g.p1 = c.y; g.root = c.z; g.nchild = c.w;
    g.draw = d.x; g.mumax = __uint_as_float(d.y); g.inv_mumax = __uint_as_float(d.z); g.ti = (int)d.w;
    g.tf = __uint_as_float(e.x); g.chan = e.y;
}

template <bool TR>
__global__ void __launch_bounds__(256, PSL_PHOTON_MIN_BLOCKS) k_photon(ArgsT<TR> A, const Particle *src, const uint32_t *n_ptr, uint32_t n_fixed,
                                                uint32_t cap, uint32_t *head, const Particle *src2,
                                                const uint32_t *n2_ptr, uint32_t cap2) {
    __shared__ FeedSmem sm;
    __shared__ uint32_t bh[NBANDS];
    __shared__ unsigned long long sled[NLEDGER];
#if PSL_PHOTON_SLOTS
    __shared__ __align__(16) uint32_t slots[FEED_WARPS * 32][SLOT_WORDS];
    uint32_t *my = slots[threadIdx.x];
    uint32_t slot = SLOT_EMPTY;
#endif
    band_hist_init(bh);
    acc_init(sled);
    __syncthreads();
    // the photons of the pass: the primaries (or a first queue), then the
    // secondaries carried over from the previous chunk (src2, may be null)
    FeedSrc fs;
    fs.p1 = src;
    fs.n1 = n_ptr ? min(*n_ptr, cap) : n_fixed;
    fs.n1p = (fs.n1 + FEED_CHUNK - 1) / FEED_CHUNK * FEED_CHUNK;
    fs.p2 = src2;
    fs.n2 = src2 ? min(*n2_ptr, cap2) : 0u;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    Acc acc = {0u, 0u, 0ull, 0ull};
    Photon g;
    Feed F;
    F.init(sm, fs, head, A.err, A.wait_polls, (A.dbg & PSL_DEBUG_FEED_STALL) != 0);
    bool alive = false, done = false, real = false;
    for (;;) {
#if PSL_PHOTON_SLOTS
        if (!alive && slot == SLOT_READY) { slot_load(my, g); slot = SLOT_EMPTY; alive = true; }
#endif
        const unsigned need = __ballot_sync(FULL, !alive && !done);
        if (need) {
            Particle p;
            const bool mine = !alive && !done;
            const bool got = F.take(sm, need, lt, mine, p, fs, head, A.err, A.wait_polls,
                                    (A.dbg & PSL_DEBUG_FEED_STALL) != 0);
            if (mine) {
                if (!got) {
                    done = true;
                } else {
                    g.x = p.x; g.y = p.y; g.z = p.z; g.u = p.u; g.v = p.v; g.w = p.w; g.e = p.e; g.wt = p.wt;
                    g.p0 = p.pid_lo; g.p1 = p.pid_hi; g.root = p.root; g.nchild = 0;
                    g.draw = 0;
                    photon_energy(A, g);
                    alive = true;
                }
            }
        }
        const unsigned live = __ballot_sync(FULL, alive);
#if PSL_PHOTON_SLOTS
        const unsigned pend = __ballot_sync(FULL, slot == SLOT_PENDING);
        if (!live && !pend) break;
        // the parked interactions run when enough lanes have one, or when
        // every live lane is blocked (its photon has an interaction too)
        const unsigned stuck = __ballot_sync(FULL, alive && real);
        if (pend && (__popc(pend) >= PSL_G_DEFER || stuck == live)) {
            if (slot == SLOT_PENDING) {
                Photon q;
                slot_load(my, q);
                if (alive) { slot_store(my, g); slot = real ? SLOT_PENDING : SLOT_READY; }
                else slot = SLOT_EMPTY;
                g = q;
                alive = photon_interact(A, acc, g, bh);
                real = false;
            }
        }
        if (alive && !real) {
            // up to PSL_G_INNER steps while the steps are virtual: the loop's
            // refill and parking bookkeeping is then paid once per few steps
            int r = photon_step(A, acc, g);
            for (int k = 1; k < PSL_G_INNER && r == G_ON; ++k) r = photon_step(A, acc, g);
            if (r == G_END) {
                alive = false;
            } else if (r == G_REAL) {
                if (slot == SLOT_EMPTY) {                     // park it, take other work
                    slot_store(my, g); slot = SLOT_PENDING; alive = false;
                } else if (slot == SLOT_READY) {              // swap with the set-aside photon
                    Photon q;
                    slot_load(my, q);
                    slot_store(my, g);
                    slot = SLOT_PENDING;
                    g = q;
                } else {
                    real = true;                              // blocked until the parked one has run
                }
            }
        }
        {
            // a blocked photon parks in another lane's empty slot
            const unsigned stk = __ballot_sync(FULL, alive && real);
            if (stk) {
                const unsigned emp = __ballot_sync(FULL, slot == SLOT_EMPTY);
                const int m = min(__popc(stk), __popc(emp));
                if (m) {
                    if (alive && real) {
                        const int k = __popc(stk & lt);
                        if (k < m) {
                            const int dst = (int)__fns(emp, 0u, k + 1);
                            slot_store(slots[(threadIdx.x & ~31u) + dst], g);
                            alive = false; real = false;
                        }
                    }
                    if (slot == SLOT_EMPTY && __popc(emp & lt) < m) slot = SLOT_PENDING;
                    __syncwarp();
                }
            }
        }
#else
        if (!live) break;
        // Real interactions wait until enough lanes have one (or every live
        // lane waits), so that the interaction code runs with most lanes
        // active; the other lanes keep taking Woodcock steps meanwhile.
        const unsigned rm = __ballot_sync(FULL, real);
        if (rm && (__popc(rm) >= PSL_G_DEFER || rm == live)) {
            if (real) { alive = photon_interact(A, acc, g, bh); real = false; }
        }
        if (alive && !real) {
            const int r = photon_step(A, acc, g);
            alive = r != G_END;
            real = r == G_REAL;
        }
#endif
    }
    flush_acc(A, acc, sled, 10, 8, 3);
    band_hist_flush(A, bh);
}

// ----------------------------------------------------------- electrons ---
struct Electron {
    float x, y, z, u, v, w, t, wt, nlam;
    float r;                   // CSDA range at t (g/cm^2), carried from step to step
    int ix, iy, iz;
    uint32_t p0, p1, root, nchild;
    int steps;
    uint32_t draw;             // draws taken from the particle's Philox stream
#if PSL_DEP_COMBINE
    uint32_t piv;              // voxel of the deposits summed in pq (not yet added to the tally)
    unsigned long long pq;
#endif
};

// The per-step deposit of an electron.  With PSL_DEP_COMBINE the deposits
// of consecutive steps in one voxel are summed in registers (the integer
// sum is the same) and added with one atomic when the voxel changes or the
// electron ends (electron_flush).
template <class AT>
__device__ __forceinline__ void electron_deposit(const AT &A, Acc &acc, Electron &s, uint32_t iv, float e) {
#if PSL_DEP_COMBINE
    const unsigned long long q = fixed_point(e, s.wt);
    if (!q) return;
    if (A.hist_dep) atomicAdd(&A.hist_dep[s.root & ROOT_INDEX_MASK], q);
    if (iv == s.piv) { s.pq += q; return; }
    if (s.pq) {
        atomicAdd(&A.tally[(uint64_t)(s.root >> ROOT_SLICE_SHIFT) * (uint64_t)A.nvox + s.piv], s.pq);
        acc.atomics++;
    }
    s.piv = iv;
    s.pq = q;
#else
    deposit(A, acc, iv, e, s.wt, s.root);
#endif
}

template <class AT>
__device__ __forceinline__ void electron_flush(const AT &A, Acc &acc, Electron &s) {
#if PSL_DEP_COMBINE
    if (s.pq) {
        atomicAdd(&A.tally[(uint64_t)(s.root >> ROOT_SLICE_SHIFT) * (uint64_t)A.nvox + s.piv], s.pq);
        acc.atomics++;
        s.pq = 0;
    }
#endif
}

__device__ __forceinline__ float highland(float T, float s, float rho) {
    const float t = s * rho * (1.0f / 36.08f);
    if (!(t > 0.0f)) return 0.0f;
    const float bcp = __fdividef(T * (T + 2.0f * F_ME), T + F_ME);
    const float f = 1.0f + 0.038f * __logf(t);
    if (!(f > 0.0f)) return 0.0f;
    return __fdividef(13.6f, bcp) * (t * rsqrtf(t)) * f;
}

// energy whose CSDA range is r (g/cm^2): ln T from the inverse range table,
// then one Newton step on the forward (Hermite) range, so that the range of
// the result is r to float precision (a step of zero length keeps T)
// (sp: the species' table offset, 0 for electrons and NT for positrons)
__device__ __forceinline__ float energy_of_range(const Tables &T, float r, int sp) {
    const int k = sp / NT;
    float x = (__logf(r) - T.lnR0[k]) * T.inv_dlnR[k];
    x = fminf(fmaxf(x, 0.0f), (float)(NT - 1) - 1e-3f);
    const int i = (int)x + sp;
    const float f = x - (float)(i - sp);
    const float a = __ldg(T.irng + i), b = __ldg(T.irng + i + 1);
    const float lt0 = a + f * (b - a);
    // forward table position of ln T0 and the Hermite range with its slope
    float xf = (lt0 - T.lnE0) * T.inv_dln;
    xf = fminf(fmaxf(xf, 0.0f), (float)(NT - 1) - 1e-3f);
    const int j = (int)xf;
    const float g = xf - (float)j;
    const float4 c = __ldg(T.rng + j + sp);
    const float rg = fmaf(g, fmaf(g, fmaf(g, c.w, c.z), c.y), c.x);
    const float dr = fmaf(g, fmaf(g, 3.0f * c.w, 2.0f * c.z), c.y);
    const float g1 = dr > 0.0f ? g + __fdividef(r - rg, dr) : g;
    return expf(T.lnE0 + ((float)j + g1) * T.dln);
}

__device__ __forceinline__ float sample_moller(float T, float wcc, Rng &rng, const uint32_t *rk, uint32_t p0,
                                               uint32_t p1, uint32_t *err) {
    const float tau = T / F_ME, ec = wcc / T;
    const float g = (tau / (tau + 1.0f)) * (tau / (tau + 1.0f));
    const float a = (2.0f * tau + 1.0f) / ((tau + 1.0f) * (tau + 1.0f));
    const float w1 = 1.0f / ec - 2.0f, w2 = 5.0f * (0.5f - ec);
    for (int it = 0; it < 1000; ++it) {
        const float r1 = rng.next(rk, p0, p1), r2 = rng.next(rk, p0, p1), r3 = rng.next(rk, p0, p1);
        const float e = (r1 * (w1 + w2) < w1) ? ec / (1.0f - r2 * (1.0f - 2.0f * ec)) : ec + r2 * (0.5f - ec);
        const float q = e / (1.0f - e);
        const float f = 1.0f + q * q + g * e * e - a * q;
        if (r3 * (1.0f + 5.0f * e * e) <= f) return e;
    }
    atomicOr(err, PSL_DEV_ERR_STEPS);
    return ec;
}

// Bhabha energy-transfer fraction x in [wcc/T, 1]: x proposed from the
// density 1/x^2 on [x0, 1] and kept with probability
// h(x) = 1 - beta^2 x (B1 - x (B2 - x (B3 - x B4))), which lies in (0, 1].
__device__ __forceinline__ float sample_bhabha(float T, float wcc, Rng &rng, const uint32_t *rk, uint32_t p0,
                                               uint32_t p1, uint32_t *err) {
    const float y = 1.0f / (T * (1.0f / F_ME) + 2.0f), q = 1.0f - 2.0f * y, q2 = q * q;
    const float b1 = 2.0f - y * y, b2 = q * (3.0f + y * y), b4 = q2 * q, b3 = b4 + q2;
    const float gm = T * (1.0f / F_ME) + 1.0f, beta2 = 1.0f - 1.0f / (gm * gm);
    const float x0 = wcc / T;
    for (int it = 0; it < 1000; ++it) {
        const float r1 = rng.next(rk, p0, p1), r2 = rng.next(rk, p0, p1);
        const float x = x0 / (1.0f - r1 * (1.0f - x0));
        const float h = 1.0f - beta2 * x * (b1 - x * (b2 - x * (b3 - x * b4)));
        if (r2 <= h) return x;
    }
    atomicOr(err, PSL_DEV_ERR_STEPS);
    return x0;
}

template <bool POS, class AT>
__device__ __forceinline__ void electron_end(const AT &A, Acc &acc, Electron &s, uint32_t iv) {
    deposit(A, acc, iv, s.t, s.wt, s.root);
    if (POS) {
        if (A.flags & PSL_PHYS_LOCAL_SECONDARIES) {
            deposit(A, acc, iv, 2.0f * F_ME, s.wt, s.root);
        } else {
            EventRng ev(s.draw);
            annihilate(A, ev.r, s.x, s.y, s.z, s.wt, s.p0, s.p1, s.nchild, s.root);
        }
    }
}

// One condensed-history step.  Returns E_END when the electron ends,
// E_HARD when the step ends at a hard event (electron_hard() runs it; the
// caller may defer it), E_ON otherwise.
enum { E_END = 0, E_ON = 1, E_HARD = 2 };

// An electron whose step ends below the cut-off (not at a hard event) ends in
// that same call, in the voxel the step ended in, so that its lane takes the
// next electron at once instead of idling through one more pass of the loop;
// the deposits and draws are those of ending at the start of the next step.
template <bool POS, class AT>
__device__ __forceinline__ int electron_step(const AT &A, Acc &acc, Electron &s) {
    uint32_t iv = ((uint32_t)s.iz * (uint32_t)A.ny + (uint32_t)s.iy) * (uint32_t)A.nx + (uint32_t)s.ix;
    if (!(s.t <= A.ecut) && ++s.steps <= MAX_E_STEPS) {
        acc.steps++;
        count_event(A, s.root);
        EventRng ev(s.draw);
        Rng &rng = ev.r;
        rng.align();                                                  // the step's draws (at most 3)
        rng.fill(A.rk, s.p0, s.p1);
        if (s.nlam < 0.0f) s.nlam = -ln_uniform(rng.take());       // a new mean free path count
        const bool hard_on = !(A.flags & PSL_PHYS_NO_HARD);
        const float rho = fabsf(__ldg(A.mrho + iv));
        int ti; float tf;
        tab_pos(A.tab, s.t, ti, tf);
        constexpr int sp = POS ? NT : 0;                           // the species' table rows
        const float4 el = lerp4(A.tab.el + sp, ti, tf);
        // hard cross sections vanish below their thresholds (guard the
        // interpolation): Moller above 2 W_cc, Bhabha above W_cc
        const float wth = sp ? A.wcc : 2.0f * A.wcc;
        const float sig = hard_on ? rho * ((s.t > wth ? el.y : 0.0f) + (s.t > A.wcb ? el.z : 0.0f)) : 0.0f;
        const float s_hard = sig > 0.0f ? __fdividef(s.nlam, sig) : INFINITY;
        // distance to the voxel boundary
        float s_bound = INFINITY;
        int axis = -1, cross = 0;
        {
            const float d[3] = {s.u, s.v, s.w}, p[3] = {s.x, s.y, s.z}, vv[3] = {A.vx, A.vy, A.vz};
            const int ii[3] = {s.ix, s.iy, s.iz};
    #pragma unroll
            for (int k = 0; k < 3; ++k) {
                float t;
                if (d[k] == 0.0f) continue;                // (the far face: ii + 1 moving up, ii moving down)
                t = __fdividef((float)(ii[k] + (d[k] > 0.0f)) * vv[k] - p[k], d[k]);
                t = fmaxf(t, 0.0f);
                if (t < s_bound) { s_bound = t; axis = k; cross = d[k] > 0.0f ? 1 : -1; }
            }
        }
        const float tlim = fmaxf(0.9f * s.t, A.ecut);
        const float rlim = range_of(A.tab, tlim, sp);
        const float s_max = __fdividef(s.r - rlim, rho);         // (a step limit: the fast division)
        int which;
        float step;
        if (s_hard <= s_bound && s_hard <= s_max) { which = 0; step = s_hard; }
        else if (s_bound <= s_max) { which = 1; step = s_bound; }
        else { which = 2; step = s_max; }
        // energy at the end of the step: the 10 % limit exactly, else from the
        // range left; the range itself is carried, not recomputed from the energy
        float tend, rend;
        if (which == 2) { tend = tlim; rend = rlim; }
        else { rend = s.r - rho * step; tend = fmaxf(energy_of_range(A.tab, rend, sp), tlim); }
        const float th0 = highland(s.t, step, rho);
        electron_deposit(A, acc, s, iv, s.t - tend);
        s.t = tend;
        s.r = rend;
        s.x += step * s.u; s.y += step * s.v; s.z += step * s.w;
        s.nlam -= step * sig;
        if (!(A.flags & PSL_PHYS_NO_MSC) && step > 0.0f) {
            const float l2 = -2.0f * ln_uniform(rng.take());
            const float th = th0 * (l2 * rsqrtf(l2));
            float st, ct, sp, cp;
            sincos_polar(th, &st, &ct);
            st = fabsf(st);
            sincos_2pi(rng.take(), &sp, &cp);
            rotate_dir(s.u, s.v, s.w, ct, st, sp, cp);
        }
        if (which == 1) {
            // the crossed axis moves to the shared face and one cell on; the
            // others stay inside the grid, so one unsigned test finds an exit
            // (selects, no branch per axis)
            const int up = cross > 0;
            const int cx = axis == 0 ? cross : 0, cy = axis == 1 ? cross : 0, cz = axis == 2 ? cross : 0;
            s.x = axis == 0 ? (float)(s.ix + up) * A.vx : s.x;
            s.y = axis == 1 ? (float)(s.iy + up) * A.vy : s.y;
            s.z = axis == 2 ? (float)(s.iz + up) * A.vz : s.z;
            s.ix += cx; s.iy += cy; s.iz += cz;
            const int out = (unsigned)s.ix >= (unsigned)A.nx || (unsigned)s.iy >= (unsigned)A.ny || (unsigned)s.iz >= (unsigned)A.nz;
            if (out) {
                electron_flush(A, acc, s);
                escape(A, acc, s.t + (POS ? 2.0f * F_ME : 0.0f), s.wt, s.root);
                return E_END;
            }
        }
        if (which == 0) return E_HARD;
        if (!(s.t <= A.ecut)) return E_ON;
        iv = ((uint32_t)s.iz * (uint32_t)A.ny + (uint32_t)s.iy) * (uint32_t)A.nx + (uint32_t)s.ix;
    }                                                         // the step's draws are committed here
    if (s.steps > MAX_E_STEPS) atomicOr(A.err, PSL_DEV_ERR_STEPS);
    electron_flush(A, acc, s);
    electron_end<POS>(A, acc, s, iv);
    return E_END;
}

// the hard event (Moller delta ray or bremsstrahlung photon) that ended the
// last step; the electron stays in the voxel of that step
template <bool POS, class AT>
__device__ __forceinline__ void electron_hard(const AT &A, Acc &acc, Electron &s, uint32_t *bh) {
    const uint32_t iv = ((uint32_t)s.iz * (uint32_t)A.ny + (uint32_t)s.iy) * (uint32_t)A.nx + (uint32_t)s.ix;
    EventRng ev(s.draw);
    Rng &rng = ev.r;
    {
        int tj; float tg;
        tab_pos(A.tab, s.t, tj, tg);
        constexpr int sp = POS ? NT : 0;
        const float4 e2 = lerp4(A.tab.el + sp, tj, tg);
        const float sm = s.t > (sp ? A.wcc : 2.0f * A.wcc) ? e2.y : 0.0f, sb = s.t > A.wcb ? e2.z : 0.0f;
        rng.align();                                            // the hard event's draws
        const float r = rng.next(A.rk, s.p0, s.p1) * (sm + sb);
        if (sm + sb > 0.0f) {
            if (r < sm) {                                         // hard Moller (e-) or Bhabha (e+)
                acc.ev += EV_HARD;
                const float eps = POS ? sample_bhabha(s.t, A.wcc, rng, A.rk, s.p0, s.p1, A.err)
                                        : sample_moller(s.t, A.wcc, rng, A.rk, s.p0, s.p1, A.err);
                const float W = eps * s.t, tp = s.t - W;
                // polar cosines of the two electrons from momentum balance;
                // their sines from the same balance without cancellation
                const float cp = sqrtf(tp * (s.t + 2.0f * F_ME) / (s.t * (tp + 2.0f * F_ME)));
                const float cd = sqrtf(W * (s.t + 2.0f * F_ME) / (s.t * (W + 2.0f * F_ME)));
                const float sp_ = sqrtf(2.0f * F_ME * W / (s.t * (tp + 2.0f * F_ME)));
                const float sd_ = sqrtf(2.0f * F_ME * tp / (s.t * (W + 2.0f * F_ME)));
                float sph, cph;
                sincos_2pi(rng.next(A.rk, s.p0, s.p1), &sph, &cph);
                float du = s.u, dv = s.v, dw = s.w;
                rotate_dir(du, dv, dw, cd, sd_, -sph, -cph);              // azimuth phi + pi
                rotate_dir(s.u, s.v, s.w, cp, sp_, sph, cph);
                emit_charged(A, acc, rng, bh, 1, W, s.x, s.y, s.z, du, dv, dw, s.wt, iv, s.p0, s.p1, s.nchild, s.root);
                s.t = tp;
            } else {                                              // hard bremsstrahlung
                const float kph = A.wcb * expf(rng.next(A.rk, s.p0, s.p1) * logf(s.t / A.wcb));
                if (A.flags & PSL_PHYS_LOCAL_SECONDARIES) deposit(A, acc, iv, kph, s.wt, s.root);
                else push_particle(A.p_out, A, 0, s.x, s.y, s.z, s.u, s.v, s.w, kph, s.wt, s.p0, s.p1, s.nchild, s.root);
                s.t -= kph;
            }
            s.r = range_of(A.tab, s.t, sp);
        }
        s.nlam = -1.0f;                                           // drawn at the next step
    }
}

// One species' queue: each lane steps one particle and takes the next
// when it ends (POS: positrons, with their own tables and Bhabha
// collisions; the electron loop compiles without the positron branches - a
// runtime species cost the electron pass 5 %).
template <bool POS, class AT>
__device__ __forceinline__ void electron_loop(const AT &A, Acc &acc, const Particle *src, uint32_t n,
                                              uint32_t *head, uint32_t *bh) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    Electron s;
    bool alive = false, done = false, hard = false;
    uint32_t cbase = 0, cleft = 0;        // the warp's claimed queue range not yet handed out
    for (;;) {
        // Hard events wait until enough lanes have one (or every live lane
        // waits), so that the long hard-event code runs with most lanes
        // active; the other lanes keep stepping meanwhile.
        const unsigned hm = __ballot_sync(FULL, hard), live0 = __ballot_sync(FULL, alive);
        if (hm && (__popc(hm) >= PSL_E_DEFER || hm == live0)) {
            if (hard) { electron_hard<POS>(A, acc, s, bh); hard = false; }
        }
        // lanes whose particle ended (in this pass's step or before) take the next
        const unsigned need = __ballot_sync(FULL, !alive && !done);
        if (need) {
            // the needing lanes take, in lane order, the rest of the warp's
            // claim and then a new claim of at least PSL_E_CLAIM entries
            // (indices past the queue's end mean it is exhausted)
            const uint32_t nn = __popc(need), k = __popc(need & lt);
            uint32_t nb = 0, c = 0;
            if (nn > cleft) {                                 // claim more (warp-uniform)
                c = max(nn - cleft, (uint32_t)PSL_E_CLAIM);
                if (lane == 0) nb = atomicAdd(head, c);
                nb = __shfl_sync(FULL, nb, 0);
            }
            const uint32_t ck = cleft, cb = cbase;
            if (nn > ck) { cbase = nb + (nn - ck); cleft = c - (nn - ck); } else { cbase += nn; cleft -= nn; }
            if (!alive && !done) {
                const uint32_t idx = k < ck ? cb + k : nb + (k - ck);
                if (idx < n) {
                    const Particle p = load_particle(src + idx);
                    s.x = p.x; s.y = p.y; s.z = p.z; s.u = p.u; s.v = p.v; s.w = p.w; s.t = p.e; s.wt = p.wt;
                    s.p0 = p.pid_lo; s.p1 = p.pid_hi; s.root = p.root; s.nchild = 0; s.steps = 0;
                    s.ix = min(max((int)floorf(s.x * A.ivx), 0), A.nx - 1);
                    s.iy = min(max((int)floorf(s.y * A.ivy), 0), A.ny - 1);
                    s.iz = min(max((int)floorf(s.z * A.ivz), 0), A.nz - 1);
                    s.draw = 0;
#if PSL_DEP_COMBINE
                    s.piv = 0xFFFFFFFFu; s.pq = 0ull;
#endif
                    s.nlam = -1.0f;                               // drawn at the first step
                    s.r = range_of(A.tab, s.t, POS ? NT : 0);
                    alive = true;
                } else {
                    done = true;
                }
            }
        }
        if (!__ballot_sync(FULL, alive)) break;
        if (alive && !hard) {
            const int r = electron_step<POS>(A, acc, s);
            alive = r != E_END;
            hard = r == E_HARD;
        }
    }
}

// The electron pass: the band-ordered electrons, then (as each warp runs out
// of electrons) the generation's positrons from their own queue.
template <bool TR>
__global__ void __launch_bounds__(256, PSL_TRANSPORT_MIN_BLOCKS) k_electron(ArgsT<TR> A, const Particle *src, const uint32_t *n_ptr, uint32_t cap,
                                                  uint32_t *head, const Particle *psrc, const uint32_t *pn_ptr,
                                                  uint32_t pcap, uint32_t *phead) {
    // electrons live for several steps and their queue reads hit L1, so
    // refills load directly (a staged feed measured 2 % slower here)
    __shared__ uint32_t bh[NBANDS];
    __shared__ unsigned long long sled[NLEDGER];
    band_hist_init(bh);
    acc_init(sled);
    __syncthreads();
    Acc acc = {0u, 0u, 0ull, 0ull};
    electron_loop<false>(A, acc, src, min(*n_ptr, cap), head, bh);
    electron_loop<true>(A, acc, psrc, min(*pn_ptr, pcap), phead, bh);
    flush_acc(A, acc, sled, 6, 9, 11);
    band_hist_flush(A, bh);
}

// Slice of every caller particle of a materialised batch: the given one, or
// (slice < 0) its history's by the particle id.
__global__ void k_assign_slices(Args A, Particle *p, int64_t nph, int64_t nel, int64_t cap, int32_t slice) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nph + nel; t += (int64_t)gridDim.x * blockDim.x) {
        Particle *q = p + (t < nph ? t : cap - 1 - (t - nph));
        const uint32_t sl = slice >= 0 ? (uint32_t)slice : history_slice(q->pid_lo, q->pid_hi, A.rk, A.n_slices);
        q->root = (sl << ROOT_SLICE_SHIFT) | (q->root & ROOT_INDEX_MASK);
    }
}

// ---------------------------------------------------------------- source ---
// Source stage of a lazy batch (histories first + i * stride): accepted
// photons are written to the primary buffer, charged primaries go straight to
// the electron queue.  Each warp locates its first history and its lanes
// reuse that (group, segment) when it is also theirs.
// Batch of every history of a window [first, first + n): the key of the
// stable sort that partitions the window batch by batch.
__global__ void __launch_bounds__(256) k_slice_keys(Args A, int64_t first_block, uint32_t n, uint32_t nb, uint32_t *keys) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        keys[i] = block_slice((uint64_t)(first_block + i), A.rk, nb);
}

__global__ void k_or_err(const uint32_t *src, uint32_t *err) {
    if (*src) atomicOr(err, *src);
}

// off[b] = first position of batch b in the sorted keys (off[nb] = n)
__global__ void k_slice_bounds(const uint32_t *keys, uint32_t n, uint32_t nb, uint32_t *off) {
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b <= nb; b += gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = n;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (keys[mid] < b) lo = mid + 1; else hi = mid;
        }
        off[b] = lo;
    }
}

// Histories first + i * stride, i < n; or (LIST, the batch-by-batch
// order) the histories of one batch of the window [first, first + stride):
// the blocks list[list_off[slice] ...] (offsets from the window's first
// batch block, sorted by batch), each block's BATCH_BLOCK consecutive ids
// clipped to the window (at most n histories: more is an overflow).
// TRACE: the instance launched while a tally records the source stage
// (psl_tally_trace_source); the production instances compile without it.
template <bool TRACE, bool LIST>
__global__ void __launch_bounds__(256, SRC_MIN_BLOCKS) k_source(Args A, PlanDev P, int64_t first, int64_t stride, uint32_t n,
                                                uint32_t root0, int32_t slice, Particle *out, uint32_t *count,
                                                const uint32_t *list, const uint32_t *list_off, SrcTraceDev T) {
    __shared__ PlanShared S;
    __shared__ uint32_t bh[NBANDS];
    __shared__ unsigned long long sled[NLEDGER];
    plan_shared_load(P, S);
    band_hist_init(bh);
    acc_init(sled);
    __syncthreads();
    const uint32_t cap = n;
    // list mode (one batch of a window, PSL_ORDER_BATCH): the batch's blocks of
    // BATCH_BLOCK consecutive histories, as offsets from the window's first
    // block (first >> BATCH_BLOCK_SHIFT); the window is [first, first + stride)
    uint32_t lbase = 0, n_runs;
    if (LIST) {
        // (bounds from a sort whose look-back gave up may be out of order:
        // then the batch is skipped, and the error word already says why)
        const uint32_t o0 = list_off[slice], o1 = list_off[slice + 1];
        n_runs = o1 >= o0 ? o1 - o0 : 0u;
        lbase = o0;
        // every block but the window's first and last is whole: more of them
        // than the pass holds is an overflow (the primary queue's own check
        // catches the rest)
        if (n_runs > 2u && (uint64_t)(n_runs - 2u) * BATCH_BLOCK > n && blockIdx.x == 0 && threadIdx.x == 0)
            atomicOr(A.err, PSL_DEV_ERR_QUEUE);
    } else {
        n_runs = (n + SRC_RUN - 1) / SRC_RUN;
    }
    static_assert(SRC_RUN == BATCH_BLOCK, "a run of the source stage is a batch block");
    Acc acc = {0u, 0u, 0ull, 0ull};
    unsigned long long emitted = 0, missed = 0;      // this thread's fixed-point energy
    const int lane = threadIdx.x & 31;
    // each warp takes runs of SRC_RUN consecutive histories, 32 at a time,
    // and each lane carries its (group, segment) to the next 32: consecutive
    // histories stay in a segment or step to the next, so the searches are
    // rare; the runs are dealt out in turn, so that all warps read nearby
    // records of the reading order at the same time
    const uint32_t n_warps = gridDim.x * (blockDim.x >> 5);
    const uint32_t gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int g = -1;
    int64_t q = -1;
    for (uint32_t run = gw; run < n_runs; run += n_warps) {
    // the run's histories: hbase + j, 0 <= j < len (call index ib0 + j)
    int64_t hbase;
    uint32_t len, ib0;
    if (LIST) {
        const int64_t blk = (first >> BATCH_BLOCK_SHIFT) + (int64_t)__ldg(list + lbase + run);
        const int64_t lo = max(blk << BATCH_BLOCK_SHIFT, first);
        const int64_t hi = min((blk + 1) << BATCH_BLOCK_SHIFT, first + stride);
        hbase = lo;
        len = hi > lo ? (uint32_t)(hi - lo) : 0u;
        ib0 = 0;
    } else {
        ib0 = run * SRC_RUN;
        hbase = first + (int64_t)ib0 * stride;
        len = min(n - ib0, (uint32_t)SRC_RUN);
    }
    for (uint32_t jb = 0; jb < len; jb += 32u * SRC_ILP) {
        // SRC_ILP histories per lane, 32 apart: their plan lookups and
        // record reads are issued together, so that their latencies overlap
        bool ok[SRC_ILP];
        int64_t h[SRC_ILP], use[SRC_ILP], qk[SRC_ILP];
        int gk[SRC_ILP];
#pragma unroll
        for (int k = 0; k < SRC_ILP; ++k) {
            const uint32_t j = jb + 32u * k + lane;
            ok[k] = j < len;
            h[k] = hbase + (int64_t)(ok[k] ? j : 0u) * (LIST ? 1 : stride);
            if (k == 0 && jb == 0) {
                if (lane == 0 && ok[0]) locate(P, S, h[0], g, q);
                g = __shfl_sync(FULL, g, 0);
                q = __shfl_sync(FULL, q, 0);
            }
            if (ok[k]) locate_hinted(P, S, h[k], g, q);
            gk[k] = g; qk[k] = q;
        }
        // the segment -> entry -> record chain of the plan lookup, as source_at
        EntryDev E[SRC_ILP];
#pragma unroll
        for (int k = 0; k < SRC_ILP; ++k) {
            if (!ok[k]) continue;
            const SegDev sg = P.seg[qk[k]];
            uint64_t rq, pidx;
            divmod_u64((uint64_t)(h[k] - S.gs[gk[k]] - sg.h), (uint64_t)sg.w, rq, pidx);
            use[k] = sg.r0 + (int64_t)rq;
            E[k] = P.ent[S.gseg[gk[k]] + (int64_t)pidx];
        }
        PslRecord R[SRC_ILP];
        int64_t ri[SRC_ILP];
#pragma unroll
        for (int k = 0; k < SRC_ILP; ++k) {
            if (!ok[k]) continue;
            uint64_t rw, rr;
            divmod_u64((uint64_t)(E[k].offset + use[k]), (uint64_t)E[k].nrec, rw, rr);
            ri[k] = E[k].start + (int64_t)rr;
            R[k] = P.rec[ri[k]];
        }
#pragma unroll
        for (int k = 0; k < SRC_ILP; ++k) {
            const uint32_t i = LIST ? 0u : ib0 + jb + 32u * k + lane;   // index in the call (traced transport)
            SrcOut o;
            o.status = -1;
            if (ok[k]) record_to_phantom(R[k], P.beams[E[k].beam], P.z_psl, P.L, P.origin, true, o);
            if (TRACE && ok[k]) {                                   // traced call (tests)
                const int64_t t = h[k] - T.first;
                if (t >= 0 && t < T.n) {
                    if (T.entry) T.entry[t] = E[k].entry;
                    if (T.use) T.use[t] = use[k];
                    if (T.rec) T.rec[t] = ri[k];
                    if (T.status) T.status[t] = (int8_t)o.status;
                    if (T.ptype) T.ptype[t] = o.ptype;
                    if (T.state && o.status == PSL_SRC_TRANSPORT)
                        for (int c = 0; c < 8; ++c) T.state[8 * t + c] = o.s[c];
                }
            }
            if (o.status == PSL_SRC_TRANSPORT || o.status == PSL_SRC_MISS) {
                const unsigned long long e = fixed_point(o.s[6], o.s[7]);
                emitted += e;
                if (o.status == PSL_SRC_MISS) missed += e;
            }
            if (o.status == PSL_SRC_TRANSPORT) {
                Particle c;
                c.x = o.s[0]; c.y = o.s[1]; c.z = o.s[2]; c.e = o.s[6];
                c.u = o.s[3]; c.v = o.s[4]; c.w = o.s[5]; c.wt = o.s[7];
                c.pid_lo = (uint32_t)h[k]; c.pid_hi = (uint32_t)((uint64_t)h[k] >> 32);
                c.type = (uint32_t)o.ptype;
                const uint32_t sl = slice >= 0 ? (uint32_t)slice : history_slice(c.pid_lo, c.pid_hi, A.rk, A.n_slices);
                c.root = (sl << ROOT_SLICE_SHIFT) | ((root0 + i) & ROOT_INDEX_MASK);
                if (o.ptype == 0) {
                    queue_push(Queue{out, count, cap}, c, A.err);
                } else {
                    if (o.ptype == 1) atomicAdd(&bh[band_of(A, c.e)], 1u);
                    queue_push(A.e_out, c, A.err);
                }
            }
        }
    }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        emitted += __shfl_xor_sync(FULL, emitted, o);
        missed += __shfl_xor_sync(FULL, missed, o);
    }
    if (lane == 0) {
        if (emitted) atomicAdd(&sled[0], emitted);
        if (missed) atomicAdd(&sled[1], missed);
    }
    flush_acc(A, acc, sled, 6, 8, -1);
    band_hist_flush(A, bh);
}

// ------------------------------------------------------------ band sort ---
__device__ __forceinline__ const Particle *pick(const Particle *a, uint32_t na, const Particle *b, uint32_t i) {
    return i < na ? a + i : b + (i - na);
}

__global__ void __launch_bounds__(256) k_band_count(Args A, const Particle *a, uint32_t na, const Particle *b,
                                                    const uint32_t *nb_ptr, uint32_t capb, uint32_t *hist) {
    __shared__ uint32_t h[NBANDS];
    if (threadIdx.x < NBANDS) h[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t n = na + min(*nb_ptr, capb);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Particle *q = pick(a, na, b, i);
        if (__ldg(&q->type) != 2u) atomicAdd(&h[band_of(A, __ldg(&q->e))], 1u);
    }
    __syncthreads();
    if (threadIdx.x < NBANDS && h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

__global__ void k_band_scan(uint32_t *hist, uint32_t *cursor, uint32_t *out_count) {
    const int t = threadIdx.x;                  // one warp
#if PSL_BAND_DESC
    // highest band first: the longest-lived electrons start first and the
    // short ones fill the lanes at the end of the pass
    const int b = NBANDS - 1 - t;
#else
    const int b = t;
#endif
    uint32_t v = hist[b], x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(FULL, x, o);
        if (t >= o) x += y;
    }
    cursor[b] = x - v;
    hist[b] = 0;
    if (t == 31) *out_count = x;
}

// Electrons go to dst in band order; positrons to the positron queue (their
// own pass, k_electron<true>).
__global__ void __launch_bounds__(256) k_band_scatter(Args A, const Particle *a, uint32_t na, const Particle *b,
                                                      const uint32_t *nb_ptr, uint32_t capb, uint32_t *cursor,
                                                      Particle *dst, uint32_t capd, Queue pos_q) {
    __shared__ uint32_t h[NBANDS], base[NBANDS];
    const uint32_t n = na + min(*nb_ptr, capb);
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i0 = blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
        if (threadIdx.x < NBANDS) h[threadIdx.x] = 0;
        __syncthreads();
        const uint32_t i = i0 + threadIdx.x;
        Particle p;
        int bnd = 0;
        uint32_t local = 0;
        const bool have = i < n;
        bool positron = false;
        if (have) {
            p = load_particle(pick(a, na, b, i));
            positron = p.type == 2u;
            bnd = band_of(A, p.e);
            if (!positron) local = atomicAdd(&h[bnd], 1u);
        }
        __syncthreads();
        if (threadIdx.x < NBANDS && h[threadIdx.x]) base[threadIdx.x] = atomicAdd(&cursor[threadIdx.x], h[threadIdx.x]);
        __syncthreads();
        if (have && positron) {
            queue_push(pos_q, p, A.err);
        } else if (have) {
            uint32_t d = base[bnd] + local;
            if (d < capd) store_particle(dst + d, p);
            else atomicOr(A.err, PSL_DEV_ERR_QUEUE);
        }
        __syncthreads();
    }
}

// after a fixed generation budget: count particles that were left undone
__global__ void k_accumulate_leftover(uint32_t *cnt) { cnt[12] += cnt[10] + cnt[11]; }

__global__ void k_ledger_add(unsigned long long *ledger, const unsigned long long *src) {
    ledger[0] += src[0];
    ledger[1] += src[1];
}

// --------------------------------------------------------------- state ---
struct TableCache {
    int device = -1;
    float wcc = -1.f, wcb = -1.f;
    float4 *ph0 = nullptr, *ph1 = nullptr, *el = nullptr;
    float4 *rng = nullptr;
    float *irng = nullptr;
    float igrid[4] = {0.f, 0.f, 0.f, 0.f};   // per species: ln R0, 1 / d ln R
};
std::mutex g_tab_mu;
std::vector<TableCache> g_tabs;

int get_tables(float wcc, float wcb, cudaStream_t st, TableCache &out) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_tab_mu);
    for (auto &t : g_tabs)
        if (t.device == dev && t.wcc == wcc && t.wcb == wcb) { out = t; return PSL_OK; }
    TableCache t;
    t.device = dev; t.wcc = wcc; t.wcb = wcb;
    PSL_CUDA(cudaMalloc((void **)&t.ph0, NT * sizeof(float4)));
    PSL_CUDA(cudaMalloc((void **)&t.ph1, NT * sizeof(float4)));
    PSL_CUDA(cudaMalloc((void **)&t.el, 2 * NT * sizeof(float4)));
    PSL_CUDA(cudaMalloc((void **)&t.rng, 2 * NT * sizeof(float4)));
    k_tables<<<(NT + 255) / 256, 256, 0, st>>>(t.ph0, t.ph1, t.el, (double)wcc, (double)wcb); PSL_NOTE_LAUNCH();
    double *iv = nullptr;
    float *ig = nullptr;
    PSL_CUDA(cudaMalloc((void **)&iv, 2 * NT * sizeof(double)));
    PSL_CUDA(cudaMalloc((void **)&ig, 4 * sizeof(float)));
    PSL_CUDA(cudaMalloc((void **)&t.irng, 2 * NT * sizeof(float)));
    k_range_intervals<<<dim3((NT + 127) / 128, 2), 128, 0, st>>>(iv, (double)wcc, (double)wcb); PSL_NOTE_LAUNCH();
    k_range_table<<<2, 1024, 0, st>>>(iv, t.rng, t.irng, ig, (double)wcc, (double)wcb); PSL_NOTE_LAUNCH();
    PSL_CUDA(cudaMemcpyAsync(t.igrid, ig, 4 * sizeof(float), cudaMemcpyDeviceToHost, st));
    PSL_CUDA(cudaStreamSynchronize(st));
    cudaFree(iv);
    cudaFree(ig);
    PSL_CUDA(cudaGetLastError());
    PSL_CUDA(cudaStreamSynchronize(st));
    g_tabs.push_back(t);
    out = t;
    return PSL_OK;
}

}  // namespace

struct Workspace {
    int device = 0;                    // the device its buffers live on
    int64_t chunk = 0;                 // primaries per pass the buffers are sized for
    uint32_t cap_p = 0, cap_e = 0, cap_s = 0, cap_q = 0;
    Particle *P[2] = {nullptr, nullptr}, *E[2] = {nullptr, nullptr}, *S = nullptr, *Q = nullptr, *Pos = nullptr;
    uint32_t *cnt = nullptr;           // [0..1] P counts, [2..3] E counts, [4] S count, [5..6] heads,
                                       // [7] primary photons, [9] err, [16..47] band hist, [48..79] cursors,
                                       // [80] positron count, [81] positron head
    int *rmax = nullptr;
    float *mrho = nullptr;             // packed material/density of the phantom
    int64_t nvox = 0;
    uint32_t *host = nullptr;          // pinned: counts read back
    // batch-by-batch order (psl_run): a window's batch keys and history
    // offsets, sorted by batch, the sort's scratch and the batch bounds
    int64_t bm_cap = 0;
    uint32_t *bm_keys[2] = {nullptr, nullptr}, *bm_vals[2] = {nullptr, nullptr}, *bm_off = nullptr;
    void *bm_scratch = nullptr;
    // cached CUDA graph of one psl_run call
    cudaGraphExec_t graph = nullptr;
    uint64_t graph_key[11] = {0};
    // cached CUDA graph of one psl_plan_replay call (reset, run, readout)
    cudaGraphExec_t plan_graph = nullptr;
    uint64_t plan_key[16] = {0};
};

void workspace_free(Workspace *w) {
    if (!w) return;
    if (w->graph) cudaGraphExecDestroy(w->graph);
    if (w->plan_graph) cudaGraphExecDestroy(w->plan_graph);
    for (int k = 0; k < 2; ++k) { if (w->P[k]) cudaFree(w->P[k]); if (w->E[k]) cudaFree(w->E[k]); }
    if (w->S) cudaFree(w->S);
    if (w->Q) cudaFree(w->Q);
    if (w->Pos) cudaFree(w->Pos);
    if (w->cnt) cudaFree(w->cnt);
    if (w->rmax) cudaFree(w->rmax);
    if (w->mrho) cudaFree(w->mrho);
    if (w->host) cudaFreeHost(w->host);
    for (int k = 0; k < 2; ++k) { if (w->bm_keys[k]) cudaFree(w->bm_keys[k]); if (w->bm_vals[k]) cudaFree(w->bm_vals[k]); }
    if (w->bm_off) cudaFree(w->bm_off);
    if (w->bm_scratch) cudaFree(w->bm_scratch);
    delete w;
}

// Queue bytes per primary of a pass: photons 2 x 3, electrons 2 x 8, the
// regrouped electrons 9, the primary photons 1 and the positrons 1 particles
constexpr int64_t WORKSPACE_BYTES_PER_PRIMARY = 33 * (int64_t)sizeof(Particle);

// Device bytes a workspace holds: the particle queues (photons 2 x cap_p,
// electrons 2 x cap_e, the regrouped electrons cap_s, the primary photons
// one chunk), the packed densities and the batch-order buffers.
int64_t workspace_bytes_of(const Workspace *w) {
    if (!w) return 0;
    const int64_t base = std::max<int64_t>(w->chunk, 4096);
    int64_t b = (2 * (int64_t)w->cap_p + 2 * (int64_t)w->cap_e + (int64_t)w->cap_s + (int64_t)w->cap_q + base) *
                (int64_t)sizeof(Particle);
    b += 128 * 4 + 2 * 4 + w->nvox * 4;
    if (w->bm_cap) b += 16 * w->bm_cap + (PSL_MAX_BATCHES + 1) * 4 + (int64_t)sort_pairs_scratch_bytes((uint32_t)w->bm_cap);
    return b;
}

// The workspace of a destroyed tally, kept for the next tally on the same
// device: its particle queues hold ~30 x chunk particles (26 GB at the
// default chunk of 2^24) and mapping them afresh cost ~14 ms per tally.  At
// most WS_CACHE_MAX are kept; psl_memory_trim frees them.
namespace {
constexpr size_t WS_CACHE_MAX = 1;
std::mutex g_ws_mu;
std::vector<Workspace *> g_ws_cache;
}  // namespace

// A destroyed tally's workspace: into the cache (after the device is idle,
// as cudaFree would wait too), or freed when the cache is full.
void workspace_release(Workspace *w) {
    if (!w) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != w->device) cudaSetDevice(w->device);
    cudaDeviceSynchronize();                         // the device the queues live on
    if (cur != w->device) cudaSetDevice(cur);
    if (w->graph) { cudaGraphExecDestroy(w->graph); w->graph = nullptr; }
    std::memset(w->graph_key, 0, sizeof(w->graph_key));
    if (w->plan_graph) { cudaGraphExecDestroy(w->plan_graph); w->plan_graph = nullptr; }
    std::memset(w->plan_key, 0, sizeof(w->plan_key));
    Workspace *drop = w;
    {
        std::lock_guard<std::mutex> lk(g_ws_mu);
        if (g_ws_cache.size() < WS_CACHE_MAX) { g_ws_cache.push_back(w); drop = nullptr; }
    }
    workspace_free(drop);
}

// Free the cached workspaces of the current device (psl_memory_trim).
void workspace_cache_trim() {
    int dev = 0;
    cudaGetDevice(&dev);
    std::vector<Workspace *> out;
    {
        std::lock_guard<std::mutex> lk(g_ws_mu);
        for (size_t i = 0; i < g_ws_cache.size();) {
            if (g_ws_cache[i]->device == dev) { out.push_back(g_ws_cache[i]); g_ws_cache.erase(g_ws_cache.begin() + i); }
            else ++i;
        }
    }
    for (Workspace *w : out) workspace_free(w);
}

// A cached workspace of this device with room for `chunk` primaries, or null.
static Workspace *workspace_take(int dev, int64_t chunk) {
    std::lock_guard<std::mutex> lk(g_ws_mu);
    for (size_t i = 0; i < g_ws_cache.size(); ++i) {
        Workspace *w = g_ws_cache[i];
        if (w->device == dev && w->chunk >= chunk) {
            g_ws_cache.erase(g_ws_cache.begin() + i);
            return w;
        }
    }
    return nullptr;
}

// Resident 256-thread blocks of the source kernel per SM: its grid is one
// wave, since each warp takes an equal contiguous run of histories.
static int source_blocks_per_sm() {
    static int nb = 0;
    if (!nb) {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_source<false, false>, 256, 0) != cudaSuccess || v < 1) v = 4;
        nb = v;
    }
    return nb;
}

// Batch-by-batch order (PSL_ORDER_BATCH): batch blocks per window, so that
// the blocks of one batch of a window (binomial, mean Wb / nb) hold at most
// one transport pass of `chunk` primaries by 8 standard deviations:
// x = Wb / nb with x + 8 sqrt(x) = chunk / BATCH_BLOCK.
static int64_t batch_window(int64_t chunk, int nb) {
    const double r = std::sqrt((double)chunk / BATCH_BLOCK + 16.0) - 4.0;
    return std::min<int64_t>(std::max<int64_t>(1, (int64_t)(r * r * nb)), (int64_t)1 << 24);
}

static bool use_batch_order(const psl_tally *t) {
    if (t->n_batches < 2 || t->order == PSL_ORDER_READING) return false;
    if (t->order == PSL_ORDER_BATCH) return true;
    int dev = 0, l2 = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    return (double)t->nvox * (double)t->n_batches * 8.0 > 0.5 * (double)l2;
}

static int batch_order_ensure(psl_tally *t, int64_t W) {
    Workspace *w = t->ws;
    if (w->bm_cap >= W) return PSL_OK;
    for (int k = 0; k < 2; ++k) {
        if (w->bm_keys[k]) cudaFree(w->bm_keys[k]);
        if (w->bm_vals[k]) cudaFree(w->bm_vals[k]);
        w->bm_keys[k] = w->bm_vals[k] = nullptr;
    }
    if (w->bm_off) cudaFree(w->bm_off);
    if (w->bm_scratch) cudaFree(w->bm_scratch);
    w->bm_off = nullptr; w->bm_scratch = nullptr; w->bm_cap = 0;
    for (int k = 0; k < 2; ++k) {
        PSL_CUDA(cudaMalloc((void **)&w->bm_keys[k], (size_t)W * 4));
        PSL_CUDA(cudaMalloc((void **)&w->bm_vals[k], (size_t)W * 4));
    }
    PSL_CUDA(cudaMalloc((void **)&w->bm_off, (PSL_MAX_BATCHES + 1) * 4));
    PSL_CUDA(cudaMalloc((void **)&w->bm_scratch, sort_pairs_scratch_bytes((uint32_t)W)));
    w->bm_cap = W;
    return PSL_OK;
}

static int workspace_ensure(psl_tally *t, int64_t chunk) {
    Workspace *w = t->ws;
    if (w && w->chunk >= chunk) return PSL_OK;
    if (w) { cudaDeviceSynchronize(); workspace_free(w); t->ws = nullptr; }
    int dev = 0;
    PSL_CUDA(cudaGetDevice(&dev));
    if ((w = workspace_take(dev, chunk))) {
        t->ws = w;
        if (w->nvox < t->nvox) {                     // the phantom's packed densities need more room
            PSL_CUDA(cudaFree(w->mrho));
            w->mrho = nullptr;
            PSL_CUDA(cudaMalloc((void **)&w->mrho, t->nvox * sizeof(float)));
            w->nvox = t->nvox;
        }
        return PSL_OK;
    }
    w = new Workspace();
    t->ws = w;
    w->device = dev;
    w->chunk = chunk;
    const int64_t base = std::max<int64_t>(chunk, 4096);
    w->cap_p = (uint32_t)std::min<int64_t>(3 * base, 0xF0000000ll);
    w->cap_e = (uint32_t)std::min<int64_t>(8 * base, 0xF0000000ll);
    w->cap_s = w->cap_e + (uint32_t)base;
    w->cap_q = (uint32_t)std::min<int64_t>(base, 0xF0000000ll);   // positrons of a generation (pairs are rare)
    PSL_CUDA(cudaMalloc((void **)&w->P[0], (size_t)w->cap_p * sizeof(Particle)));
    PSL_CUDA(cudaMalloc((void **)&w->P[1], (size_t)w->cap_p * sizeof(Particle)));
    PSL_CUDA(cudaMalloc((void **)&w->E[0], (size_t)w->cap_e * sizeof(Particle)));
    PSL_CUDA(cudaMalloc((void **)&w->E[1], (size_t)w->cap_e * sizeof(Particle)));
    PSL_CUDA(cudaMalloc((void **)&w->S, (size_t)w->cap_s * sizeof(Particle)));
    PSL_CUDA(cudaMalloc((void **)&w->Q, (size_t)base * sizeof(Particle)));
    PSL_CUDA(cudaMalloc((void **)&w->Pos, (size_t)w->cap_q * sizeof(Particle)));
    PSL_CUDA(cudaMalloc((void **)&w->cnt, 128 * sizeof(uint32_t)));
    PSL_CUDA(cudaMemset(w->cnt, 0, 128 * sizeof(uint32_t)));
    PSL_CUDA(cudaMalloc((void **)&w->rmax, 2 * sizeof(int)));
    PSL_CUDA(cudaMalloc((void **)&w->mrho, t->nvox * sizeof(float)));
    w->nvox = t->nvox;
    PSL_CUDA(cudaMallocHost((void **)&w->host, 16 * sizeof(uint32_t)));
    return PSL_OK;
}

// Secondary generations launched per pass when no host check is made
#define RUN_GENERATIONS 10

// One batch of work: either a lazy history range (source stage inside) or
// caller / materialised particles.
struct Job {
    bool lazy = false;
    PlanDev P{};
    int64_t first = 0, stride = 1, n = 0;            // lazy
    const uint32_t *list = nullptr, *list_off = nullptr;  // lazy, one batch of a sorted window (slice = the batch)
    const Particle *p = nullptr;                     // materialised
    int64_t nph = 0, nel = 0, cap = 0;
    int32_t slice = 0;
};

struct Runner {
    cudaStream_t st = nullptr;
    psl_tally *tally = nullptr;
    Workspace *w = nullptr;
    Args A{};
    bool timing = false;
    int grid_t = 0, grid_m = 0, grid_src = 0;
    int64_t chunk = 0;
    uint32_t cap_p = 0, cap_e = 0, cap_s = 0, cap_q = 0;   // queue capacities in use (a test may cap them)

    int prepare(const psl_phantom_t *ph, const psl_physics_t *phys, psl_tally *t, uint64_t seed, int64_t need,
                cudaStream_t stream, bool capturing) {
        psl_physics_t P;
        psl_physics_default(&P);
        if (phys) P = *phys;
        if (!(P.electron_cut > 0.f) || !(P.photon_cut > 0.f) || !(P.wcc > P.electron_cut) || !(P.wcb > P.photon_cut))
            return psl_fail(PSL_EINVAL, "transport: bad physics thresholds");
        st = stream;
        tally = t;
        TableCache tc;
        int rc;
        if ((rc = get_tables(P.wcc, P.wcb, st, tc))) return rc;
        chunk = std::max<int64_t>(1, std::min<int64_t>(need, t->chunk_cap));
        if ((rc = workspace_ensure(t, chunk))) return rc;
        w = t->ws;
        {
            const long long qc = psl_debug_queue_cap();       // failure-detection tests only
            cap_p = qc > 0 ? (uint32_t)std::min<long long>(w->cap_p, qc) : w->cap_p;
            cap_e = qc > 0 ? (uint32_t)std::min<long long>(w->cap_e, qc) : w->cap_e;
            cap_s = qc > 0 ? (uint32_t)std::min<long long>(w->cap_s, qc) : w->cap_s;
            cap_q = qc > 0 ? (uint32_t)std::min<long long>(w->cap_q, qc) : w->cap_q;
        }
        A.wait_polls = (uint32_t)std::min<long long>(psl_wait_polls(FEED_SPIN), 0xFFFFFFFFll);
        A.dbg = psl_debug_flags();
        const int64_t nvox = t->nvox;
        cudaMemsetAsync(w->rmax, 0, 2 * sizeof(int), st);
        k_rho_max<<<(int)std::min<int64_t>((nvox + 255) / 256, psl_sm_count() * 4), 256, 0, st>>>(ph->mat, ph->rho, nvox, w->rmax, w->mrho); PSL_NOTE_LAUNCH();
        A.nx = ph->nx; A.ny = ph->ny; A.nz = ph->nz;
        A.vx = ph->vx; A.vy = ph->vy; A.vz = ph->vz;
        A.ivx = 1.0f / ph->vx; A.ivy = 1.0f / ph->vy; A.ivz = 1.0f / ph->vz;
        A.mat = ph->mat; A.rho = ph->rho; A.mrho = w->mrho;
        A.pcut = P.photon_cut; A.ecut = P.electron_cut; A.wcc = P.wcc; A.wcb = P.wcb; A.flags = P.flags;
        A.seed = seed;
        A.k0 = (uint32_t)seed; A.k1 = (uint32_t)(seed >> 32);
        for (int r = 0; r < 10; ++r) {
            A.rk[2 * r] = A.k0 + (uint32_t)r * 0x9E3779B9u;
            A.rk[2 * r + 1] = A.k1 + (uint32_t)r * 0xBB67AE85u;
        }
        A.tab.ph0 = tc.ph0; A.tab.ph1 = tc.ph1; A.tab.el = tc.el; A.tab.rng = tc.rng; A.rmax = w->rmax;
        A.tab.irng = tc.irng;
        for (int k = 0; k < 2; ++k) { A.tab.lnR0[k] = tc.igrid[2 * k]; A.tab.inv_dlnR[k] = tc.igrid[2 * k + 1]; }
        A.tab.lnE0 = (float)log(T_LO);
        A.tab.inv_dln = (float)((NT - 1) / (log(T_HI) - log(T_LO)));
        A.tab.dln = 1.0f / A.tab.inv_dln;          // (the correctly rounded reciprocal, as __frcp_rn)
        A.ledger = t->ledger;
        A.hist_dep = nullptr; A.hist_esc = nullptr; A.hist_events = nullptr;
        A.err = w->cnt + 9;
        A.band_hist = w->cnt + 16;
        A.band_ln0 = logf(P.electron_cut);
        A.band_scale = (float)(NBANDS / log(20.0 / P.electron_cut));
        cudaMemsetAsync(w->cnt, 0, 128 * sizeof(uint32_t), st);
        timing = psl_timer_on() && !capturing;
        grid_t = psl_sm_count() * t->grid_mult;
        grid_m = psl_sm_count() * 8;
        grid_src = psl_sm_count() * source_blocks_per_sm();
        return PSL_OK;
    }

    // Queues carried from chunk to chunk (and job to job) of one call: after
    // a chunk's electron pass its secondaries (photons in P[pc ^ 1],
    // electrons in E[ec ^ 1]) are not transported generation by generation
    // at once but join the next chunk's passes; drain() finishes them after
    // the last chunk.  Particles carry their own random streams and tally
    // slices, so the order changes nothing in the result.
    int pc = 0, ec = 0, gen_now = 0;
    bool begun = false, carried = false;

    uint32_t *cP(int k) { return w->cnt + k; }
    uint32_t *cE(int k) { return w->cnt + 2 + k; }

    void tb(int k, void **tok) { if (timing) psl_timer_begin(k, st, tok); }
    void te(int k, void *tok) { if (tok) psl_timer_end(k, st, tok); }
    // generations after the first two are small: a smaller grid starts faster
    int gm() const { return gen_now >= 2 ? psl_sm_count() : grid_m; }
    int gt() const { return gen_now >= 2 ? psl_sm_count() : grid_t; }

    void band_sort(const Particle *a, uint32_t na) {
        uint32_t *hist = w->cnt + 16, *cursor = w->cnt + 48, *cS = w->cnt + 4;
        void *tk = nullptr;
        tb(PK_BAND, &tk);
        // the queue's electrons were counted by the kernels that queued them;
        // only caller electrons (a materialised batch) are counted here
        if (na) { k_band_count<<<gm(), 256, 0, st>>>(A, a, na, w->E[ec], cE(ec), 0u, hist); PSL_NOTE_LAUNCH(); }
        k_band_scan<<<1, 32, 0, st>>>(hist, cursor, cS); PSL_NOTE_LAUNCH();
        cudaMemsetAsync(w->cnt + 80, 0, 4, st);                 // positrons go to their own queue
        k_band_scatter<<<gm(), 256, 0, st>>>(A, a, na, w->E[ec], cE(ec), cap_e, cursor, w->S, cap_s,
                                             Queue{w->Pos, w->cnt + 80, cap_q}); PSL_NOTE_LAUNCH();
        te(PK_BAND, tk);
    }
    // the per-history record of transport_trace is on (the kernels' traced instances)
    bool traced() const { return A.hist_dep || A.hist_esc || A.hist_events; }
    template <bool TR> static ArgsT<TR> as_traced(const Args &a) {
        ArgsT<TR> t;
        static_cast<Args &>(t) = a;
        return t;
    }
    // one photon pass over src (its count at nptr, else nfix) and, when src2
    // is given, the photons of src2 (its count at n2ptr) after them
    void photon_pass(const Particle *src, const uint32_t *nptr, uint32_t nfix, uint32_t cap,
                     const Particle *src2 = nullptr, const uint32_t *n2ptr = nullptr, uint32_t cap2 = 0) {
        Args a2 = A;
        a2.e_out = Queue{w->E[ec], cE(ec), cap_e};
        a2.p_out = Queue{w->P[pc ^ 1], cP(pc ^ 1), cap_p};
        cudaMemsetAsync(w->cnt + 5, 0, 4, st);
        void *tk = nullptr;
        tb(PK_PHOTON, &tk);
        // (a persistent grid: no more blocks than stay resident)
        const int gp = gen_now >= 2 ? psl_sm_count() : psl_sm_count() * std::min(tally->grid_mult, PSL_PHOTON_MIN_BLOCKS);
        if (traced()) k_photon<true><<<gp, 256, 0, st>>>(as_traced<true>(a2), src, nptr, nfix, cap, w->cnt + 5, src2, n2ptr, cap2);
        else k_photon<false><<<gp, 256, 0, st>>>(as_traced<false>(a2), src, nptr, nfix, cap, w->cnt + 5, src2, n2ptr, cap2);
        PSL_NOTE_LAUNCH();
        te(PK_PHOTON, tk);
    }
    void electron_pass() {
        Args a2 = A;
        a2.e_out = Queue{w->E[ec ^ 1], cE(ec ^ 1), cap_e};
        a2.p_out = Queue{w->P[pc ^ 1], cP(pc ^ 1), cap_p};
        cudaMemsetAsync(w->cnt + 6, 0, 4, st);
        void *tk = nullptr;
        tb(PK_ELECTRON, &tk);
        cudaMemsetAsync(w->cnt + 81, 0, 4, st);
        if (traced())
            k_electron<true><<<gt(), 256, 0, st>>>(as_traced<true>(a2), w->S, w->cnt + 4, cap_s, w->cnt + 6, w->Pos,
                                                   w->cnt + 80, cap_q, w->cnt + 81);
        else
            k_electron<false><<<gt(), 256, 0, st>>>(as_traced<false>(a2), w->S, w->cnt + 4, cap_s, w->cnt + 6, w->Pos,
                                                    w->cnt + 80, cap_q, w->cnt + 81);
        PSL_NOTE_LAUNCH();
        te(PK_ELECTRON, tk);
    }

    // One job, chunk by chunk: its primaries (source stage or caller
    // particles) and the secondaries carried from the chunk before.
    int run(const Job &J) {
        A.tally = tally->t;
        A.nvox = tally->nvox;
        A.n_slices = (uint32_t)tally->n_batches;
        if (!J.lazy && J.nph + J.nel > 0) {
            // caller particles: their histories' slices go into the root words
            // (the batch's own buffer: a batch is consumed by its transport)
            k_assign_slices<<<grid_m, 256, 0, st>>>(A, const_cast<Particle *>(J.p), J.nph, J.nel, J.cap, J.slice);
            PSL_NOTE_LAUNCH();
        }
        if (!begun) {
            cudaMemsetAsync(w->cnt, 0, 5 * sizeof(uint32_t), st);
            pc = 0; ec = 0;
            begun = true;
        }
        const int64_t total = J.lazy ? J.n : std::max(J.nph, J.nel);
        for (int64_t a0 = 0; a0 < total; a0 += chunk) {
            gen_now = 0;
            if (carried) {
                // the last chunk's outputs are this chunk's inputs
                pc ^= 1; ec ^= 1;
                cudaMemsetAsync(cP(pc ^ 1), 0, 4, st);
                cudaMemsetAsync(cE(ec ^ 1), 0, 4, st);
            }
            const Particle *ca = nullptr;
            uint32_t na = 0;
            if (J.lazy) {
                const uint32_t cp = (uint32_t)std::min<int64_t>(J.n - a0, chunk);
                Args a2 = A;
                a2.e_out = Queue{w->E[ec], cE(ec), cap_e};
                cudaMemsetAsync(w->cnt + 7, 0, 4, st);
                void *tk = nullptr;
                tb(PK_SOURCE, &tk);
                auto *ks = J.list ? (tally->trace.n ? k_source<true, true> : k_source<false, true>)
                                  : (tally->trace.n ? k_source<true, false> : k_source<false, false>);
                ks<<<grid_src, 256, 0, st>>>(a2, J.P, J.list ? J.first : J.first + a0 * J.stride, J.stride, cp,
                                             (uint32_t)a0, J.slice, w->Q, w->cnt + 7, J.list, J.list_off,
                                             tally->trace);
                PSL_NOTE_LAUNCH();
                te(PK_SOURCE, tk);
                // the chunk's primaries and the carried photons in one pass
                if (carried) photon_pass(w->Q, w->cnt + 7, 0, cp, w->P[pc], cP(pc), cap_p);
                else photon_pass(w->Q, w->cnt + 7, 0, cp);
            } else {
                const uint32_t cp = (uint32_t)std::max<int64_t>(0, std::min<int64_t>(J.nph - a0, chunk));
                na = (uint32_t)std::max<int64_t>(0, std::min<int64_t>(J.nel - a0, chunk));
                ca = J.p + (J.cap - a0 - na);
                if (cp && carried) photon_pass(J.p + a0, nullptr, cp, cp, w->P[pc], cP(pc), cap_p);
                else if (cp) photon_pass(J.p + a0, nullptr, cp, cp);
                else if (carried) photon_pass(w->P[pc], cP(pc), 0, cap_p);
            }
            band_sort(ca, na);
            electron_pass();
            carried = true;
        }
        return PSL_OK;
    }

    // The generations left after the last chunk.  check_from: the first
    // generation after which the host reads the queue counts (and stops when
    // they are empty); a negative value launches RUN_GENERATIONS generations
    // with no host check (graph capture) and leaves the count of undone
    // particles for finish().
    // the device's error word: a queue that overflowed or a bounded wait that
    // gave up leaves the tally incomplete
    static int device_errors(uint32_t e) {
        if (e & PSL_DEV_ERR_QUEUE) return psl_fail(PSL_EOVERFLOW, "transport: particle queue overflow (tally incomplete)");
        if (e & PSL_DEV_ERR_TIMEOUT)
            return psl_fail(PSL_ETIMEOUT, "transport: a bounded device wait gave up (tally incomplete)");
        return PSL_OK;
    }

    int drain(int check_from) {
        int rc_err = PSL_OK;
        if (!carried) return PSL_OK;
        const bool sync_gens = check_from >= 0;
        for (int gen = 0;; ++gen) {
            if (sync_gens && gen >= check_from) {
                cudaMemcpyAsync(w->host, w->cnt, 16 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
                cudaError_t e = cudaStreamSynchronize(st);
                if (e != cudaSuccess) return psl_fail(PSL_ECUDA, std::string("transport: ") + cudaGetErrorString(e));
                if ((rc_err = device_errors(w->host[9]))) return rc_err;
                if (w->host[pc ^ 1] == 0 && w->host[2 + (ec ^ 1)] == 0) break;
                if (gen >= MAX_GEN) return psl_fail(PSL_EOVERFLOW, "transport: too many secondary generations");
            } else if (!sync_gens && gen >= RUN_GENERATIONS) {
                break;
            }
            // next generation: swap current/next, clear the new "next"
            gen_now = gen + 1;
            pc ^= 1; ec ^= 1;
            cudaMemsetAsync(cP(pc ^ 1), 0, 4, st);
            cudaMemsetAsync(cE(ec ^ 1), 0, 4, st);
            photon_pass(w->P[pc], cP(pc), 0, cap_p);
            band_sort(nullptr, 0);
            electron_pass();
        }
        if (!sync_gens) {
            // the last generation's output must be empty (checked by finish())
            cudaMemcpyAsync(w->cnt + 10, cP(pc ^ 1), 4, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(w->cnt + 11, cE(ec ^ 1), 4, cudaMemcpyDeviceToDevice, st);
            k_accumulate_leftover<<<1, 1, 0, st>>>(w->cnt); PSL_NOTE_LAUNCH();
        }
        carried = false;
        return PSL_OK;
    }

    // wait, then report device-side errors and undrained queues
    int finish() {
        cudaMemcpyAsync(w->host, w->cnt, 16 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return psl_fail(PSL_ECUDA, std::string("transport: ") + cudaGetErrorString(e));
        int rc_err = device_errors(w->host[9]);
        if (rc_err) return rc_err;
        if (w->host[12]) return psl_fail(PSL_EOVERFLOW, "transport: secondaries left after the generation budget");
        return PSL_OK;
    }
};

static int check_transport_args(const psl_phantom_t *ph, psl_tally_t *tally) {
    if (!ph || !tally) return psl_fail(PSL_EINVAL, "transport: null argument");
    if (ph->nx != tally->nx || ph->ny != tally->ny || ph->nz != tally->nz || !ph->mat || !ph->rho)
        return psl_fail(PSL_EINVAL, "transport: phantom does not match the tally");
    return PSL_OK;
}

static Job job_of(psl_batch_t *batch, int32_t slice) {
    Job J;
    J.slice = slice;
    if (batch->lazy) {
        J.lazy = true;
        J.P = make_plan_dev(batch->plan, &batch->phantom);
        J.first = batch->first_history; J.stride = batch->stride; J.n = batch->n_histories;
    } else {
        J.p = batch->p; J.nph = batch->n_photons; J.nel = batch->n_electrons; J.cap = batch->cap;
    }
    return J;
}

static int transport_impl(const psl_phantom_t *ph, const psl_physics_t *phys, psl_batch_t *batch, psl_tally_t *tally,
                          int32_t b, int64_t *hist_dep, int64_t *hist_esc, int32_t *hist_events, void *stream_) {
    int rc = check_transport_args(ph, tally);
    if (rc) return rc;
    if (!batch) return psl_fail(PSL_EINVAL, "transport_run: null batch");
    if ((b < 0 && b != PSL_SLICE_BY_HISTORY) || b >= tally->n_batches)
        return psl_fail(PSL_EINVAL, "transport_run: batch index out of range");
    if (hist_dep || hist_esc || hist_events) {
        const int64_t nt = batch->lazy ? batch->n_histories : batch->n_photons + batch->n_electrons;
        if (nt > (int64_t)ROOT_INDEX_MASK + 1) return psl_fail(PSL_EINVAL, "transport_trace: batch too large to trace");
    }
    if (batch->consumed) return psl_fail(PSL_EINVAL, "transport_run: batch already transported");
    if (batch->lazy && (batch->phantom.nx != ph->nx || batch->phantom.ny != ph->ny || batch->phantom.nz != ph->nz))
        return psl_fail(PSL_EINVAL, "transport_run: batch was sourced for another phantom");
    cudaStream_t st = as_stream(stream_);
    Runner R;
    const int64_t need = batch->lazy ? batch->n_histories : std::max(batch->n_photons, batch->n_electrons);
    if ((rc = R.prepare(ph, phys, tally, batch->seed, need, st, false))) return rc;
    R.A.hist_dep = (unsigned long long *)hist_dep;
    R.A.hist_esc = (unsigned long long *)hist_esc;
    R.A.hist_events = hist_events;
    batch->consumed = 1;
    if (!batch->lazy) { k_ledger_add<<<1, 1, 0, st>>>(tally->ledger, (const unsigned long long *)(batch->counts + 2)); PSL_NOTE_LAUNCH(); }
    if ((rc = R.run(job_of(batch, b)))) return rc;
    if ((rc = R.drain(0))) return rc;
    return R.finish();
}

extern "C" int transport_run(const psl_phantom_t *ph, const psl_physics_t *phys, psl_batch_t *batch, psl_tally_t *tally,
                             int32_t b, void *stream) {
    return transport_impl(ph, phys, batch, tally, b, nullptr, nullptr, nullptr, stream);
}

extern "C" int transport_trace(const psl_phantom_t *ph, const psl_physics_t *phys, psl_batch_t *batch,
                               psl_tally_t *tally, int32_t b, int64_t *hist_dep, int64_t *hist_esc,
                               int32_t *hist_events, void *stream) {
    return transport_impl(ph, phys, batch, tally, b, hist_dep, hist_esc, hist_events, stream);
}

// ---------------------------------------------------------------- psl_run --
// All batches of a plan's history range, without host synchronisation.
// Generations launched before the first host check in psl_run without a graph:
// most batches finish within them, so a batch usually costs one host check.
#define UNCHECKED_GENERATIONS 3

// Batch blocks per window of the batch-by-batch order for a range of n
// histories (0: the range runs in reading order).
static int64_t batch_order_window(const psl_tally *tally, int64_t n) {
    if (!use_batch_order(tally)) return 0;
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(n, tally->chunk_cap));
    return std::min<int64_t>(batch_window(chunk, tally->n_batches), n / BATCH_BLOCK + 2);
}

static int run_body(const psl_plan_t *plan, const psl_phantom_t *ph, const psl_physics_t *phys, psl_tally_t *tally,
                    int64_t first, int64_t n, cudaStream_t st, bool capturing, Runner &R) {
    // each history's deposits go to the tally slice of its id (independent
    // batches, Sec. 2.3.3); the range runs in reading order, or window by
    // window and, inside a window, batch by batch (the dose is the same)
    int rc = R.prepare(ph, phys, tally, plan->seed, n, st, capturing);
    if (rc) return rc;
    Job J;
    J.lazy = true;
    J.P = make_plan_dev(plan, ph);
    J.first = first; J.stride = 1; J.n = n; J.slice = PSL_SLICE_BY_HISTORY;
    const int check = capturing ? -1 : UNCHECKED_GENERATIONS;
    const int64_t W = batch_order_window(tally, n);
    if (W <= 0) {
        if ((rc = R.run(J))) return rc;
        return R.drain(check);
    }
    if (!capturing && (rc = batch_order_ensure(tally, W))) return rc;   // (a capture is set up beforehand)
    Workspace *w = tally->ws;
    if (w->bm_cap < W) return psl_fail(PSL_EINVAL, "psl_run: batch-order buffers not set up");
    const uint32_t nb = (uint32_t)tally->n_batches;
    const int bits = 32 - __builtin_clz(nb - 1);
    // windows of W batch blocks (B = h >> BATCH_BLOCK_SHIFT) over the range's
    // blocks; in a window the blocks are sorted by batch (a stable radix pass)
    // and each batch's blocks run as one pass, clipped to the range
    const int64_t B0 = first >> BATCH_BLOCK_SHIFT, B1 = (first + n - 1) >> BATCH_BLOCK_SHIFT;
    for (int64_t b0 = B0; b0 <= B1; b0 += W) {
        const uint32_t wb = (uint32_t)std::min<int64_t>(W, B1 - b0 + 1);
        const int64_t h_lo = std::max<int64_t>(first, b0 << BATCH_BLOCK_SHIFT);
        const int64_t h_hi = std::min<int64_t>(first + n, (b0 + wb) << BATCH_BLOCK_SHIFT);
        k_slice_keys<<<R.grid_m, 256, 0, st>>>(R.A, b0, wb, nb, w->bm_keys[0]); PSL_NOTE_LAUNCH();
        int alt = 0;
        if (sort_pairs_u32(w->bm_keys[0], w->bm_vals[0], w->bm_keys[1], w->bm_vals[1], wb, bits, nullptr, true,
                           w->bm_scratch, &alt, st))
            return psl_fail(PSL_EINVAL, "psl_run: batch sort");
        k_or_err<<<1, 1, 0, st>>>(sort_err_word(w->bm_scratch), R.A.err); PSL_NOTE_LAUNCH();
        k_slice_bounds<<<1, 256, 0, st>>>(w->bm_keys[alt], wb, nb, w->bm_off); PSL_NOTE_LAUNCH();
        for (uint32_t b = 0; b < nb; ++b) {
            Job Jb = J;
            Jb.first = h_lo;                            // the window [h_lo, h_hi)
            Jb.stride = h_hi - h_lo;
            Jb.n = std::min<int64_t>(R.chunk, h_hi - h_lo);   // one pass; k_source flags a batch larger than it
            Jb.slice = (int32_t)b;
            Jb.list = w->bm_vals[alt];
            Jb.list_off = w->bm_off;
            if ((rc = R.run(Jb))) return rc;
        }
    }
    return R.drain(check);
}

static inline uint32_t __float_as_uint_host(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

// Key of a captured graph: everything the recorded launches depend on.
static void run_key(const psl_plan_t *plan, const psl_phantom_t *ph, const psl_physics_t *phys, const psl_tally_t *tally,
                    int64_t first, int64_t n, uint64_t key[11]) {
    psl_physics_t P;
    psl_physics_default(&P);
    if (phys) P = *phys;
    const SrcTraceDev &T = tally->trace;
    const uint64_t k[11] = {(uint64_t)(uintptr_t)plan, (uint64_t)first, (uint64_t)n, (uint64_t)(uintptr_t)ph->rho,
                            (uint64_t)(uintptr_t)ph->mat, ((uint64_t)P.flags << 32) | (uint64_t)tally->grid_mult,
                            (uint64_t)tally->chunk_cap ^ ((uint64_t)tally->order << 60), (uint64_t)plan->seed,
                            (uint64_t)T.first ^ ((uint64_t)T.n << 1), (uint64_t)(uintptr_t)T.entry ^ (uint64_t)(uintptr_t)T.use ^
                                (uint64_t)(uintptr_t)T.rec ^ (uint64_t)(uintptr_t)T.status ^ (uint64_t)(uintptr_t)T.state ^
                                (uint64_t)(uintptr_t)T.ptype,
                            (uint64_t)psl_debug_flags() ^ ((uint64_t)psl_debug_queue_cap() << 8) ^
                                ((uint64_t)psl_wait_polls(0) << 40) ^ ((uint64_t)__float_as_uint_host(P.wcc) << 20) ^
                                (uint64_t)__float_as_uint_host(P.photon_cut) ^ ((uint64_t)__float_as_uint_host(P.electron_cut) << 32) ^
                                ((uint64_t)__float_as_uint_host(P.wcb) << 12)};
    memcpy(key, k, sizeof(k));
}

// The readout a psl_plan_replay graph ends with.
struct ReadoutArgs {
    double norm;
    double *dose, *sigma, *ledger;
};

// Record (once per key) and replay a graph of psl_run's body; with `ro`,
// the graph also resets the tally first and reads the dose out last.
static int graph_run(const psl_plan_t *plan, const psl_phantom_t *ph, const psl_physics_t *phys, psl_tally_t *tally,
                     int64_t first, int64_t n, const ReadoutArgs *ro, cudaStream_t st) {
    int rc;
    uint64_t key[16] = {0};
    run_key(plan, ph, phys, tally, first, n, key);
    if (ro) {
        uint64_t nb;
        memcpy(&nb, &ro->norm, 8);
        key[11] = nb; key[12] = (uint64_t)(uintptr_t)ro->dose; key[13] = (uint64_t)(uintptr_t)ro->sigma;
        key[14] = (uint64_t)(uintptr_t)ro->ledger; key[15] = (uint64_t)(uintptr_t)ph->rho;
    }
    // workspace and tables are set up outside the capture
    {
        Runner pre;
        if ((rc = pre.prepare(ph, phys, tally, plan->seed, n, st, false))) return rc;
        const int64_t W = batch_order_window(tally, n);
        if (W > 0 && (rc = batch_order_ensure(tally, W))) return rc;
        PSL_CUDA(cudaStreamSynchronize(st));
    }
    Workspace *w = tally->ws;
    cudaGraphExec_t &gx = ro ? w->plan_graph : w->graph;
    uint64_t *gk = ro ? w->plan_key : w->graph_key;
    const size_t kbytes = ro ? sizeof(w->plan_key) : sizeof(w->graph_key);
    if (!gx || memcmp(gk, key, kbytes) != 0) {
        if (gx) { cudaGraphExecDestroy(gx); gx = nullptr; }
        cudaStream_t cs;
        PSL_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            Runner C;
            rc = ro ? psl_tally_reset(tally, cs) : PSL_OK;
            if (!rc) rc = run_body(plan, ph, phys, tally, first, n, cs, true, C);
            if (!rc && ro) rc = dose_readout(tally, ph, ro->norm, ro->dose, ro->sigma, ro->ledger, cs);
            e = cudaStreamEndCapture(cs, &g);
        }
        cudaStreamDestroy(cs);
        if (rc) { if (g) cudaGraphDestroy(g); return rc; }
        if (e != cudaSuccess) return psl_fail(PSL_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&gx, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { gx = nullptr; return psl_fail(PSL_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e)); }
        memcpy(gk, key, kbytes);
    }
    PSL_CUDA(cudaGraphLaunch(gx, st));
    PSL_NOTE_LAUNCH();
    Runner R;
    R.st = st; R.w = w; R.tally = tally;
    return R.finish();
}

static int check_run_args(const psl_plan_t *plan, const psl_phantom_t *ph, psl_tally_t *tally, int64_t first,
                          int64_t n, const char *who) {
    int rc = check_transport_args(ph, tally);
    if (rc) return rc;
    if (!plan || first < 0 || n <= 0 || first + n > plan->n_histories)
        return psl_fail(PSL_EINVAL, std::string(who) + ": bad plan or history range");
    if (plan->n_groups > 1024) return psl_fail(PSL_EINVAL, std::string(who) + ": too many energy divisions");
    return PSL_OK;
}

extern "C" int psl_run(const psl_plan_t *plan, const psl_phantom_t *ph, const psl_physics_t *phys, psl_tally_t *tally,
                       int64_t first, int64_t n, int32_t use_graph, void *stream_) {
    int rc = check_run_args(plan, ph, tally, first, n, "psl_run");
    if (rc) return rc;
    cudaStream_t st = as_stream(stream_);
    if (use_graph) return graph_run(plan, ph, phys, tally, first, n, nullptr, st);
    Runner R;
    if ((rc = run_body(plan, ph, phys, tally, first, n, st, false, R))) return rc;
    return R.finish();
}

extern "C" int psl_plan_replay(const psl_plan_t *plan, const psl_phantom_t *ph, const psl_physics_t *phys,
                               psl_tally_t *tally, int64_t first, int64_t n, double norm, double *dose, double *sigma,
                               double *ledger, void *stream_) {
    int rc = check_run_args(plan, ph, tally, first, n, "psl_plan_replay");
    if (rc) return rc;
    if (!ph->rho) return psl_fail(PSL_EINVAL, "psl_plan_replay: null density");
    ReadoutArgs ro{norm, dose, sigma, ledger};
    return graph_run(plan, ph, phys, tally, first, n, &ro, as_stream(stream_));
}

// ---------------------------------------------------------------- tuning --
extern "C" int psl_autotune(const psl_plan_t *plan, const psl_phantom_t *ph, const psl_physics_t *phys,
                            psl_tally_t *tally, int64_t n_probe, int32_t *blocks_per_sm, int64_t *queue_depth,
                            void *stream_) {
    int rc = check_transport_args(ph, tally);
    if (rc) return rc;
    if (!plan || n_probe <= 0) return psl_fail(PSL_EINVAL, "psl_autotune: bad argument");
    n_probe = std::min<int64_t>(n_probe, plan->n_histories);
    cudaStream_t st = as_stream(stream_);
    const int grids[] = {2, 3, 4, 6};
    const int64_t depths[] = {1 << 21, 1 << 22, 1 << 23, 1 << 24, 1 << 25, 1 << 26};
    // A pass ends with a tail in which lanes run out of particles, so a
    // depth is timed on at least two passes of its own (a probe shorter than
    // a pass would hide the tail that a deeper queue pays less often), and
    // the candidates compare histories per second.  Depths whose workspace
    // would take more than 80 % of the free device memory (or exceed the
    // plan's histories) are not tried.
    size_t free_b = 0, total_b = 0;
    PSL_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const int64_t held = workspace_bytes_of(tally->ws);
    double best = 0.0;
    int bg = tally->grid_mult;
    int64_t bd = tally->chunk_cap;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    for (int gi : grids) {
        for (int64_t d : depths) {
            if (d != depths[0] && (d > plan->n_histories ||
                                   (double)d * WORKSPACE_BYTES_PER_PRIMARY > 0.8 * (double)(free_b + held)))
                continue;
            const int64_t np = std::min<int64_t>(plan->n_histories, std::max<int64_t>(n_probe, 2 * d));
            tally->grid_mult = gi;
            tally->chunk_cap = d;
            cudaEventRecord(a, st);
            Runner R;
            rc = run_body(plan, ph, phys, tally, 0, np, st, false, R);
            if (!rc) rc = R.finish();
            cudaEventRecord(b, st);
            if (rc) break;
            cudaEventSynchronize(b);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            const double rate = (double)np / std::max(ms, 1e-3f);
            if (rate > best) { best = rate; bg = gi; bd = d; }
        }
        if (rc) break;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    tally->grid_mult = bg;
    tally->chunk_cap = bd;
    if (rc) return rc;
    if ((rc = psl_tally_reset(tally, stream_))) return rc;
    if (blocks_per_sm) *blocks_per_sm = bg;
    if (queue_depth) *queue_depth = bd;
    return PSL_OK;
}

// Autotuner for the PSL position-bin size (the paper leaves it to
// benchmarking): for every candidate cell size, the store is built with
// square cells over the same extent, the plan created and n_probe histories
// run (once to warm up, once timed); the estimate is the plan creation plus
// the probe's time scaled to the plan's histories.
extern "C" int psl_autotune_bins(const psl_params_t *params, const psl_records_t *records, const psl_beam_t *beams,
                                 int32_t n_beams, float sad, const psl_phantom_t *ph, const psl_physics_t *phys,
                                 int64_t n_histories, uint64_t seed, int32_t n_batches, const float *cell_cm,
                                 int32_t n_cells, int64_t n_probe, float *best_cell, double *plan_seconds,
                                 void *stream_) {
    if (!params || !records || !beams || n_beams <= 0 || !ph || !cell_cm || n_cells <= 0 || n_probe <= 0 ||
        n_histories <= 0 || !params->x_edges || !params->y_edges || params->nx <= 0 || params->ny <= 0)
        return psl_fail(PSL_EINVAL, "psl_autotune_bins: bad argument");
    for (int k = 0; k < n_cells; ++k)
        if (!(cell_cm[k] > 0.f)) return psl_fail(PSL_EINVAL, "psl_autotune_bins: cell sizes must be > 0");
    cudaStream_t st = as_stream(stream_);
    const double x0 = params->x_edges[0], x1 = params->x_edges[params->nx];
    const double y0 = params->y_edges[0], y1 = params->y_edges[params->ny];
    const int64_t probe = std::min<int64_t>(n_probe, n_histories);
    psl_tally_t *tally = nullptr;
    int rc = psl_tally_create(ph, n_batches, &tally);
    if (rc) return rc;
    cudaEvent_t a, b, c;
    cudaEventCreate(&a); cudaEventCreate(&b); cudaEventCreate(&c);
    double best = 1e300;
    float best_c = cell_cm[0];
    for (int k = 0; k < n_cells && !rc; ++k) {
        const int nx = (int)std::max<long long>(1, std::llround((x1 - x0) / cell_cm[k]));
        const int ny = (int)std::max<long long>(1, std::llround((y1 - y0) / cell_cm[k]));
        std::vector<float> xe(nx + 1), ye(ny + 1);
        for (int i = 0; i <= nx; ++i) xe[i] = (float)(x0 + (x1 - x0) * i / nx);
        for (int i = 0; i <= ny; ++i) ye[i] = (float)(y0 + (y1 - y0) * i / ny);
        psl_params_t pc = *params;
        pc.nx = nx; pc.ny = ny; pc.x_edges = xe.data(); pc.y_edges = ye.data();
        psl_store_t *store = nullptr;
        psl_plan_t *plan = nullptr;
        if ((rc = psl_build(&pc, records, &store, stream_))) break;
        float ms_plan = 0.f, ms_run = 0.f;
        cudaEventRecord(a, st);
        rc = psl_plan_create(store, beams, n_beams, sad, n_histories, seed, &plan, stream_);
        cudaEventRecord(b, st);
        for (int rep = 0; rep < 2 && !rc; ++rep) {
            if (rep == 1) cudaEventRecord(b, st);
            if (!(rc = psl_tally_reset(tally, stream_))) rc = psl_run(plan, ph, phys, tally, 0, probe, 0, stream_);
            if (rep == 0 && !rc) { cudaEventSynchronize(b); cudaEventElapsedTime(&ms_plan, a, b); }
        }
        cudaEventRecord(c, st);
        if (!rc) {
            cudaEventSynchronize(c);
            cudaEventElapsedTime(&ms_run, b, c);
            const double est = 1e-3 * ((double)ms_plan + (double)ms_run * (double)n_histories / (double)probe);
            if (plan_seconds) plan_seconds[k] = est;
            if (est < best) { best = est; best_c = cell_cm[k]; }
        }
        psl_plan_destroy(plan);
        psl_store_destroy(store);
    }
    cudaEventDestroy(a); cudaEventDestroy(b); cudaEventDestroy(c);
    psl_tally_destroy(tally);
    if (rc) return rc;
    if (best_cell) *best_cell = best_c;
    return PSL_OK;
}
