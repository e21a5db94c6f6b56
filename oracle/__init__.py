"""CPU oracle of the phase-space-let (PSL) Monte Carlo dose path.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package.  The
product path (the CUDA library and its binding) never imports it, and the two
share no code: the oracle has its own Philox generator, binning, selection,
physics, transport and readout.  Inputs come from the separate seeded
generator module ``paper_1302_1861_b300.inputs``.

Layout:
  source.py     azimuthal redistribution (Sec. 2.3.1), PSL build, selection,
                history counts, reading order, jaw, fluence, MU weights,
                rotations (Sec. 2.2, 2.3.2, 2.3.3, 2.4); Methods 1 and 2 as
                an unsorted stream (Sec. 2.1, 2.2)
  stream.c      the on-the-fly type/energy bin fill of Methods 1 and 2
  transport.c   double-precision photon/electron transport and tally
                (Sec. 2.3.3 "dose counters", Sec. 2.6 cut-offs)
  readout.py    dose, batch uncertainty, normalisation (Sec. 2.3.3, 2.5),
                gamma index (Sec. 3, Table 1 criteria)
"""
from __future__ import annotations

import numpy as np

from . import _lib, readout, source  # noqa: F401
from ._lib import philox  # noqa: F401

ME = 0.51099895
PCUT = 0.010                 # photon cut-off, MeV (Sec. 2.6)
ECUT = 0.700 - ME            # electron cut-off: 0.700 MeV total energy (Sec. 2.6)
WCC = 0.200                  # hard Moller threshold, MeV
WCB = 0.200                  # hard bremsstrahlung threshold, MeV

F_LOCAL_SECONDARIES = 1
F_FIRST_INTERACTION = 2
F_NO_MSC = 4
F_NO_HARD = 8

L_EMITTED, L_ESCAPED, L_DEPOSITED, L_COMPTON, L_PHOTO, L_PAIR, L_ESTEPS, L_ERRORS, L_HARD_COLL, L_HARD_BREM = range(10)
L_N = 10


def transport(ptype, pos, dirs, e, wt, pid, phantom, seed, flags=0, nthreads=0,
              pcut=PCUT, ecut=ECUT, wcc=WCC, wcb=WCB, per_history=False):
    """Transport primaries through the phantom; returns (tally, ledger[, hist]).

    Positions are phantom-local (cm from the (0,0,0) voxel corner)."""
    L = _lib.lib()
    n = len(e)
    ptype = np.ascontiguousarray(ptype, np.int32)
    pos = np.ascontiguousarray(pos, np.float64).reshape(n, 3)
    dirs = np.ascontiguousarray(dirs, np.float64).reshape(n, 3)
    e = np.ascontiguousarray(e, np.float64)
    wt = np.ascontiguousarray(wt, np.float64)
    pid = np.ascontiguousarray(pid, np.uint64)
    nz, ny, nx = phantom.shape
    mat = np.ascontiguousarray(phantom.mat, np.uint8)
    rho = np.ascontiguousarray(phantom.rho, np.float32)
    tally = np.zeros(nx * ny * nz, np.int64)
    ledger = np.zeros(L_N, np.int64)
    hd = he = hv = hp = None
    if per_history:
        hd, he = np.zeros(n, np.int64), np.zeros(n, np.int64)
        hv, hp = np.zeros(n, np.int32), np.zeros(n, np.float64)
    P = _lib._p
    vx, vy, vz = phantom.voxel
    L.ora_transport(n, P(ptype), P(pos), P(dirs), P(e), P(wt), P(pid), nx, ny, nz,
                    float(vx), float(vy), float(vz), P(mat), P(rho), int(seed), int(flags),
                    pcut, ecut, wcc, wcb, P(tally), P(ledger), P(hd), P(he), P(hv), P(hp),
                    int(nthreads))
    tally = tally.reshape(nz, ny, nx)
    if per_history:
        return tally, ledger, dict(dep=hd, esc=he, events=hv, path=hp)
    return tally, ledger


TAG_BATCH = 4
BATCH_BLOCK = 256            # consecutive history ids that share a batch


def history_slices(h: np.ndarray, seed: int, n_batches: int) -> np.ndarray:
    """Batch of every history (Sec. 2.3.3: independent batches).  The ids
    are cut into blocks of BATCH_BLOCK consecutive histories; block
    B = h // BATCH_BLOCK goes to batch floor(r N_b / 2^32), r the first word of
    Philox(key = seed; counter = (0, TAG_BATCH, B)).  A pseudo-random
    partition of the reading order into blocks: every batch is an independent
    sample of blocks, whatever order they are read in."""
    h = np.asarray(h, np.uint64) // np.uint64(BATCH_BLOCK)
    ctr = np.zeros((len(h), 4), np.uint32)
    ctr[:, 1] = TAG_BATCH
    ctr[:, 2] = (h & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    ctr[:, 3] = (h >> np.uint64(32)).astype(np.uint32)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], np.uint32)
    r = philox(ctr, key)[:, 0].astype(np.uint64)
    return ((r * np.uint64(n_batches)) >> np.uint64(32)).astype(np.int64)


def run_plan(w, n_histories=None, first=0, n_batches=None, nthreads=0, flags=0,
             store=None, plan=None):
    """Whole path for a workload on the CPU: build, plan, source, transport
    (one tally per batch), in the order of Sec. 2.3.  Returns a dict."""
    n_sim = w.n_histories
    n_h = n_sim if n_histories is None else n_histories
    nb = w.n_batches if n_batches is None else n_batches
    if store is None:
        store = source.psl_build(w.records, w.binning)
    if plan is None:
        plan = source.make_plan(store, w.beams, n_sim, w.seed, w.z_psl, w.sad)
    nz, ny, nx = w.phantom.shape
    tallies = np.zeros((nb, nz, ny, nx), np.int64)
    ledger = np.zeros(L_N, np.int64)
    h_all = np.arange(first, first + n_h, dtype=np.int64)
    sl = history_slices(h_all, w.seed, nb)
    for b in range(nb):
        h = h_all[sl == b]                  # batch b: the histories drawn into it
        s = source.source(plan, store, w.records, w.beams, w.phantom, h, w.z_psl, w.sad)
        ledger[L_EMITTED] += s.emitted_fp
        ledger[L_ESCAPED] += s.missed_fp
        m = s.status == source.ST_TRANSPORT
        t, lg = transport(s.ptype[m], s.pos[m], s.dir[m], s.e[m], s.wt[m].astype(np.float64),
                          h[m].astype(np.uint64), w.phantom, w.seed, flags=flags, nthreads=nthreads)
        tallies[b] = t
        ledger += lg
    return dict(store=store, plan=plan, tallies=tallies, ledger=ledger)
