"""CPU oracle of the PSL source stage (TEST INFRASTRUCTURE).

Only the tests, the package smoke check and the CPU-baseline leg of the
benchmark may import this module.  It shares no code with the CUDA path.

It follows the paper's steps in order:

* Azimuthal particle redistribution, Sec. 2.3.1 (before PSL generation):
  each record is also used as K-1 copies rotated about the beam axis by
  independent uniform azimuths, position and direction cosines together.
* PSL generation, Sec. 2.3.2: split the records by particle type (photon;
  electron/positron), then by energy bin, then by dx x dy position bin.  The
  PSL store is one array sorted by the PSL id plus its bin offsets.
* PSL selection, Sec. 2.3.3 and Fig. 1: back-project the jaw opening (plus a
  margin) from SAD to the PSL plane; keep every PSL whose area overlaps it.
* Histories per PSL, Sec. 2.3.3 (the equations for N_total^psl and P_ij):
  histories proportional to the records of each selected PSL of each field.
* Reading order, Sec. 2.3.3: energy division by energy division; inside one,
  a few particles from each PSL in turn; the first read of a PSL starts at a
  random record and wraps to its start (recycling, Sec. 2.6).
* Jaw model, Sec. 2.2: accept a particle if its straight line passes inside
  both jaw openings, otherwise terminate it.
* Fluence map, Sec. 2.2 and 2.4: project to the map plane, multiply the weight
  by the map value; MU weight w' = w MU_i / MU_total (Sec. 2.3.3).
* Rotations and projection to the phantom surface, Sec. 2.3.3.

Readings where the paper is silent (also listed in the design notes): the
jaw, fluence and ROI decisions are taken in float32, the precision of the
kernel; every other quantity is float64.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

from . import _lib

F32 = np.float32

# source status codes (per history)
ST_TRANSPORT, ST_JAW, ST_FLUENCE, ST_ZERO_WEIGHT, ST_MISS = 0, 1, 2, 3, 4

TAG_OFFSET = 1
TAG_APR = 3
APR_MAX_BLOCKS = 64


# --------------------------------------------------------------------------
# Sec. 2.3.1: azimuthal particle redistribution
# --------------------------------------------------------------------------
def _apr_coord(w: np.ndarray) -> np.ndarray:
    """2 U - 1 in float32 for U = ((w >> 9) + 0.5) 2^-23 (exact)."""
    u = ((w >> np.uint32(9)).astype(F32) + F32(0.5)) * F32(2.0 ** -23)
    return F32(2.0) * u - F32(1.0)


def apr_angles(n_records: int, k: int, seed: int):
    """cos and sin (float32, [n_records, k]) of the azimuth of every copy.

    Copy 0 is the record itself (angle 0).  For copy c > 0 of record i the
    angle is the doubled polar angle of a uniform point (a, b) of the unit
    disc, found by rejection: Philox blocks with counter (blk, TAG_APR, i, c)
    under key seed, two candidate points per block, the first with
    a^2 + b^2 <= 1 taken; none in APR_MAX_BLOCKS blocks gives angle 0.  Then
    cos = (a^2 - b^2) / r^2 and sin = 2ab / r^2.  Every operation is a
    float32 operation rounded to nearest, the precision the PSL records are
    stored in."""
    cs = np.ones((n_records, k), F32)
    sn = np.zeros((n_records, k), F32)
    if k <= 1 or n_records == 0:
        return cs, sn
    ii, cc = np.meshgrid(np.arange(n_records, dtype=np.int64), np.arange(1, k, dtype=np.int64), indexing="ij")
    ii, cc = ii.ravel(), cc.ravel()
    oc = np.ones(len(ii), F32)
    os_ = np.zeros(len(ii), F32)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], np.uint32)
    pending = np.arange(len(ii))
    for blk in range(APR_MAX_BLOCKS):
        if len(pending) == 0:
            break
        ctr = np.stack([np.full(len(pending), blk), np.full(len(pending), TAG_APR), ii[pending], cc[pending]],
                       1).astype(np.uint32)
        w = _lib.philox(ctr, key)
        done = np.zeros(len(pending), bool)
        for h in range(2):
            a, b = _apr_coord(w[:, 2 * h]), _apr_coord(w[:, 2 * h + 1])
            aa, bb = a * a, b * b
            r2 = aa + bb
            take = (r2 <= F32(1.0)) & ~done
            sel = pending[take]
            oc[sel] = (aa[take] - bb[take]) / r2[take]
            os_[sel] = (F32(2.0) * (a[take] * b[take])) / r2[take]
            done |= take
        pending = pending[~done]
    cs[:, 1:] = oc.reshape(n_records, k - 1)
    sn[:, 1:] = os_.reshape(n_records, k - 1)
    return cs, sn


def apr_expand(records, k: int, seed: int):
    """The phase space after redistribution: record i becomes records
    i*k + c, c = 0..k-1; copy 0 unchanged, the others rotated about the beam
    axis: x' = x cos - y sin, y' = x sin + y cos, the same for (u, v)."""
    from paper_1302_1861_b300.inputs import Records
    if k <= 1:
        return records
    n = records.n
    cs, sn = apr_angles(n, k, seed)
    out = {}
    for name in ("e", "wt", "q"):
        out[name] = np.repeat(getattr(records, name), k)
    for a_name, b_name in (("x", "y"), ("u", "v")):
        a = np.asarray(getattr(records, a_name), F32)[:, None]
        b = np.asarray(getattr(records, b_name), F32)[:, None]
        ra = a * cs - b * sn
        rb = a * sn + b * cs
        ra[:, 0] = a[:, 0]                 # copy 0: the record as given, bit for bit
        rb[:, 0] = b[:, 0]
        out[a_name], out[b_name] = ra.ravel(), rb.ravel()
    return Records(out["x"], out["y"], out["u"], out["v"], out["e"], out["wt"], out["q"])


# --------------------------------------------------------------------------
# Sec. 2.3.2: PSL generation
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Store:
    keys: np.ndarray         # int64 [n] PSL id per input record (n_bins = invalid)
    perm: np.ndarray         # int64 [n_valid] input index of each sorted record
    offsets: np.ndarray      # int64 [n_bins + 1]
    n_bins: int
    nx: int
    ny: int
    n_ebins: int
    x_edges: np.ndarray
    y_edges: np.ndarray

    @property
    def n_valid(self) -> int:
        return int(self.offsets[-1])


def psl_keys(x, y, e, q, x_edges, y_edges, e_edges) -> np.ndarray:
    """PSL id of every record: (type * N_E + energy bin) * (nx ny) + position.

    Bins are half-open [edge_k, edge_k+1).  Positions outside the extent and
    energies <= 0 get the sentinel id n_bins.  Energies are binned by the
    interior edges only, so E below the first or above the last edge fall in
    the first or last energy bin."""
    nx, ny, ne = len(x_edges) - 1, len(y_edges) - 1, len(e_edges) - 1
    n_bins = 2 * ne * nx * ny
    bx = np.searchsorted(x_edges, x, side="right") - 1
    by = np.searchsorted(y_edges, y, side="right") - 1
    eb = np.searchsorted(e_edges[1:-1], e, side="right")
    t = (q != 0).astype(np.int64)
    valid = (bx >= 0) & (bx < nx) & (by >= 0) & (by < ny) & (e > 0)
    key = (t * ne + eb) * (nx * ny) + by * nx + bx
    return np.where(valid, key, n_bins).astype(np.int64)


def psl_build(records, binning) -> Store:
    """Sort the phase space into PSLs: stable sort by PSL id, bin offsets."""
    keys = psl_keys(records.x, records.y, records.e, records.q,
                    binning.x_edges, binning.y_edges, binning.e_edges)
    n_bins = binning.n_bins
    order = np.argsort(keys, kind="stable")
    counts = np.bincount(keys, minlength=n_bins + 1)
    offsets = np.zeros(n_bins + 1, np.int64)
    offsets[1:] = np.cumsum(counts[:n_bins])
    perm = order[: offsets[-1]].astype(np.int64)
    return Store(keys, perm, offsets, n_bins, binning.nx, binning.ny, binning.n_ebins,
                 binning.x_edges, binning.y_edges)


# --------------------------------------------------------------------------
# Sec. 2.3.3: selection, counts, reading order
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Plan:
    field: np.ndarray        # int64 [n_entries] field index of entry
    psl: np.ndarray          # int64 PSL id
    start: np.ndarray        # int64 first sorted record of the PSL
    nrec: np.ndarray         # int64 records in the PSL
    count: np.ndarray        # int64 histories assigned to the entry
    offset: np.ndarray       # int64 random start record inside the PSL
    group: np.ndarray        # int64 reading group (energy division major, type minor)
    n_total_psl: int
    n_sim: int
    group_start: np.ndarray  # int64 [n_groups + 1] first history of each group
    group_order: List[np.ndarray]   # per group: entries in visiting order
    n_ebins: int
    _literal: Dict[int, tuple] = dataclasses.field(default_factory=dict)


def roi_select(x_edges, y_edges, beam, z_psl, sad) -> np.ndarray:
    """Boolean [ny, nx]: PSL positions whose area overlaps the field's ROI.

    ROI: the jaw opening at SAD widened by the margin, back-projected from the
    source to the PSL plane (scaled by z_psl/SAD).  Overlap is strict: a PSL
    that only touches the ROI edge is not selected."""
    s = F32(z_psl) / F32(sad)
    m = F32(beam.roi_margin)
    xlo, xhi = (F32(beam.x1) - m) * s, (F32(beam.x2) + m) * s
    ylo, yhi = (F32(beam.y1) - m) * s, (F32(beam.y2) + m) * s
    sx = (x_edges[:-1] < xhi) & (x_edges[1:] > xlo)
    sy = (y_edges[:-1] < yhi) & (y_edges[1:] > ylo)
    return sy[:, None] & sx[None, :]


def psl_offsets(seed: int, field: np.ndarray, psl: np.ndarray, nrec: np.ndarray) -> np.ndarray:
    """Random first record of each (field, PSL): the 64-bit word of
    Philox(seed; field, tag, psl) scaled to [0, nrec) by (r * nrec) >> 64."""
    n = len(psl)
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = field
    ctr[:, 1] = TAG_OFFSET
    ctr[:, 2] = psl & 0xFFFFFFFF
    ctr[:, 3] = psl >> 32
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)
    r = _lib.philox(ctr, key) if n else np.zeros((0, 4), np.uint32)
    r64 = r[:, 0].astype(object) + (r[:, 1].astype(object) << 32)
    off = (r64 * nrec.astype(object)) >> 64
    return np.array(list(off), np.int64) if n else np.zeros(0, np.int64)


def make_plan(store: Store, beams, n_sim: int, seed: int, z_psl: float, sad: float) -> Plan:
    npos = store.nx * store.ny
    ne = store.n_ebins
    nrec_psl = np.diff(store.offsets)
    fields, psls = [], []
    for i, b in enumerate(beams):
        sel = np.flatnonzero(roi_select(store.x_edges, store.y_edges, b, z_psl, sad).ravel())
        # every type and energy division of every selected position, in PSL-id order
        ids = (np.arange(2 * ne)[:, None] * npos + sel[None, :]).ravel()
        fields.append(np.full(len(ids), i, np.int64))
        psls.append(ids.astype(np.int64))
    field = np.concatenate(fields)
    psl = np.concatenate(psls)
    start = store.offsets[psl]
    nrec = nrec_psl[psl].astype(np.int64)
    n_total = int(nrec.sum())
    if n_total == 0:
        raise ValueError("no phase-space records inside the selected PSLs")
    # N_ij = N_sim N_j / N_total, rounded by differencing the floor of the
    # cumulative share (exact Python integers; the counts sum to N_sim)
    cum = np.zeros(len(nrec) + 1, dtype=object)
    cum[1:] = np.cumsum(nrec.astype(object))
    fl = (cum * int(n_sim)) // n_total
    count = np.array(list(fl[1:] - fl[:-1]), np.int64)
    offset = psl_offsets(seed, field, psl, nrec)
    t = psl // (ne * npos)
    e = (psl // npos) % ne
    group = e * 2 + t
    n_groups = 2 * ne
    group_order = []
    sizes = np.zeros(n_groups, np.int64)
    for g in range(n_groups):
        idx = np.flatnonzero((group == g) & (count > 0))
        # visiting order inside one round: larger counts first, then list order
        o = idx[np.lexsort((idx, -count[idx]))]
        group_order.append(o)
        sizes[g] = count[o].sum()
    gs = np.zeros(n_groups + 1, np.int64)
    gs[1:] = np.cumsum(sizes)
    return Plan(field, psl, start, nrec, count, offset, group, n_total, n_sim, gs, group_order, ne)


def _literal_group(plan: Plan, g: int):
    """All (entry, use) pairs of group g in reading order: round k visits, in
    the group's visiting order, every entry that still has more than k
    histories to give."""
    if g not in plan._literal:
        o = plan.group_order[g]
        c = plan.count[o]
        pos = np.repeat(np.arange(len(o)), c)
        k = np.concatenate([np.arange(n) for n in c]) if len(c) else np.zeros(0, np.int64)
        order = np.lexsort((pos, k))
        plan._literal[g] = (o[pos[order]], k[order])
    return plan._literal[g]


def _group_lookup(plan: Plan, g: int, hl: np.ndarray):
    """(entry, use) of the hl-th histories of group g: the round is the
    largest r with F(r) = sum_e min(count_e, r) <= hl, and the history is
    the (hl - F(r))-th entry visited in that round (the visiting order puts
    the entries that still have histories first).  F is tabulated for every
    round r = 0 .. max count and searched for all hl at once."""
    o = plan.group_order[g]
    c = plan.count[o]
    cs = np.sort(c)
    r = np.arange(int(c.max()) + 1, dtype=np.int64)
    k = np.searchsorted(cs, r, side="left")          # entries with count < r
    below = np.concatenate([[0], np.cumsum(cs)])
    F = below[k] + r * (len(cs) - k)
    rnd = np.searchsorted(F, hl, side="right") - 1
    return o[hl - F[rnd]].astype(np.int64), rnd


def history_map(plan: Plan, h: np.ndarray, literal_limit: int = 4_000_000):
    """Entry index and use number (k-th read of that entry) of each history."""
    h = np.asarray(h, np.int64)
    g = np.searchsorted(plan.group_start, h, side="right") - 1
    entry = np.empty(len(h), np.int64)
    use = np.empty(len(h), np.int64)
    for gg in np.unique(g):
        m = g == gg
        hl = h[m] - plan.group_start[gg]
        size = plan.group_start[gg + 1] - plan.group_start[gg]
        if size <= literal_limit:
            ent, k = _literal_group(plan, int(gg))
            entry[m], use[m] = ent[hl], k[hl]
        else:
            entry[m], use[m] = _group_lookup(plan, int(gg), hl)
    return entry, use


# --------------------------------------------------------------------------
# Sec. 2.2 / 2.3.3 / 2.4: per-particle source transform
# --------------------------------------------------------------------------
def _sincosd(deg: float):
    """sin and cos of an angle in degrees, exact at multiples of 90."""
    n = int(round(deg / 90.0))
    r = math.radians(deg - 90.0 * n)
    s, c = math.sin(r), math.cos(r)
    for _ in range(n % 4):
        s, c = c, -s
    return s, c


def beam_matrix(beam) -> np.ndarray:
    """Rotation from the beam frame to the patient frame: couch (about z),
    gantry (about y) and collimator (about z), applied collimator first."""
    sc, cc = _sincosd(beam.collimator)
    sg, cg = _sincosd(beam.gantry)
    st, ct = _sincosd(beam.couch)
    Rc = np.array([[cc, -sc, 0.0], [sc, cc, 0.0], [0.0, 0.0, 1.0]])
    Rg = np.array([[cg, 0.0, sg], [0.0, 1.0, 0.0], [-sg, 0.0, cg]])
    Rt = np.array([[ct, -st, 0.0], [st, ct, 0.0], [0.0, 0.0, 1.0]])
    return Rt @ Rg @ Rc


@dataclasses.dataclass
class SourceOut:
    status: np.ndarray       # int8
    entry: np.ndarray        # int64
    use: np.ndarray          # int64
    rec: np.ndarray          # int64 sorted record index
    beam: np.ndarray         # int64
    ptype: np.ndarray        # int32 0 photon, 1 electron, 2 positron
    pos: np.ndarray          # float64 [n, 3] phantom-local entry point
    dir: np.ndarray          # float64 [n, 3]
    e: np.ndarray            # float64 MeV
    wt: np.ndarray           # float32 weight after jaw/fluence/MU
    emitted_fp: int          # sum of fixed-point E*wt over accepted histories
    missed_fp: int           # part of it that missed the phantom


def mu_ratios(beams) -> np.ndarray:
    """w'/w = MU_i / MU_total (Sec. 2.3.3), from the float32 MU values the
    plan carries, summed in beam order in double and rounded to float32."""
    mus = [float(F32(b.mu)) for b in beams]
    tot = 0.0
    for m in mus:
        tot += m
    return np.array([F32(m / tot) for m in mus], F32)


def to_phantom(x, y, u, v, e, wt0, q, beam, beams, phantom, z_psl: float, sad: float, collimate: bool = True):
    """Sec. 2.2, 2.3.3 and 2.4 for records (float32 arrays) of fields `beam`
    (index into beams): jaw model and fluence map when `collimate`, MU weight,
    rotation into the patient and entry into the phantom box.

    Returns (status, wt, pos, dirs, ptype, fixed-point energy per record)."""
    n = len(x)
    status = np.zeros(n, np.int8)
    wt = np.zeros(n, F32)
    murat = mu_ratios(beams)
    one = F32(1.0)
    # direction cosine w in float32 (decides acceptance)
    s = (one - u * u) - v * v
    ok = s > 0
    w32 = np.sqrt(np.where(ok, s, one)).astype(F32)
    status[~ok] = ST_JAW
    for i, b in enumerate(beams):
        m = (beam == i) & ok
        if not m.any():
            continue
        zjx, zjy, sadf, zp = F32(b.z_jaw_x), F32(b.z_jaw_y), F32(sad), F32(z_psl)
        ww = wt0[m].copy()
        st = np.full(m.sum(), ST_TRANSPORT, np.int8)
        if collimate:
            xlo, xhi = (F32(b.x1) * zjx) / sadf, (F32(b.x2) * zjx) / sadf
            ylo, yhi = (F32(b.y1) * zjy) / sadf, (F32(b.y2) * zjy) / sadf
            xj = x[m] + u[m] * ((zjx - zp) / w32[m])
            yj = y[m] + v[m] * ((zjy - zp) / w32[m])
            acc = (xj >= xlo) & (xj <= xhi) & (yj >= ylo) & (yj <= yhi)
            st = np.where(acc, ST_TRANSPORT, ST_JAW).astype(np.int8)
            if b.fluence is not None:
                fny, fnx = b.fluence.shape
                ti = (sadf - zp) / w32[m]
                fx = ((x[m] + u[m] * ti) - F32(b.fx0)) / F32(b.fdx)
                fy = ((y[m] + v[m] * ti) - F32(b.fy0)) / F32(b.fdy)
                ix, iy = np.floor(fx), np.floor(fy)
                inside = (ix >= 0) & (ix < fnx) & (iy >= 0) & (iy < fny)
                st = np.where(acc & ~inside, ST_FLUENCE, st).astype(np.int8)
                ixc = np.clip(ix, 0, fnx - 1).astype(np.int64)
                iyc = np.clip(iy, 0, fny - 1).astype(np.int64)
                ww = ww * b.fluence[iyc, ixc]
        ww = ww * murat[i]
        st = np.where((st == ST_TRANSPORT) & (ww == 0), ST_ZERO_WEIGHT, st).astype(np.int8)
        status[m] = st
        wt[m] = ww
    # rotations and projection to the phantom surface (float64)
    pos = np.zeros((n, 3))
    dirs = np.zeros((n, 3))
    ud, vd = u.astype(np.float64), v.astype(np.float64)
    wd = np.sqrt(np.maximum(1.0 - ud * ud - vd * vd, 0.0))
    L = np.array(phantom.shape[::-1], np.float64) * np.array(phantom.voxel, np.float64)
    origin = np.array(phantom.origin, np.float64)
    for i, b in enumerate(beams):
        m = (beam == i) & (status == ST_TRANSPORT)
        if not m.any():
            continue
        R = beam_matrix(b)
        pb = np.stack([x[m].astype(np.float64), y[m].astype(np.float64),
                       np.full(m.sum(), float(z_psl))], 1)
        pb[:, 2] -= float(sad)
        pp = pb @ R.T + np.array(b.iso, np.float64) - origin
        dd = np.stack([ud[m], vd[m], wd[m]], 1) @ R.T
        # full-line slab intersection with the box [0, L]
        with np.errstate(divide="ignore", invalid="ignore"):
            t0 = (0.0 - pp) / dd
            t1 = (L - pp) / dd
        tmin = np.where(dd != 0, np.minimum(t0, t1), -np.inf)
        tmax = np.where(dd != 0, np.maximum(t0, t1), np.inf)
        outside_par = (dd == 0) & ((pp < 0) | (pp > L))
        t_in = tmin.max(1)
        t_out = tmax.min(1)
        hit = (t_in < t_out) & ~outside_par.any(1)
        idx = np.flatnonzero(m)
        status[idx[~hit]] = ST_MISS
        pos[idx] = pp + t_in[:, None] * dd
        dirs[idx] = dd
    ptype = np.where(q == 0, 0, np.where(q < 0, 1, 2)).astype(np.int32)
    fp = np.rint(e.astype(np.float64) * wt.astype(np.float64) * 4294967296.0).astype(np.int64)
    return status, wt, pos, dirs, ptype, fp


def source(plan: Plan, store: Store, records, beams, phantom, h: np.ndarray,
           z_psl: float, sad: float) -> SourceOut:
    h = np.asarray(h, np.int64)
    entry, use = history_map(plan, h)
    nrec = plan.nrec[entry]
    rec = plan.start[entry] + (plan.offset[entry] + use) % nrec
    beam = plan.field[entry]
    src = store.perm[rec]
    x, y, u, v = records.x[src], records.y[src], records.u[src], records.v[src]
    e, wt0, q = records.e[src], records.wt[src], records.q[src]
    status, wt, pos, dirs, ptype, fp = to_phantom(x, y, u, v, e, wt0, q, beam, beams, phantom, z_psl, sad)
    accepted = (status == ST_TRANSPORT) | (status == ST_MISS)
    emitted = int(fp[accepted].sum())
    missed = int(fp[status == ST_MISS].sum())
    return SourceOut(status, entry, use, rec, beam, ptype, pos, dirs, e.astype(np.float64), wt, emitted, missed)


# --------------------------------------------------------------------------
# Sec. 2.1, 2.2: Methods 1 and 2, the phase space as an unsorted stream
# --------------------------------------------------------------------------
METHOD_PATIENT_DEPENDENT, METHOD_JAW_MODEL = 1, 2


@dataclasses.dataclass
class StreamOut:
    status: np.ndarray       # int8 [n] per history (ST_*)
    ptype: np.ndarray
    pos: np.ndarray
    dirs: np.ndarray
    e: np.ndarray
    wt: np.ndarray
    key: np.ndarray          # int32 [n] bin (type * n_ebins + energy bin), -1 if not binned
    emitted: int
    missed: int
    group_bin: np.ndarray    # int64 [groups] in the order they are sent to transport
    group_count: np.ndarray
    hist: np.ndarray         # int64 history ids of the binned particles in that order


def stream_bin(records, e_edges, beam, method: int, phantom, first: int, n: int, capacity: int,
               z_psl: float, sad: float) -> StreamOut:
    """Methods 1 and 2: history h = first + i reads record h mod N (the
    stream, recycled).  Method 2 applies the field's jaw model and fluence
    map (Sec. 2.2), method 1 takes every record as it is (the phase space
    already holds the collimation, Sec. 2.1).  The particles that pass, and
    only those, are binned by type and energy (interior edges, as in the PSL
    generation) and sent to transport in the paper's on-the-fly order."""
    h = first + np.arange(n, dtype=np.int64)
    r = h % records.n if n else h
    x, y, u, v = records.x[r], records.y[r], records.u[r], records.v[r]
    e, wt0, q = records.e[r], records.wt[r], records.q[r]
    status, wt, pos, dirs, ptype, fp = to_phantom(x, y, u, v, e, wt0, q, np.zeros(n, np.int64), [beam], phantom,
                                                  z_psl, sad, collimate=(method == METHOD_JAW_MODEL))
    ne = len(e_edges) - 1
    binned = ((status == ST_TRANSPORT) | (status == ST_MISS)) & (e > 0)
    eb = np.searchsorted(np.asarray(e_edges, F32)[1:-1], e, side="right")
    key = np.where(binned, (q != 0).astype(np.int64) * ne + eb, -1).astype(np.int32)
    gb = np.zeros(max(n, 1), np.int64)
    gc = np.zeros(max(n, 1), np.int64)
    order = np.zeros(max(n, 1), np.int64)
    key_c = np.ascontiguousarray(key)
    ng = _lib.lib().ora_stream_bin(n, _lib._p(key_c), 2 * ne, int(capacity), _lib._p(gb), _lib._p(gc),
                                   _lib._p(order))
    if ng < 0:
        raise ValueError("ora_stream_bin: bad arguments")
    nb = int(gc[:ng].sum())
    return StreamOut(status, ptype, pos, dirs, e.astype(np.float64), wt, key, int(fp[binned].sum()),
                     int(fp[binned & (status == ST_MISS)].sum()), gb[:ng].copy(), gc[:ng].copy(),
                     first + order[:nb])
