"""Oracle readout: dose, batch uncertainty, normalisation and gamma index
(TEST INFRASTRUCTURE; see the package docstring for who may import it).

* Dose counters and uncertainty, Sec. 2.3.3: the dose is the sum of the batch
  tallies; its standard error is the standard deviation of the independent
  batch estimates divided by sqrt(N_b).
* Normalisation, Sec. 2.5: D = D_o N_total^phsp / (N_total^simulated
  N_incident^phsp); the caller passes that factor as ``norm``.
* Gamma index, Sec. 3 and Table 1: 3D global gamma, dose criterion as a
  fraction of the reference maximum, distance criterion in cm, evaluated on
  reference voxels above a fraction (10 %) of the maximum.
"""
from __future__ import annotations

import numpy as np

MEV_TO_J = 1.602176634e-13
FP_SCALE = 2.0 ** -32


def dose(tallies: np.ndarray, rho: np.ndarray, voxel, norm: float = 1.0):
    """tallies: int64 [N_b, nz, ny, nx] fixed point (2^-32 MeV).  Returns
    (dose Gy * norm, sigma) as float64 arrays [nz, ny, nx]."""
    nb = tallies.shape[0]
    vol = float(voxel[0]) * float(voxel[1]) * float(voxel[2])
    mass_kg = rho.astype(np.float64) * vol * 1e-3
    with np.errstate(divide="ignore", invalid="ignore"):
        c = np.where(mass_kg > 0, FP_SCALE * MEV_TO_J / mass_kg, 0.0) * norm
    t = tallies.astype(np.float64)
    total = t.sum(0)
    d = total * c
    if nb > 1:
        mean = total / nb
        var = ((t - mean[None]) ** 2).sum(0)
        s = c * np.sqrt(nb / (nb - 1.0) * var)
    else:
        s = np.zeros_like(d)
    return d, s


def gamma_pass_rate(ref: np.ndarray, ev: np.ndarray, voxel, dose_crit=0.02, dta_cm=0.2,
                    threshold=0.10, upsample=4, max_radius_cm=None):
    """Fraction of reference voxels above `threshold` * max(ref) with gamma <= 1.

    Gamma at a reference voxel is the minimum over evaluated points r of
    sqrt(|r - r_ref|^2 / dta^2 + (D_ev(r) - D_ref)^2 / (dose_crit max ref)^2);
    D_ev between voxel centres is trilinear.  Search radius 1.5 * dta by
    default, on a grid of voxel / upsample."""
    ref = np.asarray(ref, np.float64)
    ev = np.asarray(ev, np.float64)
    dmax = ref.max()
    dd = dose_crit * dmax
    vz, vy, vx = voxel[2], voxel[1], voxel[0]
    mask = ref >= threshold * dmax
    idx = np.argwhere(mask)
    dref = ref[mask]
    rad = 1.5 * dta_cm if max_radius_cm is None else max_radius_cm
    best = ((ev[mask] - dref) / dd) ** 2
    nz, ny, nx = ev.shape
    steps = []
    for v in (vz, vy, vx):
        h = v / upsample
        m = int(np.ceil(rad / h))
        steps.append(np.arange(-m, m + 1) * h)
    for oz in steps[0]:
        for oy in steps[1]:
            for ox in steps[2]:
                r2 = oz * oz + oy * oy + ox * ox
                if r2 == 0 or r2 > rad * rad:
                    continue
                if r2 / (dta_cm * dta_cm) >= best.max():
                    continue
                fz = idx[:, 0] + oz / vz
                fy = idx[:, 1] + oy / vy
                fx = idx[:, 2] + ox / vx
                val = _trilinear(ev, fz, fy, fx)
                g2 = r2 / (dta_cm * dta_cm) + ((val - dref) / dd) ** 2
                np.minimum(best, np.where(np.isnan(g2), np.inf, g2), out=best)
    return float((best <= 1.0).mean()), int(mask.sum())


def _trilinear(a, fz, fy, fx):
    nz, ny, nx = a.shape
    out = np.full(fz.shape, np.nan)
    ok = (fz >= 0) & (fz <= nz - 1) & (fy >= 0) & (fy <= ny - 1) & (fx >= 0) & (fx <= nx - 1)
    z, y, x = fz[ok], fy[ok], fx[ok]
    z0 = np.minimum(np.floor(z).astype(np.int64), nz - 2 if nz > 1 else 0)
    y0 = np.minimum(np.floor(y).astype(np.int64), ny - 2 if ny > 1 else 0)
    x0 = np.minimum(np.floor(x).astype(np.int64), nx - 2 if nx > 1 else 0)
    tz, ty, tx = z - z0, y - y0, x - x0
    z1, y1, x1 = np.minimum(z0 + 1, nz - 1), np.minimum(y0 + 1, ny - 1), np.minimum(x0 + 1, nx - 1)
    c00 = a[z0, y0, x0] * (1 - tx) + a[z0, y0, x1] * tx
    c01 = a[z0, y1, x0] * (1 - tx) + a[z0, y1, x1] * tx
    c10 = a[z1, y0, x0] * (1 - tx) + a[z1, y0, x1] * tx
    c11 = a[z1, y1, x0] * (1 - tx) + a[z1, y1, x1] * tx
    c0 = c00 * (1 - ty) + c01 * ty
    c1 = c10 * (1 - ty) + c11 * ty
    out[ok] = c0 * (1 - tz) + c1 * tz
    return out
