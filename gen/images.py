"""Seeded image / voxel generators standing in for the paper's Poisson composites.

The paper's own specimen files are hosted elsewhere and are not used. These
generators give images of the shapes the paper's workloads have (two-phase 2D
composites with circular soft inclusions, Section 3.1 "Mode-I fracture of
Poisson composites"), plus a 3D voxel foam and batches of uneven 2D
specimens.

Phase convention: 0 = void (no particle), 1 = stiff matrix, 2 = soft
inclusion. Arrays are indexed [y, x] in 2D and [z, y, x] in 3D, so that a
C-order flatten gives x fastest (raster order).

Everything here is input preparation: random numbers, thresholds and the two
material tables. No spring, force or integration arithmetic lives here.
"""
from __future__ import annotations

import numpy as np

# Stiff matrix / soft inclusion materials used by every two-phase workload.
STIFF_K, STIFF_EPSC = 1.0, 0.05
SOFT_K, SOFT_EPSC = 0.1, 0.3


def _rng(seed):
    if isinstance(seed, (tuple, list)):
        return np.random.default_rng([int(s) for s in seed])
    return np.random.default_rng(int(seed))


def inclusion_image(nx: int, ny: int, r_min: float, r_max: float, frac: float, seed) -> np.ndarray:
    """2D two-phase image: matrix (1) with overlapping circular soft inclusions (2).

    Disks are drawn one at a time (centre uniform in [0,nx) x [0,ny), radius
    uniform in [r_min, r_max]); pixel (px, py) is soft when its centre lies in
    the disk. Drawing stops at the first disk that brings the soft area fraction
    to at least ``frac``. Returns uint8 [ny, nx].
    """
    rng = _rng(seed)
    soft = np.zeros((ny, nx), dtype=bool)
    target = frac * nx * ny
    count = 0
    while count < target:
        cx = rng.uniform(0.0, nx)
        cy = rng.uniform(0.0, ny)
        r = rng.uniform(r_min, r_max)
        x0, x1 = max(0, int(np.floor(cx - r - 1))), min(nx, int(np.ceil(cx + r + 1)))
        y0, y1 = max(0, int(np.floor(cy - r - 1))), min(ny, int(np.ceil(cy + r + 1)))
        if x0 >= x1 or y0 >= y1:
            continue
        py, px = np.mgrid[y0:y1, x0:x1]
        disk = (px + 0.5 - cx) ** 2 + (py + 0.5 - cy) ** 2 <= r * r
        sub = soft[y0:y1, x0:x1]
        count += int(np.count_nonzero(disk & ~sub))
        sub |= disk
    img = np.ones((ny, nx), dtype=np.uint8)
    img[soft] = 2
    return img


def foam_volume(n: int = 256, sigma: float = 4.0, solid_frac: float = 0.35, seed=2) -> np.ndarray:
    """3D one-phase foam: N(0,1) noise smoothed by a periodic separable Gaussian
    (sigma voxels, truncated at 4 sigma), thresholded so that ``solid_frac`` of
    the voxels are solid (phase 1); the rest are void (0). Returns uint8 [n,n,n]
    indexed [z, y, x].
    """
    from scipy.ndimage import gaussian_filter

    rng = _rng(seed)
    noise = rng.standard_normal((n, n, n), dtype=np.float64)
    field = gaussian_filter(noise, sigma=sigma, mode="wrap", truncate=4.0)
    thr = np.quantile(field, 1.0 - solid_frac)
    return (field > thr).astype(np.uint8)


def batch_specimens(count: int = 512, l_min: int = 32, l_max: int = 512, seed0: int = 3):
    """Uneven batch of square two-phase specimens.

    Specimen b uses seed (seed0, b): side L uniform integer in [l_min, l_max],
    inclusion fraction uniform in [0.10, 0.50], radii 3..8 px.
    """
    out = []
    for b in range(count):
        rng = _rng((seed0, b))
        side = int(rng.integers(l_min, l_max + 1))
        frac = float(rng.uniform(0.10, 0.50))
        img_seed = (seed0, b, 1)
        out.append(inclusion_image(side, side, 3.0, 8.0, frac, img_seed))
    return out


def warmstart_specimens(seeds, side: int = 256):
    """Two-phase side x side specimens for the learned warm start; specimen
    seed s draws its inclusion fraction uniformly in [0.10, 0.50]."""
    out = []
    for s in seeds:
        rng = _rng((4, s))
        frac = float(rng.uniform(0.10, 0.50))
        out.append(inclusion_image(side, side, 3.0, 8.0, frac, (4, s, 1)))
    return out


def two_phase_materials():
    """Per-phase-pair spring tables for the stiff/soft composite.

    Returns (k_tab, epsc_tab, mass), 2x2 row-major tables indexed by
    (phase_i - 1, phase_j - 1). The paper's Table of spring constants gives the
    stiff-soft spring its own values rather than a rule; here the interface
    spring is taken as the two half-springs in series (harmonic mean of k) and
    the mean of the two critical strains.
    """
    k_int = 2.0 * STIFF_K * SOFT_K / (STIFF_K + SOFT_K)
    e_int = 0.5 * (STIFF_EPSC + SOFT_EPSC)
    k_tab = np.array([[STIFF_K, k_int], [k_int, SOFT_K]], dtype=np.float64)
    e_tab = np.array([[STIFF_EPSC, e_int], [e_int, SOFT_EPSC]], dtype=np.float64)
    mass = np.array([1.0, 1.0], dtype=np.float64)
    return k_tab, e_tab, mass


def one_phase_materials(k: float = 1.0, epsc: float = 0.04):
    return (np.array([[k]], dtype=np.float64), np.array([[epsc]], dtype=np.float64),
            np.array([1.0], dtype=np.float64))


def paper_table_materials():
    """The paper's three linear fracture springs (stiff-stiff, soft-soft,
    stiff-soft) as k and critical strain tables with r0 = 10 (Table of spring
    constants, Section 3.1): critical strain = rc / r0 - 1."""
    k_tab = np.array([[2.00e-3, 1.25e-4], [1.25e-4, 2.00e-5]], dtype=np.float64)
    rc = np.array([[10.1, 10.4], [10.4, 11.0]], dtype=np.float64)
    return k_tab, rc / 10.0 - 1.0, np.array([1.0, 1.0])


# Named workloads (image recipe + loading schedule): the 64^2 parity case,
# the 2048^2 composite and the 256^3 foam (the batch: batch_specimens).
WORKLOADS = {
    "2d_64": dict(dim=2, nx=64, ny=64, r=(3.0, 8.0), frac=0.30, seed=0,
                  eps_max=0.10, increments=100, steps=20, dt=0.01, damping=0.1),
    "2d_2048": dict(dim=2, nx=2048, ny=2048, r=(10.0, 60.0), frac=0.30, seed=1,
                    eps_inc=1e-3, steps=20, dt=0.01, damping=0.1),
    "3d_foam_256": dict(dim=3, n=256, sigma=4.0, solid=0.35, seed=2,
                        eps_min=-0.20, increments=100, steps=20, dt=0.01, damping=0.1),
}


def workload_image(name: str):
    w = WORKLOADS[name]
    if name.startswith("3d"):
        return foam_volume(w["n"], w["sigma"], w["solid"], w["seed"])
    return inclusion_image(w["nx"], w["ny"], w["r"][0], w["r"][1], w["frac"], w["seed"])
