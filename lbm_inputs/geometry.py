"""Seeded voxel geometries and random arrays (no lattice Boltzmann arithmetic here).

Every mask is a uint8 array laid out [z][y][x] (x fastest), 1 = solid, 0 = pore,
matching the voxel images the paper's experiments use (a square tube and a
micro-CT rock sub-volume, Section 3).  The rock image itself is not available,
so seeded sphere packs stand in for it.
"""
from __future__ import annotations

import json
import os
import tempfile

import numpy as np


def duct_mask(nx: int, ny: int, nz: int, wall: int = 1) -> np.ndarray:
    """Square/rectangular duct along z: a solid ring `wall` voxels thick on the
    four lateral faces, open at z=0 (inlet) and z=nz-1 (outlet)."""
    m = np.zeros((nz, ny, nx), dtype=np.uint8)
    if wall > 0:
        m[:, :wall, :] = 1
        m[:, ny - wall:, :] = 1
        m[:, :, :wall] = 1
        m[:, :, nx - wall:] = 1
    return m


def random_mask(nx: int, ny: int, nz: int, p_solid: float, seed: int) -> np.ndarray:
    """I.i.d. Bernoulli(p_solid) solids; the inlet and outlet planes keep at
    least one pore each so that both boundary conditions have nodes."""
    rng = np.random.default_rng(seed)
    m = (rng.random((nz, ny, nx)) < p_solid).astype(np.uint8)
    for z in (0, nz - 1):
        if m[z].all():
            m[z, ny // 2, nx // 2] = 0
    return m


def keep_inlet_connected(mask: np.ndarray) -> np.ndarray:
    """Turn every pore region that is not 6-connected to the inlet plane (z=0)
    into solid, so that only cells the injected fluid can reach remain."""
    from scipy import ndimage

    pore = mask == 0
    lab, _ = ndimage.label(pore, structure=ndimage.generate_binary_structure(3, 1))
    keep = np.unique(lab[0][lab[0] > 0])
    out = np.ones_like(mask)
    out[np.isin(lab, keep)] = 0
    return out


def _place_spheres(rng, shape_zyx, rmin, rmax, target_fraction, max_tries):
    """Random sequential addition of non-overlapping spheres (centres anywhere
    in the box, spheres may cross its faces) until the nominal solid volume
    reaches `target_fraction` or `max_tries` consecutive candidates fail."""
    nz, ny, nx = shape_zyx
    vol = float(nx * ny * nz)
    cs = np.empty((0, 3))
    rs = np.empty((0,))
    solid = 0.0
    fails = 0
    while solid < target_fraction * vol and fails < max_tries:
        r = rng.uniform(rmin, rmax)
        c = rng.uniform(0.0, 1.0, 3) * np.array([nx, ny, nz], dtype=float)
        if len(rs):
            d = np.sqrt(((cs - c) ** 2).sum(axis=1))
            if np.any(d < rs + r):
                fails += 1
                continue
        cs = np.vstack([cs, c])
        rs = np.append(rs, r)
        solid += 4.0 / 3.0 * np.pi * r ** 3
        fails = 0
    return cs, rs


def sphere_pack(n: int | tuple, rmin: float, rmax: float, porosity: float, seed: int,
                reservoir: int = 0, lam_max: float = 1.8, max_tries: int = 2000, cache: bool = True):
    """Seeded synthetic sphere pack with a prescribed voxel porosity.

    Centres come from random sequential addition of non-overlapping spheres with
    radii U[rmin, rmax].  Random addition jams well above porosity 0.35, so all
    radii are then scaled by one common factor lam, chosen as the quantile of the
    per-voxel distance ratio min_s |x - c_s| / r_s that gives the requested
    porosity (spheres may then overlap).  A voxel is solid when its centre lies
    inside a scaled sphere.  `reservoir` pure-pore layers are cleared at each z
    end and pores not connected to the inlet are filled.

    Returns (mask, info) with info = {porosity, lam, n_spheres, seed}.  Results
    are cached under the system temporary directory (keyed by every argument)
    because large packs take tens of seconds to generate.
    """
    if isinstance(n, int):
        nx = ny = nz = n
    else:
        nx, ny, nz = n
    key = "pack_%d_%d_%d_%g_%g_%g_%d_%d_%g_%d" % (nx, ny, nz, rmin, rmax, porosity, seed, reservoir,
                                                  lam_max, max_tries)
    path = os.path.join(tempfile.gettempdir(), "lbm_inputs_cache", key + ".npz")
    if cache and os.path.exists(path):
        with np.load(path, allow_pickle=False) as z:
            return z["mask"].copy(), json.loads(str(z["info"]))
    rng = np.random.default_rng(seed)
    cs, rs = _place_spheres(rng, (nz, ny, nx), rmin, rmax, 0.40, max_tries)
    ratio = np.full((nz, ny, nx), np.inf, dtype=np.float32)
    for c, r in zip(cs, rs):
        h = lam_max * r
        lo = np.maximum(np.floor(c - h).astype(int), 0)
        hi = np.minimum(np.ceil(c + h).astype(int) + 1, [nx, ny, nz])
        if np.any(hi <= lo):
            continue
        xs = np.arange(lo[0], hi[0]) + 0.5 - c[0]
        ys = np.arange(lo[1], hi[1]) + 0.5 - c[1]
        zs = np.arange(lo[2], hi[2]) + 0.5 - c[2]
        d = np.sqrt(zs[:, None, None] ** 2 + ys[None, :, None] ** 2 + xs[None, None, :] ** 2) / r
        sub = ratio[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
        np.minimum(sub, d.astype(np.float32), out=sub)
    body = ratio[reservoir:nz - reservoir] if reservoir else ratio
    lam = float(np.quantile(body, 1.0 - porosity))
    if not np.isfinite(lam) or lam >= lam_max:
        raise ValueError("sphere_pack: porosity target not reachable with lam_max=%g" % lam_max)
    mask = (ratio <= lam).astype(np.uint8)
    if reservoir:
        mask[:reservoir] = 0
        mask[nz - reservoir:] = 0
    mask = keep_inlet_connected(mask)
    body = mask[reservoir:nz - reservoir] if reservoir else mask
    info = {"porosity": float(1.0 - body.mean()), "lam": lam, "n_spheres": int(len(rs)),
            "seed": int(seed), "reservoir": int(reservoir)}
    if cache:
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = path + ".%d.tmp.npz" % os.getpid()
            np.savez(tmp, mask=mask, info=json.dumps(info))
            os.replace(tmp, path)
        except OSError:
            pass
    return mask, info


def uniform_field(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Seeded i.i.d. U[lo, hi) float64 array (used to perturb initial states)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=shape)
