"""Seeded synthetic inputs shaped like the paper's workloads.

This module builds geometry only: cell types, fill levels, density and
velocity fields, plus the physical parameters of each workload.  It holds none
of the method's arithmetic (no distributions, no mass exchange, no bubble
volumes), so both the CUDA library and the CPU oracle can take their inputs
from it.

Lattice conventions: arrays have shape (nz, ny, nx) and flatten to the linear
index i = x + nx*(y + ny*z); cell (x, y, z) covers [x, x+1) x [y, y+1) x
[z, z+1) and its centre is (x+0.5, y+0.5, z+0.5).  Every axis wraps; walls are
obstacle cells inside the box.  Fill levels (the liquid fraction, Sec. 2.2 of
the paper) are the fraction of sub x sub x sub sample points of the cell that
lie outside every gas region.

Workloads (paper Sec. 3 stands behind 2 and 3):
  static_bubble       32^3 periodic box, one spherical bubble of radius 8.
  gas_thread          256x64x64, gas cylinder along x with a sinusoidal radius
                      perturbation (capillary breakup of a gas thread, Sec. 3.1).
  orifice             128x128x256 bubble formation at a submerged orifice fed by
                      a gas reservoir (Sec. 3.2).
  bubble_population   many independent small domains with random bubbles.
  foam                512^3 dense lognormal bubble packing under a moving lid.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional, Tuple

import numpy as np

LIQUID, INTERFACE, GAS, OBSTACLE, LID = 0, 1, 2, 3, 4
BGK, TRT = 0, 1

# the 18 non-rest neighbour offsets (dx, dy, dz) of the D3Q19 neighbourhood
_N18 = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
        if 0 < abs(dx) + abs(dy) + abs(dz) <= 2]


@dataclasses.dataclass
class Scenario:
    """One lattice: geometry arrays plus its physical parameters."""
    name: str
    nx: int
    ny: int
    nz: int
    flags: np.ndarray          # uint8 (nz, ny, nx)
    fill: np.ndarray           # float64 (nz, ny, nx)
    rho: np.ndarray            # float64 (nz, ny, nx)
    u: np.ndarray              # float64 (3, nz, ny, nx)
    collision: int = BGK
    tau: float = 0.8
    magic: float = 3.0 / 16.0
    sigma: float = 0.0
    gravity: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    eps: float = 1e-3
    lid: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    normal_rule: int = 1
    lonely_rule: int = 1
    # (seed cell, extra volume, volume drain per step, constant pressure)
    sources: List[Tuple[int, float, float, int]] = dataclasses.field(default_factory=list)
    steps: int = 0

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    def params(self) -> dict:
        return dict(nx=self.nx, ny=self.ny, nz=self.nz, collision=self.collision, tau=self.tau,
                    magic=self.magic, sigma=self.sigma, gravity=tuple(self.gravity), eps=self.eps,
                    lid=tuple(self.lid), normal_rule=self.normal_rule, lonely_rule=self.lonely_rule)

    def linear(self, x: int, y: int, z: int) -> int:
        return int(x + self.nx * (y + self.ny * z))


# ------------------------------------------------------------------ helpers

def _centres(shape):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64) + 0.5,
                          np.arange(ny, dtype=np.float64) + 0.5,
                          np.arange(nx, dtype=np.float64) + 0.5, indexing="ij")
    return x, y, z


def liquid_fraction(shape, sdf: Callable, sub: int = 4, band: float = 1.0) -> np.ndarray:
    """Fraction of sub^3 sample points per cell where sdf(x, y, z) >= 0.

    sdf < 0 marks gas; it must grow no faster than about one unit per cell, so
    that cells whose centre value exceeds `band` in magnitude are entirely on
    one side and only the band around the surface is sub-sampled.
    """
    x, y, z = _centres(shape)
    d = sdf(x, y, z)
    fill = (d >= 0.0).astype(np.float64)
    near = np.abs(d) <= band
    if not near.any():
        return fill
    xs, ys, zs = x[near], y[near], z[near]
    cnt = np.zeros(xs.shape, dtype=np.int64)
    offs = (np.arange(sub, dtype=np.float64) + 0.5) / sub - 0.5
    for oz in offs:
        for oy in offs:
            for ox in offs:
                cnt += (sdf(xs + ox, ys + oy, zs + oz) >= 0.0)
    fill[near] = cnt / float(sub ** 3)
    return fill


def _any_neighbour(mask: np.ndarray) -> np.ndarray:
    out = np.zeros_like(mask)
    for dx, dy, dz in _N18:
        out |= np.roll(mask, shift=(-dz, -dy, -dx), axis=(0, 1, 2))
    return out


def classify(fill: np.ndarray, obstacle: Optional[np.ndarray] = None,
             lid: Optional[np.ndarray] = None) -> np.ndarray:
    """Cell types from fill levels, closing the interface layer.

    Full cells are liquid, empty cells gas, partial cells interface; a liquid
    cell with a gas neighbour becomes interface, so interface cells always
    separate liquid from gas (Sec. 2.2).
    """
    flags = np.full(fill.shape, INTERFACE, dtype=np.uint8)
    flags[fill >= 1.0] = LIQUID
    flags[fill <= 0.0] = GAS
    if obstacle is not None:
        flags[obstacle] = OBSTACLE
    if lid is not None:
        flags[lid] = LID
    gas = flags == GAS
    close = (flags == LIQUID) & _any_neighbour(gas)
    flags[close] = INTERFACE
    return flags


def _finish(name, flags, fill, rho=None, u=None, **kw) -> Scenario:
    nz, ny, nx = flags.shape
    fill = np.where(flags == LIQUID, 1.0, np.where(flags == INTERFACE, fill, 0.0))
    if rho is None:
        rho = np.ones(flags.shape)
    if u is None:
        u = np.zeros((3,) + flags.shape)
    return Scenario(name=name, nx=nx, ny=ny, nz=nz, flags=np.ascontiguousarray(flags),
                    fill=np.ascontiguousarray(fill, dtype=np.float64),
                    rho=np.ascontiguousarray(rho, dtype=np.float64),
                    u=np.ascontiguousarray(u, dtype=np.float64), **kw)


def _spheres_sdf(centres: np.ndarray, radii: np.ndarray):
    """Signed distance to a union of spheres (negative inside gas)."""
    def sdf(x, y, z):
        d = np.full(np.shape(x), np.inf)
        for (cx, cy, cz), r in zip(centres, radii):
            d = np.minimum(d, np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) - r)
        return d
    return sdf


def _wall_shell(shape, axes) -> np.ndarray:
    nz, ny, nx = shape
    obs = np.zeros(shape, dtype=bool)
    if 0 in axes:
        obs[:, :, 0] = obs[:, :, nx - 1] = True
    if 1 in axes:
        obs[:, 0, :] = obs[:, ny - 1, :] = True
    if 2 in axes:
        obs[0, :, :] = obs[nz - 1, :, :] = True
    return obs


# ---------------------------------------------------------------- workloads

def static_bubble(n: int = 32, radius: float = 8.0, sigma: float = 1e-3, tau: float = 0.8,
                  collision: int = BGK, steps: int = 200) -> Scenario:
    """Periodic n^3 box of liquid at rest with one spherical bubble at the centre."""
    c = n / 2.0
    sdf = _spheres_sdf(np.array([[c, c, c]]), np.array([radius]))
    fill = liquid_fraction((n, n, n), sdf)
    flags = classify(fill)
    return _finish(f"static_bubble_{n}_r{radius:g}", flags, fill, collision=collision, tau=tau,
                   sigma=sigma, steps=steps)


def gas_thread(nx: int = 256, ny: int = 64, nz: int = 64, radius: float = 8.0, amp: float = 0.1,
               wavelength: float = 64.0, sigma: float = 5e-3, tau: float = 0.8,
               collision: int = TRT, steps: int = 20000) -> Scenario:
    """Gas cylinder along x with radius R(x) = R (1 + amp sin(2 pi x / wavelength)),
    periodic in x, no-slip walls on the other four sides (paper Sec. 3.1)."""
    cy, cz = ny / 2.0, nz / 2.0

    def sdf(x, y, z):
        r = np.sqrt((y - cy) ** 2 + (z - cz) ** 2)
        return r - radius * (1.0 + amp * np.sin(2.0 * np.pi * x / wavelength))

    shape = (nz, ny, nx)
    fill = liquid_fraction(shape, sdf, band=1.2)
    obs = _wall_shell(shape, axes=(1, 2))
    flags = classify(fill, obstacle=obs)
    return _finish(f"gas_thread_{nx}x{ny}x{nz}", flags, fill, collision=collision, tau=tau,
                   sigma=sigma, steps=steps)


def orifice(nx: int = 128, ny: int = 128, nz: int = 256, plate_z: int = 8, hole_radius: float = 6.0,
            depth: int = 200, cap_radius: float = 6.0, drain: float = 0.02, reservoir: float = 2e4,
            gravity: float = 1e-5, sigma: float = 2e-3, tau: float = 0.8, steps: int = 100000) -> Scenario:
    """Bubble formation at a submerged circular orifice (paper Sec. 3.2).

    No-slip box; a plate at z = plate_z with a circular hole; gas reservoir
    below the plate whose volume shrinks by `drain` cells^3 per step; liquid up
    to z = plate_z + depth with a constant-pressure gas layer above; a
    hemispherical gas cap of radius `cap_radius` sits on the hole.  Density is
    hydrostatic, rho = 1 + 3 g (h - z), h the liquid surface height.
    """
    shape = (nz, ny, nx)
    x, y, z = _centres(shape)
    hx, hy = nx / 2.0, ny / 2.0
    top = plate_z + 1 + depth
    obs = _wall_shell(shape, axes=(0, 1, 2))
    rr = np.sqrt((x - hx) ** 2 + (y - hy) ** 2)
    plate = (np.floor(z) == plate_z) & (rr > hole_radius)
    obs |= plate

    def sdf(xx, yy, zz):
        below = plate_z + 0.5 - zz           # > 0 below the plate centre: reservoir gas
        above = zz - top                      # > 0 in the atmosphere
        cap = cap_radius - np.sqrt((xx - hx) ** 2 + (yy - hy) ** 2 + (zz - (plate_z + 1.0)) ** 2)
        hole = np.where(np.abs(zz - (plate_z + 0.5)) <= 0.5, hole_radius - np.sqrt((xx - hx) ** 2 + (yy - hy) ** 2), -np.inf)
        gas = np.maximum(np.maximum(below, above), np.maximum(cap, hole))
        return -gas

    fill = liquid_fraction(shape, sdf, band=1.5)
    flags = classify(fill, obstacle=obs)
    rho = 1.0 + 3.0 * gravity * (top - z)
    rho = np.where((flags == LIQUID) | (flags == INTERFACE), rho, 1.0)
    seed = int(hx) + nx * (int(hy) + ny * 2)
    atm = int(hx) + nx * (int(hy) + ny * (nz - 3))
    return _finish(f"orifice_{nx}x{ny}x{nz}", flags, fill, rho=rho, collision=TRT, tau=tau,
                   sigma=sigma, gravity=(0.0, 0.0, -gravity), steps=steps,
                   sources=[(seed, reservoir, drain, 0), (atm, 0.0, 0.0, 1)])


def _rsa(rng, dims, radii, gap, max_attempts, periodic=True):
    """Random sequential addition of non-overlapping spheres with a liquid gap:
    each sphere in turn draws random centres until one keeps the gap to every
    sphere placed so far; all draws together are capped at max_attempts."""
    dims = np.asarray(dims, dtype=np.float64)
    pc = np.zeros((len(radii), 3))
    pr = np.zeros(len(radii))
    n = 0
    attempts = 0
    for r in radii:
        placed = False
        while attempts < max_attempts and not placed:
            # a batch of candidate centres tested against all placed spheres
            batch = int(min(256, max_attempts - attempts))
            cand = rng.uniform(0.0, 1.0, (batch, 3)) * dims
            if n == 0:
                ok = np.ones(batch, dtype=bool)
            else:
                d = cand[:, None, :] - pc[None, :n, :]
                if periodic:
                    d -= dims * np.round(d / dims)
                dist = np.sqrt((d * d).sum(-1))
                ok = (dist >= (r + pr[:n] + gap)[None, :]).all(1)
            hit = np.nonzero(ok)[0]
            if hit.size:
                attempts += int(hit[0]) + 1
                pc[n] = cand[hit[0]]
                pr[n] = r
                n += 1
                placed = True
            else:
                attempts += batch
        if attempts >= max_attempts:
            break
    return pc[:n].copy(), pr[:n].copy()


def _stamp_spheres(shape, centres, radii, sub: int = 4) -> np.ndarray:
    """Liquid fraction of a periodic box holding non-overlapping gas spheres:
    each sphere is sub-sampled only inside its own bounding box."""
    nz, ny, nx = shape
    fill = np.ones(shape)
    offs = (np.arange(sub, dtype=np.float64) + 0.5) / sub - 0.5
    for c, r in zip(centres, radii):
        lo = np.floor(np.asarray(c) - r - 1).astype(int)
        hi = np.ceil(np.asarray(c) + r + 1).astype(int)
        zi = np.arange(lo[2], hi[2]); yi = np.arange(lo[1], hi[1]); xi = np.arange(lo[0], hi[0])
        zz, yy, xx = np.meshgrid(zi, yi, xi, indexing="ij")
        cnt = np.zeros(zz.shape)
        for oz in offs:
            for oy in offs:
                for ox in offs:
                    d2 = (xx + 0.5 + ox - c[0]) ** 2 + (yy + 0.5 + oy - c[1]) ** 2 + (zz + 0.5 + oz - c[2]) ** 2
                    cnt += d2 < r * r
        sl = (np.mod(zz, nz), np.mod(yy, ny), np.mod(xx, nx))
        fill[sl] = np.minimum(fill[sl], 1.0 - cnt / float(sub ** 3))
    return fill


def _periodic_spheres_sdf(centres, radii, dims):
    dims = np.asarray(dims, dtype=np.float64)

    def sdf(x, y, z):
        d = np.full(np.shape(x), np.inf)
        for c, r in zip(centres, radii):
            dx = x - c[0]; dx -= dims[0] * np.round(dx / dims[0])
            dy = y - c[1]; dy -= dims[1] * np.round(dy / dims[1])
            dz = z - c[2]; dz -= dims[2] * np.round(dz / dims[2])
            d = np.minimum(d, np.sqrt(dx * dx + dy * dy + dz * dz) - r)
        return d
    return sdf


def random_bubbles(nx: int, ny: int, nz: int, n_bubbles: int, r_min: float, r_max: float,
                   u_max: float, sigma: float, seed: int, gap: float = 2.0,
                   collision: int = TRT, tau: float = 0.8, max_attempts: int = 10000,
                   steps: int = 2000) -> Scenario:
    """Periodic box with randomly placed bubbles and a smooth random velocity field
    (one Fourier mode per component, |u| <= u_max)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    radii = rng.uniform(r_min, r_max, n_bubbles)
    centres, radii = _rsa(rng, (nx, ny, nz), radii, gap, max_attempts)
    shape = (nz, ny, nx)
    fill = _stamp_spheres(shape, centres, radii)
    flags = classify(fill)
    x, y, z = _centres(shape)
    u = np.zeros((3,) + shape)
    k = rng.integers(1, 3, size=(3, 3))
    ph = rng.uniform(0.0, 2.0 * np.pi, size=3)
    amp = u_max * rng.uniform(0.3, 1.0) / math.sqrt(3.0)
    for c in range(3):
        arg = 2.0 * np.pi * (k[c, 0] * x / nx + k[c, 1] * y / ny + k[c, 2] * z / nz) + ph[c]
        u[c] = amp * np.sin(arg)
    u[:, (flags == GAS)] = 0.0
    return _finish(f"random_bubbles_{nx}x{ny}x{nz}_s{seed}", flags, fill, u=u, collision=collision,
                   tau=tau, sigma=sigma, steps=steps)


def bubble_population(n_domains: int = 64, seed: int = 0, sides=(32, 48, 64, 96), steps: int = 2000):
    """Independent domains, each axis drawn from `sides`, 20-200 bubbles of radius
    U[3, 10] per domain by random sequential addition (attempt cap 10^4),
    |u0| <= 0.02, sigma ~ U[1e-3, 5e-3]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for d in range(n_domains):
        nx, ny, nz = (int(v) for v in rng.choice(sides, 3))
        nb = int(rng.integers(20, 201))
        sig = float(rng.uniform(1e-3, 5e-3))
        out.append(random_bubbles(nx, ny, nz, nb, 3.0, 10.0, 0.02, sig, seed=int(rng.integers(1 << 31)),
                                  steps=steps))
    return out


def _rsa_grid(rng, box_lo, box_hi, radii, gap, max_attempts, periodic):
    """Random sequential addition: sphere k (in the given order) draws uniform
    centres until one keeps a liquid gap of `gap` to every sphere placed so
    far, all draws together capped at max_attempts.  On a periodic axis the
    centre ranges over [lo, hi) and distances take the minimum image; on a
    bounded axis it ranges over [lo + r, hi - r].

    Candidates are drawn in batches and the first acceptable one in draw order
    is taken (the others count as drawn).  Two filters make a draw cheap: a
    coarse grid of 2-cell voxels marks voxels lying entirely within
    r_j + gap + r_min of a placed centre (no sphere of the list may be centred
    there), and the exact test looks only at the spheres of the 27 buckets
    around the candidate (bucket edge >= the largest centre distance of two
    spheres that can conflict)."""
    lo = np.asarray(box_lo, dtype=np.float64)
    hi = np.asarray(box_hi, dtype=np.float64)
    per = np.asarray(periodic, dtype=bool)
    L = hi - lo
    radii = np.asarray(radii, dtype=np.float64)
    if radii.size == 0:
        return np.zeros((0, 3)), np.zeros(0)
    rmin = float(radii.min())
    reach = 2.0 * float(radii.max()) + gap
    nb = np.maximum(1, np.floor(L / reach).astype(np.int64))
    h = L / nb
    nbk = int(np.prod(nb))
    members = np.full((nbk, 16), -1, dtype=np.int64)
    fillc = np.zeros(nbk, dtype=np.int64)
    pc = np.zeros((len(radii) + 1, 3))
    pr = np.zeros(len(radii) + 1)
    pc[-1] = 1e30                      # member slot -1: a sphere far away
    offs = [np.arange(-1, 2) if nb[a] >= 3 else None for a in range(3)]
    # coarse exclusion grid: voxel edge 2, voxel v covers [lo + 2 v, lo + 2 v + 2)
    nv = np.maximum(1, np.ceil(L / 2.0).astype(np.int64))
    excl = np.zeros(int(np.prod(nv)), dtype=bool)

    def neighbour_buckets(bi):         # (k, 3) bucket coordinates -> (k, <= 27) bucket ids
        ax = []
        for a in range(3):
            if offs[a] is None:
                v = np.broadcast_to(np.arange(nb[a]), (bi.shape[0], nb[a]))
            elif per[a]:
                v = (bi[:, a:a + 1] + offs[a][None, :]) % nb[a]
            else:
                v = np.clip(bi[:, a:a + 1] + offs[a][None, :], 0, nb[a] - 1)
            ax.append(v)
        return (ax[0][:, :, None, None] + nb[0] * (ax[1][:, None, :, None] + nb[1] * ax[2][:, None, None, :])
                ).reshape(bi.shape[0], -1)

    def voxel_ids(p):                  # (k, 3) points -> (k,) coarse voxel ids
        v = np.minimum(((p - lo) / 2.0).astype(np.int64), nv - 1)
        return v[:, 0] + nv[0] * (v[:, 1] + nv[1] * v[:, 2])

    def exclude(c, r):                 # mark voxels entirely within r + gap + rmin of c
        R = r + gap + rmin
        m = int(np.ceil(R / 2.0)) + 1
        o = np.arange(-m, m + 1)
        vc = np.floor((c - lo) / 2.0).astype(np.int64)
        axes = []
        for a in range(3):
            v = vc[a] + o
            ctr = lo[a] + 2.0 * v + 1.0 - c[a]          # voxel centre relative to c (before wrapping)
            if per[a]:
                v = np.mod(v, nv[a])
                keep = np.ones(v.shape, dtype=bool)
            else:
                keep = (v >= 0) & (v < nv[a])
            axes.append((v[keep], ctr[keep]))
        (vx, cx_), (vy, cy_), (vz, cz_) = axes
        d2 = cz_[:, None, None] ** 2 + cy_[None, :, None] ** 2 + cx_[None, None, :] ** 2
        inside = np.sqrt(d2) + np.sqrt(3.0) <= R
        ids = vx[None, None, :] + nv[0] * (vy[None, :, None] + nv[1] * vz[:, None, None])
        excl[ids[inside]] = True

    n = 0
    attempts = 0
    batch = 8
    for r in radii:
        clo = np.where(per, lo, lo + r)
        chi = np.where(per, hi, hi - r)
        if np.any(chi <= clo):
            continue
        placed = False
        while attempts < max_attempts and not placed:
            k = int(min(batch, max_attempts - attempts))
            cand = clo + rng.uniform(0.0, 1.0, (k, 3)) * (chi - clo)
            free = np.nonzero(~excl[voxel_ids(cand)])[0]
            hit = -1
            if free.size:
                cf = cand[free]
                bi = np.minimum(((cf - lo) / h).astype(np.int64), nb - 1)
                idx = members[neighbour_buckets(bi)].reshape(free.size, -1)     # (kf, M)
                d = cf[:, None, :] - pc[idx]
                for a in range(3):
                    if per[a]:
                        d[:, :, a] -= L[a] * np.round(d[:, :, a] / L[a])
                ok = np.all((d * d).sum(-1) >= (r + pr[idx] + gap) ** 2, axis=1)
                w = np.nonzero(ok)[0]
                if w.size:
                    hit = int(free[w[0]])
            if hit >= 0:
                attempts += hit + 1
                c = cand[hit]
                pc[n] = c
                pr[n] = r
                bj = np.minimum(((c - lo) / h).astype(np.int64), nb - 1)
                b = int(bj[0] + nb[0] * (bj[1] + nb[1] * bj[2]))
                if fillc[b] == members.shape[1]:
                    members = np.concatenate([members, np.full_like(members, -1)], 1)
                members[b, fillc[b]] = n
                fillc[b] += 1
                exclude(c, r)
                n += 1
                placed = True
                batch = max(8, batch // 2)
            else:
                attempts += k
                batch = min(1 << 14, 2 * batch)
        if attempts >= max_attempts:
            break
    return pc[:n].copy(), pr[:n].copy()


def _stamp_spheres_banded(shape, centres, radii, sub: int = 4, chunk_cells: int = 1 << 22) -> np.ndarray:
    """Liquid fraction of a box (every axis wrapping) holding non-overlapping gas
    spheres: the fraction of sub^3 sample points of each cell outside every
    sphere.  Cells whose centre lies more than the sample points' reach
    (sqrt(3)/2 (1 - 1/sub)) inside a sphere are all gas, those as far outside
    are untouched; only the band between is sub-sampled.  Spheres are handled
    in chunks of equal bounding-box size, all with numpy array operations."""
    nz, ny, nx = shape
    fill = np.ones(nz * ny * nx)
    offs = (np.arange(sub, dtype=np.float64) + 0.5) / sub - 0.5
    reach = 0.5 * np.sqrt(3.0) * (1.0 - 1.0 / sub) + 1e-9
    centres = np.asarray(centres, dtype=np.float64)
    radii = np.asarray(radii, dtype=np.float64)
    box = np.ceil(2.0 * radii + 3.0).astype(np.int64)
    order = np.argsort(box, kind="stable")
    for b in np.unique(box):
        sel = order[box[order] == b]
        per = max(1, chunk_cells // int(b) ** 3)
        o = np.arange(b, dtype=np.float64)
        for s0 in range(0, len(sel), per):
            ids = sel[s0:s0 + per]
            c = centres[ids]
            r = radii[ids]
            base = np.floor(c - r[:, None] - 1.0)                    # (M, 3) first cell of the box
            X = base[:, 0:1] + o[None, :]                             # (M, b) cell corners
            Y = base[:, 1:2] + o[None, :]
            Z = base[:, 2:3] + o[None, :]
            dx2 = (X + 0.5 - c[:, 0:1]) ** 2
            dy2 = (Y + 0.5 - c[:, 1:2]) ** 2
            dz2 = (Z + 0.5 - c[:, 2:3]) ** 2
            dist = np.sqrt(dz2[:, :, None, None] + dy2[:, None, :, None] + dx2[:, None, None, :]) - r[:, None, None, None]
            xi = np.mod(X.astype(np.int64), nx)
            yi = np.mod(Y.astype(np.int64), ny)
            zi = np.mod(Z.astype(np.int64), nz)
            flat = xi[:, None, None, :] + nx * (yi[:, None, :, None] + ny * zi[:, :, None, None])
            inside = dist < -reach
            fill[flat[inside]] = 0.0
            m, k, j, i = np.nonzero(np.abs(dist) <= reach)
            if m.size == 0:
                continue
            ax = (X[m, i][:, None] + 0.5 + offs[None, :] - c[m, 0][:, None]) ** 2     # (NB, sub)
            ay = (Y[m, j][:, None] + 0.5 + offs[None, :] - c[m, 1][:, None]) ** 2
            az = (Z[m, k][:, None] + 0.5 + offs[None, :] - c[m, 2][:, None]) ** 2
            d2 = az[:, :, None, None] + ay[:, None, :, None] + ax[:, None, None, :]
            cnt = np.count_nonzero((d2 < (r[m] ** 2)[:, None, None, None]).reshape(m.size, -1), axis=1)
            fb = flat[m, k, j, i]
            fill[fb] = np.minimum(fill[fb], 1.0 - cnt / float(sub ** 3))
    return fill.reshape(shape)


def foam(n: int = 512, gas_fraction: float = 0.4, seed: int = 0, lid_speed: float = 0.05,
         gravity: float = 1e-5, sigma: float = 3e-3, max_attempts: Optional[int] = None, gap: float = 2.0,
         steps: int = 10000) -> Scenario:
    """Dense bubble packing: lognormal radii (median 8, sigma_log 0.3, clipped to
    [4, 16]) drawn until their volume reaches `gas_fraction` of the box, placed
    largest first by random sequential addition with a liquid gap of `gap`
    cells between bubbles and to the walls (attempts capped, so a jammed
    packing stops short of the target); periodic in x and y, no-slip bottom
    wall at z = 0, lid at z = n - 1 moving at u_x = lid_speed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    target = gas_fraction * n ** 3
    radii = []
    vol = 0.0
    while vol < target:
        r = float(np.clip(np.exp(np.log(8.0) + 0.3 * rng.standard_normal()), 4.0, 16.0))
        radii.append(r)
        vol += 4.0 / 3.0 * np.pi * r ** 3
    radii = np.sort(np.array(radii))[::-1]
    if max_attempts is None:
        max_attempts = 100 * len(radii)
    centres, radii = _rsa_grid(rng, (0.0, 0.0, 1.0 + gap), (float(n), float(n), n - 1.0 - gap), radii, gap,
                               max_attempts, (True, True, False))
    shape = (n, n, n)
    fill = _stamp_spheres_banded(shape, centres, radii)
    obs = np.zeros(shape, dtype=bool)
    obs[0] = True
    lid = np.zeros(shape, dtype=bool)
    lid[n - 1] = True
    flags = classify(fill, obstacle=obs, lid=lid)
    sc = _finish(f"foam_{n}", flags, fill, collision=TRT, sigma=sigma, gravity=(0.0, 0.0, -gravity),
                 lid=(lid_speed, 0.0, 0.0), steps=steps)
    sc.bubbles_placed = int(len(radii))
    return sc


# the thread-rupture case of the paper (Sec. 3.1): its physical quantities
RUPTURE_DX = 1.25e-5       # m, lattice spacing
RUPTURE_NU = 1e-6          # m^2/s, kinematic viscosity of the liquid
RUPTURE_RHO = 1000.0       # kg/m^3, liquid density
RUPTURE_SIGMAS = (0.072, 0.018)   # N/m, the two surface tensions
RUPTURE_FRAMES_MS = {0.072: (22, 38, 46, 68, 324), 0.018: (22, 65, 76, 90, 324)}
RUPTURE_PIECES = {0.072: 5, 0.018: 6}


def rupture_units(sigma_si: float, dt: float = 5e-7, tau: Optional[float] = 0.8, nu_si: float = RUPTURE_NU,
                  dx: float = RUPTURE_DX, rho_si: float = RUPTURE_RHO) -> dict:
    """Lattice parameters of the thread-rupture case for an assumed time step
    dt (the paper gives dx, nu, rho and sigma but no time step):
    sigma_lb = sigma dt^2 / (rho dx^3).  With tau=None the viscosity is the
    paper's, tau = 3 nu dt / dx^2 + 1/2 (0.5096 at dt = 5e-7 s); otherwise tau
    is taken as given and the viscosity it implies, nu = (tau - 1/2) dx^2 /
    (3 dt), is reported."""
    if tau is None:
        nu_lb = nu_si * dt / dx ** 2
        tau = 3.0 * nu_lb + 0.5
    nu_lb = (tau - 0.5) / 3.0
    return {"dt": dt, "tau": tau, "nu_lb": nu_lb, "nu_si": nu_lb * dx ** 2 / dt,
            "sigma_lb": sigma_si * dt ** 2 / (rho_si * dx ** 3)}


def thread_rupture(sigma_si: float = 0.072, dt: float = 5e-7, tau: Optional[float] = 0.8, nx: int = 360,
                   ny: int = 40, nz: int = 40, gas=(336, 8, 8), collision: int = TRT) -> Scenario:
    """Rupture of a thin gas thread (paper Sec. 3.1): a 360 x 40 x 40 domain of
    liquid at rest holding a centred rectangular gas block of 336 x 8 x 8 cells.
    No-slip walls close all six faces (a one-cell obstacle shell inside the
    box); no gravity.  The block's faces lie on cell faces, so fill levels are
    0 or 1 and the closed interface layer is the liquid cells touching gas.
    tau and sigma in lattice units follow from the paper's dx, rho, sigma and
    the assumed dt (rupture_units)."""
    p = rupture_units(sigma_si, dt, tau)
    shape = (nz, ny, nx)
    gx, gy, gz = gas
    x0, y0, z0 = (nx - gx) // 2, (ny - gy) // 2, (nz - gz) // 2
    fill = np.ones(shape)
    fill[z0:z0 + gz, y0:y0 + gy, x0:x0 + gx] = 0.0
    obs = _wall_shell(shape, axes=(0, 1, 2))
    flags = classify(fill, obstacle=obs)
    sc = _finish(f"thread_rupture_{nx}x{ny}x{nz}_sigma{sigma_si:g}", flags, fill, collision=collision,
                 tau=p["tau"], sigma=p["sigma_lb"], steps=int(round(324e-3 / dt)))
    sc.units = p
    return sc
