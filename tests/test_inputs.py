"""The seeded input generators (shared by the oracle and the CUDA path, and
holding none of the method's arithmetic) against the workload recipes: sizes,
gas volumes, walls, parameters, the closed interface layer every generator
must produce (no liquid cell next to a gas cell), and determinism in the seed."""
import numpy as np
import pytest

from paper_1604_01632_gb300 import scenarios as S

# the 18 neighbour offsets of D3Q19 (faces and edges)
OFFS = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
        if 0 < abs(dx) + abs(dy) + abs(dz) <= 2]


def _liquid_touches_gas(flags: np.ndarray) -> int:
    """Liquid cells with a gas cell among their 18 neighbours (periodic wrap)."""
    gas = flags == S.GAS
    near = np.zeros_like(gas)
    for dx, dy, dz in OFFS:
        near |= np.roll(gas, shift=(dz, dy, dx), axis=(0, 1, 2))
    return int(np.count_nonzero(near & (flags == S.LIQUID)))


def _gas_volume(sc) -> float:
    """Gas cells count 1, interface cells 1 - fill level."""
    g = sc.flags == S.GAS
    i = sc.flags == S.INTERFACE
    return float(np.count_nonzero(g) + np.sum(1.0 - sc.fill[i]))


def test_static_bubble_recipe():
    sc = S.static_bubble()
    assert (sc.nx, sc.ny, sc.nz) == (32, 32, 32)
    assert sc.collision == S.BGK and sc.tau == 0.8 and sc.sigma == 1e-3
    assert not np.any(sc.flags == S.OBSTACLE)          # periodic box
    assert _gas_volume(sc) == pytest.approx(4.0 / 3.0 * np.pi * 8.0 ** 3, rel=1e-2)
    assert _liquid_touches_gas(sc.flags) == 0


def test_gas_thread_recipe():
    sc = S.gas_thread()
    assert (sc.nx, sc.ny, sc.nz) == (256, 64, 64)
    assert sc.collision == S.TRT and sc.sigma == 5e-3
    obs = sc.flags == S.OBSTACLE
    # walls on the four sides parallel to x, none across x (periodic there)
    assert obs[:, 0, :].all() and obs[:, -1, :].all() and obs[0, :, :].all() and obs[-1, :, :].all()
    assert not obs[1:-1, 1:-1, :].any()
    # R(x) = 8 (1 + 0.1 sin(2 pi x / 64)): mean cross-section pi 64 (1 + 0.01 / 2)
    want = np.pi * 64.0 * (1.0 + 0.005) * 256
    assert _gas_volume(sc) == pytest.approx(want, rel=1e-2)
    assert _liquid_touches_gas(sc.flags) == 0


def test_orifice_recipe_reduced():
    sc = S.orifice(nx=32, ny=32, nz=48, plate_z=4, hole_radius=3.0, depth=30, cap_radius=3.0,
                   reservoir=500.0, drain=0.05, gravity=1e-4, sigma=2e-3)
    obs = sc.flags == S.OBSTACLE
    plate = obs[4, 1:-1, 1:-1]
    assert plate.mean() > 0.9 and not obs[4, 16, 16]     # a plate with a hole at its centre
    assert sc.gravity == (0.0, 0.0, -1e-4)
    (seed, extra, drain, constp), (atm, _, _, constp2) = sc.sources
    assert (extra, drain, constp, constp2) == (500.0, 0.05, 0, 1)
    assert sc.flags.reshape(-1)[seed] in (S.GAS, S.INTERFACE)
    assert sc.flags.reshape(-1)[atm] in (S.GAS, S.INTERFACE)
    liq = sc.flags == S.LIQUID
    z = np.nonzero(liq)[0]
    # hydrostatic: denser at the bottom of the liquid than at its top
    assert sc.rho[liq][z == z.min()].mean() > sc.rho[liq][z == z.max()].mean()
    assert _liquid_touches_gas(sc.flags) == 0


def test_bubble_population_recipe():
    scs = S.bubble_population(n_domains=6, seed=0)
    assert len(scs) == 6
    for sc in scs:
        assert {sc.nx, sc.ny, sc.nz} <= {32, 48, 64, 96}
        assert 1e-3 <= sc.sigma <= 5e-3 and sc.collision == S.TRT
        assert np.abs(sc.u).max() <= 0.02 + 1e-12
        assert np.count_nonzero(sc.flags == S.GAS) > 0
        assert _liquid_touches_gas(sc.flags) == 0


def test_foam_recipe_reduced():
    sc = S.foam(n=40, gas_fraction=0.3, seed=1, max_attempts=20000)
    obs = sc.flags == S.OBSTACLE
    assert obs[0].all() and not obs[1:].any()             # no-slip bottom only
    assert sc.lid == (0.05, 0.0, 0.0)
    assert _gas_volume(sc) / sc.n > 0.1
    assert _liquid_touches_gas(sc.flags) == 0


def test_generators_are_deterministic_in_the_seed():
    a = S.random_bubbles(24, 20, 16, n_bubbles=6, r_min=2.5, r_max=4.5, u_max=0.06, sigma=5e-3, seed=3)
    b = S.random_bubbles(24, 20, 16, n_bubbles=6, r_min=2.5, r_max=4.5, u_max=0.06, sigma=5e-3, seed=3)
    c = S.random_bubbles(24, 20, 16, n_bubbles=6, r_min=2.5, r_max=4.5, u_max=0.06, sigma=5e-3, seed=4)
    assert np.array_equal(a.flags, b.flags) and np.array_equal(a.fill, b.fill) and np.array_equal(a.u, b.u)
    assert not np.array_equal(a.flags, c.flags)


def test_thread_rupture_recipe():
    """Paper Sec. 3.1: 360 x 40 x 40 with a centred 336 x 8 x 8 gas block, walls on
    all faces; the lattice units follow from dx, rho, sigma and the assumed dt."""
    sc = S.thread_rupture(0.072)
    assert (sc.nx, sc.ny, sc.nz) == (360, 40, 40)
    f = sc.flags
    assert (f == S.GAS).sum() == 336 * 8 * 8
    gas = np.argwhere(f == S.GAS)
    assert gas.min(0).tolist() == [16, 16, 12] and gas.max(0).tolist() == [23, 23, 347]
    for ax in range(3):
        assert (np.take(f, 0, axis=ax) == S.OBSTACLE).all() and (np.take(f, -1, axis=ax) == S.OBSTACLE).all()
    assert _liquid_touches_gas(f) == 0
    assert (sc.fill[f == S.INTERFACE] == 1.0).all()
    # sigma dt^2 / (rho dx^3) and tau = 3 nu dt / dx^2 + 1/2 by hand for dt = 5e-7 s
    u = S.rupture_units(0.072, tau=None)
    assert u["sigma_lb"] == pytest.approx(0.072 * 2.5e-13 / (1000.0 * 1.953125e-15), rel=1e-12)
    assert u["tau"] == pytest.approx(0.5 + 3.0 * 1e-6 * 5e-7 / 1.5625e-10, rel=1e-12)
    assert sc.tau == 0.8 and sc.units["nu_si"] == pytest.approx(0.1 * 1.5625e-10 / 5e-7, rel=1e-12)
    assert S.thread_rupture(0.018).sigma == pytest.approx(sc.sigma / 4.0, rel=1e-12)
    assert sc.steps == 648000
