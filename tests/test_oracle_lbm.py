"""Pins of the oracle's lattice Boltzmann core (paper Sec. 2.1) against facts
fixed by the mathematics: lattice isotropy, moments of the equilibrium (Eqs.
3-5), conservation and relaxation rates of the collision (Eq. 6), Guo's force
moments, the exact Poiseuille profile of TRT with Lambda = 3/16, and the decay
rate of a shear wave (viscosity (tau - 1/2)/3)."""
import itertools

import numpy as np
import pytest

from paper_1604_01632_gb300 import scenarios as S


def test_d3q19_isotropy(oracle_mod):
    c, w, opp = oracle_mod.lattice()
    c = c.astype(np.float64)
    assert len({tuple(v) for v in c}) == 19
    norms = (c * c).sum(1)
    assert sorted(norms.tolist()) == [0] + [1] * 6 + [2] * 12
    assert np.all(c[opp] == -c)
    assert np.all(opp[opp] == np.arange(19))
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.abs((w[:, None] * c).sum(0)).max() < 1e-16
    second = np.einsum("a,ai,aj->ij", w, c, c)
    assert np.abs(second - np.eye(3) / 3.0).max() < 1e-15
    third = np.einsum("a,ai,aj,ak->ijk", w, c, c, c)
    assert np.abs(third).max() < 1e-16
    fourth = np.einsum("a,ai,aj,ak,al->ijkl", w, c, c, c, c)
    d = np.eye(3)
    iso = (np.einsum("ij,kl->ijkl", d, d) + np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)) / 9.0
    assert np.abs(fourth - iso).max() < 1e-15


def test_equilibrium_moments(oracle_mod):
    c, w, _ = oracle_mod.lattice()
    c = c.astype(np.float64)
    rng = np.random.default_rng(1)
    for _ in range(50):
        rho = rng.uniform(0.8, 1.2)
        u = rng.uniform(-0.1, 0.1, 3)
        f = oracle_mod.feq(rho, u)
        assert abs(f.sum() - rho) < 1e-14
        assert np.abs(c.T @ f - rho * u).max() < 1e-15
        pi = np.einsum("a,ai,aj->ij", f, c, c)
        assert np.abs(pi - (rho / 3.0 * np.eye(3) + rho * np.outer(u, u))).max() < 1e-14
    # at rest the equilibrium is the weights times rho
    assert np.abs(oracle_mod.feq(1.3, np.zeros(3)) - 1.3 * w).max() < 1e-16


@pytest.mark.parametrize("collision", [S.BGK, S.TRT])
def test_collision_invariants(oracle_mod, collision):
    c, w, opp = oracle_mod.lattice()
    c = c.astype(np.float64)
    rng = np.random.default_rng(2)
    tau = 0.7
    for _ in range(20):
        rho = rng.uniform(0.9, 1.1)
        u = rng.uniform(-0.05, 0.05, 3)
        fe = oracle_mod.feq(rho, u)
        # equilibrium is a fixed point
        out, r = oracle_mod.collide(fe, collision=collision, tau=tau)
        assert abs(r - rho) < 1e-14
        assert np.abs(out - fe).max() < 1e-15
        # mass and momentum conserved for an arbitrary state
        fin = fe + rng.normal(0.0, 1e-3, 19)
        out, _ = oracle_mod.collide(fin, collision=collision, tau=tau)
        assert abs(out.sum() - fin.sum()) < 1e-14
        assert np.abs(c.T @ out - c.T @ fin).max() < 1e-15


def test_relaxation_rates(oracle_mod):
    """A non-equilibrium part with zero mass and momentum relaxes by (1 - omega+) in
    its even part and by (1 - omega-) in its odd part; BGK is omega- = omega+."""
    c, w, opp = oracle_mod.lattice()
    c = c.astype(np.float64)
    tau, lam = 0.9, 3.0 / 16.0
    om_p = 1.0 / tau
    om_m = 1.0 / (lam / (tau - 0.5) + 0.5)
    rng = np.random.default_rng(3)
    rho, u = 1.0, np.array([0.02, -0.01, 0.03])
    fe = oracle_mod.feq(rho, u)
    # project a random vector onto the complement of {1, c_x, c_y, c_z}
    basis = np.stack([np.ones(19), c[:, 0], c[:, 1], c[:, 2]], 1)
    q, _ = np.linalg.qr(basis)
    d = rng.normal(0.0, 1e-3, 19)
    d -= q @ (q.T @ d)
    even = 0.5 * (d + d[opp])
    odd = 0.5 * (d - d[opp])
    out, _ = oracle_mod.collide(fe + d, collision=S.TRT, tau=tau, magic=lam)
    expect = fe + (1.0 - om_p) * even + (1.0 - om_m) * odd
    assert np.abs(out - expect).max() < 1e-15
    out_b, _ = oracle_mod.collide(fe + d, collision=S.BGK, tau=tau)
    assert np.abs(out_b - (fe + (1.0 - om_p) * d)).max() < 1e-15
    # TRT whose magic parameter gives omega- = omega+ is BGK
    out_t, _ = oracle_mod.collide(fe + d, collision=S.TRT, tau=tau, magic=(tau - 0.5) ** 2)
    assert np.abs(out_t - out_b).max() < 1e-15


@pytest.mark.parametrize("collision", [S.BGK, S.TRT])
def test_guo_force_moments(oracle_mod, collision):
    """Guo forcing adds exactly the force to the momentum and nothing to the mass."""
    c, _, _ = oracle_mod.lattice()
    c = c.astype(np.float64)
    rng = np.random.default_rng(4)
    g = np.array([1e-4, -2e-4, 3e-5])
    for _ in range(10):
        rho = rng.uniform(0.95, 1.05)
        fin = oracle_mod.feq(rho, rng.uniform(-0.05, 0.05, 3)) + rng.normal(0.0, 1e-4, 19)
        out, r = oracle_mod.collide(fin, collision=collision, tau=0.8, gravity=tuple(g))
        assert abs(out.sum() - fin.sum()) < 1e-14
        assert np.abs(c.T @ out - (c.T @ fin + r * g)).max() < 1e-15


def _channel(oracle_mod, H, tau, g, collision, magic, steps):
    nx, nz = 2, 2
    ny = H + 2
    flags = np.zeros((nz, ny, nx), dtype=np.uint8)
    flags[:, 0, :] = S.OBSTACLE
    flags[:, ny - 1, :] = S.OBSTACLE
    fill = np.where(flags == 0, 1.0, 0.0)
    o = oracle_mod.Oracle(nx=nx, ny=ny, nz=nz, collision=collision, tau=tau, magic=magic,
                          gravity=(g, 0.0, 0.0))
    assert o.init(flags, fill, np.ones(flags.shape), np.zeros((3,) + flags.shape)) == 0
    o.step(steps)
    f = o.f()
    c, _, _ = oracle_mod.lattice()
    rho = f.sum(0)
    jx = c[:, 0].astype(np.float64) @ f
    # stored PDFs are post-collision: u = (j_post - F/2) / rho
    ux = (jx - 0.5 * rho * g) / rho
    ux = ux.reshape(nz, ny, nx)[0, 1:ny - 1, 0]
    yy = np.arange(1, ny - 1, dtype=np.float64)
    nu = (tau - 0.5) / 3.0
    # walls half-way between the wall cells and the first fluid cells
    exact = g / (2.0 * nu) * (yy - 0.5) * (H + 0.5 - yy)
    return ux, exact


def test_poiseuille_trt_exact(oracle_mod):
    """Force-driven channel, TRT with Lambda = 3/16 and half-way bounce-back: the
    parabolic profile is reproduced to round-off."""
    ux, exact = _channel(oracle_mod, H=8, tau=0.8, g=1e-5, collision=S.TRT, magic=3.0 / 16.0, steps=6000)
    assert np.abs(ux - exact).max() / exact.max() < 1e-9


def test_poiseuille_bgk_second_order(oracle_mod):
    ux, exact = _channel(oracle_mod, H=16, tau=0.8, g=1e-6, collision=S.BGK, magic=0.0, steps=16000)
    assert np.abs(ux - exact).max() / exact.max() < 2e-2


def test_shear_wave_viscosity(oracle_mod):
    """u_x = A sin(2 pi y / L) decays as exp(-nu k^2 t) with nu = (tau - 1/2)/3."""
    L, tau, A, steps = 32, 0.8, 1e-4, 200
    nx, nz = 2, 2
    shape = (nz, L, nx)
    y = (np.arange(L) + 0.0)
    u = np.zeros((3,) + shape)
    u[0] = A * np.sin(2 * np.pi * y / L)[None, :, None]
    o = oracle_mod.Oracle(nx=nx, ny=L, nz=nz, collision=S.BGK, tau=tau)
    assert o.init(np.zeros(shape, np.uint8), np.ones(shape), np.ones(shape), u) == 0
    o.step(steps)
    c, _, _ = oracle_mod.lattice()
    f = o.f()
    ux = (c[:, 0].astype(np.float64) @ f / f.sum(0)).reshape(shape)[0, :, 0]
    amp = 2.0 / L * (ux * np.sin(2 * np.pi * y / L)).sum()
    nu = (tau - 0.5) / 3.0
    k = 2 * np.pi / L
    expect = A * np.exp(-nu * k * k * steps)
    # second-order lattice effects and the start-up from f = f_eq stay well below 1 %;
    # nu = tau/3 or a missing factor would be off by tens of percent
    assert abs(amp / expect - 1.0) < 1e-2


def test_uniform_flow_is_steady(oracle_mod):
    shape = (4, 5, 6)
    u = np.zeros((3,) + shape)
    u[0], u[1], u[2] = 0.03, -0.02, 0.01
    o = oracle_mod.Oracle(nx=6, ny=5, nz=4, collision=S.TRT, tau=0.6)
    assert o.init(np.zeros(shape, np.uint8), np.ones(shape), np.ones(shape), u) == 0
    f0 = o.f()
    o.step(20)
    assert np.abs(o.f() - f0).max() < 1e-15
