"""Pins of the oracle's cell conversion (paper Sec. 2.2, cell conversion), on
lattices small enough to work out one step without the oracle.

With BGK at tau = 1 (omega = 1) the post-collision PDFs of a cell are the
equilibrium of the moments of what streamed in, and from rest equilibria
f_a = w_a rho0 every incoming PDF is known in closed form: w_a rho0(x - c_a)
from a liquid or interface source, and, from a gas source with the gas density
3 p0 = 1 (Eqs. 8, 12-14 at V* = V, sigma = 0) and the cell's own velocity 0,
the reconstruction f_eq,a + f_eq,abar - f*_abar (Eq. 11) = 2 w_a - w_a rho0(x).
The tests build the expected post-step state from that alone (numpy), then
check the conversion rules the oracle reads into the paper:

  * a gas cell claimed by a filled neighbour becomes an interface cell with
    f = f_eq(mean rho, mean u) over its liquid and non-emptied interface
    neighbours (emptied ones excluded), starting from m = 0 (it then takes
    its share of the excess mass like any interface cell);
  * an interface cell without a gas neighbour fills, one without a liquid
    neighbour empties (the lonely-cell rule), and neither converts with the
    rule off.

A dropped division, a neighbour set that includes the gas or the emptied
cell, or a velocity left out of the equilibrium fails the first test."""
import numpy as np
import pytest

from paper_1604_01632_gb300 import scenarios as S

# D3Q19 velocities and weights in the documented order (written out here,
# independently of the oracle's tables)
C = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
              [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1], [1, 0, -1], [-1, 0, 1],
              [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]])
W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def feq(rho, u):
    """Second-order equilibrium w rho (1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u)."""
    cu = C @ u
    return W * rho * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * (u @ u))


def _layered(nx=8, ny=6, nz=8):
    """Liquid z = 0..2 and 7, interface layers z = 3 and 6, gas z = 4..5
    (every axis periodic); fill 0.5 on the interface layers."""
    flags = np.full((nz, ny, nx), S.LIQUID, np.uint8)
    flags[3] = flags[6] = S.INTERFACE
    flags[4:6] = S.GAS
    fill = np.where(flags == S.LIQUID, 1.0, np.where(flags == S.INTERFACE, 0.5, 0.0))
    return flags, fill


def _one_step_tau1(flags, rho0):
    """Post-collision PDFs after one step from f = w rho0, BGK tau = 1,
    gas density 1 and gas-side velocity 0: f*' = f_eq(rho', u') of the
    streamed-in PDFs (liquid and interface cells; NaN elsewhere)."""
    nz, ny, nx = flags.shape
    fin = np.zeros((19, nz, ny, nx))
    for a in range(19):
        src_rho = np.roll(rho0, shift=(C[a, 2], C[a, 1], C[a, 0]), axis=(0, 1, 2))     # rho0(x - c_a)
        src_gas = np.roll(flags == S.GAS, shift=(C[a, 2], C[a, 1], C[a, 0]), axis=(0, 1, 2))
        fin[a] = np.where(src_gas, 2 * W[a] - W[a] * rho0, W[a] * src_rho)
    rho = fin.sum(0)
    u = np.einsum("ad,azyx->dzyx", C.astype(float), fin) / rho
    out = np.full((19, nz, ny, nx), np.nan)
    fluid = (flags == S.LIQUID) | (flags == S.INTERFACE)
    for z, y, x in zip(*np.nonzero(fluid)):
        out[:, z, y, x] = feq(rho[z, y, x], u[:, z, y, x])
    return out, rho, u


def _oracle(oracle_mod, flags, fill, rho0, lonely=1):
    nz, ny, nx = flags.shape
    o = oracle_mod.Oracle(nx=nx, ny=ny, nz=nz, collision=S.BGK, tau=1.0, sigma=0.0, normal_rule=0,
                          lonely_rule=lonely)
    assert o.init(flags, fill, rho0, np.zeros((3,) + flags.shape)) == 0
    return o


def test_new_interface_cell_from_gas_takes_the_mean_of_its_eligible_neighbours(oracle_mod):
    flags, fill = _layered()
    nz, ny, nx = flags.shape
    rng = np.random.Generator(np.random.PCG64(7))
    rho0 = np.where(flags == S.GAS, 1.0, 1.0 + 0.02 * rng.uniform(-1, 1, flags.shape))
    F, E, G = (3, 2, 2), (3, 2, 4), (4, 2, 3)          # (z, y, x): filled, emptied, claimed gas
    fill[F] = 1.3                                       # m = 1.3 rho0 > (1 + eps) rho: filled
    fill[E] = -0.3                                      # m < -eps rho: emptied (not next to F)
    want_f, rho1, u1 = _one_step_tau1(flags, rho0)
    o = _oracle(oracle_mod, flags, fill, rho0)
    o.step(1)
    fl = o.flags().reshape(flags.shape)
    assert fl[F] == S.LIQUID and fl[E] == S.GAS and fl[G] == S.INTERFACE
    # G's liquid and interface neighbours at the start of the conversion:
    # (z=3) its cell below, F, and the two beside them; E (emptied, with no
    # filled neighbour to cancel the mark) does not count
    elig = [(3, 2, 3), F, (3, 1, 3), (3, 3, 3)]
    rbar = np.mean([rho1[c] for c in elig])
    ubar = np.mean([u1[(slice(None),) + c] for c in elig], axis=0)
    got = o.f().reshape((19,) + flags.shape)[(slice(None),) + G]
    np.testing.assert_allclose(got, feq(rbar, ubar), rtol=0, atol=1e-15)
    # and the expected state is not degenerate: E's or the gas's inclusion,
    # or no division, would move the density by far more than the tolerance
    wrong = np.mean([rho1[c] for c in elig + [E]])
    assert abs(wrong - rbar) > 1e-4 and np.abs(ubar).max() > 1e-4
    # the neighbours themselves follow the closed form (pins the model above)
    for c in elig:
        if c != F:
            np.testing.assert_allclose(o.f().reshape((19,) + flags.shape)[(slice(None),) + c],
                                       want_f[(slice(None),) + c], rtol=0, atol=1e-15)


@pytest.mark.parametrize("lonely", [1, 0])
def test_interface_cell_without_gas_neighbour_fills(oracle_mod, lonely):
    """One interface cell inside liquid (no gas neighbour), fill 0.5: with the
    rule it becomes liquid after one step; without it stays interface."""
    n = 6
    flags = np.full((n, n, n), S.LIQUID, np.uint8)
    flags[3, 3, 3] = S.INTERFACE
    fill = np.where(flags == S.LIQUID, 1.0, 0.5)
    o = _oracle(oracle_mod, flags, fill, np.ones(flags.shape), lonely)
    o.step(1)
    fl = o.flags().reshape(flags.shape)
    assert fl[3, 3, 3] == (S.LIQUID if lonely else S.INTERFACE)
    assert np.count_nonzero(fl == S.INTERFACE) == (0 if lonely else 1)


@pytest.mark.parametrize("lonely", [1, 0])
def test_interface_cell_without_liquid_neighbour_empties(oracle_mod, lonely):
    """One interface cell inside gas (no liquid neighbour), fill 0.5: with the
    rule it becomes gas after one step (its mass goes to the pool, as no
    interface neighbour is left to take it); without it stays interface."""
    n = 6
    flags = np.full((n, n, n), S.GAS, np.uint8)
    flags[2, 3, 1] = S.INTERFACE
    fill = np.where(flags == S.INTERFACE, 0.5, 0.0)
    o = _oracle(oracle_mod, flags, fill, np.ones(flags.shape), lonely)
    o.step(1)
    fl = o.flags().reshape(flags.shape)
    assert fl[2, 3, 1] == (S.GAS if lonely else S.INTERFACE)
    if lonely:
        assert o.pool_fx() * 2.0 ** -40 == pytest.approx(0.5, abs=1e-9)
        assert len(o.bubbles()) == 1
