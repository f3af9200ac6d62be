"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on
the same seeded inputs.  FP64 storage: cell types and bubble ids bit-identical,
PDFs, mass and fill level within 1e-12, bubble table V and V* identical in
fixed point.  Reduced-precision storage: stated tolerances."""
import numpy as np
import pytest

from paper_1604_01632_gb300 import scenarios as S

from parity_util import compare_exact, gpu_state, macro, oracle_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fsl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_01632_gb300 import build, fsl as F
    build.build()
    return F


def _pair(fsl, oracle_mod, sc, precision="fp64"):
    sim = fsl.Simulation.from_scenarios([sc], precision=precision)
    o = oracle_mod.Oracle.from_scenario(sc)
    return sim, o


def _run_compare(fsl, oracle_mod, sc, checkpoints, what):
    sim, o = _pair(fsl, oracle_mod, sc)
    compare_exact(gpu_state(sim), oracle_state(o), what=f"{what} init")
    done = 0
    for k in checkpoints:
        sim.step(k - done)
        o.step(k - done)
        done = k
        compare_exact(gpu_state(sim), oracle_state(o), what=f"{what} step {k}")
    sim.sync()
    assert o.status == 0
    return sim, o


def test_static_bubble_fp64_bitexact(fsl, oracle_mod):
    """32^3 periodic box, bubble R = 8, sigma = 1e-3, BGK tau = 0.8, 200 steps."""
    sc = S.static_bubble()
    _run_compare(fsl, oracle_mod, sc, [1, 2, 3, 50, 200], "static bubble")


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_bubbles_with_conversions(fsl, oracle_mod, seed):
    """Moving liquid with several bubbles: conversions every step, merges and
    splits; state compared after every step for the first 10, then sparser."""
    sc = S.random_bubbles(24, 20, 16, n_bubbles=6, r_min=2.5, r_max=4.5, u_max=0.06, sigma=5e-3, seed=seed)
    _run_compare(fsl, oracle_mod, sc, list(range(1, 11)) + [20, 40, 80], f"random bubbles {seed}")


def test_thread_breakup_split(fsl, oracle_mod):
    sc = S.gas_thread(nx=48, ny=20, nz=20, radius=3.0, amp=0.25, wavelength=24, sigma=0.05, steps=0)
    sim, o = _run_compare(fsl, oracle_mod, sc, [50, 80, 85, 88, 89, 90, 92, 100, 150], "thread breakup")
    assert len(o.bubbles()) == 2


def test_buoyant_merge(fsl, oracle_mod):
    nx, ny, nz, g = 16, 16, 32, 5e-4
    shape = (nz, ny, nx)
    cen = np.array([[8.0, 8.0, 24.5], [8.0, 8.0, 13.5]])
    fill = S.liquid_fraction(shape, S._spheres_sdf(cen, np.array([4.0, 4.0])))
    flags = S.classify(fill, obstacle=S._wall_shell(shape, axes=(2,)))
    x, y, z = S._centres(shape)
    sc = S._finish("merge", flags, fill, rho=1.0 + 3.0 * g * (nz - 1 - z), collision=S.TRT, sigma=0.002,
                   gravity=(0.0, 0.0, -g))
    sim, o = _run_compare(fsl, oracle_mod, sc, [100, 200, 240, 245, 246, 247, 248, 250, 300], "buoyant merge")
    assert len(o.bubbles()) == 1


def test_droplet_in_atmosphere_and_reservoir(fsl, oracle_mod):
    n, R = 24, 6.0
    fill = S.liquid_fraction((n, n, n), lambda x, y, z: R - np.sqrt((x - 12) ** 2 + (y - 12) ** 2 + (z - 12) ** 2))
    sc = S._finish("drop", S.classify(fill), fill, sigma=2e-3, collision=S.TRT, sources=[(0, 0.0, 0.0, 1)])
    _run_compare(fsl, oracle_mod, sc, [1, 10, 60], "droplet")
    sc2 = S.static_bubble(n=24, radius=5.0, sigma=2e-3)
    sc2.sources = [(sc2.linear(12, 12, 12), 100.0, 0.5, 0)]
    _run_compare(fsl, oracle_mod, sc2, [1, 10, 60], "reservoir")


def test_gravity_lid_and_ragged_sizes(fsl, oracle_mod):
    """Odd domain sizes (not a multiple of the 256-cell block), gravity, a moving lid."""
    nx, ny, nz = 13, 11, 17
    shape = (nz, ny, nx)
    fill = S.liquid_fraction(shape, S._spheres_sdf(np.array([[6.5, 5.5, 7.0]]), np.array([3.2])))
    obs = np.zeros(shape, bool)
    obs[0] = True
    lid = np.zeros(shape, bool)
    lid[nz - 1] = True
    flags = S.classify(fill, obstacle=obs, lid=lid)
    sc = S._finish("lid", flags, fill, collision=S.TRT, sigma=3e-3, gravity=(0.0, 0.0, -2e-5), lid=(0.05, 0.0, 0.0))
    _run_compare(fsl, oracle_mod, sc, [1, 5, 30, 120], "lid")


def test_batched_domains_match_separate_oracles(fsl, oracle_mod):
    scs = [S.random_bubbles(20, 16, 12, n_bubbles=3, r_min=2.5, r_max=4.0, u_max=0.05, sigma=4e-3, seed=s)
           for s in range(3)]
    scs.append(S.static_bubble(n=16, radius=4.0))
    sim = fsl.Simulation.from_scenarios(scs, precision="fp64")
    oras = [oracle_mod.Oracle.from_scenario(s) for s in scs]
    prev = 0
    for k in (1, 7, 40):
        sim.step(k - prev)
        for o in oras:
            o.step(k - prev)
        prev = k
        for d, o in enumerate(oras):
            compare_exact(gpu_state(sim, d), oracle_state(o), what=f"domain {d} step {k}")


def test_full_size_gas_thread_sampled(fsl, oracle_mod):
    """The full 256x64x64 gas-thread lattice (the benchmark workload) for a few
    steps in FP64: identical to the oracle."""
    sc = S.gas_thread()
    _run_compare(fsl, oracle_mod, sc, [1, 3], "gas thread 256x64x64")


def test_geometry_error_is_reported(fsl):
    sc = S.static_bubble(n=16, radius=4.0)
    bad = sc.flags.copy().reshape(-1)
    # a liquid cell next to a gas cell breaks the closed interface layer
    gas = np.nonzero(bad == S.GAS)[0][0]
    itf = np.nonzero(bad == S.INTERFACE)[0]
    bad[itf] = S.LIQUID
    sim = fsl.Simulation([sc.params()], precision="fp64")
    with pytest.raises(fsl.FslError) as e:
        sim.init_geometry(0, bad, sc.fill, sc.rho, sc.u)
    assert e.value.status == -2
    assert gas >= 0


# FP32 stores f itself (values ~w_a), so each step rounds at ~1e-8 and the
# density drifts by a few 1e-6 over 200 steps; the shifted 16-bit forms store
# only f_a - w_a and round that small deviation instead
@pytest.mark.parametrize("precision,tol_u,tol_rho,tol_v", [("fp32", 3e-5, 3e-5, 1e-4), ("f16s", 2e-4, 2e-4, 1e-3),
                                                            ("bf16s", 2e-3, 2e-3, 1e-2)])
def test_reduced_precision_static_bubble(fsl, oracle_mod, precision, tol_u, tol_rho, tol_v):
    """FP32 collide with FP32 / FP16-shifted / BF16-shifted storage against the FP64
    oracle on the static bubble (200 steps): L-infinity errors of rho and u on fluid
    cells and the relative error of the bubble volume."""
    sc = S.static_bubble()
    sim, o = _pair(fsl, oracle_mod, sc, precision)
    sim.step(200)
    o.step(200)
    g, r = gpu_state(sim), oracle_state(o)
    fl = np.isin(r["flags"], (S.LIQUID, S.INTERFACE)) & np.isin(g["flags"], (S.LIQUID, S.INTERFACE))
    rg, ug = macro(g["f"][:, fl])
    rr, ur = macro(r["f"][:, fl])
    print(f"{precision}: |drho| {np.abs(rg - rr).max():.3e} |du| {np.abs(ug - ur).max():.3e} "
          f"dV/V {abs(g['bubbles']['volume'][0] / r['bubbles']['volume'][0] - 1.0):.3e} "
          f"flag agreement {(g['flags'] == r['flags']).mean():.6f}")
    assert np.abs(rg - rr).max() < tol_rho
    assert np.abs(ug - ur).max() < tol_u
    assert len(g["bubbles"]) == len(r["bubbles"]) == 1
    assert abs(g["bubbles"]["volume"][0] / r["bubbles"]["volume"][0] - 1.0) < tol_v
    assert (g["flags"] == r["flags"]).mean() > 0.999


@pytest.mark.parametrize("form", [-1, 5])
def test_batched_bubble_population_parity(fsl, oracle_mod, form):
    """Three domains of the bubble-population workload (axes from {32, 48}) in one
    handle against three oracles: the tuned stream-collide form, and the
    two-kernel form, whose normals pass takes the batch through its tile table
    (every domain holds a whole 32 x 8 x 8 tile)."""
    scs = S.bubble_population(n_domains=3, seed=5, sides=(32, 48))
    sim = fsl.Simulation.from_scenarios(scs, precision="fp64")
    if form >= 0:
        sim.set_stream_form(form)
    oras = [oracle_mod.Oracle.from_scenario(s) for s in scs]
    prev = 0
    for k in (1, 6):
        sim.step(k - prev)
        for o in oras:
            o.step(k - prev)
        prev = k
        for d, o in enumerate(oras):
            compare_exact(gpu_state(sim, d), oracle_state(o), what=f"population domain {d} step {k}")


def test_orifice_reduced_parity(fsl, oracle_mod):
    """Orifice workload at reduced size: walls, plate with a hole, gravity,
    draining reservoir below, constant-pressure atmosphere above."""
    sc = S.orifice(nx=32, ny=32, nz=48, plate_z=4, hole_radius=3.0, depth=30, cap_radius=3.0, reservoir=500.0,
                   drain=0.05, gravity=1e-4, sigma=2e-3)
    _run_compare(fsl, oracle_mod, sc, [1, 10, 40], "orifice 32x32x48")


def test_foam_reduced_parity(fsl, oracle_mod):
    """Foam workload at reduced size: lognormal bubbles, moving lid, gravity."""
    sc = S.foam(n=40, gas_fraction=0.3, seed=1, max_attempts=20000)
    _run_compare(fsl, oracle_mod, sc, [1, 10, 30], "foam 40^3")


def test_nan_density_is_reported(fsl):
    sc = S.static_bubble(n=16, radius=4.0)
    rho = sc.rho.copy()
    liq = np.argwhere(sc.flags == S.LIQUID)[0]
    rho[tuple(liq)] = np.nan
    sim = fsl.Simulation([sc.params()], precision="fp64")
    sim.init_geometry(0, sc.flags, sc.fill, rho, sc.u)
    sim.step(1)
    with pytest.raises(fsl.FslError) as e:
        sim.sync()
    assert e.value.status == -4


@pytest.mark.parametrize("precision", ["fp32", "f16s", "bf16s"])
def test_reduced_precision_thread_breakup(fsl, oracle_mod, precision):
    """Dynamic topology in reduced precision: the small perturbed gas thread breaks
    into the same two bubbles within a few steps of the FP64 oracle, with the
    bubble volumes within 1 %."""
    sc = S.gas_thread(nx=48, ny=20, nz=20, radius=3.0, amp=0.25, wavelength=24, sigma=0.05, steps=0)
    o = oracle_mod.Oracle.from_scenario(sc)
    sim = fsl.Simulation.from_scenarios([sc], precision=precision)
    t_o = t_g = None
    for k in range(1, 131):
        o.step(1)
        sim.step(1)
        if t_o is None and len(o.bubbles()) > 1:
            t_o = k
        if t_g is None and len(sim.bubbles()) > 1:
            t_g = k
    assert t_o is not None and t_g is not None
    print(f"{precision}: breakup step gpu {t_g} oracle {t_o}")
    assert abs(t_g - t_o) <= 5
    gb, ob = sim.bubbles(), o.bubbles()
    assert len(gb) == len(ob) == 2
    assert np.allclose(np.sort(gb["volume"]), np.sort(ob["volume"]), rtol=1e-2)


def test_rayleigh_plateau_gas_thread_full_size(fsl):
    """Physics check on the full gas-thread lattice (256x64x64, four wavelengths of
    a radius perturbation of half the radius, k R = 2 pi 8 / 64 < 1 is unstable):
    the thread pinches into four equal bubbles.  (With the 10 % perturbation of
    the benchmark workload the thread stays whole at this resolution: the
    digitised curvature scatters by about 0.02 per cell against a 0.012 signal.)"""
    sc = S.gas_thread(amp=0.5)
    sim = fsl.Simulation.from_scenarios([sc], precision="fp32")
    n0 = len(sim.bubbles())
    sim.step(3000)
    sim.sync()
    b = sim.bubbles()
    print(f"bubbles: {n0} -> {len(b)}, labelling runs {sim.labelling_runs}, volumes {np.round(b['volume'], 1)}")
    assert n0 == 1
    assert len(b) == 4
    assert np.allclose(b["volume"], b["volume"].mean(), rtol=1e-3)


def test_accuracy_report_reduced_forms(fsl, oracle_mod):
    """The accuracy figures of the FP32-collide forms against the FP64 oracle on a
    gas thread of the benchmark's shape at a quarter of its size (128x32x32,
    R = 4(1 + 0.1 sin(2 pi x/32)), sigma = 5e-3, TRT), 300 steps: relative L2 and
    L-infinity errors of the pressure p = rho/3 and of the velocity on cells that
    are fluid on both sides, the worst per-bubble relative volume error, the
    relative drift of the total liquid mass against the oracle's, and the bubble
    counts.  Printed as one line per storage form; the asserts are loose bounds
    (the figures themselves go to the design notes)."""
    import json
    sc = S.gas_thread(nx=128, ny=32, nz=32, radius=4.0, wavelength=32.0)
    o = oracle_mod.Oracle.from_scenario(sc)
    m0 = o.total_mass()
    o.step(300)
    r = oracle_state(o)
    mo = o.total_mass()
    rr, ur = macro(r["f"])
    for precision in ("fp32", "f16s", "bf16s"):
        sim = fsl.Simulation.from_scenarios([sc], precision=precision)
        sim.step(300)
        g = gpu_state(sim)
        fl = np.isin(r["flags"], (S.LIQUID, S.INTERFACE)) & np.isin(g["flags"], (S.LIQUID, S.INTERFACE))
        rg, ug = macro(g["f"])
        pg, pr = rg[fl] / 3.0, rr[fl] / 3.0
        du = ug[:, fl] - ur[:, fl]
        umax = np.abs(ur[:, fl]).max()
        lm = np.isin(g["flags"], (S.LIQUID,))
        mg = float(rg[lm].sum() + g["mass"][g["flags"] == S.INTERFACE].sum())
        gb, rb = g["bubbles"], r["bubbles"]
        dv = 0.0
        if len(gb) == len(rb):
            dv = float(np.max(np.abs(np.sort(gb["volume"]) / np.sort(rb["volume"]) - 1.0)))
        rep = {"storage": precision,
               "p_rel_l2": float(np.linalg.norm(pg - pr) / np.linalg.norm(pr)),
               "p_rel_linf": float(np.abs(pg - pr).max() / np.abs(pr).max()),
               "u_rel_l2": float(np.linalg.norm(du) / max(np.linalg.norm(ur[:, fl]), 1e-300)),
               "u_linf_over_umax": float(np.abs(du).max() / max(umax, 1e-300)),
               "bubble_volume_rel_max": dv,
               "mass_drift_vs_oracle": float((mg - mo) / mo),
               "oracle_mass_drift": float((mo - m0) / m0),
               "bubbles_gpu": int(len(gb)), "bubbles_oracle": int(len(rb)),
               "flag_agreement": float((g["flags"] == r["flags"]).mean())}
        print("ACCURACY " + json.dumps(rep))
        assert rep["bubbles_gpu"] == rep["bubbles_oracle"]
        assert rep["p_rel_linf"] < 1e-2
        assert rep["bubble_volume_rel_max"] < 2e-2
        assert abs(rep["mass_drift_vs_oracle"]) < 1e-2
        sim.close()


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-13), ("fp32", 1e-5), ("f16s", 1e-5)])
def test_total_mass_against_oracle(fsl, oracle_mod, precision, rtol):
    """fsl_total_mass (rho over liquid cells + m over interface cells + pool,
    summed on the device in a fixed order) against the oracle's liquid mass on
    moving bubbles with conversions, after 0 and 40 steps; the FP64 path
    differs only by summation order, the FP32-collide forms by their rounding.
    Summed twice, the value is the same bit for bit."""
    sc = S.random_bubbles(24, 20, 16, n_bubbles=6, r_min=2.5, r_max=4.5, u_max=0.06, sigma=5e-3, seed=1)
    sim, o = _pair(fsl, oracle_mod, sc, precision)
    for k in (0, 40):
        if k:
            sim.step(k)
            o.step(k)
        got, want = sim.total_mass(), o.total_mass()
        assert got == sim.total_mass()
        assert abs(got / want - 1.0) < rtol, (k, got, want)
    sim.close()


@pytest.mark.parametrize("form", [1, 2, 3, 5, 8])
def test_persistent_stream_forms_bitexact(fsl, oracle_mod, form):
    """The persistent stream-collide forms (1, 2 or 4 tiles per liquid item,
    interface chunks interleaved) and the two-kernel forms (liquid kernel and
    one thread per interface cell, one after the other or side by side on two
    streams) give the oracle's state bit for bit: a batch
    of moving-bubble domains with conversions, merges and splits, and a single
    domain with a moving lid and gravity."""
    scs = [S.random_bubbles(24, 20, 16, n_bubbles=6, r_min=2.5, r_max=4.5, u_max=0.06, sigma=5e-3, seed=s)
           for s in (0, 1)]
    scs.append(S.static_bubble(n=16, radius=4.0))
    sim = fsl.Simulation.from_scenarios(scs, precision="fp64")
    sim.set_stream_form(form)
    assert sim.stream_form == form
    oras = [oracle_mod.Oracle.from_scenario(s) for s in scs]
    prev = 0
    for k in (1, 5, 30):
        sim.step(k - prev)
        for o in oras:
            o.step(k - prev)
        prev = k
        for d, o in enumerate(oras):
            compare_exact(gpu_state(sim, d), oracle_state(o), what=f"form {form} domain {d} step {k}")
    sim.close()
    sc = S.foam(n=40, gas_fraction=0.3, seed=1, max_attempts=20000)
    sim = fsl.Simulation.from_scenarios([sc], precision="fp64")
    sim.set_stream_form(form)
    o = oracle_mod.Oracle.from_scenario(sc)
    for k in (1, 10):
        sim.step(k if k == 1 else 9)
        o.step(k if k == 1 else 9)
        compare_exact(gpu_state(sim), oracle_state(o), what=f"form {form} foam step {k}")
    sim.close()


@pytest.mark.parametrize("form", [0, 1, 4, 5])
def test_cell_ordered_interface_list_bitexact(fsl, oracle_mod, form):
    """The interface list rebuilt in cell order after every conversion (two
    passes over the cell types inside the conversion kernel) changes only the
    order of the work: the oracle's state bit for bit, split, persistent and
    slab stream-collide forms."""
    scs = [S.random_bubbles(24, 20, 16, n_bubbles=6, r_min=2.5, r_max=4.5, u_max=0.06, sigma=5e-3, seed=s)
           for s in (2, 3)]
    sim = fsl.Simulation.from_scenarios(scs, precision="fp64")
    sim.set_interface_order(1)
    sim.set_stream_form(form)
    assert sim.interface_order == 1
    oras = [oracle_mod.Oracle.from_scenario(s) for s in scs]
    prev = 0
    for k in (1, 4, 25):
        sim.step(k - prev)
        for o in oras:
            o.step(k - prev)
        prev = k
        for d, o in enumerate(oras):
            compare_exact(gpu_state(sim, d), oracle_state(o), what=f"ordered list form {form} domain {d} step {k}")
    sim.close()


def _paper_trigger_cases():
    scs = [S.gas_thread(nx=48, ny=20, nz=20, radius=3.0, amp=0.25, wavelength=24, sigma=0.05, steps=0)]
    scs += [S.random_bubbles(24, 20, 16, n_bubbles=6, r_min=2.5, r_max=4.5, u_max=0.06, sigma=5e-3, seed=s)
            for s in (0, 1, 2)]
    scs += S.bubble_population(n_domains=2, seed=5, sides=(32, 48))
    return scs


def test_paper_split_trigger_against_exact_trigger_and_oracle(fsl, oracle_mod):
    """The paper's split trigger (anti-parallel normals around a cell that
    fills, Sec. 2.3.2) against the exact local test and the oracle (which
    labels every step), on the thread breakup, moving bubbles with merges and
    splits, and two bubble-population domains, over 120 steps.  The exact
    trigger must match the oracle everywhere.  For the paper's trigger the
    first checkpoint at which each domain departs from the oracle (a split it
    missed: ids and bubble table differ) is recorded and printed with the
    number of labelling passes of each trigger; the thread's pinch-off is a
    split the paper's criterion, as read here, does not catch."""
    import json
    scs = _paper_trigger_cases()
    exact = fsl.Simulation.from_scenarios(scs, precision="fp64")
    paper = fsl.Simulation.from_scenarios(scs, precision="fp64", split_trigger=1)
    oras = [oracle_mod.Oracle.from_scenario(s) for s in scs]
    first_miss = [None] * len(scs)
    prev = 0
    for k in (10, 40, 80, 90, 100, 120):
        for sim in (exact, paper):
            sim.step(k - prev)
        for o in oras:
            o.step(k - prev)
        prev = k
        for d, o in enumerate(oras):
            r = oracle_state(o)
            compare_exact(gpu_state(exact, d), r, what=f"exact trigger domain {d} step {k}")
            if first_miss[d] is None:
                try:
                    compare_exact(gpu_state(paper, d), r, what="")
                except AssertionError:
                    first_miss[d] = k
    rep = {"labelling_passes_exact": exact.labelling_runs, "labelling_passes_paper": paper.labelling_runs,
           "first_step_paper_trigger_departs": first_miss,
           "domains": ["thread breakup 48x20x20", "moving bubbles s0", "moving bubbles s1", "moving bubbles s2",
                       "population 0", "population 1"]}
    print("PAPER_TRIGGER " + json.dumps(rep))
    exact.close()
    paper.close()


@pytest.mark.parametrize("form", [6, 7])
@pytest.mark.parametrize("precision", ["fp32", "f16s"])
def test_tile_fused_forms_match_split_form(fsl, form, precision):
    """The tile-fused stream-collide forms (liquid cells, then the tile's
    interface cells one per thread) against the split form on moving bubbles
    and a small foam, 30 steps, FP32 and FP16-shifted storage.  Both run the
    same steps per cell; with FMA contraction in these forms the two code
    paths may round differently, so the states must agree within rounding:
    cell types on > 99.9 % of the cells, density and velocity relative L2
    below 1e-5 and 1e-3, the same bubble count, bubble volumes within 1e-5
    (the FP64 form of the shared one-thread-per-cell code is compared with the
    oracle bit for bit through form 5)."""
    scs = [S.random_bubbles(24, 20, 16, n_bubbles=6, r_min=2.5, r_max=4.5, u_max=0.06, sigma=5e-3, seed=1),
           S.foam(n=40, gas_fraction=0.3, seed=1, max_attempts=20000)]
    for sc in scs:
        ref = fsl.Simulation.from_scenarios([sc], precision=precision)
        ref.set_stream_form(0)
        sim = fsl.Simulation.from_scenarios([sc], precision=precision)
        sim.set_stream_form(form)
        ref.step(30)
        sim.step(30)
        a, b = gpu_state(ref), gpu_state(sim)
        assert (a["flags"] == b["flags"]).mean() > 0.999, sc.name
        fl = np.isin(a["flags"], FLUID_T) & np.isin(b["flags"], FLUID_T)
        ra, ua = macro(a["f"][:, fl])
        rb, ub = macro(b["f"][:, fl])
        assert np.linalg.norm(ra - rb) / np.linalg.norm(ra) < 1e-5, sc.name
        assert np.linalg.norm(ua - ub) / max(np.linalg.norm(ua), 1e-30) < 1e-3, sc.name
        assert len(a["bubbles"]) == len(b["bubbles"]), sc.name
        assert np.allclose(a["bubbles"]["volume"], b["bubbles"]["volume"], rtol=1e-5), sc.name
        ref.close()
        sim.close()


FLUID_T = (S.LIQUID, S.INTERFACE)
