"""The gas-thread workload (256x64x64, periodic in x, walls elsewhere, gas
cylinder R(x) = 8 (1 + 0.1 sin(2 pi x / 64)), sigma = 5e-3, TRT) in the forms
and over the horizons of its recipe:

  * the benchmark's own form (FP16-shifted storage, FP32 collision, CUDA
    graphs, tuned stream-collide form) on the full lattice, element-wise
    against the FP64 oracle (its OpenMP build) after 60 steps;
  * per-bubble volume and pressure against the oracle at a 400-step horizon,
    FP32 and FP16-shifted storage;
  * the recipe's full 20,000 steps in FP32 and FP16-shifted storage, with the
    bubble count and the liquid-mass drift reported.

At this resolution the 10 % perturbation does not pinch the thread within
20,000 steps; the test reports the final state rather than asserting a
breakup the recipe only expects (the full-size Rayleigh-Plateau breakup with a
larger perturbation is checked in test_parity_gpu.py)."""
import json

import numpy as np
import pytest

from paper_1604_01632_gb300 import scenarios as S

from parity_util import macro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fsl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_01632_gb300 import build, fsl as F
    build.build()
    return F


@pytest.fixture(scope="module")
def thread():
    return S.gas_thread()


def _oracle(oracle_mod, sc):
    try:
        return oracle_mod.Oracle.from_scenario(sc, openmp=True)
    except RuntimeError:
        return oracle_mod.Oracle.from_scenario(sc)


def test_benchmark_form_full_size_against_oracle(fsl, oracle_mod, thread):
    """FP16-shifted storage on the full lattice, 60 steps: cell types agree on
    more than 99.99 % of the cells; on cells fluid in both runs the density
    within relative L2 1e-5 and L-infinity 1e-4, the velocity within relative
    L2 5e-2 of a field whose maximum is ~1e-3 (spurious currents round a
    resting thread; measured 0.029); one bubble on both sides, volumes within
    1e-5."""
    sim = fsl.Simulation.from_scenarios([thread], precision="f16s")
    o = _oracle(oracle_mod, thread)
    sim.step(60)
    o.step(60)
    g = sim.fields(0, ("flags", "pdf"))
    rf = o.flags()
    assert (g["flags"] == rf).mean() > 0.9999
    fl = np.isin(rf, (S.LIQUID, S.INTERFACE)) & np.isin(g["flags"], (S.LIQUID, S.INTERFACE))
    rg, ug = macro(g["pdf"][:, fl])
    rr, ur = macro(o.f()[:, fl])
    rel_rho = np.linalg.norm(rg - rr) / np.linalg.norm(rr)
    inf_rho = np.abs(rg - rr).max() / np.abs(rr).max()
    rel_u = np.linalg.norm(ug - ur) / max(np.linalg.norm(ur), 1e-30)
    gb, ob = sim.bubbles(0), o.bubbles()
    print("FULLSIZE_F16S " + json.dumps({"rho_rel_l2": float(rel_rho), "rho_rel_linf": float(inf_rho),
                                         "u_rel_l2": float(rel_u), "u_max": float(np.abs(ur).max()),
                                         "flag_agreement": float((g["flags"] == rf).mean()),
                                         "bubbles": [len(gb), len(ob)]}))
    assert rel_rho < 1e-5 and inf_rho < 1e-4
    assert rel_u < 5e-2
    assert len(gb) == len(ob) == 1
    assert abs(gb["volume"][0] / ob["volume"][0] - 1.0) < 1e-5
    sim.close()


def test_bubble_volume_and_pressure_at_400_steps(fsl, oracle_mod, thread):
    o = _oracle(oracle_mod, thread)
    o.step(400)
    ob = o.bubbles()
    for precision in ("fp32", "f16s"):
        sim = fsl.Simulation.from_scenarios([thread], precision=precision)
        sim.step(400)
        gb = sim.bubbles(0)
        rep = {"storage": precision, "bubbles": [len(gb), len(ob)],
               "V_rel": [float(gb["volume"][k] / ob["volume"][k] - 1.0) for k in range(min(len(gb), len(ob)))],
               "p_rel": [float(gb["pressure"][k] / ob["pressure"][k] - 1.0) for k in range(min(len(gb), len(ob)))]}
        print("HORIZON400 " + json.dumps(rep))
        assert len(gb) == len(ob)
        # FP32 storage rounds f itself each step (measured 7.4e-6 in V and p)
        assert max(abs(v) for v in rep["V_rel"]) < 1e-4
        assert max(abs(v) for v in rep["p_rel"]) < 1e-4
        sim.close()


def test_recipe_horizon_20000_steps(fsl, thread):
    out = {}
    for precision in ("fp32", "f16s"):
        sim = fsl.Simulation.from_scenarios([thread], precision=precision)
        m0 = sim.total_mass()
        counts = []
        for _ in range(20):
            sim.step(1000)
            counts.append(len(sim.bubbles(0)))
        b = sim.bubbles(0)
        m1 = sim.total_mass()
        out[precision] = {"bubble_count_every_1000_steps": counts, "final_volumes": np.round(b["volume"], 2).tolist(),
                          "final_pressures": np.round(b["pressure"], 7).tolist(),
                          "mass_drift_rel": float((m1 - m0) / m0), "labelling_runs": sim.labelling_runs}
        sim.close()
        # FP32 storage: ~1e-8 per step, measured 2.3e-4 over the 20,000 steps
        assert abs((m1 - m0) / m0) < 1e-3
    print("HORIZON20000 " + json.dumps(out))
    assert out["fp32"]["bubble_count_every_1000_steps"][-1] == out["f16s"]["bubble_count_every_1000_steps"][-1]
