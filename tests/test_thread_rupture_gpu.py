"""Rupture of a thin gas thread (paper Sec. 3.1): a 360 x 40 x 40 domain with a
rectangular gas block of 336 x 8 x 8 cells, surface tension 72 mN/m and
18 mN/m, dx = 1.25e-5 m, nu = 1e-6 m^2/s, rho = 1000 kg/m^3.

The paper gives no time step; the scenario assumes dt = 5e-7 s, which gives
sigma = 9.2e-3 (72 mN/m) or 2.3e-3 (18 mN/m) in lattice units.  With the
paper's viscosity the same dt gives tau = 0.5096, at which this TRT scheme
diverged (a NaN within the first 500 steps); the replay takes tau = 0.8, a
viscosity of 3.1e-5 m^2/s (31 times water's), and keeps the two surface
tensions and their ratio.  The paper's piece counts (5 and 6 bubbles after
324 ms) are context, not a pin: they depend on its unstated time step and
collision model.  The tests check what the method fixes here:

  * the FP64 path against the FP64 oracle on the full lattice, bit for bit in
    flags and bubble ids, over the first steps of the rupture run;
  * that the thread ruptures under both surface tensions (a NaN or any other
    device error raises from the syncing calls), with the bubble count
    recorded at the paper's frame times (22 ... 324 ms).
"""
import json

import numpy as np
import pytest

from paper_1604_01632_gb300 import scenarios as S

from parity_util import compare_exact, gpu_state, oracle_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fsl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_01632_gb300 import build, fsl as F
    build.build()
    return F


def _oracle(oracle_mod, sc):
    try:
        return oracle_mod.Oracle.from_scenario(sc, openmp=True)
    except RuntimeError:
        return oracle_mod.Oracle.from_scenario(sc)


@pytest.mark.parametrize("sigma_si", S.RUPTURE_SIGMAS)
def test_full_size_fp64_against_oracle(fsl, oracle_mod, sigma_si):
    sc = S.thread_rupture(sigma_si)
    sim = fsl.Simulation.from_scenarios([sc], precision="fp64")
    o = _oracle(oracle_mod, sc)
    done = 0
    for k in (1, 9, 30):
        sim.step(k)
        o.step(k)
        done += k
        compare_exact(gpu_state(sim), oracle_state(o), what=f"sigma {sigma_si} step {done}")
    sim.close()


def test_sigma_sweep_ruptures(fsl):
    out = {}
    for sigma_si in S.RUPTURE_SIGMAS:
        sc = S.thread_rupture(sigma_si)
        dt = sc.units["dt"]
        sim = fsl.Simulation.from_scenarios([sc], precision="fp32")
        b0 = sim.bubbles(0)
        frames, counts = S.RUPTURE_FRAMES_MS[sigma_si], []
        done, first_split = 0, None
        # to the first frame in coarse strides, recording the first split
        probe = 500
        for t_ms in frames:
            target = int(round(t_ms * 1e-3 / dt))
            while done < target:
                k = min(probe, target - done)
                sim.step(k)
                done += k
                if first_split is None and len(sim.bubbles(0)) > 1:
                    first_split = done
            counts.append(len(sim.bubbles(0)))
        b = sim.bubbles(0)
        out[f"{sigma_si:g}"] = {
            "tau": sc.tau, "sigma_lb": sc.sigma, "nu_si": sc.units["nu_si"], "steps": done,
            "bubbles_at_frames_ms": dict(zip([str(t) for t in frames], counts)),
            "first_split_step": first_split,
            "first_split_ms": None if first_split is None else round(first_split * dt * 1e3, 2),
            "paper_pieces": S.RUPTURE_PIECES[sigma_si],
            "V0": float(b0["volume"].sum()), "V_end": float(b["volume"].sum()),
            "Vstar_end": float(b["init_volume"].sum()),
            "labelling_runs": sim.labelling_runs}
        sim.close()
        assert counts[-1] >= 2, f"sigma {sigma_si}: the thread did not rupture ({counts})"
    print("RUPTURE " + json.dumps(out))
