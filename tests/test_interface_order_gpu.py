"""The interface list rebuilt in cell order after every conversion
(fsl_set_interface_order): the same results as the appended list, bit for
bit, in every storage form; the FP64 path still identical to the oracle,
also with several domains of ragged sizes (padding cells between them)."""
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


def test_ordered_list_fp64_matches_oracle(fsl, oracle_mod):
    """Moving bubbles with conversions, merges and splits every few steps."""
    sc = S.random_bubbles(24, 20, 16, n_bubbles=6, r_min=2.5, r_max=4.5, u_max=0.06, sigma=5e-3, seed=1)
    sim = fsl.Simulation.from_scenarios([sc], precision="fp64")
    sim.set_interface_order(1)
    assert sim.interface_order == 1
    o = oracle_mod.Oracle.from_scenario(sc)
    done = 0
    for k in (1, 2, 3, 10, 40):
        sim.step(k - done)
        o.step(k - done)
        done = k
        compare_exact(gpu_state(sim), oracle_state(o), what=f"ordered list step {k}")


def test_ordered_list_batched_ragged_fp64(fsl, oracle_mod):
    """Domains whose sizes are not multiples of 256 cells, one handle."""
    scs = [S.random_bubbles(21, 15, 13, n_bubbles=3, r_min=2.5, r_max=3.5, u_max=0.05, sigma=4e-3, seed=s)
           for s in range(3)]
    scs.append(S.static_bubble(n=17, radius=4.5))
    sim = fsl.Simulation.from_scenarios(scs, precision="fp64")
    sim.set_interface_order(1)
    oras = [oracle_mod.Oracle.from_scenario(s) for s in scs]
    prev = 0
    for k in (1, 5, 25):
        sim.step(k - prev)
        for o in oras:
            o.step(k - prev)
        prev = k
        for d, o in enumerate(oras):
            compare_exact(gpu_state(sim, d), oracle_state(o), what=f"ordered list domain {d} step {k}")


@pytest.mark.parametrize("precision", ["f16s", "fp32", "bf16s"])
def test_order_modes_give_identical_results(fsl, precision):
    """Four domains of the bubble-population workload, 30 steps with the list
    as appended and with the list in cell order: every field identical."""
    scs = S.bubble_population(n_domains=4, seed=3, sides=(32, 48))
    states = []
    for mode in (0, 1):
        sim = fsl.Simulation.from_scenarios(scs, precision=precision)
        sim.set_interface_order(mode)
        assert sim.interface_order == mode
        sim.step(30)
        sim.sync()
        states.append([gpu_state(sim, d) for d in range(len(scs))])
        sim.close()
    for d in range(len(scs)):
        a, b = states[0][d], states[1][d]
        for key in ("flags", "ids", "phi", "mass", "f"):
            assert np.array_equal(a[key], b[key], equal_nan=key not in ("flags", "ids")), f"domain {d}: {key}"
        for col in ("id", "n_cells", "volume", "init_volume", "pressure"):
            assert np.array_equal(a["bubbles"][col], b["bubbles"][col]), f"domain {d}: bubble {col}"


def test_default_order_follows_lattice_size(fsl):
    """Default: decided per step (rule 2) when the two PDF arrays exceed twice
    the L2 cache, else never (rule 0)."""
    import torch
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    sc = S.static_bubble(n=112, radius=20.0)
    cells = 112 ** 3
    for precision, fbytes in (("fp64", 8), ("f16s", 2)):
        sim = fsl.Simulation.from_scenarios([sc], precision=precision)
        want = 2 if 2 * 19 * cells * fbytes > 2 * l2 else 0
        assert sim.interface_order == want
        for mode in (0, 1):
            sim.set_interface_order(mode)
            assert sim.interface_order == mode
        sim.set_interface_order(-1)
        assert sim.interface_order == want
        with pytest.raises(fsl.FslError):
            sim.set_interface_order(2)
        sim.close()


def test_default_order_on_a_large_population_gives_identical_results(fsl):
    """Twelve bubble-population domains in FP64 (PDF arrays above twice the L2
    cache, about a tenth of the cells in the interface): the default rule
    rebuilds the list every step; 8 steps identical to the appended list."""
    scs = S.bubble_population(n_domains=12, seed=7, sides=(48, 64))
    states = []
    for mode in (0, -1):
        sim = fsl.Simulation.from_scenarios(scs, precision="fp64")
        sim.set_interface_order(mode)
        states.append(sim)
    assert states[1].interface_order == 2
    for sim in states:
        sim.step(8)
        sim.sync()
    for d in range(len(scs)):
        a, b = gpu_state(states[0], d), gpu_state(states[1], d)
        for key in ("flags", "ids", "phi", "mass", "f"):
            assert np.array_equal(a[key], b[key], equal_nan=key not in ("flags", "ids")), f"domain {d}: {key}"
    for sim in states:
        sim.close()
