"""Failure reporting of bounded device waits, made to run out on purpose in
forms that fault and hang nothing: the labelling's union / find loops with
their iteration cap set to 1 (any bubble of three or more cells needs more),
and the conversion kernel's grid barriers told to wait for one block more
than the grid holds, with a poll limit of a few thousand.  Each must come back
as its status from the next synchronising call (and again from the ones
after it: the status latches)."""
import pytest

from paper_1604_01632_gb300 import scenarios as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fsl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_01632_gb300 import build, fsl as F
    build.build()
    return F


def _status(fsl, fn):
    with pytest.raises(fsl.FslError) as e:
        fn()
    return e.value.status


def test_initial_labelling_cap_reports_not_converged(fsl):
    sim = fsl.Simulation.from_scenarios([S.static_bubble(n=16, radius=4.0)], precision="fp64")
    sim.set_limits(ccl_max_iter=1)
    assert _status(fsl, lambda: (sim.step(1), sim.sync())) == -5      # FSL_ERR_CCL_NOT_CONVERGED
    assert _status(fsl, sim.sync) == -5                                # latched: reported again
    sim.close()


def test_labelling_cap_inside_the_conversion_kernel(fsl):
    """Moving bubbles: the labelling inside the conversion kernel (run on a
    step whose conversions may merge or split) hits the cap."""
    sc = S.random_bubbles(24, 20, 16, n_bubbles=6, r_min=2.5, r_max=4.5, u_max=0.06, sigma=5e-3, seed=0)
    sim = fsl.Simulation.from_scenarios([sc], precision="fp64")
    sim.step(1)
    sim.sync()                                        # initial labelling with the default cap
    runs0 = sim.labelling_runs
    sim.set_limits(ccl_max_iter=1)
    status = 0
    for _ in range(40):
        sim.step(1)
        try:
            sim.sync()
        except fsl.FslError as e:
            status = e.status
            break
    assert status == -5
    assert sim.labelling_runs > runs0
    sim.close()


@pytest.mark.parametrize("graphs", [True, False])
def test_barrier_that_cannot_complete_reports_sync_error(fsl, graphs):
    sim = fsl.Simulation.from_scenarios([S.static_bubble(n=16, radius=4.0)], precision="f16s")
    sim.set_graphs(graphs)
    sim.step(2)
    sim.sync()
    sim.set_limits(barrier_polls=4000, barrier_absent=True)
    assert _status(fsl, lambda: (sim.step(1), sim.sync())) == -8      # FSL_ERR_SYNC
    sim.close()
