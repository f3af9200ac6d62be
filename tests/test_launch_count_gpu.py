"""The library's launch count (the bench reports it as the kernels of the
timed steps): exactly two kernels per step, the stream-collide kernel and the
cooperative conversion kernel, with and without CUDA graphs."""
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


@pytest.mark.parametrize("graphs", [True, False])
def test_two_kernels_per_step(fsl, graphs):
    sim = fsl.Simulation.from_scenarios([S.static_bubble(n=16, radius=4.0)], precision="f16s")
    sim.set_graphs(graphs)
    sim.step(1)   # the first step also runs the initial labelling and list
    sim.sync()
    l0 = sim.launches
    sim.step(5)
    sim.sync()
    assert sim.launches - l0 == 10
    sim.close()
