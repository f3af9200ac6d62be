"""The library's launch count (the bench reports it as the kernels of the
timed steps): per step the stream-collide kernel (two kernels in the
two-kernel forms: liquid cells, then interface cells), the normals pass in the
forms that take interface cells one per thread (5-8) and the cooperative
conversion kernel, with and without CUDA graphs, in every stream-collide form."""
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


@pytest.mark.parametrize("form", list(range(9)))
@pytest.mark.parametrize("graphs", [True, False])
def test_kernels_per_step(fsl, graphs, form):
    sim = fsl.Simulation.from_scenarios([S.static_bubble(n=16, radius=4.0)], precision="f16s")
    sim.set_graphs(graphs)
    if form == 4:
        sim.set_interface_order(1)
    sim.set_stream_form(form)
    sim.step(1)   # the first step also runs the initial labelling and list
    sim.sync()
    l0 = sim.launches
    sim.step(5)
    sim.sync()
    per_step = 4 if form in (5, 8) else 3 if form in (6, 7) else 2
    assert sim.launches - l0 == 5 * per_step
    sim.close()


def test_labelling_counters(fsl):
    """The labelling passes and the bubbles they take: a pass runs only on steps
    whose conversions may have merged or split a bubble, and takes only the
    bubbles marked then (at least one, never more than exist)."""
    scs = S.bubble_population(n_domains=3, seed=5, sides=(32, 48))
    sim = fsl.Simulation.from_scenarios(scs, precision="f16s")
    sim.step(1)
    r0, b0 = sim.labelling_runs, sim.relabelled_bubbles
    sim.step(40)
    runs, took = sim.labelling_runs - r0, sim.relabelled_bubbles - b0
    nb = sum(len(sim.bubbles(d)) for d in range(len(scs)))
    assert 0 < runs <= 40
    assert runs <= took
    assert took / runs <= nb + 50   # bubbles that merged away in a pass no longer count at the end
    sim.close()
