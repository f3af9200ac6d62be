"""Host transfers through the C ABI: the handle's staging buffer grows when a
call needs more and is reused otherwise; caller-supplied (pinned) output
arrays receive the same values as arrays the binding allocates."""
import numpy as np
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


def test_fields_into_pinned_buffers_and_growing_staging(fsl):
    import torch
    scs = [S.static_bubble(n=16, radius=4.0), S.static_bubble(n=24, radius=6.0)]
    sim = fsl.Simulation.from_scenarios(scs, precision="f16s")
    sim.step(3)
    small = sim.fields(0, ("flags",))                       # smallest staging need first
    full = sim.fields(1, ("flags", "fill", "mass", "id", "rho", "u", "pdf"))   # grows it
    again = sim.fields(0, ("flags", "fill", "pdf"))         # reuses it
    assert np.array_equal(small["flags"], again["flags"])
    n1 = scs[1].n
    out = {}
    for k, (dt, m) in (("fill", (np.float64, 1)), ("pdf", (np.float64, 19)), ("id", (np.int64, 1))):
        t = torch.empty(m * n1, dtype=getattr(torch, np.dtype(dt).name), pin_memory=True)
        out[k] = t.numpy()
    got = sim.fields(1, ("fill", "pdf", "id", "flags"), out=out)
    assert got["fill"].ctypes.data == out["fill"].ctypes.data
    for k in ("fill", "pdf", "id", "flags"):
        assert np.array_equal(got[k], full[k], equal_nan=k in ("fill", "pdf")), k
    with pytest.raises(ValueError):
        sim.fields(1, ("fill",), out={"fill": np.empty(n1 + 1)})
    sim.close()
