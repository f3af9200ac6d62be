"""The allocation-free labelling entry point (for callers that cannot allocate
device memory) against the library's own labels.

fsl_label_bubbles_static labels gas/interface components with a fixed scratch
array compiled into the library instead of allocating.  Its labels must equal
the bubble ids fsl_fields reports after fsl_init_geometry, on two calls in a
row (the second call reuses the scratch the first one left behind).  This file
is collected last so that a failure here stops a -x run only after every other
test has run."""
import numpy as np
import pytest

from paper_1604_01632_gb300 import scenarios as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1604_01632_gb300 import build, fsl
    build.build()
    return torch, fsl


def _cases():
    return [S.random_bubbles(24, 20, 16, n_bubbles=6, r_min=2.5, r_max=4.5, u_max=0.05, sigma=5e-3, seed=3),
            S.gas_thread(nx=48, ny=20, nz=20, radius=3.0, amp=0.25, wavelength=24, sigma=0.05, steps=0),
            S.static_bubble(n=16, radius=4.0)]


def test_static_labels_match_library_ids_twice(env):
    torch, fsl = env
    for sc in _cases():
        sim = fsl.Simulation.from_scenarios([sc], precision="fp64")
        want = sim.fields(0, ("id",))["id"]
        sim.close()
        flags = torch.from_numpy(np.ascontiguousarray(sc.flags.reshape(-1))).cuda()
        for _ in range(2):
            out = torch.full((sc.n,), -7, dtype=torch.int64, device="cuda")
            fsl.label_bubbles_static(flags, sc.nx, sc.ny, sc.nz, out)
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy(), want), sc.name


def test_static_labels_reject_oversized_lattice(env):
    """A lattice above the fixed scratch (2^21 cells) is refused by the library
    itself, with buffers large enough to pass the binding's own checks."""
    torch, fsl = env
    n = 256 * 128 * 65                                      # 2^21 + 2^15 cells
    flags = torch.zeros(n, dtype=torch.uint8, device="cuda")
    out = torch.zeros(n, dtype=torch.int64, device="cuda")
    with pytest.raises(fsl.FslError) as e:
        fsl.label_bubbles_static(flags, 256, 128, 65, out)
    assert e.value.status == -1
