"""fsl_init_geometry from page-locked host buffers (read by the initialisation
kernel in place) gives the state that pageable buffers (staged by copies)
give: FP64, every field identical after 0 and 5 steps."""
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


def _pinned_copy(a):
    import torch
    t = torch.empty(a.size, dtype=getattr(torch, a.dtype.name), pin_memory=True)
    v = t.numpy()
    np.copyto(v, a.reshape(-1))
    return t, v


def test_pinned_and_pageable_initial_states_agree(fsl):
    sc = S.random_bubbles(24, 20, 16, n_bubbles=6, r_min=2.5, r_max=4.5, u_max=0.06, sigma=5e-3, seed=2)
    a = fsl.Simulation([sc.params()], precision="fp64")
    a.init_geometry(0, sc.flags, sc.fill, sc.rho, sc.u)
    keep = [_pinned_copy(x) for x in (sc.flags, sc.fill, sc.rho, sc.u)]
    b = fsl.Simulation([sc.params()], precision="fp64")
    b.init_geometry(0, *(v for _, v in keep))
    for k in (0, 5):
        if k:
            a.step(k)
            b.step(k)
        fa, fb = a.fields(0), b.fields(0)
        for name in fa:
            assert np.array_equal(fa[name], fb[name]), f"{name} differs after {k} steps"
    a.close()
    b.close()
