"""Argument checks of the Python binding that run before any call into the
library: the allocation-free labelling entry point refuses host arrays, host
tensors, wrong dtypes, non-contiguous views and buffers shorter than the
lattice, so that a bad buffer never reaches its kernels (no GPU needed)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1604_01632_gb300 import fsl


def _refused(flags, labels, dims=(4, 4, 4)):
    with pytest.raises(ValueError):
        fsl.label_bubbles_static(flags, *dims, labels)


def test_host_arrays_and_tensors_are_refused(monkeypatch):
    # the library must not even be loaded for a refused call
    monkeypatch.setattr(fsl, "load_library", lambda: pytest.fail("library called with a bad buffer"))
    n = 64
    _refused(np.zeros(n, np.uint8), np.zeros(n, np.int64))
    _refused(torch.zeros(n, dtype=torch.uint8), torch.zeros(n, dtype=torch.int64))


def test_dimensions_must_be_positive(monkeypatch):
    monkeypatch.setattr(fsl, "load_library", lambda: pytest.fail("library called with bad dimensions"))
    with pytest.raises(ValueError):
        fsl.label_bubbles_static(None, 0, 4, 4, None)


@pytest.mark.gpu
def test_short_or_mistyped_device_buffers_are_refused(monkeypatch):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    monkeypatch.setattr(fsl, "load_library", lambda: pytest.fail("library called with a bad buffer"))
    n = 64
    ok_f = torch.zeros(n, dtype=torch.uint8, device="cuda")
    ok_l = torch.zeros(n, dtype=torch.int64, device="cuda")
    _refused(ok_f[: n - 1], ok_l)                                   # flags shorter than the lattice
    _refused(ok_f, ok_l[: n - 1])                                   # labels shorter than the lattice
    _refused(ok_f.to(torch.int32), ok_l)                            # wrong flag type
    _refused(ok_f, ok_l.to(torch.int32))                            # wrong label type
    _refused(ok_f, torch.zeros(2 * n, dtype=torch.int64, device="cuda")[::2])   # not contiguous
