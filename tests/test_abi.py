"""The C ABI library builds, loads and exports every entry point declared in
include/fsl.h (no GPU needed: nothing here calls into the device)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(fsl_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_1604_01632_gb300 import build
    try:
        build.nvcc()
    except RuntimeError:
        if not os.path.exists(build.LIB):
            pytest.skip("no nvcc and no prebuilt library")
        return build.LIB
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("fsl_create", "fsl_init_geometry", "fsl_step", "fsl_bubbles", "fsl_fields", "fsl_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_lists_match_header():
    from paper_1604_01632_gb300 import fsl
    assert set(fsl.EXPORTS) <= set(_declared())


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1604_01632_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "fsl_oracle" not in txt, f


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_1604_01632_gb300 import fsl
    monkeypatch.setattr(fsl, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(fsl, "_lib", None)
    with pytest.raises(RuntimeError):
        fsl.load_library()
