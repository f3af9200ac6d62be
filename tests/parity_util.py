"""Helpers shared by the GPU parity tests: run the CUDA library and the oracle
on the same seeded inputs and compare their states."""
import numpy as np

from paper_1604_01632_gb300 import scenarios as S

FLUID = (S.LIQUID, S.INTERFACE)


def gpu_state(sim, d=0):
    fl = sim.fields(d, ("flags", "fill", "mass", "id", "pdf"))
    return dict(flags=fl["flags"], phi=fl["fill"], mass=fl["mass"], ids=fl["id"], f=fl["pdf"], bubbles=sim.bubbles(d))


def oracle_state(o):
    return dict(flags=o.flags(), phi=o.phi(), mass=o.mass(), ids=o.ids(), f=o.f(), bubbles=o.bubbles())


def compare_exact(g, r, f_tol=1e-12, what=""):
    """FP64 path: flags and bubble ids bit-identical, PDFs / mass / fill within
    f_tol, bubble table V and V* identical (fixed point), pressure to 1e-12."""
    assert np.array_equal(g["flags"], r["flags"]), f"{what}: flags differ at {np.nonzero(g['flags'] != r['flags'])[0][:10]}"
    assert np.array_equal(g["ids"], r["ids"]), f"{what}: bubble ids differ"
    fl = np.isin(r["flags"], FLUID)
    df = np.abs(g["f"][:, fl] - r["f"][:, fl]).max() if fl.any() else 0.0
    assert df <= f_tol, f"{what}: max |f_gpu - f_oracle| = {df}"
    itf = r["flags"] == S.INTERFACE
    if itf.any():
        assert np.abs(g["mass"][itf] - r["mass"][itf]).max() <= f_tol, f"{what}: interface mass"
        assert np.abs(g["phi"][itf] - r["phi"][itf]).max() <= f_tol, f"{what}: fill level"
    gb, rb = g["bubbles"], r["bubbles"]
    assert len(gb) == len(rb), f"{what}: {len(gb)} bubbles on the GPU, {len(rb)} in the oracle"
    assert np.array_equal(gb["id"], rb["id"]), f"{what}: bubble ids"
    assert np.array_equal(gb["n_cells"], rb["n_cells"]), f"{what}: bubble cell counts"
    assert np.array_equal(gb["volume"], rb["volume"]), f"{what}: bubble volumes"
    assert np.array_equal(gb["init_volume"], rb["init_volume"]), f"{what}: bubble V*"
    assert np.allclose(gb["pressure"], rb["pressure"], rtol=1e-12, atol=0), f"{what}: bubble pressure"
    return df


def macro(f):
    c = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                  [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1], [1, 0, -1], [-1, 0, 1],
                  [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]], dtype=np.float64)
    rho = f.sum(0)
    with np.errstate(invalid="ignore", divide="ignore"):
        u = (c.T @ f) / rho
    return rho, u
