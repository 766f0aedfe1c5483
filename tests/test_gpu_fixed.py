"""AP_FIXED: FP32 pair and PME arithmetic with 64-bit fixed-point accumulation of fields,
forces, torque terms, the energy and the PME grid (the paper's fixed-point mode, Sec. 2.4).
Parity with the FP64 oracle at the mixed mode's tolerances, and bitwise reproducibility:
two independent runs, and runs with different launch shapes, give identical bits."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import Oracle, Params
from paper_2011_01207_gb300 import binding, synth

pytestmark = pytest.mark.gpu
DEBYE = 4.80321


def _rel_rms(a, b):
    return float(np.sqrt(np.mean((a - b) ** 2) / np.mean(b ** 2)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2011_01207_gb300 import build
    build.build_library()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _step(s, grid, tune=False):
    c = binding.Context(s, cutoff=7.0, buffer=2.0, beta=0.5446, grid=grid, precision=binding.AP_FIXED)
    c.build()
    c.permanent_field()
    if tune:
        binding.ap_autotune(c.ctx, 2)
        c.permanent_field()
    info = c.solve(tol=1e-6, max_iter=100)
    e, f = c.energy_forces(c.mu)
    out = {"field": c.field.cpu().numpy().copy(), "mu": c.mu.cpu().numpy().copy(),
           "energy": e.cpu().numpy().copy(), "forces": f.cpu().numpy().copy(), "iters": info.iterations}
    v = torch.tensor(np.random.default_rng(3).normal(size=(s.n, 3)) * 0.1, device="cuda")
    tv = torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")
    c.matvec(v, tv)
    out["Tv"] = tv.cpu().numpy().copy()
    c.close()
    return out


@pytest.mark.parametrize("which", ["water", "chain"])
def test_fixed_point_parity(which):
    if which == "water":
        s, grid = synth.water_box(216, 18.64, 1001), (24, 24, 24)
    else:
        s, grid = synth.solvated_chain(60, 180, 26.0, 1103), (32, 32, 32)
    r = _step(s, grid)
    o = Oracle(s, Params(beta=0.5446, grid=grid, cutoff=7.0))
    E = o.permanent_field()
    assert _rel_rms(r["field"], E) < 2e-5
    v = np.random.default_rng(3).normal(size=(s.n, 3)) * 0.1
    assert _rel_rms(r["Tv"], o.apply_T(v)) < 1e-5
    mu = r["mu"]
    assert o.residual_eps(E - o.apply_A(mu)) < 1.5e-6
    mu_star, _ = o.pcg(E, tol=1e-10)
    assert DEBYE * np.sqrt(np.mean(np.sum((mu - mu_star) ** 2, axis=1))) < 1e-5
    e_o = o.energy(mu, E)
    assert abs(float(r["energy"][0]) - e_o) < 1e-5 * abs(e_o)
    assert _rel_rms(r["forces"], o.forces(mu)) < 1e-4


def test_fixed_point_is_bitwise_reproducible():
    s = synth.solvated_chain(60, 180, 26.0, 1103)
    grid = (32, 32, 32)
    a = _step(s, grid)
    b = _step(s, grid)
    c = _step(s, grid, tune=True)     # other launch shapes of the pair and PME kernels
    for k in ("field", "mu", "energy", "forces", "Tv"):
        assert np.array_equal(a[k], b[k]), k
        assert np.array_equal(a[k], c[k]), k
    assert a["iters"] == b["iters"] == c["iters"]
