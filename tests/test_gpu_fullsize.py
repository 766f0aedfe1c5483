"""GPU parity at the full sizes of the benchmark's water box (96,000 atoms, 98.7 A, grid
100), the solvated-chain box (23,558 atoms, 62.2 A, grid 64) and the large water box
(1,065,000 atoms, 221.6 A, grid 224), in the mixed precision the benchmark runs (FP32 pair
and PME arithmetic, FP64 accumulation), through the C-ABI and in the benchmark's launch
configuration (7 A + 2 A lists, tile shifts, list filtering, graph solve).

The 96,000- and 23,558-atom boxes are checked atom by atom against the full FP64 oracle:
permanent field, the true residual of the solved dipoles (and at 23,558 atoms their
distance to the oracle's solution and the nine components of the virial), the energy and
every force at those dipoles. At a
million atoms the oracle evaluates sampled rows: the permanent field and the true residual
of the solved dipoles at 200 atoms."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import Oracle, Params, model
from paper_2011_01207_gb300 import binding, synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
DEBYE = 4.80321


def _rel_rms(a, b):
    return float(np.sqrt(np.mean((a - b) ** 2) / np.mean(b ** 2)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2011_01207_gb300 import build
    build.build_library()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def test_water_96000_atoms_full():
    s = synth.water_box(32000, 98.7, 1002)
    grid = (100, 100, 100)
    c = binding.Context(s, cutoff=7.0, buffer=2.0, beta=0.5446, grid=grid, precision=binding.AP_MIXED)
    c.build()
    c.permanent_field()
    tol = 1e-5
    info = c.solve(tol=tol, max_iter=100)
    assert info.status == 0 and info.eps_debye <= tol
    e, f = c.energy_forces(c.mu)
    torch.cuda.synchronize()
    o = Oracle(s, Params(beta=0.5446, grid=grid, cutoff=7.0))
    E = o.permanent_field()
    assert _rel_rms(c.field.cpu().numpy(), E) < 1e-5
    mu = c.mu.cpu().numpy()
    assert o.residual_eps(E - o.apply_A(mu)) < 1.5 * tol
    e_o = o.energy(mu, E)
    assert abs(float(e.cpu()[0]) - e_o) < 1e-5 * abs(e_o)
    F_o = o.forces(mu)
    assert _rel_rms(f.cpu().numpy(), F_o) < 1e-4
    c.close()


def test_solvated_chain_23558_atoms():
    s = synth.solvated_chain(2489, 7023, 62.2, 1003)
    assert s.n == 23558
    grid = (64, 64, 64)
    c = binding.Context(s, cutoff=7.0, buffer=2.0, beta=0.5446, grid=grid, precision=binding.AP_MIXED)
    c.build()
    c.permanent_field()
    o = Oracle(s, Params(beta=0.5446, grid=grid, cutoff=7.0))
    E = o.permanent_field()
    assert _rel_rms(c.field.cpu().numpy(), E) < 2e-5
    tol = 1e-5
    info = c.solve(tol=tol, max_iter=100)
    assert info.status == 0 and info.eps_debye <= tol
    mu = c.mu.cpu().numpy()
    assert o.residual_eps(E - o.apply_A(mu)) < 1.5 * tol
    mu_star, _ = o.pcg(E, tol=1e-9)
    err_debye = DEBYE * np.sqrt(np.mean(np.sum((mu - mu_star) ** 2, axis=1)))
    assert err_debye < 10 * tol
    e, f, V = c.energy_forces(c.mu, virial=True)
    e_o = o.energy(mu, E)
    assert abs(float(e.cpu()[0]) - e_o) < 1e-5 * abs(e_o)
    assert _rel_rms(f.cpu().numpy(), o.forces(mu)) < 1e-4
    V_o = o.virial(mu)
    assert np.abs(V.cpu().numpy() - V_o).max() < 1e-4 * np.abs(V_o).max()
    c.close()


def test_water_1065000_atoms_sampled_rows():
    s = synth.water_box(355000, 221.6, 1004)
    grid = (224, 224, 224)
    c = binding.Context(s, cutoff=7.0, buffer=2.0, beta=0.5446, grid=grid, precision=binding.AP_MIXED)
    c.build()
    c.permanent_field()
    info = c.solve(tol=1e-5, max_iter=100)
    assert info.status == 0
    rows = np.random.default_rng(11).choice(s.n, 200, replace=False)
    mu = c.mu.cpu().numpy()
    E_o, Tmu = model.row_fields(s, Params(beta=0.5446, grid=grid, cutoff=7.0), rows, mu)
    assert _rel_rms(c.field.cpu().numpy()[rows], E_o) < 1e-5
    resid = E_o - (mu[rows] / s.alpha[rows, None] - Tmu)
    eps = DEBYE * np.sqrt(np.mean(np.sum((s.alpha[rows, None] * resid) ** 2, axis=1)))
    assert eps < 1.5e-5
    c.close()
