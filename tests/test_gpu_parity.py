"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle on the same seeded
inputs. FP64 mode must agree to rounding (1e-9 relative); the mixed mode (FP32 pair and
PME arithmetic, FP64 accumulation) within the stated tolerances: field 1e-5 RMS-relative,
energy 1e-5 relative, forces 1e-4 RMS-relative, dipoles within the PCG tolerance."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import Oracle, Params
from paper_2011_01207_gb300 import binding, synth

pytestmark = pytest.mark.gpu
DEBYE = 4.80321


def _rel_rms(a, b):
    return float(np.sqrt(np.mean((a - b) ** 2) / np.mean(b ** 2)))


def _rel_max(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2011_01207_gb300 import build
    build.build_library()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


@pytest.fixture(scope="module")
def c1():
    return synth.water_box(216, 18.64, 1001)


@pytest.fixture(scope="module")
def chain():
    return synth.solvated_chain(60, 180, 26.0, 1103)


def _ctx(s, prec, cutoff=7.0, buffer=2.0, grid=(24, 24, 24)):
    c = binding.Context(s, cutoff=cutoff, buffer=buffer, beta=0.5446, grid=grid, precision=prec)
    c.build()
    c.permanent_field()
    return c


def _oracle(s, cutoff=7.0, grid=(24, 24, 24)):
    return Oracle(s, Params(beta=0.5446, grid=grid, cutoff=cutoff))


@pytest.mark.parametrize("prec,tol", [(binding.AP_FP64, 1e-9), (binding.AP_MIXED, 1e-5)])
def test_permanent_field(c1, prec, tol):
    c = _ctx(c1, prec)
    E = c.field.cpu().numpy()
    Eo = _oracle(c1).permanent_field()
    assert _rel_rms(E, Eo) < tol
    c.close()


@pytest.mark.parametrize("prec,tol", [(binding.AP_FP64, 1e-9), (binding.AP_MIXED, 1e-5)])
def test_dipole_matvec(c1, prec, tol):
    c = _ctx(c1, prec)
    v = np.random.default_rng(4).normal(size=(c1.n, 3)) * 0.1
    out = torch.zeros((c1.n, 3), dtype=torch.float64, device="cuda")
    c.matvec(torch.tensor(v, device="cuda"), out)
    Tv = out.cpu().numpy()
    Tvo = _oracle(c1).apply_T(v)
    assert _rel_rms(Tv, Tvo) < tol
    c.close()


def test_pcg_fp64_matches_oracle_iterates(c1):
    """FP64: same algorithm, same start, same stopping rule -> same iteration count and
    dipoles to rounding."""
    c = _ctx(c1, binding.AP_FP64)
    info = c.solve(tol=1e-6, max_iter=100)
    mu = c.mu.cpu().numpy()
    o = _oracle(c1)
    E = o.permanent_field()
    mu_o, info_o = o.pcg(E, tol=1e-6)
    assert info.iterations == info_o["iters"]
    assert abs(info.eps_debye - info_o["eps"]) < 1e-6 * info_o["eps"]
    assert _rel_max(mu, mu_o) < 1e-8
    c.close()


def test_pcg_mixed_converges_to_tolerance(c1):
    tol = 1e-5
    c = _ctx(c1, binding.AP_MIXED)
    info = c.solve(tol=tol, max_iter=100)
    assert info.status == 0 and info.eps_debye <= tol
    mu = c.mu.cpu().numpy()
    o = _oracle(c1)
    E = o.permanent_field()
    true_eps = o.residual_eps(E - o.apply_A(mu))
    assert true_eps < 1.5 * tol
    mu_star, _ = o.pcg(E, tol=1e-10)
    err_debye = DEBYE * np.sqrt(np.mean(np.sum((mu - mu_star) ** 2, axis=1)))
    assert err_debye < 10 * tol
    c.close()


@pytest.mark.parametrize("prec,etol,ftol", [(binding.AP_FP64, 1e-9, 1e-8), (binding.AP_MIXED, 1e-5, 1e-4)])
def test_energy_forces(c1, prec, etol, ftol):
    c = _ctx(c1, prec)
    o = _oracle(c1)
    E = o.permanent_field()
    mu_star, _ = o.pcg(E, tol=1e-10)
    mu_t = torch.tensor(mu_star, device="cuda")
    e, f = c.energy_forces(mu_t)
    e_o = o.energy(mu_star, E)
    F_o = o.forces(mu_star)
    assert abs(float(e.cpu()[0]) - e_o) < etol * abs(e_o)
    assert _rel_rms(f.cpu().numpy(), F_o) < ftol
    c.close()


@pytest.mark.parametrize("prec,field_tol,etol,ftol", [(binding.AP_FP64, 1e-9, 1e-9, 1e-8),
                                                      (binding.AP_MIXED, 2e-5, 1e-5, 1e-4)])
def test_chain_exclusions_and_global_frames(chain, prec, field_tol, etol, ftol):
    """Chain atoms (global-frame multipoles, 1-2/1-3 exclusions) among waters. The field of
    the mixed mode is held to 2e-5: the chain's charges of ~0.3 e next to each other cancel
    in the field of the waters around them, so the relative error of the smaller field is
    larger than in pure water; energy and forces at the stated 1e-5 / 1e-4."""
    grid = (32, 32, 32)
    c = _ctx(chain, prec, grid=grid)
    o = _oracle(chain, grid=grid)
    E = o.permanent_field()
    assert _rel_rms(c.field.cpu().numpy(), E) < field_tol
    mu_star, _ = o.pcg(E, tol=1e-10)
    e, f = c.energy_forces(torch.tensor(mu_star, device="cuda"))
    assert abs(float(e.cpu()[0]) - o.energy(mu_star, E)) < etol * abs(o.energy(mu_star, E))
    assert _rel_rms(f.cpu().numpy(), o.forces(mu_star)) < ftol
    c.close()


@pytest.mark.parametrize("n_mol,box,cutoff,buffer,grid", [
    (1, 11.0, 4.0, 1.5, (8, 8, 8)),        # one molecule: a single, mostly padded block
    (11, 12.0, 4.5, 1.5, (12, 10, 8)),     # 33 atoms: one full block and a 1-atom tail
    (37, 15.0, 5.0, 2.0, (16, 16, 16)),    # non-cubic grid, ragged last block
])
def test_small_and_ragged(n_mol, box, cutoff, buffer, grid):
    s = synth.water_box(n_mol, box, 77 + n_mol, dmin_inter=1.6)
    c = _ctx(s, binding.AP_FP64, cutoff=cutoff, buffer=buffer, grid=grid)
    o = _oracle(s, cutoff=cutoff, grid=grid)
    E = o.permanent_field()
    assert _rel_rms(c.field.cpu().numpy(), E) < 1e-9
    info = c.solve(tol=1e-8, max_iter=200)
    mu_o, info_o = o.pcg(E, tol=1e-8)
    assert info.iterations == info_o["iters"]
    assert _rel_max(c.mu.cpu().numpy(), mu_o) < 1e-7
    c.close()


def test_zero_guess_and_given_guess(c1):
    c = _ctx(c1, binding.AP_FP64)
    o = _oracle(c1)
    E = o.permanent_field()
    for guess in (np.zeros((c1.n, 3)), 0.9 * c1.alpha[:, None] * E):
        info = c.solve(tol=1e-6, max_iter=100, guess=torch.tensor(guess, device="cuda"))
        mu_o, info_o = o.pcg(E, guess=guess, tol=1e-6)
        assert info.iterations == info_o["iters"]
        assert _rel_max(c.mu.cpu().numpy(), mu_o) < 1e-8
    c.close()


def test_max_iter_reports_not_converged(c1):
    c = _ctx(c1, binding.AP_MIXED)
    info = c.solve(tol=1e-12, max_iter=3)
    assert info.status == binding.AP_NOT_CONVERGED and info.iterations == 3
    c.close()


def test_dipole_matvec_after_drift_without_rebuild(c1):
    """Lists built at one configuration, field and dipole products at a drifted one (every
    atom within buffer/2): the filtered chunks and pair masks follow the configuration."""
    c = _ctx(c1, binding.AP_FP64)
    s2 = synth.perturb(c1, 31, sigma_t=0.2, sigma_r=0.05)
    disp = np.linalg.norm(s2.xyz - c1.xyz, axis=1)
    assert disp.max() < 1.0
    c.set_positions(s2.xyz)
    c.permanent_field()
    o = _oracle(s2)
    assert _rel_rms(c.field.cpu().numpy(), o.permanent_field()) < 1e-9
    v = np.random.default_rng(6).normal(size=(c1.n, 3)) * 0.1
    out = torch.zeros((c1.n, 3), dtype=torch.float64, device="cuda")
    c.matvec(torch.tensor(v, device="cuda"), out)
    assert _rel_rms(out.cpu().numpy(), o.apply_T(v)) < 1e-9
    c.close()
