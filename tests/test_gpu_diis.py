"""GPU parity of the Jacobi/DIIS solver (induced_dipoles_diis) through the C-ABI against the
oracle's Oracle.jacobi_diis on the same seeded inputs. FP64 mode runs the same algorithm from
the same start with the same stopping rule, so the update count must match and the dipoles
agree to rounding; the mixed and fixed-point modes must reach the tolerance in the true
residual, evaluated by the oracle."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import Oracle, Params
from paper_2011_01207_gb300 import binding, synth

pytestmark = pytest.mark.gpu
DEBYE = 4.80321


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


@pytest.fixture(scope="module")
def oracle_c1(c1):
    o = Oracle(c1, Params(beta=0.5446, grid=(24, 24, 24), cutoff=7.0))
    return o, o.permanent_field()


def _ctx(s, prec, grid=(24, 24, 24)):
    c = binding.Context(s, cutoff=7.0, buffer=2.0, beta=0.5446, grid=grid, precision=prec)
    c.build()
    c.permanent_field()
    return c


@pytest.mark.parametrize("depth", [4, 6, 8])
def test_fp64_matches_oracle_iterates(c1, oracle_c1, depth):
    o, E = oracle_c1
    c = _ctx(c1, binding.AP_FP64)
    info = c.solve_diis(tol=1e-6, max_iter=200, depth=depth)
    mu_o, info_o = o.jacobi_diis(E, tol=1e-6, depth=depth)
    assert info.status == 0
    assert info.iterations == info_o["iters"]
    assert abs(info.eps_debye - info_o["eps"]) < 1e-6 * info_o["eps"]
    assert abs(info.eps_initial - info_o["history"][0]) < 1e-9 * info_o["history"][0]
    assert _rel_max(c.mu.cpu().numpy(), mu_o) < 1e-8
    c.close()


def test_plain_jacobi_iterates(c1, oracle_c1):
    """depth 1: plain Jacobi, which on liquid water contracts slowly (spectral radius of
    alpha T close to 1): compare the 25th iterate, not a converged one."""
    o, E = oracle_c1
    c = _ctx(c1, binding.AP_FP64)
    info = c.solve_diis(tol=1e-6, max_iter=25, depth=1)
    mu_o, info_o = o.jacobi_diis(E, tol=1e-6, depth=1, maxiter=25)
    assert info.status == binding.AP_NOT_CONVERGED and info.iterations == 25 == info_o["iters"]
    assert abs(info.eps_debye - info_o["eps"]) < 1e-8 * info_o["eps"]
    assert _rel_max(c.mu.cpu().numpy(), mu_o) < 1e-9
    c.close()


def test_max_iter_returns_the_last_update(c1, oracle_c1):
    o, E = oracle_c1
    c = _ctx(c1, binding.AP_FP64)
    info = c.solve_diis(tol=1e-12, max_iter=3, depth=4)
    mu_o, info_o = o.jacobi_diis(E, tol=1e-12, depth=4, maxiter=3)
    assert info.status == binding.AP_NOT_CONVERGED and info.iterations == 3 == info_o["iters"]
    assert _rel_max(c.mu.cpu().numpy(), mu_o) < 1e-9
    c.close()


def test_given_guess_and_zero_guess(c1, oracle_c1):
    o, E = oracle_c1
    c = _ctx(c1, binding.AP_FP64)
    for g in (np.zeros((c1.n, 3)), 0.9 * o.alpha[:, None] * E):
        info = c.solve_diis(tol=1e-6, max_iter=200, depth=6, guess=torch.tensor(g, device="cuda"))
        mu_o, info_o = o.jacobi_diis(E, guess=g, tol=1e-6, depth=6)
        assert info.iterations == info_o["iters"]
        assert _rel_max(c.mu.cpu().numpy(), mu_o) < 1e-8
    c.close()


def test_host_loop_equals_graph(c1):
    """The WHILE-node graph and the host-driven loop launch the same kernels."""
    c = _ctx(c1, binding.AP_FP64)
    a = c.solve_diis(tol=1e-6, max_iter=200, depth=6)
    mu_a = c.mu.cpu().numpy()
    c.close()
    old = os.environ.get("AP_SOLVE_GRAPH")
    os.environ["AP_SOLVE_GRAPH"] = "0"
    try:
        c = _ctx(c1, binding.AP_FP64)
        b = c.solve_diis(tol=1e-6, max_iter=200, depth=6)
        mu_b = c.mu.cpu().numpy()
        c.close()
    finally:
        if old is None:
            del os.environ["AP_SOLVE_GRAPH"]
        else:
            os.environ["AP_SOLVE_GRAPH"] = old
    assert a.iterations == b.iterations
    assert _rel_max(mu_b, mu_a) < 1e-12


@pytest.mark.parametrize("prec", [binding.AP_MIXED, binding.AP_FIXED])
def test_reduced_precision_reaches_tolerance(c1, oracle_c1, prec):
    o, E = oracle_c1
    tol = 1e-5
    c = _ctx(c1, prec)
    info = c.solve_diis(tol=tol, max_iter=200, depth=6)
    assert info.status == 0 and info.eps_debye <= tol
    mu = c.mu.cpu().numpy()
    assert o.residual_eps(E - o.apply_A(mu)) < 1.5 * tol
    mu_star, _ = o.pcg(E, tol=1e-10)
    assert DEBYE * np.sqrt(np.mean(np.sum((mu - mu_star) ** 2, axis=1))) < 10 * tol
    c.close()


def test_fixed_point_is_bitwise_reproducible(c1):
    out = []
    for _ in range(2):
        c = _ctx(c1, binding.AP_FIXED)
        info = c.solve_diis(tol=1e-6, max_iter=200, depth=6)
        out.append((info.iterations, c.mu.cpu().numpy().tobytes()))
        c.close()
    assert out[0] == out[1]


def test_chain_exclusions_and_global_frames(chain):
    o = Oracle(chain, Params(beta=0.5446, grid=(24, 24, 24), cutoff=7.0))
    E = o.permanent_field()
    c = _ctx(chain, binding.AP_FP64)
    info = c.solve_diis(tol=1e-6, max_iter=200, depth=6)
    mu_o, info_o = o.jacobi_diis(E, tol=1e-6, depth=6)
    assert info.iterations == info_o["iters"]
    assert _rel_max(c.mu.cpu().numpy(), mu_o) < 1e-8
    c.close()


def test_window_growth_and_argument_errors(c1, oracle_c1):
    """A longer window on a context that already holds shorter rings regrows them; bad
    arguments are rejected before any launch."""
    o, E = oracle_c1
    c = _ctx(c1, binding.AP_FP64)
    c.solve_diis(tol=1e-6, max_iter=200, depth=2)
    info = c.solve_diis(tol=1e-6, max_iter=200, depth=7)
    _, info_o = o.jacobi_diis(E, tol=1e-6, depth=7)
    assert info.iterations == info_o["iters"]
    for depth in (0, 9):
        with pytest.raises(binding.ApError):
            c.solve_diis(tol=1e-6, max_iter=10, depth=depth)
    with pytest.raises(binding.ApError):
        c.solve_diis(tol=0.0, max_iter=10, depth=4)
    c.close()


@pytest.mark.parametrize("n_mol,box,cutoff,buffer,grid", [
    (1, 11.0, 4.0, 1.5, (8, 8, 8)),        # one molecule: a single, mostly padded block
    (11, 12.0, 4.5, 1.5, (12, 10, 8)),     # 33 atoms: one full block and a 1-atom tail
])
def test_small_and_ragged(n_mol, box, cutoff, buffer, grid):
    s = synth.water_box(n_mol, box, 77 + n_mol, dmin_inter=1.6)
    c = binding.Context(s, cutoff=cutoff, buffer=buffer, beta=0.5446, grid=grid, precision=binding.AP_FP64)
    c.build()
    c.permanent_field()
    o = Oracle(s, Params(beta=0.5446, grid=grid, cutoff=cutoff))
    E = o.permanent_field()
    info = c.solve_diis(tol=1e-8, max_iter=200, depth=5)
    mu_o, info_o = o.jacobi_diis(E, tol=1e-8, depth=5)
    assert info.iterations == info_o["iters"]
    assert _rel_max(c.mu.cpu().numpy(), mu_o) < 1e-7
    c.close()
