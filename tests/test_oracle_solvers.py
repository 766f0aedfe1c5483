"""Pins of the oracle's Jacobi/DIIS solver against mathematics that does not share its
code: the dense Jacobi iteration, a least-squares solution of the DIIS minimisation with
the constraint eliminated, the dense linear solve, and the identity e_k = alpha r_k that
makes its convergence measure the PCG's."""
import numpy as np
import pytest

from oracle import Oracle, Params
from paper_2011_01207_gb300 import synth


@pytest.fixture(scope="module")
def small():
    s = synth.water_box(8, 12.0, 5, dmin_inter=1.6)
    o = Oracle(s, Params(beta=0.5446, grid=(12, 12, 12), cutoff=5.0))
    E = o.permanent_field()
    A = o.dense_A()
    return s, o, E, A


def test_depth_one_is_dense_jacobi(small):
    s, o, E, A = small
    a = np.repeat(s.alpha, 3)
    T = np.diag(1.0 / a) - A
    x = a * E.ravel()
    for k in range(1, 5):
        x = a * (E.ravel() + T @ x)
        mu, info = o.jacobi_diis(E, tol=0.0, depth=1, maxiter=k)
        assert info["iters"] == k
        assert np.allclose(mu.ravel(), x, rtol=0, atol=1e-12)


def test_diis_steps_against_constraint_eliminated_least_squares(small):
    """The oracle's first three DIIS steps (depth 3), rebuilt with dense T and, for each
    window, c = (1 - sum d, d) with d from an unconstrained least-squares fit."""
    s, o, E, A = small
    a = np.repeat(s.alpha, 3)
    T = np.diag(1.0 / a) - A
    g = lambda x: a * (E.ravel() + T @ x)
    x = a * E.ravel()
    ys, es = [], []
    for k in range(3):
        y = g(x)
        ys.append(y)
        es.append(y - x)
        if len(es) == 1:
            c = np.array([1.0])
        else:
            M = np.stack([e - es[0] for e in es[1:]], 1)
            d, *_ = np.linalg.lstsq(M, -es[0], rcond=None)
            c = np.r_[1.0 - d.sum(), d]
        x = sum(ci * yi for ci, yi in zip(c, ys))
        mu, info = o.jacobi_diis(E, tol=0.0, depth=3, maxiter=k + 1)
        assert info["iters"] == k + 1
        assert np.allclose(mu.ravel(), x, rtol=0, atol=1e-11)


def test_converges_to_the_dense_solution_with_the_pcg_measure(small):
    s, o, E, A = small
    mu_star = np.linalg.solve(A, E.ravel()).reshape(-1, 3)
    for depth in (1, 4, 8):
        mu, info = o.jacobi_diis(E, tol=1e-10, depth=depth)
        assert info["converged"]
        assert np.abs(mu - mu_star).max() < 1e-9
        assert abs(info["eps"] - o.residual_eps(E - o.apply_A(mu))) < 1e-12 + 1e-9 * info["eps"]
    _, i1 = o.jacobi_diis(E, tol=1e-8, depth=1)
    _, i6 = o.jacobi_diis(E, tol=1e-8, depth=6)
    assert i6["iters"] < i1["iters"]
