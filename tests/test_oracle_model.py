"""Pins for the oracle's field, operator, solver, energy and forces.

Each check is fixed by mathematics, not by the oracle itself: independence of the total
from the Ewald splitting parameter, minus the finite-difference gradient of the energy,
zero net force and rotation invariance of the exact Ewald sum, the closed-form induced
dipoles of an isolated Thole-damped pair, a dense solve, symmetry and definiteness of A,
and the variational property of the energy."""
import numpy as np
import pytest

from oracle import Oracle, Params, model, radial
from oracle.model import F_COUL


def _exact_params(beta):
    return Params(beta=beta, cutoff=5.6 / beta + 0.5, mode="exact", images=True)


def test_beta_independence(water_small):
    res = []
    for beta in (0.35, 0.45, 0.5446, 0.65):
        o = Oracle(water_small, _exact_params(beta))
        E = o.permanent_field()
        mu, info = o.pcg(E, tol=1e-12)
        assert info["converged"]
        res.append((E, o.energy(mu, E), o.forces(mu)))
    E0, e0, F0 = res[2]
    for E, e, F in res:
        np.testing.assert_allclose(E, E0, rtol=0, atol=1e-10 * np.abs(E0).max())
        assert abs(e - e0) < 1e-10 * abs(e0)
        np.testing.assert_allclose(F, F0, rtol=0, atol=1e-10 * np.abs(F0).max())


def _fd_forces(sysobj, params, h=1e-4):
    F = np.zeros_like(sysobj.xyz)
    for i in range(sysobj.n):
        for a in range(3):
            xp = sysobj.xyz.copy()
            xm = sysobj.xyz.copy()
            xp[i, a] += h
            xm[i, a] -= h
            F[i, a] = -(model.solve_energy(sysobj, params, xp, 1e-12)
                        - model.solve_energy(sysobj, params, xm, 1e-12)) / (2 * h)
    return F


@pytest.mark.parametrize("mode", ["exact", "spme"])
def test_forces_match_finite_differences(water_small, mode):
    from paper_2011_01207_gb300 import synth
    s = synth.water_box(2, 7.5, 11, dmin_inter=1.9) if mode == "exact" else water_small
    p = _exact_params(0.5446) if mode == "exact" else Params(beta=0.5446, cutoff=3.7, grid=(10, 10, 10))
    o = Oracle(s, p)
    E = o.permanent_field()
    mu, _ = o.pcg(E, tol=1e-12)
    F = o.forces(mu)
    Ffd = _fd_forces(s, p)
    np.testing.assert_allclose(F, Ffd, rtol=0, atol=1e-7 * np.abs(F).max())
    if mode == "exact":
        np.testing.assert_allclose(F.sum(0), 0.0, atol=1e-12 * np.abs(F).max())


def test_chain_atoms_forces_match_finite_differences():
    """Global-frame chain atoms with 1-2 / 1-3 exclusions next to waters."""
    from paper_2011_01207_gb300 import synth
    s = synth.solvated_chain(5, 2, 12.0, 21)
    p = Params(beta=0.5446, cutoff=5.9, grid=(12, 12, 12))
    o = Oracle(s, p)
    E = o.permanent_field()
    mu, _ = o.pcg(E, tol=1e-12)
    F = o.forces(mu)
    np.testing.assert_allclose(F, _fd_forces(s, p), rtol=0, atol=1e-7 * np.abs(F).max())


def test_rotation_invariance_exact(water_small):
    """A 90-degree rotation about z maps the cubic lattice onto itself; the waters'
    local frames rotate with them, so the energy must not change."""
    p = _exact_params(0.5446)
    o = Oracle(water_small, p)
    E = o.permanent_field()
    mu, _ = o.pcg(E, tol=1e-12)
    e0 = o.energy(mu, E)
    x = water_small.xyz
    rot = np.stack([-x[:, 1], x[:, 0], x[:, 2]], 1)
    o2 = Oracle(water_small, p, xyz=rot)
    E2 = o2.permanent_field()
    mu2, _ = o2.pcg(E2, tol=1e-12)
    assert abs(o2.energy(mu2, E2) - e0) < 1e-11 * abs(e0)
    np.testing.assert_allclose(mu2[:, 0], -mu[:, 1], atol=1e-10)
    np.testing.assert_allclose(mu2[:, 1], mu[:, 0], atol=1e-10)


def test_isolated_damped_pair_closed_form():
    """Two charges on z, open boundary: mu_1z = alpha_1 (E_1 + t alpha_2 E_2) /
    (1 - t^2 alpha_1 alpha_2) with the axial coupling t = (3 lambda_5 - lambda_3)/r^3."""
    class S:
        pass
    for r, a1, a2, q1, q2 in ((2.3, 1.1, 0.7, 0.4, -0.3), (1.6, 0.837, 0.496, -0.5, 0.25)):
        s = S()
        s.xyz = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, r]])
        s.box = np.array([100.0, 100.0, 100.0])
        s.q, s.alpha = np.array([q1, q2]), np.array([a1, a2])
        s.dip, s.quad = np.zeros((2, 3)), np.zeros((2, 6))
        s.frame = np.array([[0, -1, -1], [0, -1, -1]])
        s.excl = np.zeros((0, 2), int)
        o = Oracle(s, Params(mode="open", thole_a=0.39))
        mu, _ = o.pcg(o.permanent_field(), tol=1e-14)
        oml = radial.thole_one_minus_lambda(radial.thole_s(r, a1, a2, 0.39))
        l3, l5 = 1 - oml[0], 1 - oml[1]
        t = (3 * l5 - l3) / r ** 3
        E1, E2 = -q2 * r * l3 / r ** 3, q1 * r * l3 / r ** 3
        m1 = a1 * (E1 + t * a2 * E2) / (1 - t * t * a1 * a2)
        m2 = a2 * (E2 + t * a1 * E1) / (1 - t * t * a1 * a2)
        np.testing.assert_allclose(mu[:, 2], [m1, m2], rtol=1e-12)
        np.testing.assert_allclose(mu[:, :2], 0.0, atol=1e-15)


def test_dense_solve_symmetry_definiteness(water_small):
    p = Params(beta=0.5446, cutoff=3.7, grid=(10, 10, 10))
    o = Oracle(water_small, p)
    A = o.dense_A()
    np.testing.assert_allclose(A, A.T, rtol=0, atol=1e-12 * np.abs(A).max())
    np.linalg.cholesky(A)                                   # SPD
    E = o.permanent_field()
    mu_dense = np.linalg.solve(A, E.ravel()).reshape(-1, 3)
    mu, info = o.pcg(E, tol=1e-12)
    np.testing.assert_allclose(mu, mu_dense, rtol=0, atol=1e-11)
    # PCG in exact arithmetic needs at most 3N iterations
    assert info["iters"] <= 3 * o.n


def test_energy_is_variational_minimum(water_small):
    p = Params(beta=0.5446, cutoff=3.7, grid=(10, 10, 10))
    o = Oracle(water_small, p)
    E = o.permanent_field()
    mu, _ = o.pcg(E, tol=1e-13)

    def g(m):
        return F_COUL * (0.5 * np.sum(m * o.apply_A(m)) - np.sum(m * E))
    e = o.energy(mu, E)
    assert abs(g(mu) - e) < 1e-10 * abs(e)
    rng = np.random.default_rng(0)
    for _ in range(3):
        d = rng.normal(size=mu.shape) * 1e-3
        assert g(mu + d) > e


def test_pcg_residual_is_true_residual():
    from paper_2011_01207_gb300 import synth
    s = synth.water_box(216, 18.64, 1001)
    o = Oracle(s, Params(beta=0.5446, cutoff=7.0, grid=(24, 24, 24)))
    E = o.permanent_field()
    mu, info = o.pcg(E, tol=1e-6)
    assert info["converged"] and 5 <= info["iters"] <= 30
    assert o.residual_eps(E - o.apply_A(mu)) < 1.01e-6


def test_row_fields_match_full_oracle():
    from paper_2011_01207_gb300 import synth
    s = synth.water_box(64, 12.5, 5)
    p = Params(beta=0.5446, cutoff=6.0, grid=(16, 16, 16))
    o = Oracle(s, p)
    v = np.random.default_rng(1).normal(size=(s.n, 3))
    rows = np.array([0, 7, 100, s.n - 1])
    Er, Tv = model.row_fields(s, p, rows, v)
    np.testing.assert_allclose(Er, o.permanent_field()[rows], rtol=0, atol=1e-12)
    np.testing.assert_allclose(Tv, o.apply_T(v)[rows], rtol=0, atol=1e-12)


def test_two_readings_of_the_threshold():
    """The alpha-weighted measure (the stopping rule) and the unweighted field residual
    differ per atom by the factor 1/alpha_i, so their ratio lies in [1/max alpha,
    1/min alpha]; and the PCG's recursive residual is the true one, so the field reading
    of a tightly converged solve is tiny too."""
    from paper_2011_01207_gb300 import synth
    s = synth.water_box(27, 9.3, 11)
    o = Oracle(s, Params(beta=0.5446, cutoff=4.5, grid=(12, 12, 12)))
    E = o.permanent_field()
    for tol in (1e-3, 1e-5, 1e-10):
        mu, info = o.pcg(E, tol=tol)
        ea = o.residual_eps(E - o.apply_A(mu))
        ratio = info["eps_field"] / ea
        assert 1 / s.alpha.max() - 1e-9 <= ratio <= 1 / s.alpha.min() + 1e-9
        assert info["eps_field"] < 3 * tol / s.alpha.min()
