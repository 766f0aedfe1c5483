"""Pins for the oracle's two-dipole-set methods (AMOEBA's d and p sets): the reduction to
the single-set model when both scale tables agree, a closed-form isolated pair, minus the
finite-difference gradient of E_pol = -(f/2) mu_d . E_p (which is not variational in
either set, so it checks the mu_p-weighted response terms), the identity
mu_d . E_p = mu_p . E_d that the symmetry of A implies, independence from the Ewald
splitting parameter, and a dense solve of both systems."""
import numpy as np
import pytest

from oracle import Oracle, Params, model, radial
from paper_2011_01207_gb300 import synth


@pytest.fixture(scope="module")
def chain_dp():
    s = synth.solvated_chain(9, 2, 12.0, 21)
    sd, pairs, scales = synth.dp_system(s, 5, 3, 5)
    return sd, (pairs, scales)


def _exact_params(beta):
    return Params(beta=beta, cutoff=5.6 / beta + 0.5, mode="exact", images=True)


def test_scale_table_has_every_kind(chain_dp):
    _, (pairs, scales) = chain_dp
    kinds = {tuple(x) for x in scales}
    assert {(0.0, 0.0), (0.0, 0.5), (0.0, 1.0), (1.0, 0.0)} <= kinds
    assert np.all(pairs[:, 0] < pairs[:, 1])


def test_equal_tables_reduce_to_the_single_set(water_small):
    """d and p scales both 0 on the exclusion list: both sets are the single-set model."""
    s = water_small
    dp = (s.excl, np.zeros((len(s.excl), 2)))
    p = Params(beta=0.5446, cutoff=3.7, grid=(10, 10, 10))
    o = Oracle(s, p, dp=dp)
    E = o.permanent_field()
    E_d, E_p = o.permanent_field_dp()
    tiny = 1e-14 * np.abs(E).max()
    np.testing.assert_allclose(E_d, E, rtol=0, atol=tiny)
    np.testing.assert_allclose(E_p, E, rtol=0, atol=tiny)
    mu, info = o.pcg(E, tol=1e-9)
    mu_d, mu_p, info2 = o.pcg_dp(E_d, E_p, tol=1e-9)
    assert info2["iters"] == info["iters"]
    np.testing.assert_allclose(mu_d, mu, rtol=0, atol=1e-12 * np.abs(mu).max())
    np.testing.assert_allclose(mu_p, mu, rtol=0, atol=1e-12 * np.abs(mu).max())
    assert abs(o.energy_dp(mu_d, E_p) - o.energy(mu, E)) < 1e-12 * abs(o.energy(mu, E))
    F, F2 = o.forces(mu), o.forces_dp(mu, mu)
    np.testing.assert_allclose(F2, F, rtol=0, atol=1e-12 * np.abs(F).max())


def test_isolated_pair_closed_form():
    """Two charges on z, open boundary, pair scales d = 0 and p = 1/2: E_d = 0 and E_p is
    half the Thole-damped Coulomb field, q_j R lambda_3 / r^3; mu_p follows the closed
    form of the coupled pair and mu_d = 0."""
    class S:
        pass
    r, a1, a2, q1, q2 = 2.1, 1.1, 0.7, 0.4, -0.3
    s = S()
    s.xyz = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, r]])
    s.box = np.array([100.0, 100.0, 100.0])
    s.q, s.alpha = np.array([q1, q2]), np.array([a1, a2])
    s.dip, s.quad = np.zeros((2, 3)), np.zeros((2, 6))
    s.frame = np.array([[0, -1, -1], [0, -1, -1]])
    s.excl = np.zeros((0, 2), int)
    o = Oracle(s, Params(mode="open", thole_a=0.39), dp=(np.array([[0, 1]]), np.array([[0.0, 0.5]])))
    E_d, E_p = o.permanent_field_dp()
    assert np.all(E_d == 0.0)
    l3 = 1.0 - np.exp(-0.39 * r ** 3 / np.sqrt(a1 * a2))
    E1, E2 = -0.5 * q2 * l3 / r ** 2, 0.5 * q1 * l3 / r ** 2
    np.testing.assert_allclose(E_p[:, 2], [E1, E2], rtol=1e-13)
    mu_d, mu_p, _ = o.pcg_dp(E_d, E_p, tol=1e-14)
    oml = radial.thole_one_minus_lambda(radial.thole_s(r, a1, a2, 0.39))
    t = (3 * (1 - oml[1]) - (1 - oml[0])) / r ** 3
    m1 = a1 * (E1 + t * a2 * E2) / (1 - t * t * a1 * a2)
    m2 = a2 * (E2 + t * a1 * E1) / (1 - t * t * a1 * a2)
    np.testing.assert_allclose(mu_p[:, 2], [m1, m2], rtol=1e-12)
    assert np.all(mu_d == 0.0)


def test_forces_match_finite_differences(chain_dp):
    s, dp = chain_dp
    p = Params(beta=0.5446, cutoff=5.9, grid=(12, 12, 12))
    o = Oracle(s, p, dp=dp)
    E_d, E_p = o.permanent_field_dp()
    mu_d, mu_p, _ = o.pcg_dp(E_d, E_p, tol=1e-12)
    F = o.forces_dp(mu_d, mu_p)
    h = 1e-4
    Ffd = np.zeros_like(F)
    for i in range(s.n):
        for a in range(3):
            xp, xm = s.xyz.copy(), s.xyz.copy()
            xp[i, a] += h
            xm[i, a] -= h
            Ffd[i, a] = -(model.solve_energy_dp(s, p, dp, xp, 1e-12)
                          - model.solve_energy_dp(s, p, dp, xm, 1e-12)) / (2 * h)
    np.testing.assert_allclose(F, Ffd, rtol=0, atol=1e-7 * np.abs(F).max())
    # the d/p forces differ from the single-set forces at either set
    assert np.abs(F - o.forces(mu_d)).max() > 1e-3 * np.abs(F).max()


def test_cross_energy_symmetry(chain_dp):
    s, dp = chain_dp
    o = Oracle(s, Params(beta=0.5446, cutoff=5.9, grid=(12, 12, 12)), dp=dp)
    E_d, E_p = o.permanent_field_dp()
    mu_d, mu_p, _ = o.pcg_dp(E_d, E_p, tol=1e-13)
    a, b = np.sum(mu_d * E_p), np.sum(mu_p * E_d)
    assert abs(a - b) < 1e-11 * abs(a)
    assert np.abs(E_d - E_p).max() > 1e-2 * np.abs(E_p).max()


def test_beta_independence(chain_dp):
    s, dp = chain_dp
    res = []
    for beta in (0.4, 0.5446, 0.65):
        o = Oracle(s, _exact_params(beta), dp=dp)
        E_d, E_p = o.permanent_field_dp()
        mu_d, mu_p, info = o.pcg_dp(E_d, E_p, tol=1e-12)
        assert info["converged"]
        res.append((E_d, E_p, o.energy_dp(mu_d, E_p), o.forces_dp(mu_d, mu_p)))
    Ed0, Ep0, e0, F0 = res[1]
    for Ed, Ep, e, F in res:
        np.testing.assert_allclose(Ed, Ed0, rtol=0, atol=1e-10 * np.abs(Ed0).max())
        np.testing.assert_allclose(Ep, Ep0, rtol=0, atol=1e-10 * np.abs(Ep0).max())
        assert abs(e - e0) < 1e-10 * abs(e0)
        np.testing.assert_allclose(F, F0, rtol=0, atol=1e-9 * np.abs(F0).max())


def test_lockstep_pcg_matches_dense_solves(chain_dp):
    s, dp = chain_dp
    o = Oracle(s, Params(beta=0.5446, cutoff=5.9, grid=(12, 12, 12)), dp=dp)
    E_d, E_p = o.permanent_field_dp()
    A = o.dense_A()
    mu_d, mu_p, info = o.pcg_dp(E_d, E_p, tol=1e-11)
    assert info["eps"] == max(info["eps_d"], info["eps_p"]) <= 1e-11
    np.testing.assert_allclose(mu_d.ravel(), np.linalg.solve(A, E_d.ravel()), rtol=0, atol=1e-10)
    np.testing.assert_allclose(mu_p.ravel(), np.linalg.solve(A, E_p.ravel()), rtol=0, atol=1e-10)


def test_scale_table_follows_its_definition():
    """Every chain pair's (d, p) scales against the rule written out pair by pair: d = 0
    inside a polarization group; p = 0 at bond separation 1 or 2, 1/2 at separation 3
    inside a group, 1 otherwise; waters: both 0 inside a molecule. Pairs absent from the
    table must have (1, 1)."""
    s = synth.solvated_chain(14, 3, 14.0, 77)
    pairs, scales = synth.dp_scales(s, synth.polarization_groups(s, 4, 3, 6))
    table = {(int(a), int(b)): tuple(v) for (a, b), v in zip(pairs, scales)}
    g = synth.polarization_groups(s, 4, 3, 6)
    chain = [i for i in range(s.n) if s.rigid[i] == 0]
    for x in range(s.n):
        for y in range(x + 1, s.n):
            if x in chain and y in chain:
                sep = abs(chain.index(x) - chain.index(y))
                same = g[x] == g[y]
                d = 0.0 if same else 1.0
                p = 0.0 if sep <= 2 else (0.5 if sep == 3 and same else 1.0)
            elif s.mol[x] == s.mol[y] and s.rigid[x] == 1:
                d, p = 0.0, 0.0
            else:
                d, p = 1.0, 1.0
            assert table.get((x, y), (1.0, 1.0)) == (d, p), (x, y)
