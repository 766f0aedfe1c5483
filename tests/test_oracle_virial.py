"""Pins of the oracle's polarization virial V_ab = dE_pol/de_ab (homogeneous deformation
x -> (I + e) x of positions and box, dipoles re-solved), against facts that do not share
its code:
  * an isolated cluster: V = sum_i x_i (dE/dx_i)^T exactly, from the (separately pinned)
    forces, all nine components;
  * periodic boxes: the diagonal equals the central finite difference of the re-solved
    energy under a stretch of one box side with the positions, in exact-Ewald and
    smooth-PME modes, water and a chain with global-frame atoms;
  * the total does not depend on the Ewald splitting parameter (every component);
  * with every multipole carried by a local frame the energy is rotation invariant, so V
    is symmetric (a transposed term breaks this);
  * the two-dipole-set virial: the same finite differences and symmetry, and with equal
    d and p tables it is the single-set virial.
A dropped term (pair, frame, structure-factor or multipole-component share) fails the
finite differences or the cluster identity; a transposed one fails the symmetry."""
import numpy as np
import pytest

from oracle import Oracle, Params, model
from paper_2011_01207_gb300 import synth


class _Cfg:
    """The same molecules at other positions and box (for strained copies)."""

    def __init__(self, s, xyz, box):
        for k in ("q", "alpha", "dip", "quad", "frame", "excl", "n"):
            setattr(self, k, getattr(s, k))
        self.xyz = np.asarray(xyz, np.float64)
        self.box = np.asarray(box, np.float64)


def _solved(s, p, dp=None):
    o = Oracle(s, p, dp=dp)
    if dp is None:
        E = o.permanent_field()
        mu, _ = o.pcg(E, tol=1e-12, maxiter=2000)
        return o, mu
    E_d, E_p = o.permanent_field_dp()
    mu_d, mu_p, _ = o.pcg_dp(E_d, E_p, tol=1e-12, maxiter=2000)
    return o, (mu_d, mu_p)


def _fd_diagonal(s, p, dp=None, h=1e-5):
    out = []
    for a in range(3):
        e = []
        for sign in (1.0, -1.0):
            sc = np.ones(3)
            sc[a] += sign * h
            c = _Cfg(s, s.xyz * sc, np.asarray(s.box) * sc)
            e.append(model.solve_energy(c, p, tol=1e-12) if dp is None
                     else model.solve_energy_dp(c, p, dp, tol=1e-12))
        out.append((e[0] - e[1]) / (2 * h))
    return np.array(out)


def _exact(beta):
    return Params(beta=beta, cutoff=5.6 / beta + 0.5, mode="exact", images=True)


@pytest.mark.parametrize("kind", ["water", "chain"])
def test_isolated_cluster_virial_is_position_times_gradient(water_small, kind):
    s = water_small if kind == "water" else synth.solvated_chain(5, 2, 12.0, 21)
    c = _Cfg(s, s.xyz, (100.0, 100.0, 100.0))
    o, mu = _solved(c, Params(mode="open"))
    V = o.virial(mu)
    want = np.einsum("ia,ib->ab", -o.forces(mu), c.xyz)
    np.testing.assert_allclose(V, want, rtol=0, atol=1e-11 * np.abs(want).max())


@pytest.mark.parametrize("case", ["exact_water", "spme_water", "spme_chain"])
def test_diagonal_matches_finite_differences(water_small, case):
    if case == "exact_water":
        s, p = synth.water_box(2, 7.5, 11, dmin_inter=1.9), _exact(0.5446)
    elif case == "spme_water":
        s, p = water_small, Params(beta=0.5446, cutoff=3.7, grid=(10, 10, 10))
    else:
        s, p = synth.solvated_chain(5, 2, 12.0, 21), Params(beta=0.5446, cutoff=5.9, grid=(12, 12, 12))
    o, mu = _solved(s, p)
    V = o.virial(mu)
    fd = _fd_diagonal(s, p)
    np.testing.assert_allclose(np.diag(V), fd, rtol=0, atol=1e-7 * np.abs(V).max())


def test_beta_independence_every_component(water_small):
    Vs = []
    for beta in (0.35, 0.45, 0.5446, 0.65):
        o, mu = _solved(water_small, _exact(beta))
        Vs.append(o.virial(mu))
    for V in Vs:
        np.testing.assert_allclose(V, Vs[2], rtol=0, atol=1e-10 * np.abs(Vs[2]).max())


@pytest.mark.parametrize("mode", ["exact", "spme"])
def test_symmetric_when_every_multipole_is_framed(water_small, mode):
    p = _exact(0.5446) if mode == "exact" else Params(beta=0.5446, cutoff=3.7, grid=(10, 10, 10))
    o, mu = _solved(water_small, p)
    V = o.virial(mu)
    np.testing.assert_allclose(V, V.T, rtol=0, atol=1e-11 * np.abs(V).max())
    assert np.abs(V - np.diag(np.diag(V))).max() > 1e-3 * np.abs(V).max()   # off-diagonals not trivially 0


def _water_dp(s):
    """Intramolecular pairs with d-scale 0 and seeded p-scales in (0.2, 0.8)."""
    pairs = np.asarray(s.excl)
    rng = np.random.default_rng(1)
    return pairs, np.stack([np.zeros(len(pairs)), rng.uniform(0.2, 0.8, len(pairs))], 1)


def test_two_sets_diagonal_matches_finite_differences():
    s0 = synth.solvated_chain(5, 2, 12.0, 21)
    s, pairs, scales = synth.dp_system(s0, 11, 3, 5)
    p = Params(beta=0.5446, cutoff=5.9, grid=(12, 12, 12))
    o, (mu_d, mu_p) = _solved(s, p, dp=(pairs, scales))
    V = o.virial_dp(mu_d, mu_p)
    fd = _fd_diagonal(s, p, dp=(pairs, scales))
    np.testing.assert_allclose(np.diag(V), fd, rtol=0, atol=1e-7 * np.abs(V).max())


def test_two_sets_symmetric_and_reduce_to_one_set(water_small):
    p = Params(beta=0.5446, cutoff=3.7, grid=(10, 10, 10))
    pairs, scales = _water_dp(water_small)
    o, (mu_d, mu_p) = _solved(water_small, p, dp=(pairs, scales))
    assert np.abs(mu_d - mu_p).max() > 1e-3 * np.abs(mu_p).max()
    V = o.virial_dp(mu_d, mu_p)
    np.testing.assert_allclose(V, V.T, rtol=0, atol=1e-11 * np.abs(V).max())
    # equal tables (the context's exclusions with both scales 0): the single-set virial
    eq = (np.asarray(water_small.excl), np.zeros((len(water_small.excl), 2)))
    o2, (md2, mp2) = _solved(water_small, p, dp=eq)
    o1, mu1 = _solved(water_small, p)
    np.testing.assert_allclose(o2.virial_dp(md2, mp2), o1.virial(mu1), rtol=0,
                               atol=1e-10 * np.abs(o1.virial(mu1)).max())
