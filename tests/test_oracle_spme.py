"""Pins for the oracle's reciprocal sums: B-spline identities, the rock-salt Madelung
constant through both reciprocal modes, SPME convergence to the exact Ewald sum at the
rate of its B-spline order, and exact invariance under a whole-grid-cell translation."""
import json
import os

import numpy as np
import pytest

from oracle import Oracle, Params, ewald, spme

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_bspline_values_and_partition():
    # M_5 at the integers 1..4 is (1, 11, 11, 1)/24 (cardinal B-spline of order 5)
    np.testing.assert_allclose(spme.cardinal_bspline(5, np.arange(1.0, 5.0)),
                               np.array([1, 11, 11, 1]) / 24.0, rtol=1e-15)
    w = np.linspace(0, 1, 11, endpoint=False)
    t = np.arange(5)
    vals = spme.cardinal_bspline(5, w[:, None] + t[None, :])
    np.testing.assert_allclose(vals.sum(1), 1.0, rtol=1e-14)
    for k in (1, 2, 3):
        d = spme.cardinal_bspline_deriv(5, w[:, None] + t[None, :], k)
        np.testing.assert_allclose(d.sum(1), 0.0, atol=1e-13)
    # derivative vs central difference
    x = np.linspace(0.3, 4.7, 9)
    h = 1e-6
    for k in (1, 2, 3):
        fd = (spme.cardinal_bspline_deriv(5, x + h, k - 1) - spme.cardinal_bspline_deriv(5, x - h, k - 1)) / (2 * h)
        np.testing.assert_allclose(spme.cardinal_bspline_deriv(5, x, k), fd, rtol=1e-6, atol=1e-8)


def test_moduli_singular_point():
    b = spme.bspline_moduli(24, 5)
    assert np.all(np.isfinite(b)) and np.all(b > 0)
    assert b[12] == pytest.approx(0.5 * (b[11] + b[13]))
    assert b[0] == pytest.approx(1.0)                  # sum of M_5 at the integers is 1


def _rock_salt():
    class S:
        pass
    s = S()
    f = np.array([[0, 0, 0], [1, 1, 0], [1, 0, 1], [0, 1, 1]], float)
    s.xyz = np.concatenate([f, f + np.array([1.0, 0, 0])])
    s.box = np.array([2.0, 2.0, 2.0])
    s.q = np.array([1.0] * 4 + [-1.0] * 4)
    s.dip = np.zeros((8, 3))
    s.quad = np.zeros((8, 6))
    s.alpha = np.ones(8)
    s.frame = np.tile(np.array([0, -1, -1]), (8, 1))
    s.excl = np.zeros((0, 2), int)
    return s


@pytest.mark.parametrize("mode", ["exact", "spme"])
def test_madelung_rock_salt(mode):
    with open(os.path.join(GOLDEN, "madelung_rock_salt.json")) as fh:
        want = json.load(fh)["madelung_nearest_neighbour"]
    s = _rock_salt()
    grid = (32, 32, 32)
    o = Oracle(s, Params(beta=2.0, cutoff=3.6, grid=grid, mode=mode, images=True))
    phi = o.charge_potential()
    # potential at a cation, nearest-neighbour distance 1: -M
    tol = 1e-9 if mode == "exact" else 1e-6
    np.testing.assert_allclose(-phi[:4], want, rtol=tol)
    np.testing.assert_allclose(phi[4:], want, rtol=tol)


def test_spme_converges_to_exact_at_spline_order(water_small):
    """Charges and dipoles: doubling K cuts the SPME field error by ~2^5 (order 5)."""
    o = Oracle(water_small, Params(mode="exact", cutoff=3.7))
    z3, z33 = np.zeros((o.n, 3)), np.zeros((o.n, 3, 3))
    for q, d in ((o.q, z3), (0 * o.q, o.dip)):
        ex = ewald.recip_derivs(o.xyz, o.box, 0.5446, q, d, z33, 1)[1]
        errs = []
        for K in (10, 20):
            sp = spme.recip_derivs(o.xyz, o.box, 0.5446, (K, K, K), 5, q, d, z33, 1)[1]
            errs.append(np.sqrt(np.mean((sp - ex) ** 2) / np.mean(ex ** 2)))
        assert errs[1] < 3e-4
        assert errs[0] / errs[1] > 16.0


def test_spme_grid_translation_invariance(water_small):
    """Moving every atom by one grid spacing shifts the grid: identical field and energy."""
    p = Params(beta=0.5446, cutoff=3.7, grid=(10, 12, 14), mode="spme")
    o1 = Oracle(water_small, p)
    E1 = o1.permanent_field()
    shift = water_small.box / np.array(p.grid) * np.array([1, 2, -3])
    o2 = Oracle(water_small, p, xyz=water_small.xyz + shift)
    E2 = o2.permanent_field()
    np.testing.assert_allclose(E2, E1, rtol=0, atol=1e-12 * np.abs(E1).max())
