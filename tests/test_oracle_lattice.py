"""Pins of the oracle's Ewald machinery against sums that use no Ewald splitting at all:

  * the spherical lattice sum: adding whole image cells in order of |n| (Thole-damped
    multipole fields written out from their textbook form, intramolecular pairs of the
    central cell left out) converges to the exact-Ewald field minus (4 pi / 3V) M, M the
    cell's dipole moment sum(q x + d) - the tin-foil / vacuum-sphere shape term - and
    likewise for the field of arbitrary dipoles, T v;
  * the smooth-PME convolution against the plain discrete Fourier sum on a small grid
    (sign and normalisation of the transforms);
  * the closed-form induced dipoles of an isolated Thole-damped pair, reproduced by the
    periodic smooth-PME path in a 200 A box within the 1/L^3 size of the image terms.
A dropped shape term, a wrong transform sign or scale, or a wrong Ewald split of any
multipole order fails one of these."""
import numpy as np

from oracle import Oracle, Params, radial, spme


def _damped_multipole_field(R, q, d, Q, ai, aj, a=0.39):
    """Field at R from (q, d, Q), phi = q/r + d.R/r^3 + R.Q.R/r^5, with the 1/r^3, 1/r^5,
    1/r^7 terms scaled by Thole's lambda_3, lambda_5, lambda_7 (s = a r^3 / sqrt(ai aj))."""
    r = np.sqrt(np.einsum("pa,pa->p", R, R))
    s = a * r ** 3 / np.sqrt(ai * aj)
    e = np.exp(-s)
    l3, l5, l7 = 1 - e, 1 - (1 + s) * e, 1 - (1 + s + 0.6 * s * s) * e
    dR = np.einsum("pa,pa->p", d, R)
    QR = np.einsum("pab,pb->pa", Q, R)
    RQR = np.einsum("pa,pa->p", QR, R)
    return ((q * l3 / r ** 3 + 3 * l5 * dR / r ** 5 + 5 * l7 * RQR / r ** 7)[:, None] * R
            - (l3 / r ** 3)[:, None] * d - (2 * l5 / r ** 5)[:, None] * QR)


def _spherical_sum(x, L, q, d, Q, alpha, skip, R_cells):
    """sum over image cells n with |n| <= R_cells (whole cells) and atoms j of the damped
    field at atom i, leaving out i = j and the pairs in `skip` within the central cell."""
    n = len(x)
    ii, jj = (a.ravel() for a in np.meshgrid(np.arange(n), np.arange(n), indexing="ij"))
    keep0 = (ii != jj) & ~skip[ii, jj]
    base = x[ii] - x[jj]
    c = np.stack(np.meshgrid(*[np.arange(-R_cells, R_cells + 1)] * 3, indexing="ij"), -1).reshape(-1, 3)
    c = c[np.einsum("ca,ca->c", c, c) <= R_cells * R_cells]
    E = np.zeros((n, 3))
    for cell in c:
        sel = keep0 if not cell.any() else np.ones_like(keep0)
        R = base[sel] + cell * L
        np.add.at(E, ii[sel], _damped_multipole_field(R, q[jj[sel]], d[jj[sel]], Q[jj[sel]],
                                                       alpha[ii[sel]], alpha[jj[sel]]))
    return E


def test_spherical_lattice_sum_of_field_and_operator(water_small):
    s = water_small
    o = Oracle(s, Params(beta=0.5446, cutoff=5.6 / 0.5446 + 0.5, mode="exact", images=True))
    L, V, n = o.box, float(np.prod(o.box)), o.n
    skip = np.zeros((n, n), bool)
    ex = np.asarray(s.excl)
    skip[ex[:, 0], ex[:, 1]] = skip[ex[:, 1], ex[:, 0]] = True
    # permanent field: intramolecular pairs of the central cell left out
    E_ex = o.permanent_field()
    M = np.einsum("j,ja->a", o.q, o.xyz) + o.dip.sum(0)
    want = E_ex - (4 * np.pi / (3 * V)) * M
    got = _spherical_sum(o.xyz, L, o.q, o.dip, o.quad, o.alpha, skip, 20)
    scale = np.abs(want).max()
    assert np.abs((4 * np.pi / (3 * V)) * M).max() > 0.05 * scale          # the shape term matters
    np.testing.assert_allclose(got, want, rtol=0, atol=2e-6 * scale)
    # the dipole-field operator: every pair at scale 1, so only i = j is left out
    v = np.random.default_rng(4).normal(size=(n, 3)) * 0.1
    Tv = o.apply_T(v)
    want = Tv - (4 * np.pi / (3 * V)) * v.sum(0)
    got = _spherical_sum(o.xyz, L, np.zeros(n), v, np.zeros((n, 3, 3)), o.alpha, np.zeros((n, n), bool), 20)
    np.testing.assert_allclose(got, want, rtol=0, atol=2e-6 * np.abs(want).max())


def test_convolution_against_the_plain_dft():
    """phi_k = sum_m G(m) Q^(m) exp(+2 pi i m.k/K) with Q^(m) = sum_k' Q_k' exp(-2 pi i m.k'/K)."""
    K, box, beta = (4, 5, 6), np.array([6.0, 7.0, 8.0]), 0.6
    rng = np.random.default_rng(2)
    grid = rng.normal(size=K)
    G = spme.influence(box, K, 5, beta)
    ks = np.stack(np.meshgrid(*[np.arange(k) for k in K], indexing="ij"), -1).reshape(-1, 3)
    ph = np.exp(-2j * np.pi * (ks / np.array(K)) @ ks.T)                  # [m, k']
    Qm = ph @ grid.ravel()
    phi = np.real(np.conj(ph).T @ (G.ravel() * Qm))
    np.testing.assert_allclose(spme.convolve(grid, box, K, 5, beta).ravel(), phi, rtol=0,
                               atol=1e-12 * np.abs(phi).max())


def test_isolated_pair_in_a_large_periodic_box():
    """Two polarizable charges 2.3 A apart on z in a 200 A box (smooth PME, beta 0.1,
    grid 80^3): the induced dipoles equal the open-boundary closed form up to the fields
    of the periodic images, of order (4 pi / 3V) |p| with p ~ 0.7 e A the pair's dipole:
    about 6e-6 of the pair's own field (measured 4.5e-6), inside the 1e-5 margin."""
    class S:
        pass
    r, a1, a2, q1, q2 = 2.3, 1.1, 0.7, 0.4, -0.3
    s = S()
    s.xyz = np.array([[100.0, 100.0, 100.0], [100.0, 100.0, 100.0 + r]])
    s.box = np.array([200.0, 200.0, 200.0])
    s.q, s.alpha = np.array([q1, q2]), np.array([a1, a2])
    s.dip, s.quad = np.zeros((2, 3)), np.zeros((2, 6))
    s.frame = np.array([[0, -1, -1], [0, -1, -1]])
    s.excl = np.zeros((0, 2), int)
    o = Oracle(s, Params(beta=0.1, cutoff=60.0, grid=(80, 80, 80), thole_a=0.39))
    mu, _ = o.pcg(o.permanent_field(), tol=1e-14)
    oml = radial.thole_one_minus_lambda(radial.thole_s(r, a1, a2, 0.39))
    l3, l5 = 1 - oml[0], 1 - oml[1]
    t = (3 * l5 - l3) / r ** 3
    E1, E2 = -q2 * l3 / r ** 2, q1 * l3 / r ** 2
    m1 = a1 * (E1 + t * a2 * E2) / (1 - t * t * a1 * a2)
    m2 = a2 * (E2 + t * a1 * E1) / (1 - t * t * a1 * a2)
    np.testing.assert_allclose(mu[:, 2], [m1, m2], rtol=1e-5)
    np.testing.assert_allclose(mu[:, :2], 0.0, atol=1e-6 * abs(m1))
