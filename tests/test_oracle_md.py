"""Pins of the oracle's minimal rigid-water MD (oracle/md.py) against facts that do not share
its code: the force-shifted Lennard-Jones pair's closed form (minimum -eps at 2^(1/6) sigma
before the shift, zero energy and force at the cutoff) and forces equal to minus the
finite-difference gradient of the energy; the constraints hold after SHAKE and the
constrained relative velocities are orthogonal to the bonds after RATTLE; velocity Verlet
conserves the total energy with an error that shrinks as dt^2 (halving dt cuts it ~4x; a
wrong kick factor breaks this), runs backwards to its start when the velocities are
reversed, and keeps the total momentum under pairwise forces; with the polarization forces
of the model the total energy is conserved too (a sign or unit error in those forces, or
in their use, would heat or cool the system)."""
import numpy as np

from oracle import Oracle, Params, md
from paper_2011_01207_gb300 import synth

EPS_O, SIG_O = 0.1521, 3.1507


def _lj_params(n):
    eps = np.zeros(n)
    sig = np.ones(n)
    eps[0::3] = EPS_O
    sig[0::3] = SIG_O
    return eps, sig


def test_lj_pair_closed_form():
    rc = 6.0
    rmin = 2.0 ** (1.0 / 6.0) * SIG_O
    V, F = md.lj_pair(np.array([rmin, rc]), EPS_O, SIG_O, rc)
    Vc, Fc = md.lj_pair(np.array([rc]), EPS_O, SIG_O, 1e9)      # unshifted values at rc
    Vc = Vc + 0.0   # (shift at a huge cutoff is negligible)
    s6 = (SIG_O / rc) ** 6
    F_rc = 24 * EPS_O * (2 * s6 * s6 - s6) / rc
    V_rc = 4 * EPS_O * (s6 * s6 - s6)
    assert abs(V[0] - (-EPS_O - V_rc + (rmin - rc) * F_rc)) < 1e-12
    assert abs(F[0] - (0.0 - F_rc)) < 1e-12
    assert abs(V[1]) < 1e-15 and abs(F[1]) < 1e-15
    r = np.linspace(2.8, 5.9, 50)
    h = 1e-6
    Vp, _ = md.lj_pair(r + h, EPS_O, SIG_O, rc)
    Vm, _ = md.lj_pair(r - h, EPS_O, SIG_O, rc)
    _, Fr = md.lj_pair(r, EPS_O, SIG_O, rc)
    np.testing.assert_allclose(Fr, -(Vp - Vm) / (2 * h), rtol=1e-6, atol=1e-9)


def test_lj_forces_are_minus_gradient():
    s = synth.water_box(27, 10.5, 31, dmin_inter=1.9)
    eps, sig = _lj_params(s.n)
    U, F = md.lj_energy_forces(s.xyz, s.box, eps, sig, 5.0)
    rng = np.random.default_rng(2)
    h = 1e-6
    for i in rng.choice(np.arange(0, s.n, 3), 6, replace=False):
        for c in range(3):
            xp, xm = s.xyz.copy(), s.xyz.copy()
            xp[i, c] += h
            xm[i, c] -= h
            d = (md.lj_energy_forces(xp, s.box, eps, sig, 5.0)[0] - md.lj_energy_forces(xm, s.box, eps, sig, 5.0)[0]) / (2 * h)
            assert abs(F[i, c] + d) < 1e-6 * max(1.0, abs(d))
    assert np.abs(F.sum(axis=0)).max() < 1e-12 * np.abs(F).max() * s.n


def _lj_run(dt, steps, n_mol=64, box=13.0, T=300.0):
    s = synth.water_box(n_mol, box, 41)
    eps, sig = _lj_params(s.n)
    m = md.water_masses(s.n)
    mol, lengths = md.water_constraints(s)
    v0 = md.rattle(synth.water_velocities(s, T, 5), s.xyz, mol, lengths, 1.0 / m)
    force = lambda x: md.lj_energy_forces(x, s.box, eps, sig, 6.0)
    return s, m, mol, lengths, md.run(s.xyz.copy(), v0, m, dt, steps, force, mol, lengths), force


def test_constraints_hold():
    s, m, mol, lengths, (xs, vs, es), _ = _lj_run(1.0, 10)
    for x, v in zip(xs, vs):
        for a, b, k in md.PAIRS:
            r = x[mol[:, a]] - x[mol[:, b]]
            assert np.abs(np.linalg.norm(r, axis=1) - lengths[k]).max() < 1e-9
            assert np.abs(np.einsum("ij,ij->i", r, v[mol[:, a]] - v[mol[:, b]])).max() < 1e-9


def test_energy_error_scales_as_dt_squared_and_momentum_is_kept():
    *_, (x1, v1, e1), _ = _lj_run(1.0, 100)
    s, m, *_ , (x2, v2, e2), _ = _lj_run(0.5, 200)
    err1 = np.abs(e1 - e1[0]).max()
    err2 = np.abs(e2 - e2[0]).max()
    kin = md.kinetic(v1[0], m)
    assert err1 < 2e-3 * kin
    assert 2.5 < err1 / err2 < 6.0, (err1, err2)
    p = np.einsum("i,tij->tj", m, v2)
    assert np.abs(p - p[0]).max() < 1e-10 * np.abs(m[:, None] * v2[0]).sum()


def test_time_reversible():
    s, m, mol, lengths, (xs, vs, es), force = _lj_run(1.0, 30)
    xb, vb, _ = md.run(xs[-1].copy(), -vs[-1], m, 1.0, 30, force, mol, lengths)
    assert np.abs(xb[-1] - xs[0]).max() < 1e-7


def test_energy_conserved_with_polarization_forces():
    s = synth.water_box(64, 13.0, 43)
    eps, sig = _lj_params(s.n)
    m = md.water_masses(s.n)
    mol, lengths = md.water_constraints(s)
    p = Params(beta=0.6, grid=(16, 16, 16), cutoff=6.0)

    class _At:                       # the same molecules at positions x
        def __init__(self, x):
            for k in ("q", "alpha", "dip", "quad", "frame", "excl", "n", "box"):
                setattr(self, k, getattr(s, k))
            self.xyz = x

    def force(x):
        o = Oracle(_At(x), p)
        E = o.permanent_field()
        mu, _ = o.pcg(E, tol=1e-11, maxiter=500)
        U_lj, F_lj = md.lj_energy_forces(x, s.box, eps, sig, 6.0)
        return o.energy(mu, E) + U_lj, o.forces(mu) + F_lj

    v0 = md.rattle(synth.water_velocities(s, 300.0, 7), s.xyz, mol, lengths, 1.0 / m)
    U0, F0 = force(s.xyz)
    assert np.abs(F0).max() > 0
    xs, vs, es = md.run(s.xyz.copy(), v0, m, 0.5, 20, force, mol, lengths)
    kin = md.kinetic(vs[0], m)
    assert np.abs(es - es[0]).max() < 2e-3 * kin
    # without the polarization forces (but its energy counted) the energy would drift
    def wrong(x):
        U, F = force(x)
        return U, md.lj_energy_forces(x, s.box, eps, sig, 6.0)[1]
    _, _, ew = md.run(s.xyz.copy(), v0, m, 0.5, 20, wrong, mol, lengths)
    assert np.abs(ew - ew[0]).max() > 5 * np.abs(es - es[0]).max()
