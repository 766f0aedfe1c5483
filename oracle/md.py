"""Minimal rigid-water molecular dynamics (oracle, FP64; test infrastructure only).

An MD step is one call of an integrator that moves positions and velocities from one
time step to the next under the forces (paper Sec. 1.1); the paper's default integrator is
velocity Verlet (Sec. 2.5 validates with it, Sec. 2.6 lists it with the multiple-time-step
ones), and its benchmarks run RESPA with a 2 fs outer step (Sec. 2.7). This module is the
plainest such step for rigid three-site waters (atoms O, H, H of each molecule):

  * velocity Verlet in the kick-drift-kick form, with the three distance constraints of a
    molecule (O-H1, O-H2, H1-H2) held by SHAKE after the drift (Ryckaert, Ciccotti and
    Berendsen 1977) and by RATTLE on the velocities after the second kick (Andersen 1983);
  * forces: the polarization forces of model.Oracle plus a Lennard-Jones term between
    oxygen sites, force-shifted at the cutoff so that energy and force are continuous
    there (the paper's force field has a van der Waals term; this minimal model keeps the
    liquid from collapsing under the attractive polarization energy).

Units: A, fs, amu, kcal/mol; a force of 1 kcal/mol/A on 1 amu is an acceleration of
ACC = 4.184e-4 A/fs^2 (1 kcal/mol = 4184 J/mol; 1 amu = 1e-3 kg/mol; 1 m^2/s^2 = 1e-10
A^2/fs^2).
"""
import numpy as np

from .pairs import pairs_min_image

ACC = 4.184e-4            # A/fs^2 per (kcal/mol/A)/amu
MASS_O, MASS_H = 15.999, 1.008
KB = 0.0019872041         # kcal/mol/K


def lj_pair(r, eps, sigma, rc):
    """Force-shifted Lennard-Jones: V(r) = 4 eps [(s/r)^12 - (s/r)^6]; returns
    (V(r) - V(rc) + (r - rc) F(rc), F(r) - F(rc)) with F = -dV/dr, both zero at rc."""
    def V(x):
        s6 = (sigma / x) ** 6
        return 4.0 * eps * (s6 * s6 - s6)

    def F(x):
        s6 = (sigma / x) ** 6
        return 24.0 * eps * (2.0 * s6 * s6 - s6) / x

    return V(r) - V(rc) + (r - rc) * F(rc), F(r) - F(rc)


def lj_energy_forces(xyz, box, eps, sigma, rc, excl=None):
    """Energy and forces of the force-shifted Lennard-Jones term over every pair within rc
    (minimum image), Lorentz-Berthelot combination (sigma_ij = (s_i + s_j)/2,
    eps_ij = sqrt(e_i e_j)); pairs in `excl` (either order) are left out."""
    xyz = np.asarray(xyz, np.float64)
    n = xyz.shape[0]
    I, J, R = pairs_min_image(xyz, box, rc)
    half = I < J                                 # each unordered pair once
    I, J, R = I[half], J[half], R[half]
    e_ij = np.sqrt(eps[I] * eps[J])
    keep = e_ij > 0.0
    if excl is not None and len(excl):
        ex = {(min(a, b), max(a, b)) for a, b in np.asarray(excl)}
        keep &= np.array([(min(a, b), max(a, b)) not in ex for a, b in zip(I, J)], bool)
    I, J, R, e_ij = I[keep], J[keep], R[keep], e_ij[keep]
    s_ij = 0.5 * (sigma[I] + sigma[J])
    r = np.linalg.norm(R, axis=1)
    V, Fr = lj_pair(r, e_ij, s_ij, rc)
    f = (Fr / r)[:, None] * R                   # force on I (R = x_I - x_J)
    F = np.zeros((n, 3))
    np.add.at(F, I, f)
    np.add.at(F, J, -f)
    return float(np.sum(V)), F


def water_masses(n):
    m = np.full(n, MASS_H)
    m[0::3] = MASS_O
    return m


def water_constraints(s):
    """[n_mol][3] atom indices (O, H1, H2) and the three lengths (O-H, O-H, H-H) of the
    rigid waters of s (every atom in a water)."""
    mol = np.arange(s.n).reshape(-1, 3)
    d = s.xyz[mol[0]]
    return mol, np.array([np.linalg.norm(d[1] - d[0]), np.linalg.norm(d[2] - d[0]), np.linalg.norm(d[2] - d[1])])


PAIRS = ((0, 1, 0), (0, 2, 1), (1, 2, 2))      # (atom a, atom b, length index) within a molecule


def shake(x_new, x_old, mol, lengths, inv_m, tol=1e-12, maxit=1000):
    """Positions after the drift moved along the old bond vectors until every constraint
    |x_a - x_b| = d holds (relative tolerance tol on |r|^2 - d^2)."""
    x = x_new.copy()
    for _ in range(maxit):
        worst = 0.0
        for a, b, k in PAIRS:
            ia, ib = mol[:, a], mol[:, b]
            d2 = lengths[k] ** 2
            r = x[ia] - x[ib]
            diff = np.einsum("ij,ij->i", r, r) - d2
            worst = max(worst, float(np.max(np.abs(diff))) / d2)
            ro = x_old[ia] - x_old[ib]
            g = diff / (2.0 * (inv_m[ia] + inv_m[ib]) * np.einsum("ij,ij->i", r, ro))
            x[ia] -= (g * inv_m[ia])[:, None] * ro
            x[ib] += (g * inv_m[ib])[:, None] * ro
        if worst < tol:
            return x
    raise RuntimeError("SHAKE did not converge")


def rattle(v, x, mol, lengths, inv_m, tol=1e-12, maxit=1000):
    """Velocities projected until every constrained pair has r . (v_a - v_b) = 0."""
    v = v.copy()
    for _ in range(maxit):
        worst = 0.0
        for a, b, k in PAIRS:
            ia, ib = mol[:, a], mol[:, b]
            r = x[ia] - x[ib]
            rv = np.einsum("ij,ij->i", r, v[ia] - v[ib])
            d2 = lengths[k] ** 2
            worst = max(worst, float(np.max(np.abs(rv))) / d2)
            g = rv / ((inv_m[ia] + inv_m[ib]) * d2)
            v[ia] -= (g * inv_m[ia])[:, None] * r
            v[ib] += (g * inv_m[ib])[:, None] * r
        if worst < tol:
            return v
    raise RuntimeError("RATTLE did not converge")


def kick_drift(x, v, f, m, dt, mol, lengths):
    """First half of a step: v(t + dt/2) = v + dt/2 a, x(t + dt) = x + dt v(t + dt/2),
    SHAKE, and the half-step velocities that the constrained drift implies."""
    inv_m = 1.0 / m
    vh = v + 0.5 * dt * ACC * f * inv_m[:, None]
    xn = shake(x + dt * vh, x, mol, lengths, inv_m)
    return xn, (xn - x) / dt


def kick(x, vh, f, m, dt, mol, lengths):
    """Second half: v(t + dt) = v(t + dt/2) + dt/2 a(t + dt), then RATTLE."""
    inv_m = 1.0 / m
    return rattle(vh + 0.5 * dt * ACC * f * inv_m[:, None], x, mol, lengths, inv_m)


def kinetic(v, m):
    """Kinetic energy, kcal/mol."""
    return 0.5 * float(np.sum(m[:, None] * v * v)) / ACC


def run(x, v, m, dt, steps, force_fn, mol, lengths):
    """Velocity-Verlet trajectory: force_fn(x) -> (potential energy, forces). Returns the
    positions, velocities and total energies of every step (step 0 first)."""
    U, f = force_fn(x)
    xs, vs, es = [x.copy()], [v.copy()], [U + kinetic(v, m)]
    for _ in range(steps):
        x, vh = kick_drift(x, v, f, m, dt, mol, lengths)
        U, f = force_fn(x)
        v = kick(x, vh, f, m, dt, mol, lengths)
        xs.append(x.copy())
        vs.append(v.copy())
        es.append(U + kinetic(v, m))
    return np.array(xs), np.array(vs), np.array(es)
