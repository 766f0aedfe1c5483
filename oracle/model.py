"""The polarization model end to end (oracle, FP64).

Permanent field (right-hand side), the linear system A mu = E with
A = alpha^-1 - T, its diagonally preconditioned conjugate-gradient solution (Sec. 1.3,
"Optimizations opportunities": PCG with one matrix-vector product per iteration;
Sec. 3: diagonal preconditioner, 1e-5 threshold), the polarization energy and forces.

Readings where the paper is silent:
  * units: f = 332.063713 kcal A / (mol e^2); 1 e A = 4.80321 D;
  * E_i = sum_j E_real(j -> i; sigma_d) + E_rec,i + (4 beta^3 / (3 sqrt(pi))) d_i,
    sigma_d = 0 for listed (bonded / intramolecular) pairs, 1 otherwise;
  * (T p)_i = sum_{j != i} [-R1 p_j + R2 (p_j.R) R] + (T_rec p)_i + (4 beta^3/(3 sqrt(pi))) p_i,
    mutual scale 1 for every pair;
  * PCG: M^-1 = diag(alpha); convergence measure eps = 4.80321 sqrt(sum_i |alpha_i r_i|^2 / N)
    (Debye RMS of the preconditioned residual); stop when eps <= tol;
  * E_pol = -(f/2) sum_i mu_i . E_i ; forces are -dE_pol/dx at fixed mu (variational).
Modes: 'spme' (the GPU's method), 'exact' (classical Ewald k-sum), 'open' (isolated
cluster: beta = 0, no reciprocal or self terms, all pairs).
"""
from dataclasses import dataclass, field

import numpy as np

from . import ewald, frames, pairs, realspace, spme

F_COUL = 332.063713
DEBYE = 4.80321


@dataclass
class Params:
    beta: float = 0.5446
    grid: tuple = (24, 24, 24)
    order: int = 5
    cutoff: float = 7.0
    thole_a: float = 0.39
    mode: str = "spme"          # 'spme' | 'exact' | 'open'
    images: bool = False        # sum real space over all images within cutoff (cutoff may exceed L/2)

    @property
    def self_coef(self):
        return 0.0 if self.mode == "open" else 4.0 * self.beta ** 3 / (3.0 * np.sqrt(np.pi))


class Oracle:
    """FP64 reference for one configuration of a System-like object."""

    def __init__(self, sysobj, params: Params, xyz=None):
        self.s = sysobj
        self.p = params
        self.xyz = np.asarray(sysobj.xyz if xyz is None else xyz, np.float64)
        self.box = np.asarray(sysobj.box, np.float64)
        self.n = self.xyz.shape[0]
        self.alpha = np.asarray(sysobj.alpha, np.float64)
        self.q = np.asarray(sysobj.q, np.float64)
        self.dip, self.quad, _ = frames.rotate_multipoles(
            self.xyz, self.box, sysobj.frame, sysobj.dip, sysobj.quad)
        if params.mode == "open":
            self.I, self.J, self.R = pairs.pairs_open(self.xyz)
            self.sigma = pairs.scale_of_pairs(self.I, self.J, sysobj.excl, self.n)
        else:
            if params.images:
                self.I, self.J, self.R = pairs.pairs_images(self.xyz, self.box, params.cutoff)
            else:
                self.I, self.J, self.R = pairs.pairs_min_image(self.xyz, self.box, params.cutoff)
            self.sigma = pairs.scale_of_pairs(self.I, self.J, sysobj.excl, self.n, self.R, self.box)
        self.beta = 0.0 if params.mode == "open" else params.beta

    # ---- reciprocal part -------------------------------------------------------------
    def recip(self, q, dip, quad, order):
        """phi derivatives [0..order] at atoms from sources (q, dip, quad); zeros if open."""
        p = self.p
        if p.mode == "open":
            n = self.n
            return [np.zeros(n), np.zeros((n, 3)), np.zeros((n, 3, 3)), np.zeros((n, 3, 3, 3))][: order + 1]
        if p.mode == "exact":
            return ewald.recip_derivs(self.xyz, self.box, p.beta, q, dip, quad, order)
        return spme.recip_derivs(self.xyz, self.box, p.beta, p.grid, p.order, q, dip, quad, order)

    # ---- fields and the operator -----------------------------------------------------
    def permanent_field(self):
        E = realspace.real_field(self.n, self.I, self.J, self.R, self.sigma, self.q, self.dip,
                                 self.quad, self.alpha, self.beta, self.p.thole_a)
        E += -self.recip(self.q, self.dip, self.quad, 1)[1]
        E += self.p.self_coef * self.dip
        return E

    def apply_T(self, v):
        v = np.asarray(v, np.float64).reshape(self.n, 3)
        out = realspace.real_dipole_field(self.n, self.I, self.J, self.R, v, self.alpha, self.beta,
                                          self.p.thole_a)
        out += -self.recip(np.zeros(self.n), v, np.zeros((self.n, 3, 3)), 1)[1]
        out += self.p.self_coef * v
        return out

    def apply_A(self, v):
        v = np.asarray(v, np.float64).reshape(self.n, 3)
        return v / self.alpha[:, None] - self.apply_T(v)

    def residual_eps(self, r):
        """Debye RMS of alpha r."""
        z = self.alpha[:, None] * r
        return DEBYE * np.sqrt(np.sum(z * z) / self.n)

    def pcg(self, E, guess=None, tol=1e-6, maxiter=500):
        """Diagonal-preconditioned CG on A mu = E. Returns (mu, info dict)."""
        a = self.alpha[:, None]
        mu = a * E if guess is None else np.array(guess, np.float64).reshape(self.n, 3)
        r = E - self.apply_A(mu)
        z = a * r
        p = z.copy()
        rz = np.sum(r * z)
        eps = DEBYE * np.sqrt(np.sum(z * z) / self.n)
        hist = [eps]
        it = 0
        while eps > tol and it < maxiter:
            qv = self.apply_A(p)
            gamma = rz / np.sum(p * qv)
            mu = mu + gamma * p
            r = r - gamma * qv
            z = a * r
            it += 1
            eps = DEBYE * np.sqrt(np.sum(z * z) / self.n)
            hist.append(eps)
            if eps <= tol:
                break
            rz_new = np.sum(r * z)
            p = z + (rz_new / rz) * p
            rz = rz_new
        return mu, {"iters": it, "eps": eps, "history": hist, "converged": eps <= tol}

    def jacobi_diis(self, E, guess=None, tol=1e-6, depth=6, maxiter=500):
        """Jacobi iteration accelerated by DIIS (one of the solvers the paper's method builds
        on, Lipparini 2014): the Jacobi map g(x) = alpha (E + T x) (the splitting
        A = alpha^-1 - T) with Pulay's direct inversion in the iterative subspace over the
        last `depth` steps.

        Step k: y_k = g(x_k) and e_k = y_k - x_k, which equals alpha r_k with r_k = E - A x_k,
        so the convergence measure is the PCG's (Debye RMS of alpha r); stop when it is
        <= tol and return x_k. Otherwise take c minimising |sum_i c_i e_i| over the window
        subject to sum_i c_i = 1 (the bordered normal equations of B_ij = e_i . e_j) and set
        x_{k+1} = sum_i c_i y_i. depth = 1 is plain Jacobi. Returns (mu, info dict) with
        "iters" the number of steps taken (each costs one application of T after the first)."""
        a = self.alpha[:, None]
        x = a * E if guess is None else np.array(guess, np.float64).reshape(self.n, 3)
        ys, es = [], []
        hist = []
        it = 0
        while True:
            y = a * (E + self.apply_T(x))
            e = y - x
            eps = DEBYE * np.sqrt(np.sum(e * e) / self.n)
            hist.append(eps)
            if eps <= tol or it >= maxiter:
                break
            ys.append(y)
            es.append(e)
            ys, es = ys[-depth:], es[-depth:]
            m = len(es)
            B = np.empty((m + 1, m + 1))
            for i in range(m):
                for j in range(m):
                    B[i, j] = np.sum(es[i] * es[j])
            B[:m, m] = B[m, :m] = -1.0
            B[m, m] = 0.0
            rhs = np.zeros(m + 1)
            rhs[m] = -1.0
            c = np.linalg.solve(B, rhs)[:m]
            x = sum(ci * yi for ci, yi in zip(c, ys))
            it += 1
        return x, {"iters": it, "eps": eps, "history": hist, "converged": eps <= tol}

    def dense_A(self):
        """A as a dense 3N x 3N matrix, column by column (tiny systems only)."""
        m = 3 * self.n
        A = np.empty((m, m))
        for k in range(m):
            e = np.zeros(m)
            e[k] = 1.0
            A[:, k] = self.apply_A(e).ravel()
        return A

    # ---- energy and forces -----------------------------------------------------------
    @staticmethod
    def energy(mu, E):
        return -0.5 * F_COUL * float(np.sum(mu * E))

    def forces(self, mu):
        """-dE_pol/dx at fixed mu: real-space pairs, reciprocal, self, frame torques."""
        f = F_COUL
        mu = np.asarray(mu, np.float64).reshape(self.n, 3)
        grad, g_dip, g_quad = realspace.real_forces(
            self.n, self.I, self.J, self.R, self.sigma, self.q, self.dip, self.quad, self.alpha,
            mu, self.beta, self.p.thole_a, f)
        if self.p.mode != "open":
            zq, zQ = np.zeros(self.n), np.zeros((self.n, 3, 3))
            phM = self.recip(self.q, self.dip, self.quad, 2)
            phU = self.recip(zq, mu, zQ, 3)
            hess_tot = phM[2] + phU[2]
            grad += f * (np.einsum("nab,nb->na", hess_tot, mu)
                         + self.q[:, None] * phU[1]
                         + np.einsum("nab,nb->na", phU[2], self.dip)
                         + np.einsum("nabc,nbc->na", phU[3], self.quad) / 3.0)
            g_dip += f * phU[1]
            g_quad += (f / 3.0) * phU[2]
            g_dip += -f * self.p.self_coef * mu
        grad += frames.frame_gradient(self.xyz, self.box, self.s.frame, self.s.dip, self.s.quad,
                                      g_dip, g_quad)
        return -grad

    def charge_potential(self):
        """Electrostatic potential at each site from all charges (Madelung checks)."""
        from .radial import ewald_b
        phi = np.zeros(self.n)
        r = np.linalg.norm(self.R, axis=1)
        np.add.at(phi, self.I, self.q[self.J] * ewald_b(r, self.beta, 0)[0])
        if self.p.mode != "open":
            zero3 = np.zeros((self.n, 3))
            phi += self.recip(self.q, zero3, np.zeros((self.n, 3, 3)), 0)[0]
            phi -= 2.0 * self.beta / np.sqrt(np.pi) * self.q
        return phi


def solve_energy(sysobj, params, xyz=None, tol=1e-11):
    """E_pol with mu converged tightly (finite-difference checks)."""
    o = Oracle(sysobj, params, xyz)
    E = o.permanent_field()
    mu, _ = o.pcg(E, tol=tol, maxiter=2000)
    return o.energy(mu, E)


def row_fields(sysobj, params, rows, vec=None):
    """Permanent field E_i and, if vec is given, (T vec)_i for the atoms in `rows` only.

    Real space by brute force over all atoms (minimum image) for each listed row, the
    reciprocal part from one full smooth-PME evaluation gathered at the rows, plus the
    self terms. For spot checks of large systems, where pairs of every atom would not fit.
    """
    from .radial import damped_r
    xyz = np.asarray(sysobj.xyz, np.float64)
    box = np.asarray(sysobj.box, np.float64)
    n = xyz.shape[0]
    rows = np.asarray(rows)
    dip, quad, _ = frames.rotate_multipoles(xyz, box, sysobj.frame, sysobj.dip, sysobj.quad)
    q = np.asarray(sysobj.q, np.float64)
    alpha = np.asarray(sysobj.alpha, np.float64)
    I, J, R = [], [], []
    for i in rows:
        d = xyz[i] - xyz
        d -= box * np.round(d / box)
        r2 = np.einsum("ij,ij->i", d, d)
        keep = (r2 < params.cutoff ** 2) & (np.arange(n) != i)
        js = np.nonzero(keep)[0]
        I.append(np.full(len(js), i))
        J.append(js)
        R.append(d[js])
    I, J, R = np.concatenate(I), np.concatenate(J), np.concatenate(R)
    sigma = pairs.scale_of_pairs(I, J, sysobj.excl, n, R, box)
    E = realspace.real_field(n, I, J, R, sigma, q, dip, quad, alpha, params.beta, params.thole_a)[rows]
    sub = xyz[rows]
    grid = spme.spread(xyz, box, params.grid, params.order, q, dip, quad)
    phi = spme.convolve(grid, box, params.grid, params.order, params.beta)
    E += -spme.gather(phi, sub, box, params.grid, params.order, 1)[1]
    E += params.self_coef * dip[rows]
    if vec is None:
        return E, None
    v = np.asarray(vec, np.float64)
    Tv = realspace.real_dipole_field(n, I, J, R, v, alpha, params.beta, params.thole_a)[rows]
    gv = spme.spread(xyz, box, params.grid, params.order, np.zeros(n), v, np.zeros((n, 3, 3)))
    phv = spme.convolve(gv, box, params.grid, params.order, params.beta)
    Tv += -spme.gather(phv, sub, box, params.grid, params.order, 1)[1]
    Tv += params.self_coef * v[rows]
    return E, Tv
