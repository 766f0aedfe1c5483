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
  * E_pol = -(f/2) sum_i mu_i . E_i ; forces are -dE_pol/dx at fixed mu (variational);
  * virial V_ab = dE_pol/de_ab under x -> (I + e) x of positions and box (local-frame
    multipoles carried by the deformed frames, mu re-solved), in kcal/mol; the sign is
    that of the strain derivative, so the pressure tensor's share is -V / volume;
  * two dipole sets (AMOEBA's d and p, the three scale factors of Sec. 2.3): E_d and E_p
    use the direct and the polarization scale factors of the listed pairs, T uses scale 1;
    mu_d = A^-1 E_d, mu_p = A^-1 E_p; E_pol = -(f/2) sum_i mu_d,i . E_p,i.
Modes: 'spme' (the GPU's method), 'exact' (classical Ewald k-sum), 'open' (isolated
cluster: beta = 0, no reciprocal or self terms, all pairs).
"""
from dataclasses import dataclass

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

    def __init__(self, sysobj, params: Params, xyz=None, dp=None):
        """dp = (pairs [M,2], scales [M,2]): AMOEBA's direct (d) and polarization (p) scale
        factors of the listed pairs (others 1), for the two-dipole-set methods (*_dp)."""
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
        if dp is not None:
            tp, tv = np.asarray(dp[0]), np.asarray(dp[1], np.float64)
            img = (None, None) if params.mode == "open" else (self.R, self.box)
            self.sigma_d = pairs.scales_from_table(self.I, self.J, tp, tv[:, 0], self.n, *img)
            self.sigma_p = pairs.scales_from_table(self.I, self.J, tp, tv[:, 1], self.n, *img)

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
        return mu, {"iters": it, "eps": eps, "history": hist, "converged": eps <= tol,
                    "eps_field": self.field_residual_debye(E, mu)}

    def field_residual_debye(self, E, mu):
        """The other reading of the threshold: 4.80321 sqrt(sum_i |r_i|^2 / N) with the true
        residual r = E - A mu (a field, unweighted by alpha), as Tinker logs it."""
        r = E - self.apply_A(mu)
        return DEBYE * float(np.sqrt(np.sum(r * r) / self.n))

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

    # ---- AMOEBA's two induced-dipole sets (d and p) ----------------------------------
    def permanent_field_dp(self):
        """(E_d, E_p): the permanent field with the direct and the polarization scale
        factors in real space; the reciprocal and self parts are unscaled and shared."""
        rec = -self.recip(self.q, self.dip, self.quad, 1)[1] + self.p.self_coef * self.dip
        out = []
        for sig in (self.sigma_d, self.sigma_p):
            E = realspace.real_field(self.n, self.I, self.J, self.R, sig, self.q, self.dip,
                                     self.quad, self.alpha, self.beta, self.p.thole_a)
            out.append(E + rec)
        return out[0], out[1]

    def pcg_dp(self, E_d, E_p, guess_d=None, guess_p=None, tol=1e-6, maxiter=500):
        """A mu_d = E_d and A mu_p = E_p by two diagonal-preconditioned CG recurrences run
        in lockstep (one iteration updates both) until the larger of the two convergence
        measures is <= tol. A recurrence whose r.z is exactly zero is left as it is.
        Returns (mu_d, mu_p, info) with info["iters"], info["eps"] = the larger measure,
        and info["eps_d"], info["eps_p"]."""
        a = self.alpha[:, None]
        mus, rs, ps, rzs = [], [], [], []
        for E, g in ((E_d, guess_d), (E_p, guess_p)):
            mu = a * E if g is None else np.array(g, np.float64).reshape(self.n, 3)
            r = E - self.apply_A(mu)
            mus.append(mu)
            rs.append(r)
            ps.append(a * r)
            rzs.append(np.sum(r * a * r))
        epsk = [self.residual_eps(r) for r in rs]
        it = 0
        while max(epsk) > tol and it < maxiter:
            for k in range(2):
                if rzs[k] == 0.0:
                    continue
                qv = self.apply_A(ps[k])
                gamma = rzs[k] / np.sum(ps[k] * qv)
                mus[k] = mus[k] + gamma * ps[k]
                rs[k] = rs[k] - gamma * qv
            it += 1
            epsk = [self.residual_eps(r) for r in rs]
            if max(epsk) <= tol:
                break
            for k in range(2):
                if rzs[k] == 0.0:
                    continue
                z = a * rs[k]
                rz_new = np.sum(rs[k] * z)
                ps[k] = z + (rz_new / rzs[k]) * ps[k]
                rzs[k] = rz_new
        return mus[0], mus[1], {"iters": it, "eps": max(epsk), "eps_d": epsk[0], "eps_p": epsk[1],
                                "converged": max(epsk) <= tol}

    @staticmethod
    def energy_dp(mu_d, E_p):
        """E_pol = -(f/2) sum_i mu_d,i . E_p,i (d-set dipoles in the p-scaled field)."""
        return -0.5 * F_COUL * float(np.sum(mu_d * E_p))

    def forces_dp(self, mu_d, mu_p):
        """-dE_pol/dx of E_pol = -(f/2) mu_d . E_p with mu_d = A^-1 E_d and mu_p = A^-1 E_p
        (converged): -(f/2) [mu_p . dE_d + mu_d . dE_p + mu_p . dT mu_d], including the
        multipole frames' rotation. Reciprocal part, with mu_s = (mu_d + mu_p)/2 and phi_X
        the reciprocal potential of sources X:
            U_rec = f mu_s . grad phi_M + (f/2) mu_p . grad phi_{mu_d}
        whose gradient is f [H(phi_M) mu_s + q grad phi_s + H(phi_s) d + D3(phi_s):Q/3]
        + (f/2) [H(phi_d) mu_p + H(phi_p) mu_d]."""
        f = F_COUL
        mu_d = np.asarray(mu_d, np.float64).reshape(self.n, 3)
        mu_p = np.asarray(mu_p, np.float64).reshape(self.n, 3)
        grad, g_dip, g_quad = realspace.real_forces_dp(
            self.n, self.I, self.J, self.R, self.sigma_d, self.sigma_p, self.q, self.dip, self.quad,
            self.alpha, mu_d, mu_p, self.beta, self.p.thole_a, f)
        if self.p.mode != "open":
            zq, zQ = np.zeros(self.n), np.zeros((self.n, 3, 3))
            mu_s = 0.5 * (mu_d + mu_p)
            phM = self.recip(self.q, self.dip, self.quad, 2)
            phS = self.recip(zq, mu_s, zQ, 3)
            phD = self.recip(zq, mu_d, zQ, 2)
            phP = self.recip(zq, mu_p, zQ, 2)
            grad += f * (np.einsum("nab,nb->na", phM[2], mu_s)
                         + self.q[:, None] * phS[1]
                         + np.einsum("nab,nb->na", phS[2], self.dip)
                         + np.einsum("nabc,nbc->na", phS[3], self.quad) / 3.0)
            grad += 0.5 * f * (np.einsum("nab,nb->na", phD[2], mu_p) + np.einsum("nab,nb->na", phP[2], mu_d))
            g_dip += f * phS[1]
            g_quad += (f / 3.0) * phS[2]
            g_dip += -f * self.p.self_coef * mu_s
        grad += frames.frame_gradient(self.xyz, self.box, self.s.frame, self.s.dip, self.s.quad,
                                      g_dip, g_quad)
        return -grad

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

    # ---- virial ----------------------------------------------------------------------
    def recip_strain(self, src_a, src_b):
        """Structure-factor share of the strain derivative of the bilinear reciprocal energy
        of two source sets (ewald.strain_sum / spme.strain_sum)."""
        p = self.p
        if p.mode == "exact":
            return ewald.strain_sum(self.xyz, self.box, p.beta, src_a, src_b)
        return spme.strain_sum(self.xyz, self.box, p.beta, p.grid, p.order, src_a, src_b)

    def virial(self, mu):
        """The virial that the paper's real-space pair loop updates with the energy and the
        forces (Sec. 1.2.1) and accumulates in double precision (Sec. 2.2); the paper
        prints no formula, so it is written here from its definition:
        V_ab = dE_pol/de_ab [3,3] (kcal/mol) under the homogeneous deformation
        x -> (I + e) x of positions and box, with the local-frame multipoles carried by the
        deformed frames and mu re-solved; because E_pol is stationary in mu this is the
        derivative of U = -f mu.E - (f/2) mu.T mu at fixed mu (global components):
          real space: sum over ordered pairs of (dU/dR)_a R_b;
          frames:     sum over frame vectors of (dU/dv)_a v_b;
          reciprocal: U_rec = f [B(mu, M) + B(mu, mu)/2], B(X, Y) = sum_m C Re[S_X conj S_Y];
                      the change of C (volume, |m|) gives the structure-factor sums, and the
                      change of m in the dipole and quadrupole factors of S gives
                      -f sum_j [dphi_{M+mu}/dx_a mu_j,b + dphi_mu/dx_a d_j,b
                                + (2/3) (H(phi_mu) Q_j)_ab];
          self terms: no dependence at fixed global components.
        The pressure tensor's polarization share is -V / volume."""
        f = F_COUL
        mu = np.asarray(mu, np.float64).reshape(self.n, 3)
        _, g_dip, g_quad, V = realspace.real_forces(
            self.n, self.I, self.J, self.R, self.sigma, self.q, self.dip, self.quad, self.alpha,
            mu, self.beta, self.p.thole_a, f, virial=True)
        if self.p.mode != "open":
            zq, zQ = np.zeros(self.n), np.zeros((self.n, 3, 3))
            M, U = (self.q, self.dip, self.quad), (zq, mu, zQ)
            phM = self.recip(*M, 1)
            phU = self.recip(*U, 2)
            g_dip += f * phU[1]
            g_quad += (f / 3.0) * phU[2]
            g_dip += -f * self.p.self_coef * mu
            V += f * (self.recip_strain(U, M) + 0.5 * self.recip_strain(U, U))
            V -= f * (np.einsum("ja,jb->ab", phM[1] + phU[1], mu) + np.einsum("ja,jb->ab", phU[1], self.dip)
                      + (2.0 / 3.0) * np.einsum("jac,jcb->ab", phU[2], self.quad))
        V += frames.frame_virial(self.xyz, self.box, self.s.frame, self.s.dip, self.s.quad, g_dip, g_quad)
        return V

    def virial_dp(self, mu_d, mu_p):
        """dE_pol/de [3,3] of E_pol = -(f/2) mu_d . E_p with both dipole sets converged,
        term by term as in `virial`: real space from real_forces_dp, reciprocal from
        U_rec = f [B(mu_s, M) + B(mu_p, mu_d)/2] with mu_s = (mu_d + mu_p)/2, frames from
        the same multipole derivatives as forces_dp."""
        f = F_COUL
        mu_d = np.asarray(mu_d, np.float64).reshape(self.n, 3)
        mu_p = np.asarray(mu_p, np.float64).reshape(self.n, 3)
        _, g_dip, g_quad, V = realspace.real_forces_dp(
            self.n, self.I, self.J, self.R, self.sigma_d, self.sigma_p, self.q, self.dip, self.quad,
            self.alpha, mu_d, mu_p, self.beta, self.p.thole_a, f, virial=True)
        if self.p.mode != "open":
            zq, zQ = np.zeros(self.n), np.zeros((self.n, 3, 3))
            mu_s = 0.5 * (mu_d + mu_p)
            M, S, D, P = (self.q, self.dip, self.quad), (zq, mu_s, zQ), (zq, mu_d, zQ), (zq, mu_p, zQ)
            phM = self.recip(*M, 1)
            phS = self.recip(*S, 2)
            phD = self.recip(*D, 1)
            phP = self.recip(*P, 1)
            g_dip += f * phS[1]
            g_quad += (f / 3.0) * phS[2]
            g_dip += -f * self.p.self_coef * mu_s
            V += f * (self.recip_strain(S, M) + 0.5 * self.recip_strain(P, D))
            V -= f * (np.einsum("ja,jb->ab", phM[1], mu_s) + np.einsum("ja,jb->ab", phS[1], self.dip)
                      + (2.0 / 3.0) * np.einsum("jac,jcb->ab", phS[2], self.quad))
            V -= 0.5 * f * (np.einsum("ja,jb->ab", phD[1], mu_p) + np.einsum("ja,jb->ab", phP[1], mu_d))
        V += frames.frame_virial(self.xyz, self.box, self.s.frame, self.s.dip, self.s.quad, g_dip, g_quad)
        return V

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


def solve_energy_dp(sysobj, params, dp, xyz=None, tol=1e-11):
    """E_pol = -(f/2) mu_d . E_p with both dipole sets converged tightly (finite-difference
    checks of forces_dp)."""
    o = Oracle(sysobj, params, xyz, dp=dp)
    E_d, E_p = o.permanent_field_dp()
    mu_d, _, _ = o.pcg_dp(E_d, E_p, tol=tol, maxiter=2000)
    return o.energy_dp(mu_d, E_p)


def row_fields(sysobj, params, rows, vec=None):
    """Permanent field E_i and, if vec is given, (T vec)_i for the atoms in `rows` only.

    Real space by brute force over all atoms (minimum image) for each listed row, the
    reciprocal part from one full smooth-PME evaluation gathered at the rows, plus the
    self terms. For spot checks of large systems, where pairs of every atom would not fit.
    """
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
