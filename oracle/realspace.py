"""Real-space pair sums (oracle, FP64).

Site J carries a permanent multipole (q, d, Q) with the potential
    phi(R) = q/R + d.R/R^3 + R.Q.R/R^5        (Q traceless, R = x_target - x_J),
i.e. the operator (q - d.grad + (1/3) Q:grad grad) applied to 1/R. With the screened
and damped radial functions R_n of `radial.damped_r`, the field at the target is
    E = q R R1 - d R1 + (d.R) R R2 - (2/3) (Q R) R2 + (1/3) (R.Q.R) R R3,
and the field of a dipole p is T p with T = -R1 I + R2 R R^T.
Pairs come from `pairs` as ordered (I, J, R); contributions go to the target I.
"""
import numpy as np

from .radial import damped_r

CHUNK = 400_000


def _chunks(m):
    for s in range(0, m, CHUNK):
        yield slice(s, min(m, s + CHUNK))


def multipole_field(R, Rn, q, d, Q):
    """Field at R from multipoles (q [P], d [P,3], Q [P,3,3]); Rn = (R1, R2, R3)."""
    R1, R2, R3 = Rn[0], Rn[1], Rn[2]
    dR = np.einsum("pa,pa->p", d, R)
    QR = np.einsum("pab,pb->pa", Q, R)
    RQR = np.einsum("pa,pa->p", QR, R)
    return ((q * R1 + dR * R2 + RQR * R3 / 3.0)[:, None] * R
            - R1[:, None] * d - (2.0 / 3.0) * R2[:, None] * QR)


def multipole_field_gradient(R, Rn, q, d, Q):
    """G[p, a, b] = dE_b/dR_a of `multipole_field`; Rn = (R1, R2, R3, R4)."""
    R1, R2, R3, R4 = Rn[0], Rn[1], Rn[2], Rn[3]
    eye = np.eye(3)[None]
    RR = np.einsum("pa,pb->pab", R, R)
    dR = np.einsum("pa,pa->p", d, R)
    QR = np.einsum("pab,pb->pa", Q, R)
    RQR = np.einsum("pa,pa->p", QR, R)
    g = (q * R1)[:, None, None] * eye - (q * R2)[:, None, None] * RR
    g += R2[:, None, None] * (np.einsum("pa,pb->pab", R, d) + np.einsum("pa,pb->pab", d, R))
    g += (dR * R2)[:, None, None] * eye - (dR * R3)[:, None, None] * RR
    g += -(2.0 / 3.0) * R2[:, None, None] * Q
    g += (2.0 / 3.0) * R3[:, None, None] * (np.einsum("pa,pb->pab", R, QR) + np.einsum("pa,pb->pab", QR, R))
    g += (RQR * R3 / 3.0)[:, None, None] * eye - (RQR * R4 / 3.0)[:, None, None] * RR
    return g


def real_field(n, I, J, R, sigma, q, dip, quad, alpha, beta, thole_a):
    """Real-space permanent field at every atom (d/p scale sigma per pair)."""
    E = np.zeros((n, 3))
    for s in _chunks(len(I)):
        r = np.linalg.norm(R[s], axis=1)
        Rn = damped_r(r, beta, alpha[I[s]], alpha[J[s]], thole_a, sigma[s], nmax=3)
        js = J[s]
        np.add.at(E, I[s], multipole_field(R[s], Rn, q[js], dip[js], quad[js]))
    return E


def real_dipole_field(n, I, J, R, p, alpha, beta, thole_a):
    """Real-space part of T p (mutual scale 1 for every pair)."""
    E = np.zeros((n, 3))
    for s in _chunks(len(I)):
        r = np.linalg.norm(R[s], axis=1)
        Rn = damped_r(r, beta, alpha[I[s]], alpha[J[s]], thole_a, 1.0, nmax=2)
        pj = p[J[s]]
        pr = np.einsum("pa,pa->p", pj, R[s])
        np.add.at(E, I[s], -Rn[0][:, None] * pj + (Rn[1] * pr)[:, None] * R[s])
    return E


def real_forces(n, I, J, R, sigma, q, dip, quad, alpha, mu, beta, thole_a, fconst, virial=False):
    """Real-space part of the polarization gradient at fixed induced dipoles mu.

    Each ordered pair (I, J) carries
        U_IJ = -f mu_I . E(R; multipole J) - (f/2) mu_I . T(R) mu_J,
    whose sum over ordered pairs is the position-dependent real-space energy.
    Returns (dU/dx [n,3] from the pair distances, dU/d(global dipole) [n,3],
    dU/d(global quadrupole) [n,3,3]) - the last two feed the frame chain rule - and, with
    virial=True, the pairs' share of dU/d(strain) [3,3]: a homogeneous deformation
    x -> (I + e) x maps every pair vector R (images included) to (I + e) R, so it is
    sum over ordered pairs of (dU_IJ/dR)_a R_b at fixed global multipoles.
    """
    grad = np.zeros((n, 3))
    g_dip = np.zeros((n, 3))
    g_quad = np.zeros((n, 3, 3))
    V = np.zeros((3, 3))
    for s in _chunks(len(I)):
        Rs = R[s]
        r = np.linalg.norm(Rs, axis=1)
        Ii, Jj = I[s], J[s]
        Rd = damped_r(r, beta, alpha[Ii], alpha[Jj], thole_a, sigma[s], nmax=4)
        Ru = damped_r(r, beta, alpha[Ii], alpha[Jj], thole_a, 1.0, nmax=3)
        mi, mj = mu[Ii], mu[Jj]
        # permanent-induced: gradient of mu_I . E(R; M_J)
        G = multipole_field_gradient(Rs, Rd, q[Jj], dip[Jj], quad[Jj])
        gR = -fconst * np.einsum("pab,pb->pa", G, mi)
        # mutual: gradient of mu_I . T mu_J with T = -R1 I + R2 R R^T
        mij = np.einsum("pa,pa->p", mi, mj)
        mir = np.einsum("pa,pa->p", mi, Rs)
        mjr = np.einsum("pa,pa->p", mj, Rs)
        dT = ((Ru[1] * mij - Ru[2] * mir * mjr)[:, None] * Rs
              + Ru[1][:, None] * (mi * mjr[:, None] + mj * mir[:, None]))
        gR += -0.5 * fconst * dT
        np.add.at(grad, Ii, gR)
        np.add.at(grad, Jj, -gR)
        V += np.einsum("pa,pb->ab", gR, Rs)
        # dependence on the source multipole J (global components)
        np.add.at(g_dip, Jj, -fconst * (-Rd[0][:, None] * mi + (Rd[1] * mir)[:, None] * Rs))
        sym = np.einsum("pa,pb->pab", mi, Rs)
        sym = sym + np.swapaxes(sym, 1, 2)
        gq = -fconst * (-(Rd[1] / 3.0)[:, None, None] * sym
                        + (Rd[2] * mir / 3.0)[:, None, None] * np.einsum("pa,pb->pab", Rs, Rs))
        np.add.at(g_quad, Jj, gq)
    return (grad, g_dip, g_quad, V) if virial else (grad, g_dip, g_quad)


def real_forces_dp(n, I, J, R, sigma_d, sigma_p, q, dip, quad, alpha, mu_d, mu_p, beta, thole_a, fconst,
                   virial=False):
    """Real-space part of the polarization gradient with AMOEBA's two induced-dipole sets:
    mu_d induced by the direct field (pair scale sigma_d), mu_p by the polarization field
    (sigma_p), mutual scale 1. Each ordered pair (I, J) carries
        U_IJ = -(f/2) [mu_p,I . E(R; M_J, sigma_d) + mu_d,I . E(R; M_J, sigma_p)]
               -(f/2) mu_p,I . T(R) mu_d,J,
    whose sum over ordered pairs is the position-dependent real-space part of
    -(f/2) mu_d . E_p at fixed dipoles, with the response of mu_d folded in through mu_p
    (A symmetric). With sigma_d = sigma_p and mu_d = mu_p it is real_forces' U_IJ.
    Returns (dU/dx, dU/d(global dipole), dU/d(global quadrupole)) and, with virial=True,
    the pairs' share of dU/d(strain) as in real_forces."""
    grad = np.zeros((n, 3))
    g_dip = np.zeros((n, 3))
    g_quad = np.zeros((n, 3, 3))
    V = np.zeros((3, 3))
    h = 0.5 * fconst
    for s in _chunks(len(I)):
        Rs = R[s]
        r = np.linalg.norm(Rs, axis=1)
        Ii, Jj = I[s], J[s]
        Rd = damped_r(r, beta, alpha[Ii], alpha[Jj], thole_a, sigma_d[s], nmax=4)
        Rp = damped_r(r, beta, alpha[Ii], alpha[Jj], thole_a, sigma_p[s], nmax=4)
        Ru = damped_r(r, beta, alpha[Ii], alpha[Jj], thole_a, 1.0, nmax=3)
        pI, dI = mu_p[Ii], mu_d[Ii]
        dJ = mu_d[Jj]
        Gd = multipole_field_gradient(Rs, Rd, q[Jj], dip[Jj], quad[Jj])
        Gp = multipole_field_gradient(Rs, Rp, q[Jj], dip[Jj], quad[Jj])
        gR = -h * (np.einsum("pab,pb->pa", Gd, pI) + np.einsum("pab,pb->pa", Gp, dI))
        # mutual: gradient of mu_p,I . T mu_d,J
        pd = np.einsum("pa,pa->p", pI, dJ)
        pr = np.einsum("pa,pa->p", pI, Rs)
        dr = np.einsum("pa,pa->p", dJ, Rs)
        dT = ((Ru[1] * pd - Ru[2] * pr * dr)[:, None] * Rs
              + Ru[1][:, None] * (pI * dr[:, None] + dJ * pr[:, None]))
        gR += -h * dT
        np.add.at(grad, Ii, gR)
        np.add.at(grad, Jj, -gR)
        V += np.einsum("pa,pb->ab", gR, Rs)
        # dependence on the source multipole J: d(mu . E)/d d_J = -R1 mu + R2 (mu.R) R,
        # d(mu . E)/d Q_J = -(R2/3) sym(mu R^T) + (R3/3)(mu.R) R R^T
        dIr = np.einsum("pa,pa->p", dI, Rs)
        gd = (-Rd[0][:, None] * pI + (Rd[1] * pr)[:, None] * Rs
              - Rp[0][:, None] * dI + (Rp[1] * dIr)[:, None] * Rs)
        np.add.at(g_dip, Jj, -h * gd)
        RR = np.einsum("pa,pb->pab", Rs, Rs)
        symp = np.einsum("pa,pb->pab", pI, Rs)
        symp = symp + np.swapaxes(symp, 1, 2)
        symd = np.einsum("pa,pb->pab", dI, Rs)
        symd = symd + np.swapaxes(symd, 1, 2)
        gq = (-(Rd[1] / 3.0)[:, None, None] * symp + (Rd[2] * pr / 3.0)[:, None, None] * RR
              - (Rp[1] / 3.0)[:, None, None] * symd + (Rp[2] * dIr / 3.0)[:, None, None] * RR)
        np.add.at(g_quad, Jj, -h * gq)
    return (grad, g_dip, g_quad, V) if virial else (grad, g_dip, g_quad)
