"""Classical Ewald reciprocal sum for multipoles (oracle, FP64, EXACT mode).

The reciprocal potential at x from all sites and their periodic images (tin-foil
boundary, no m = 0 term):
    phi(x) = sum_{m != 0} C(m) Re[ S(m) exp(2 pi i m.x) ],
    C(m)   = exp(-pi^2 |m|^2 / beta^2) / (pi V |m|^2),
    S(m)   = sum_j (q_j - 2 pi i d_j.m - (4 pi^2 / 3) m.Q_j.m) exp(-2 pi i m.x_j),
with m = (m1/L1, m2/L2, m3/L3) for integer m_a. The multipole factor is the site
operator (q - d.grad + (1/3) Q:grad grad) acting on exp(2 pi i m.(x - x_j)).
Each derivative of phi brings down a factor 2 pi i m. This is the definition that the
smooth PME of the paper approximates (Sec. 1.2.2).
"""
import numpy as np


def kvectors(box, beta, tol=1e-17):
    """Integer m != 0 with exp(-pi^2 |m|^2/beta^2) above tol along each axis."""
    mmax = np.ceil(beta * box * np.sqrt(-np.log(tol)) / np.pi).astype(int)
    grids = np.meshgrid(*[np.arange(-k, k + 1) for k in mmax], indexing="ij")
    m = np.stack(grids, -1).reshape(-1, 3)
    return m[np.any(m != 0, axis=1)]


def recip_derivs(xyz, box, beta, q, dip, quad, order, chunk=1500):
    """phi and its Cartesian derivatives up to `order` (<= 3) at every atom.

    Returns a list [phi [N], grad [N,3], hess [N,3,3], third [N,3,3,3]][: order+1].
    """
    xyz = np.asarray(xyz, np.float64)
    box = np.asarray(box, np.float64)
    n = xyz.shape[0]
    vol = float(np.prod(box))
    ms = kvectors(box, beta)
    out = [np.zeros(n), np.zeros((n, 3)), np.zeros((n, 3, 3)), np.zeros((n, 3, 3, 3))][: order + 1]
    tp = 2.0 * np.pi
    for s in range(0, len(ms), chunk):
        mt = ms[s:s + chunk] / box
        m2 = np.einsum("ma,ma->m", mt, mt)
        C = np.exp(-np.pi ** 2 * m2 / beta ** 2) / (np.pi * vol * m2)
        arg = tp * (mt @ xyz.T)                                  # [M, N]
        fac = (q[None, :] - 1j * tp * (mt @ dip.T)
               - (4.0 * np.pi ** 2 / 3.0) * np.einsum("ma,nab,mb->mn", mt, quad, mt))
        S = np.sum(fac * np.exp(-1j * arg), axis=1)              # [M]
        Z = (C * S)[:, None] * np.exp(1j * arg)                  # [M, N]
        out[0] += np.real(Z.sum(0))
        if order >= 1:
            out[1] += np.real(np.einsum("ma,mn->na", 1j * tp * mt, Z))
        if order >= 2:
            out[2] += np.real(np.einsum("ma,mb,mn->nab", 1j * tp * mt, 1j * tp * mt, Z))
        if order >= 3:
            out[3] += np.real(np.einsum("ma,mb,mc,mn->nabc", 1j * tp * mt, 1j * tp * mt, 1j * tp * mt, Z))
    return out


def strain_sum(xyz, box, beta, src_a, src_b, chunk=1500):
    """sum_{m != 0} C(m) Re[S_a(m) conj S_b(m)] K(m) [3,3] for two source sets
    src = (q [N], dip [N,3], quad [N,3,3]), with
        K(m)_ab = -delta_ab + 2 (1/|m|^2 + pi^2/beta^2) m_a m_b,
    the logarithmic derivative of C(m) under the homogeneous deformation x -> (I + e) x
    (V -> V det(I + e), m -> (I + e)^-T m; the phases m.x_j do not change). It is the
    structure-factor share of the strain derivative of sum_m C Re[S_a conj S_b]."""
    xyz = np.asarray(xyz, np.float64)
    box = np.asarray(box, np.float64)
    vol = float(np.prod(box))
    ms = kvectors(box, beta)
    tp = 2.0 * np.pi
    out = np.zeros((3, 3))
    for s in range(0, len(ms), chunk):
        mt = ms[s:s + chunk] / box
        m2 = np.einsum("ma,ma->m", mt, mt)
        C = np.exp(-np.pi ** 2 * m2 / beta ** 2) / (np.pi * vol * m2)
        ph = np.exp(-1j * tp * (mt @ xyz.T))                     # [M, N]
        S = []
        for q, dip, quad in (src_a, src_b):
            fac = (q[None, :] - 1j * tp * (mt @ dip.T)
                   - (4.0 * np.pi ** 2 / 3.0) * np.einsum("ma,nab,mb->mn", mt, quad, mt))
            S.append(np.sum(fac * ph, axis=1))
        w = C * np.real(S[0] * np.conj(S[1]))
        out += -np.sum(w) * np.eye(3)
        out += 2.0 * np.einsum("m,ma,mb->ab", w * (1.0 / m2 + np.pi ** 2 / beta ** 2), mt, mt)
    return out
