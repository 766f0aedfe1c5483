"""Ewald-screened and Thole-damped radial functions (oracle, FP64).

The paper names the electrostatics it accelerates (AMOEBA multipoles with Thole-damped
induced dipoles, smooth PME; Sec. 1.2 and its citations) without printing the formulas;
these are the standard definitions.

Screened functions, for n >= 1:
    B_0 = erfc(beta r)/r,
    B_n = [(2n-1) B_{n-1} + (2 beta^2)^n exp(-beta^2 r^2) / (beta sqrt(pi))] / r^2.
Undamped Coulomb derivatives: U_n = (2n-1)!! / r^(2n+1).
Thole damping (AMOEBA): s = a r^3 / sqrt(alpha_i alpha_j), and
    1 - lambda_3 = e^-s
    1 - lambda_5 = (1 + s) e^-s
    1 - lambda_7 = (1 + s + 3/5 s^2) e^-s
    1 - lambda_9 = (1 + s + 18/35 s^2 + 9/35 s^3) e^-s.
Real-space kernel with scale sigma in {0, 1}:  R_n = B_n - (1 - sigma lambda_{2n+1}) U_n.
All three families obey X_{n+1} = -(1/r) dX_n/dr, which the tests check numerically.
"""
import numpy as np
from scipy.special import erfc

SQRT_PI = np.sqrt(np.pi)


def ewald_b(r, beta, nmax):
    """B_0..B_nmax at distances r (array). beta = 0 gives the bare U_n."""
    r = np.asarray(r, dtype=np.float64)
    out = np.empty((nmax + 1,) + r.shape)
    r2 = r * r
    if beta == 0.0:
        out[0] = 1.0 / r
        for n in range(1, nmax + 1):
            out[n] = (2 * n - 1) * out[n - 1] / r2
        return out
    out[0] = erfc(beta * r) / r
    g = np.exp(-beta * beta * r2) / (beta * SQRT_PI)
    for n in range(1, nmax + 1):
        out[n] = ((2 * n - 1) * out[n - 1] + (2.0 * beta * beta) ** n * g) / r2
    return out


def coulomb_u(r, nmax):
    """U_0..U_nmax = (2n-1)!! / r^(2n+1)."""
    return ewald_b(r, 0.0, nmax)


def thole_s(r, alpha_i, alpha_j, a):
    """Thole argument s = a r^3 / sqrt(alpha_i alpha_j); inf where either alpha is 0."""
    prod = np.asarray(alpha_i, dtype=np.float64) * np.asarray(alpha_j, dtype=np.float64)
    with np.errstate(divide="ignore"):
        return np.where(prod > 0.0, a * r ** 3 / np.sqrt(np.where(prod > 0.0, prod, 1.0)), np.inf)


def thole_one_minus_lambda(s):
    """[1-lambda_3, 1-lambda_5, 1-lambda_7, 1-lambda_9] as an array [4, ...]."""
    s = np.asarray(s, dtype=np.float64)
    e = np.exp(-s)
    e = np.where(np.isinf(s), 0.0, e)
    s_ = np.where(np.isinf(s), 0.0, s)
    return np.stack([
        e,
        (1.0 + s_) * e,
        (1.0 + s_ + 0.6 * s_ ** 2) * e,
        (1.0 + s_ + (18.0 / 35.0) * s_ ** 2 + (9.0 / 35.0) * s_ ** 3) * e,
    ])


def damped_r(r, beta, alpha_i, alpha_j, a, sigma, nmax=4):
    """R_1..R_nmax (index n-1) with R_n = B_n - (1 - sigma lambda_{2n+1}) U_n.

    sigma is the pair's scale (array or scalar, 0 or 1). nmax <= 4.
    """
    b = ewald_b(r, beta, nmax)
    u = coulomb_u(r, nmax)
    oml = thole_one_minus_lambda(thole_s(r, alpha_i, alpha_j, a))   # 1 - lambda
    sigma = np.asarray(sigma, dtype=np.float64)
    out = []
    for n in range(1, nmax + 1):
        one_minus_sl = 1.0 - sigma * (1.0 - oml[n - 1])
        out.append(b[n] - one_minus_sl * u[n])
    return np.stack(out)
