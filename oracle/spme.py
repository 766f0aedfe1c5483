"""Smooth particle-mesh Ewald for multipoles (oracle, FP64, SPME mode).

The five steps of Sec. 1.2.2 ("Reciprocal space scheme"): spread the multipolar
density on a K1 x K2 x K3 grid with order-p cardinal B-splines, forward FFT, multiply
by the reciprocal kernel, backward FFT, and gather the potential and its derivatives
with B-spline derivatives. The FFT is NumPy's.

Conventions shared with the GPU path (readings, since the paper prints no formulas):
  * fractional coordinate u_a = K_a x_a / L_a; with b = floor(u) and w = u - b, the
    stencil points are k = (b - t) mod K for t = 0..p-1 with weight M_p(w + t);
  * a site at x_j spreads (q + d.grad_j + (1/3) Q:grad_j grad_j) W(x_j; k), with
    W(x; k) = prod_a M_p(u_a - k_a) periodised and grad_j acting on x_j, so each
    Cartesian derivative is (K_a / L_a) d/du_a;
  * phi_grid = IDFT[ B(m) C(m) DFT[Q] ] (unnormalised inverse), with
    C(m) = exp(-pi^2 |m|^2 / beta^2) / (pi V |m|^2), m aliased to [-K/2, K/2), C(0) = 0,
    B(m) = prod_a |b_a(m_a)|^2, |b(m)|^2 = 1 / |sum_{k=0}^{p-2} M_p(k+1) e^{2 pi i m k/K}|^2;
  * for odd p the sum vanishes at m = K/2 (even K); there |b|^2 is the mean of its two
    neighbours.
"""
import numpy as np
from math import comb


def cardinal_bspline(n, x):
    """M_n(x) by the recursion M_n(x) = [x M_{n-1}(x) + (n - x) M_{n-1}(x - 1)] / (n - 1),
    M_2(x) = 1 - |x - 1| on [0, 2] and 0 elsewhere."""
    x = np.asarray(x, np.float64)
    if n == 2:
        return np.where((x >= 0.0) & (x <= 2.0), 1.0 - np.abs(x - 1.0), 0.0)
    return (x * cardinal_bspline(n - 1, x) + (n - x) * cardinal_bspline(n - 1, x - 1.0)) / (n - 1)


def cardinal_bspline_deriv(n, x, k):
    """k-th derivative: M_n^(k)(x) = sum_l (-1)^l C(k, l) M_{n-k}(x - l), n - k >= 2."""
    if k == 0:
        return cardinal_bspline(n, x)
    return sum((-1) ** l * comb(k, l) * cardinal_bspline(n - k, np.asarray(x) - l) for l in range(k + 1))


def stencil(xyz, box, K, order, nderiv):
    """Grid indices [N, 3, p] and weights theta[d][N, 3, p] = d-th u-derivative of
    M_p(w + t), for d = 0..nderiv."""
    u = np.asarray(xyz) * (np.asarray(K) / np.asarray(box))
    b = np.floor(u)
    w = u - b
    t = np.arange(order)
    idx = (b[:, :, None].astype(np.int64) - t[None, None, :]) % np.asarray(K)[None, :, None]
    theta = [cardinal_bspline_deriv(order, w[:, :, None] + t[None, None, :], d) for d in range(nderiv + 1)]
    return idx, theta


def _deriv_weights(theta, box, K, nx, ny, nz):
    """Stencil weights [N, p, p, p] of d^(nx,ny,nz) W / dx^nx dy^ny dz^nz."""
    s = np.asarray(K) / np.asarray(box)
    return (s[0] ** nx * s[1] ** ny * s[2] ** nz) * np.einsum(
        "na,nb,nc->nabc", theta[nx][:, 0], theta[ny][:, 1], theta[nz][:, 2])


def _flat_index(idx, K):
    ix, iy, iz = idx[:, 0], idx[:, 1], idx[:, 2]
    return (ix[:, :, None, None] * K[1] + iy[:, None, :, None]) * K[2] + iz[:, None, None, :]


def spread(xyz, box, K, order, q, dip, quad, chunk=20000):
    """Grid Q[K1, K2, K3] of the multipolar density."""
    K = np.asarray(K)
    grid = np.zeros(int(np.prod(K)))
    for s in range(0, xyz.shape[0], chunk):
        sl = slice(s, s + chunk)
        idx, th = stencil(xyz[sl], box, K, order, 2)
        Qs = quad[sl]
        w = q[sl][:, None, None, None] * _deriv_weights(th, box, K, 0, 0, 0)
        for a, (nx, ny, nz) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
            w = w + dip[sl][:, a, None, None, None] * _deriv_weights(th, box, K, nx, ny, nz)
        for (a, b), (nx, ny, nz) in (((0, 0), (2, 0, 0)), ((1, 1), (0, 2, 0)), ((2, 2), (0, 0, 2)),
                                     ((0, 1), (1, 1, 0)), ((0, 2), (1, 0, 1)), ((1, 2), (0, 1, 1))):
            mult = 1.0 if a == b else 2.0
            w = w + (mult / 3.0) * Qs[:, a, b, None, None, None] * _deriv_weights(th, box, K, nx, ny, nz)
        np.add.at(grid, _flat_index(idx, K).ravel(), w.ravel())
    return grid.reshape(tuple(K))


def bspline_moduli(K, order):
    """|b(m)|^2 for m = 0..K-1, with the mean-of-neighbours rule where it is singular."""
    m = np.arange(K)
    k = np.arange(order - 1)
    mk = cardinal_bspline(order, k + 1.0)
    den = np.abs(np.sum(mk[None, :] * np.exp(2j * np.pi * np.outer(m, k) / K), axis=1)) ** 2
    out = np.empty(K)
    bad = den < 1e-10
    out[~bad] = 1.0 / den[~bad]
    for i in np.nonzero(bad)[0]:
        out[i] = 0.5 * (out[(i - 1) % K] + out[(i + 1) % K])
    return out


def influence(box, K, order, beta):
    """B(m) C(m) on the full grid [K1, K2, K3]."""
    K = np.asarray(K)
    box = np.asarray(box, np.float64)
    vol = float(np.prod(box))
    ms = [np.where(np.arange(k) < (k + 1) // 2, np.arange(k), np.arange(k) - k) / L for k, L in zip(K, box)]
    mx, my, mz = np.meshgrid(*ms, indexing="ij")
    m2 = mx ** 2 + my ** 2 + mz ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        C = np.exp(-np.pi ** 2 * m2 / beta ** 2) / (np.pi * vol * m2)
    C[0, 0, 0] = 0.0
    b = [bspline_moduli(k, order) for k in K]
    return C * b[0][:, None, None] * b[1][None, :, None] * b[2][None, None, :]


def convolve(grid, box, K, order, beta):
    """phi_grid = IDFT[B C DFT[Q]] with the unnormalised inverse transform."""
    G = influence(box, K, order, beta)
    return np.real(np.fft.ifftn(G * np.fft.fftn(grid))) * float(np.prod(K))


def gather(phi, xyz, box, K, order, max_order, chunk=20000):
    """Interpolated phi and its Cartesian derivatives up to max_order (<= 3) at atoms."""
    K = np.asarray(K)
    n = xyz.shape[0]
    out = [np.zeros(n), np.zeros((n, 3)), np.zeros((n, 3, 3)), np.zeros((n, 3, 3, 3))][: max_order + 1]
    flat = phi.ravel()
    for s in range(0, n, chunk):
        sl = slice(s, min(n, s + chunk))
        idx, th = stencil(xyz[sl], box, K, order, max_order)
        vals = flat[_flat_index(idx, K)]
        for tot in range(max_order + 1):
            for nx in range(tot + 1):
                for ny in range(tot - nx + 1):
                    nz = tot - nx - ny
                    v = np.einsum("nabc,nabc->n", _deriv_weights(th, box, K, nx, ny, nz), vals)
                    axes = [0] * nx + [1] * ny + [2] * nz
                    _assign_symmetric(out[tot], sl, axes, v)
    return out


def _assign_symmetric(arr, sl, axes, v):
    """Write v into every permutation of the derivative index tuple `axes`."""
    from itertools import permutations
    if len(axes) == 0:
        arr[sl] = v
        return
    for perm in set(permutations(axes)):
        arr[(sl,) + tuple(perm)] = v


def recip_derivs(xyz, box, beta, K, order, q, dip, quad, max_order):
    """SPME phi and derivatives at every atom from all sites (the EXACT-mode analogue)."""
    grid = spread(xyz, box, K, order, q, dip, quad)
    phi = convolve(grid, box, K, order, beta)
    return gather(phi, xyz, box, K, order, max_order)


def strain_sum(xyz, box, beta, K, order, src_a, src_b):
    """sum_m B(m) C(m) Re[F_a(m) conj F_b(m)] K(m) [3,3], F = DFT of the spread grid of
    each source set src = (q, dip, quad), K(m)_ab = -delta_ab + 2 (1/|m|^2 + pi^2/beta^2)
    m_a m_b: the smooth-PME counterpart of `ewald.strain_sum`. The B-spline moduli B(m)
    depend on the integer index only and the grid follows the fractional coordinates, so
    a homogeneous deformation changes only the volume and the Cartesian m."""
    K = np.asarray(K)
    box = np.asarray(box, np.float64)
    Fa = np.fft.fftn(spread(xyz, box, K, order, *src_a))
    Fb = np.fft.fftn(spread(xyz, box, K, order, *src_b))
    w = influence(box, K, order, beta) * np.real(Fa * np.conj(Fb))
    ms = [np.where(np.arange(k) < (k + 1) // 2, np.arange(k), np.arange(k) - k) / L for k, L in zip(K, box)]
    m = np.stack(np.meshgrid(*ms, indexing="ij"), -1)
    m2 = np.einsum("xyza,xyza->xyz", m, m)
    m2[0, 0, 0] = 1.0                                    # w is zero there
    out = -np.sum(w) * np.eye(3)
    out += 2.0 * np.einsum("xyz,xyza,xyzb->ab", w * (1.0 / m2 + np.pi ** 2 / beta ** 2), m, m)
    return out
