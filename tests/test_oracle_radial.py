"""Pins for the oracle's radial functions: each family satisfies the derivative
recursion X_{n+1} = -(1/r) dX_n/dr, checked by central differences, plus limits."""
import numpy as np
import pytest

from oracle import radial


def _fd_next(fun, r, h=1e-5):
    return -(fun(r + h) - fun(r - h)) / (2 * h) / r


@pytest.mark.parametrize("beta", [0.0, 0.35, 0.5446])
def test_screened_recursion(beta):
    r = np.linspace(0.8, 8.0, 23)
    for n in range(4):
        fd = _fd_next(lambda x: radial.ewald_b(x, beta, 4)[n], r)
        np.testing.assert_allclose(fd, radial.ewald_b(r, beta, 4)[n + 1], rtol=2e-7)


def test_screened_b0_is_erfc_over_r():
    from math import erfc
    r = np.array([0.7, 2.0, 7.0])
    want = np.array([erfc(0.5446 * x) / x for x in r])
    np.testing.assert_allclose(radial.ewald_b(r, 0.5446, 0)[0], want, rtol=1e-14)


@pytest.mark.parametrize("sigma", [0.0, 1.0])
def test_damped_recursion(sigma):
    """R_n = B_n - (1 - sigma lambda_{2n+1}) U_n: R_{n+1} = -(1/r) dR_n/dr for n = 1..3,
    which ties lambda_5, lambda_7 and lambda_9 to lambda_3."""
    r = np.linspace(0.9, 6.0, 17)
    ai, aj, a = 0.837, 0.496, 0.39
    full = radial.damped_r(r, 0.5446, ai, aj, a, sigma, nmax=4)
    for n in range(3):
        fd = _fd_next(lambda x: radial.damped_r(x, 0.5446, ai, aj, a, sigma, nmax=4)[n], r)
        np.testing.assert_allclose(fd, full[n + 1], rtol=5e-7, atol=1e-12)


def test_thole_limits():
    oml = radial.thole_one_minus_lambda(np.array([0.0, 60.0, np.inf]))
    np.testing.assert_allclose(oml[:, 0], 1.0)        # fully damped at contact
    assert np.all(np.abs(oml[:, 1:]) < 1e-20)         # undamped far away / alpha = 0
