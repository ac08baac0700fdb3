"""Pins of the inhomogeneous-medium oracle (oracle/inhom.py) against what the
paper and the mathematics fix, on the CPU."""
import math

import numpy as np
import pytest

import oracle
from oracle import inhom


def test_constant_mu_t_reduces_to_the_homogeneous_operator():
    """mu_t constant: every off-diagonal entry is h^2 e^{-mu_t r}/(2 pi r)
    exactly (the line integral of a constant); the diagonal is the exact cell
    integral D_0 to the 15 x 15 rule's accuracy (its smooth part has a |r|
    kink at the centre, so the tensor rule converges like q^-3: 2.3e-5 at
    mu_t h = 0.75)."""
    n, h, mu_t = 6, 1.0 / 6, 3.0
    mu = np.full((n, n), mu_t)
    D = inhom.diag_2d(mu, h)
    M = inhom.matrix_2d(mu, h, D=D)
    d0 = oracle.cell_weights_2d(mu_t, h, 0)[0]
    np.testing.assert_allclose(D, d0, rtol=5e-5)
    N = n * n
    ref = np.empty((N, N))
    for j in range(N):
        e = np.zeros((1, n, n), complex)
        e[0].flat[j] = 1.0
        ref[:, j] = oracle.ktilde_2d(n, h, mu_t, e, 0, D=np.array([d0])).real.reshape(-1)
    off = ~np.eye(N, dtype=bool)
    np.testing.assert_allclose(M[off], ref[off], rtol=1e-13)


def test_linear_mu_t_optical_depth_is_exact():
    """mu_t = a + b x + c y: bilinear interpolation and 5-point Gauss-Legendre
    are exact on segments between cell centres, so E_ij = exp(-r (mu_i + mu_j)/2).
    The grid is not symmetric in x and y, so a transposed sample index fails."""
    n = 7
    h = 1.0 / n
    a, b, c = 2.0, 5.0, -1.5
    xc = (np.arange(n) + 0.5) * h
    mu = a + b * xc[None, :] + c * xc[:, None]  # [i2, i1]
    M = inhom.matrix_2d(mu, h, D=np.zeros((n, n)))
    idx = np.arange(n * n)
    cx, cy = xc[idx % n], xc[idx // n]
    mui = a + b * cx + c * cy
    for i in (0, 9, 24, 48):
        r = np.hypot(cx - cx[i], cy - cy[i])
        mask = r > 0
        want = h * h * np.exp(-r[mask] * 0.5 * (mui[i] + mui[mask])) / (2 * math.pi * r[mask])
        np.testing.assert_allclose(M[i, mask], want, rtol=1e-13)


def test_diagonal_neighbour_optical_depth_by_hand():
    """Between the centres of diagonal neighbours the interpolant is
    (1-s)^2 m00 + s(1-s)(m10 + m01) + s^2 m11, a quadratic that 5-point
    Gauss-Legendre integrates exactly: m00/3 + (m10 + m01)/6 + m11/3."""
    n, h = 3, 0.25
    mu = np.array([[1.0, 4.0, 2.0], [3.0, 7.0, 5.0], [6.0, 0.5, 8.0]])  # [i2, i1]
    tau, r = inhom.optical_depth(mu, h, 0.5 * h, 0.5 * h, 1.5 * h, 1.5 * h)
    want = math.sqrt(2) * h * (mu[0, 0] / 3 + (mu[0, 1] + mu[1, 0]) / 6 + mu[1, 1] / 3)
    assert float(tau) == pytest.approx(want, rel=1e-14)
    # a horizontal neighbour: the x neighbour of sample [0, 0] is [0, 1]
    tau, r = inhom.optical_depth(mu, h, 0.5 * h, 0.5 * h, 1.5 * h, 0.5 * h)
    assert float(tau) == pytest.approx(h * (mu[0, 0] + mu[0, 1]) / 2, rel=1e-14)


def test_matrix_is_symmetric():
    """E(x, y) = E(y, x): the 5-point nodes are symmetric about s = 1/2."""
    n, h = 5, 0.2
    rng = np.random.default_rng(3)
    mu = 1.0 + 4.0 * rng.random((n, n))
    M = inhom.matrix_2d(mu, h, D=np.zeros((n, n)))
    np.testing.assert_allclose(M, M.T, rtol=1e-13, atol=0)


def test_diagonal_zero_mu_t_and_rule_convergence():
    """mu_t = 0: K~_ii = (2h/pi) ln(1 + sqrt 2) exactly.  A varying mu_t
    (mu_t h <= 1): the q-point rules converge -- 15 points within 5e-4 of 81
    (the interpolated mu_t has kinks along the centre lines, so the rule
    converges like q^-2.4 here), 41 points at least three times closer."""
    n, h = 4, 0.25
    D = inhom.diag_2d(np.zeros((n, n)), h)
    np.testing.assert_allclose(D, 2 * h / math.pi * math.log(1 + math.sqrt(2)), rtol=1e-15)
    n, h = 6, 1.0 / 6
    rng = np.random.default_rng(5)
    mu = 1.0 + 5.0 * rng.random((n, n))
    d15, d41, d81 = (inhom.diag_2d(mu, h, q=q) for q in (15, 41, 81))
    e15 = np.abs(d15 - d81) / d81
    e41 = np.abs(d41 - d81) / d81
    assert e15.max() < 5e-4
    assert e41.max() < e15.max() / 3
