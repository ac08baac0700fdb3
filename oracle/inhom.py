"""Oracle: the inhomogeneous-medium isotropic Nystrom matrix in 2D, evaluated
directly.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 2.3, Eq. iso_discretization: for i != j the entry is the kernel at the
two cell centres times the cell area,

    K~_ij = h^2 E(x_i, x_j) / (2 pi |x_i - x_j|),
    E(x, y) = exp(-|x - y| int_0^1 mu_t(x - s (x - y)) ds)

(the kernel of Eq. iso_Fredholm2_2 with |S^1| = 2 pi), the line integral taken
by 5-point Gauss-Legendre on [0, 1] (Sec. 2.3, the paragraph after Eq. iso_AU).
The diagonal entry is the kernel's integral over the cell, split as the paper
does into the mean of 1/(2 pi r), known in closed form, and the smooth rest
(E - 1)/(2 pi r) by 15-point Gauss-Legendre:

    K~_ii = (2h/pi) ln(1 + sqrt 2) + int_cell (E(x_i, y) - 1) / (2 pi |x_i - y|) dy.

Readings (the paper is silent on them): mu_t at a point comes from its
cell-centred samples by bilinear interpolation, the sample index clamped to
the grid (constant beyond the outer centres); the 15-point rule is the tensor
rule on the cell, and at its centre node (r = 0) the smooth integrand takes its
limit -mu_t(x_i) / (2 pi).

Pins (tests/test_oracle_inhom.py): constant mu_t reduces to the homogeneous
oracle (``ktilde_2d`` with L = 0 and its exact cell weight, the diagonal to the
15-point rule's accuracy); mu_t linear in x, where bilinear interpolation and
5-point Gauss-Legendre are exact, gives E = exp(-|x - y| (mu_t(x) + mu_t(y))/2);
K~ is symmetric; a two-valued mu_t against a hand-integrated optical depth.

Field layout: real arrays (n, n) indexed [i2, i1], x index fastest; cell
(i1, i2) has its centre at ((i1 + 1/2) h, (i2 + 1/2) h).
"""
import math

import numpy as np

LN1P_SQRT2 = math.log(1.0 + math.sqrt(2.0))


def gauss_legendre_01(q):
    """q-point Gauss-Legendre nodes and weights on [0, 1] (numpy's rule on [-1, 1], mapped)."""
    x, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (x + 1.0), 0.5 * w


def mu_at(mu, h, px, py):
    """mu_t at points (px, py) by bilinear interpolation of the cell-centred
    samples mu[i2, i1], the sample index clamped to the grid."""
    mu = np.asarray(mu, dtype=np.float64)
    n = mu.shape[0]
    px = np.asarray(px, dtype=np.float64)
    py = np.asarray(py, dtype=np.float64)
    if n == 1:
        return np.full(np.broadcast(px, py).shape, mu[0, 0])
    u = px / h - 0.5
    v = py / h - 0.5
    i0 = np.clip(np.floor(u), 0, n - 2).astype(np.int64)
    j0 = np.clip(np.floor(v), 0, n - 2).astype(np.int64)
    t = np.clip(u - i0, 0.0, 1.0)
    s = np.clip(v - j0, 0.0, 1.0)
    return ((1 - t) * (1 - s) * mu[j0, i0] + t * (1 - s) * mu[j0, i0 + 1]
            + (1 - t) * s * mu[j0 + 1, i0] + t * s * mu[j0 + 1, i0 + 1])


def optical_depth(mu, h, x0, y0, x1, y1, q=5):
    """|p1 - p0| int_0^1 mu_t(p0 - s (p0 - p1)) ds by q-point Gauss-Legendre."""
    s, w = gauss_legendre_01(q)
    dx = np.asarray(x1, dtype=np.float64) - x0
    dy = np.asarray(y1, dtype=np.float64) - y0
    r = np.hypot(dx, dy)
    acc = 0.0
    for sq, wq in zip(s, w):
        acc = acc + wq * mu_at(mu, h, x0 + sq * dx, y0 + sq * dy)
    return r * acc, r


def diag_2d(mu, h, q=15):
    """K~_ii for every cell: (2h/pi) ln(1 + sqrt 2) plus the smooth part by the
    q x q tensor Gauss-Legendre rule on the cell (limit -mu_t(x_i)/(2 pi) at r = 0)."""
    mu = np.asarray(mu, dtype=np.float64)
    n = mu.shape[0]
    xg, wg = np.polynomial.legendre.leggauss(q)
    ya, yb = np.meshgrid(xg, xg, indexing="ij")  # node (a, b): offsets (xg[a], xg[b]) h/2
    wab = np.outer(wg, wg)
    out = np.empty((n, n))
    for i2 in range(n):
        for i1 in range(n):
            cx, cy = (i1 + 0.5) * h, (i2 + 0.5) * h
            tau, r = optical_depth(mu, h, cx, cy, cx + 0.5 * h * ya, cy + 0.5 * h * yb)
            r_safe = np.where(r > 0, r, 1.0)
            g = np.where(r > 0, np.expm1(-tau) / (2 * math.pi * r_safe),
                         -float(mu_at(mu, h, cx, cy)) / (2 * math.pi))
            out[i2, i1] = (2 * h / math.pi) * LN1P_SQRT2 + (0.5 * h) ** 2 * float(np.sum(wab * g))
    return out


def apply_2d(mu, h, x, rows=None, D=None):
    """y = K~ x (the direct O(N^2) sum), optionally only at the flat cell
    indices ``rows``; D = diag_2d(mu, h) may be passed in to reuse it."""
    mu = np.asarray(mu, dtype=np.float64)
    n = mu.shape[0]
    x = np.asarray(x, dtype=np.float64).reshape(-1)
    D = diag_2d(mu, h) if D is None else D
    idx = np.arange(n * n)
    cx = (idx % n + 0.5) * h
    cy = (idx // n + 0.5) * h
    rows = idx if rows is None else np.asarray(rows)
    out = np.empty(len(rows))
    for k, i in enumerate(rows):
        tau, r = optical_depth(mu, h, cx[i], cy[i], cx, cy)
        r_safe = np.where(r > 0, r, 1.0)
        kij = h * h * np.exp(-tau) / (2 * math.pi * r_safe)
        kij[i] = D.reshape(-1)[i]
        out[k] = kij @ x
    return out


def matrix_2d(mu, h, D=None):
    """The dense N x N matrix K~ (small n only)."""
    mu = np.asarray(mu, dtype=np.float64)
    n = mu.shape[0]
    D = diag_2d(mu, h) if D is None else D
    N = n * n
    M = np.empty((N, N))
    idx = np.arange(N)
    cx = (idx % n + 0.5) * h
    cy = (idx // n + 0.5) * h
    for i in range(N):
        tau, r = optical_depth(mu, h, cx[i], cy[i], cx, cy)
        r_safe = np.where(r > 0, r, 1.0)
        M[i] = h * h * np.exp(-tau) / (2 * math.pi * r_safe)
        M[i, i] = D.reshape(-1)[i]
    return M
