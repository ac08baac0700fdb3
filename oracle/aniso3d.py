"""Oracle: the 3D anisotropic-scattering Nystrom operator in real spherical
harmonics, evaluated directly.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 3.1.2 expands the angular density and the phase function in spherical
harmonics and keeps the degrees l <= L of the phase function.  Written for a
real orthonormal basis Y_a, a = (l, m), index a = l^2 + l + m, M = (L+1)^2
channels, and the moments u_a(x) = (4 pi)^{-1/2} int_{S^2} Phi(x, v) Y_a(v) dv
(so u_0 is the mean density of the isotropic case), integrating the transport
equation along v (y = x - s v, dy = s^2 ds dv) gives the system of Fredholm
equations of the second kind

    u_a(x) = sum_b int K(x, y) W_ab(v) mu_s sigma_hat_{l_b} u_b(y) dy
           + int K(x, y) W_a0(v) f(y) dy,
    K(x, y) = exp(-mu_t |x - y|) / (4 pi |x - y|^2),   v = (x - y)/|x - y|,
    W_ab(v) = 4 pi Y_a(v) Y_b(v),

with sigma_hat_l the Legendre moments of the phase function (sigma_hat_0 = 1;
the paper's coefficient of Y_l^0 times sqrt(4 pi/(2l+1)), the factor of its
operator A; Henyey-Greenstein: g^l).  L = 0 is the isotropic equation of
Sec. 2.1.  The Nystrom rule (Sec. 2.3) takes the kernel at cell centres times
h^3 off the diagonal; the diagonal block is the kernel's integral over the
cell, D_ab = int_cell K(0, y) W_ab(y/|y|) dy (the cell is symmetric under
y -> -y, so the sign of v does not matter there).

Readings (the paper is silent or garbled on them): the real basis below
(no Condon-Shortley phase; the channel order a = l^2 + l + m); sigma_hat as
the Legendre moments; D_ab by the split into the six faces of the cube:
(1/4 pi) int_{S^2} W_ab(w) (1 - exp(-mu_t R(w)))/mu_t dw, each face
parametrised by its points (dw = a dx dy / rho^3), a q x q Gauss-Legendre
rule on each face (the face integrand is analytic there).

Real basis: Y_{l,0} = Y_l^0, Y_{l,m} = sqrt2 (-1)^m Re Y_l^m (m > 0),
Y_{l,-m} = sqrt2 (-1)^m Im Y_l^m (m > 0), from scipy's complex harmonics;
so Y_{1,-1}, Y_{1,0}, Y_{1,1} = sqrt(3/4pi) (y, z, x).

Pins (tests/test_oracle_aniso3d.py): the textbook closed forms for l <= 2,
orthonormality by a product rule exact for the degree, the addition theorem
against Legendre polynomials; D_00 against the isotropic oracle's cell
weight (QUADPACK in spherical coordinates), sum_m D_{lm,lm} = (2l+1) D_00,
the parity zeros; L = 0 against the isotropic direct sum; the discrete
parity-transpose symmetry; the outward first moment of a point source; a
solve with sigma_hat_1 = 0 whose mean density is the isotropic solution; one
transport step taken through the angular density instead (the
Henyey-Greenstein function integrated by brute-force sphere quadrature), which
fixes the normalisation of sigma_hat, the 4 pi of W_ab and the direction of v.

Field layout: real arrays (M, n, n, n) indexed [a, iz, iy, ix], x fastest.
"""
import math

import numpy as np
from scipy import special


def n_channels(L):
    return (L + 1) ** 2


def channel_l(L):
    """Degree l of every channel a = l^2 + l + m."""
    return np.concatenate([np.full(2 * l + 1, l) for l in range(L + 1)])


def real_sh(L, v):
    """Real orthonormal spherical harmonics Y_a(v), a = 0..(L+1)^2-1, at unit
    vectors v (..., 3) -> (..., M)."""
    v = np.asarray(v, dtype=np.float64)
    x, y, z = v[..., 0], v[..., 1], v[..., 2]
    # polar angle by arctan2: arccos(z) loses half the digits near the poles
    theta = np.arctan2(np.hypot(x, y), z)
    phi = np.arctan2(y, x)
    out = np.empty(v.shape[:-1] + (n_channels(L),))
    for l in range(L + 1):
        out[..., l * l + l] = special.sph_harm_y(l, 0, theta, phi).real
        for m in range(1, l + 1):
            c = special.sph_harm_y(l, m, theta, phi)
            s = math.sqrt(2.0) * (-1.0) ** m
            out[..., l * l + l + m] = s * c.real
            out[..., l * l + l - m] = s * c.imag
    return out


def pair_kernel(L, v):
    """W_ab(v) = 4 pi Y_a(v) Y_b(v) -> (..., M, M)."""
    Y = real_sh(L, v)
    return 4.0 * math.pi * Y[..., :, None] * Y[..., None, :]


def cell_weights(L, mu_t, h, q=40):
    """D_ab = int_cell exp(-mu_t r)/(4 pi r^2) W_ab(y/r) dy -> (M, M): over
    each face of the cube, (1/4pi) int W_ab(w) (1 - e^{-mu_t rho})/mu_t
    a dx dy / rho^3 with w = p/rho, p the face point, rho = |p|, a = h/2."""
    a = 0.5 * h
    t, w = np.polynomial.legendre.leggauss(q)
    X, Yy = np.meshgrid(a * t, a * t, indexing="ij")
    Wt = np.outer(w, w) * a * a
    rho = np.sqrt(X * X + Yy * Yy + a * a)
    rad = rho if mu_t == 0.0 else -np.expm1(-mu_t * rho) / mu_t
    base = Wt * rad * a / rho ** 3 / (4.0 * math.pi)
    M = n_channels(L)
    D = np.zeros((M, M))
    A = np.full_like(X, a)
    for axis in range(3):
        for sgn in (1.0, -1.0):
            p = [None, None, None]
            p[axis] = sgn * A
            others = [k for k in range(3) if k != axis]
            p[others[0]] = X
            p[others[1]] = Yy
            P = np.stack(p, axis=-1) / rho[..., None]
            D += np.einsum("ij,ijab->ab", base, pair_kernel(L, P))
    return D


def _offset_tables(n, h, mu_t, L):
    """kappa h^3 and Y_a at every cell offset o = x_i - x_j, |o_k| <= n-1,
    indexed [oz + n-1, oy + n-1, ox + n-1] (zero kernel at o = 0)."""
    o = np.arange(-(n - 1), n)
    OZ, OY, OX = np.meshgrid(o, o, o, indexing="ij")
    off = np.stack([OX, OY, OZ], axis=-1).astype(np.float64)
    r = h * np.sqrt((off ** 2).sum(-1))
    zero = r == 0
    r_safe = np.where(zero, 1.0, r)
    kap = np.where(zero, 0.0, h ** 3 * np.exp(-mu_t * r) / (4.0 * math.pi * r_safe ** 2))
    v = off / np.where(zero, 1.0, np.sqrt((off ** 2).sum(-1)))[..., None]
    v[zero] = (0.0, 0.0, 1.0)
    return kap, real_sh(L, v)


def ktilde(n, h, mu_t, L, x, rows=None, D=None):
    """out[a, i] = sum_b sum_j K~^{ab}_{ij} x[b, j] (the direct Nystrom sum),
    optionally only at the flat cell indices ``rows`` -> (M, len(rows))."""
    M = n_channels(L)
    N = n ** 3
    x = np.asarray(x, dtype=np.float64).reshape(M, N)
    D = cell_weights(L, mu_t, h) if D is None else D
    kap, Yo = _offset_tables(n, h, mu_t, L)
    idx = np.arange(N)
    jx, jy, jz = idx % n, (idx // n) % n, idx // (n * n)
    rows = idx if rows is None else np.asarray(rows)
    out = np.empty((M, len(rows)))
    for k, i in enumerate(rows):
        ix, iy, iz = i % n, (i // n) % n, i // (n * n)
        sel = (iz - jz + n - 1, iy - jy + n - 1, ix - jx + n - 1)
        kj = kap[sel]                      # (N,)
        Yj = Yo[sel]                       # (N, M)
        s = (Yj * x.T).sum(-1) * kj        # sum_b Y_b(v_ij) x_b(j) kappa_ij
        out[:, k] = 4.0 * math.pi * (Yj * s[:, None]).sum(0) + D @ x[:, i]
    return out


def apply_K(n, h, mu_t, mu_s, sigma_hat, u, rows=None, D=None):
    """(K u)_a = sum_b K~^{ab} mu_s sigma_hat_{l_b} u_b."""
    L = len(sigma_hat) - 1
    c = mu_s * np.asarray(sigma_hat, dtype=np.float64)[channel_l(L)]
    u = np.asarray(u, dtype=np.float64).reshape(n_channels(L), -1)
    return ktilde(n, h, mu_t, L, c[:, None] * u, rows=rows, D=D)


def rhs(n, h, mu_t, L, f, rows=None, D=None):
    """b_a = sum_j K~^{a0}_{ij} f_j (the source is isotropic)."""
    x = np.zeros((n_channels(L), n ** 3))
    x[0] = np.asarray(f, dtype=np.float64).reshape(-1)
    return ktilde(n, h, mu_t, L, x, rows=rows, D=D)


def assemble(n, h, mu_t, L, D=None):
    """Dense K~ as an (M N) x (M N) matrix, row index a N + i (small n only):
    entry (a i, b j) = 4 pi kappa_ij h^3 Y_a(v_ij) Y_b(v_ij), D_ab at i = j."""
    M, N = n_channels(L), n ** 3
    D = cell_weights(L, mu_t, h) if D is None else D
    kap, Yo = _offset_tables(n, h, mu_t, L)
    idx = np.arange(N)
    jx, jy, jz = idx % n, (idx // n) % n, idx // (n * n)
    out = np.empty((M, N, M, N))
    for i in range(N):
        ix, iy, iz = i % n, (i // n) % n, i // (n * n)
        sel = (iz - jz + n - 1, iy - jy + n - 1, ix - jx + n - 1)
        Yj = Yo[sel]
        T = 4.0 * math.pi * kap[sel][:, None, None] * Yj[:, :, None] * Yj[:, None, :]
        out[:, i, :, :] = T.transpose(1, 2, 0)
        out[:, i, :, i] += D
    return out.reshape(M * N, M * N)


def solve_dense(n, h, mu_t, mu_s, sigma_hat, f, Kt=None):
    """u = (I - K)^{-1} b by LU on the dense matrix -> (M, n, n, n)."""
    L = len(sigma_hat) - 1
    M, N = n_channels(L), n ** 3
    Kt = assemble(n, h, mu_t, L) if Kt is None else Kt
    c = mu_s * np.asarray(sigma_hat, dtype=np.float64)[channel_l(L)]
    A = np.eye(M * N) - Kt * np.repeat(c, N)[None, :]
    b = np.zeros(M * N)
    b[:] = Kt[:, :N] @ np.asarray(f, dtype=np.float64).reshape(-1)
    return np.linalg.solve(A, b).reshape(M, n, n, n)
