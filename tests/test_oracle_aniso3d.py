"""Pins of the 3D anisotropic oracle (oracle/aniso3d.py) against what the
paper and the mathematics fix, on the CPU."""
import math

import numpy as np
import pytest
from scipy import special

import oracle
from oracle import aniso3d as A


def _unit(rng, k):
    v = rng.standard_normal((k, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def test_real_harmonics_closed_forms():
    """Textbook Cartesian forms for l <= 2 (no Condon-Shortley phase):
    Y_1 = sqrt(3/4pi) (y, z, x); Y_2 = sqrt(15/4pi) (xy, yz, (3z^2-1)/(2 sqrt3), xz, (x^2-y^2)/2),
    also at and next to the poles (a polar angle from arccos(z) is off by
    1e-8 there once z has rounded to 1)."""
    v = _unit(np.random.default_rng(1), 50)
    # the poles and points 1e-9 off them, where z rounds to +-1 exactly
    v = np.concatenate([v, [[0, 0, 1], [0, 0, -1], [1e-9, 0, 1], [0, -1e-9, -1], [1e-9, 1e-9, 1]]])
    x, y, z = v.T
    Y = A.real_sh(2, v)
    c1, c2 = math.sqrt(3 / (4 * math.pi)), math.sqrt(15 / (4 * math.pi))
    want = np.stack([np.full_like(x, 1 / math.sqrt(4 * math.pi)),
                     c1 * y, c1 * z, c1 * x,
                     c2 * x * y, c2 * y * z, c2 * (3 * z * z - 1) / (2 * math.sqrt(3)), c2 * x * z,
                     c2 * (x * x - y * y) / 2], axis=1)
    np.testing.assert_allclose(Y, want, atol=1e-14)


def test_real_harmonics_orthonormal_and_addition_theorem():
    """Orthonormal on S^2 (Gauss-Legendre in cos(theta) x uniform in psi, exact
    for degree <= 8) and sum_m Y_lm(u) Y_lm(v) = (2l+1)/(4 pi) P_l(u.v)."""
    L = 4
    t, w = np.polynomial.legendre.leggauss(12)
    psi = 2 * math.pi * np.arange(24) / 24
    T, P = np.meshgrid(t, psi, indexing="ij")
    s = np.sqrt(1 - T * T)
    v = np.stack([s * np.cos(P), s * np.sin(P), T], axis=-1).reshape(-1, 3)
    wt = np.repeat(w, 24) * (2 * math.pi / 24)
    Y = A.real_sh(L, v)
    G = (Y * wt[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(A.n_channels(L)), atol=1e-13)
    rng = np.random.default_rng(2)
    u, v2 = _unit(rng, 30), _unit(rng, 30)
    Yu, Yv = A.real_sh(L, u), A.real_sh(L, v2)
    cosg = (u * v2).sum(1)
    for l in range(L + 1):
        sl = slice(l * l, (l + 1) * (l + 1))
        np.testing.assert_allclose((Yu[:, sl] * Yv[:, sl]).sum(1),
                                   (2 * l + 1) / (4 * math.pi) * special.eval_legendre(l, cosg), atol=1e-14)


@pytest.mark.parametrize("mu_t,h", [(3.0, 0.1), (0.0, 0.25), (40.0, 1.0 / 16)])
def test_cell_weights(mu_t, h):
    """D_00 is the isotropic cell weight (QUADPACK in spherical coordinates);
    sum over m of D_{lm,lm} is (2l+1) D_00 (the addition theorem at u = v);
    the cube's reflections make D_ab = 0 unless W_ab is even in x, y and z,
    and its rotations make the three l = 1 entries equal."""
    L = 3
    D = A.cell_weights(L, mu_t, h)
    d0 = oracle.cell_weight_3d(mu_t, h)
    assert D[0, 0] == pytest.approx(d0, rel=1e-13)
    for l in range(L + 1):
        sl = slice(l * l, (l + 1) * (l + 1))
        assert np.trace(D[sl, sl]) == pytest.approx((2 * l + 1) * d0, rel=1e-13)
    np.testing.assert_allclose(np.diag(D)[1:4], d0, rtol=1e-13)
    # parity of Y_a under x, y, z reflection from its values at mirrored points
    v = _unit(np.random.default_rng(3), 8)
    Y = A.real_sh(L, v)
    even = np.ones((A.n_channels(L),) * 2, bool)
    for k in range(3):
        m = v.copy()
        m[:, k] *= -1
        p = np.sign(np.round(A.real_sh(L, m)[0] / Y[0], 6))
        even &= np.outer(p, p) > 0
    assert np.abs(D[~even]).max() < 1e-12 * d0


def test_isotropic_reduction():
    """L = 0: the operator is the isotropic 3D direct sum (Sec. 2.1)."""
    n, h, mu_t = 5, 0.2, 4.0
    x = np.random.default_rng(4).standard_normal((n, n, n))
    got = A.ktilde(n, h, mu_t, 0, x[None]).reshape(n, n, n)
    want = oracle.ktilde_3d(n, h, mu_t, x)
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-15 * np.abs(want).max())


def test_parity_transpose_symmetry_and_direct_sum():
    """W_ab(-v) = (-1)^(l_a + l_b) W_ab(v), so with P = diag((-1)^l_a),
    P K~ P = K~^T; the assembled matrix agrees with the row sums."""
    n, h, mu_t, L = 3, 1.0 / 3, 2.0, 2
    K = A.assemble(n, h, mu_t, L)
    N = n ** 3
    p = np.repeat((-1.0) ** A.channel_l(L), N)
    np.testing.assert_allclose(p[:, None] * K * p[None, :], K.T, atol=1e-15)
    x = np.random.default_rng(5).standard_normal(A.n_channels(L) * N)
    np.testing.assert_allclose(A.ktilde(n, h, mu_t, L, x).reshape(-1), K @ x, rtol=1e-13, atol=1e-15)


def test_point_source_first_moment_points_outward():
    """A point source at cell j: b_(1,m)(x_i) = sqrt3 b_0(x_i) v_ij with
    v_ij = (x_i - x_j)/|x_i - x_j| (the flux leaves the source), and the
    l = 2 moments are the matching quadratic forms."""
    n, h, mu_t = 5, 0.2, 1.5
    f = np.zeros((n, n, n))
    f[2, 1, 3] = 1.0  # [z, y, x]
    b = A.rhs(n, h, mu_t, 2, f).reshape(9, n, n, n)
    iz, iy, ix = np.meshgrid(range(n), range(n), range(n), indexing="ij")
    off = np.stack([ix - 3, iy - 1, iz - 2], -1).astype(float)
    r = np.linalg.norm(off, axis=-1)
    m = r > 0
    v = off[m] / r[m, None]
    b0 = b[0][m]
    assert (b0 > 0).all()
    np.testing.assert_allclose(b[3][m], math.sqrt(3) * b0 * v[:, 0], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(b[1][m], math.sqrt(3) * b0 * v[:, 1], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(b[2][m], math.sqrt(3) * b0 * v[:, 2], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(b[4][m], math.sqrt(15) * b0 * v[:, 0] * v[:, 1], rtol=1e-12, atol=1e-15)


def test_solve_with_no_anisotropy_matches_isotropic_solution():
    """sigma_hat = (1, 0): the l = 1 moments do not scatter, so the mean
    density solves the isotropic equation; the first moments follow from it
    by one application of K~^{a0} to mu_s u_0 + f."""
    n, h, mu_t, mu_s = 4, 0.25, 5.0, 4.5
    f = np.random.default_rng(6).random((n, n, n))
    u = A.solve_dense(n, h, mu_t, mu_s, [1.0, 0.0], f)
    u0, _ = oracle.solve_dense_3d(n, h, mu_t, mu_s, f)
    np.testing.assert_allclose(u[0], u0, rtol=1e-11)
    b = A.rhs(n, h, mu_t, 1, mu_s * u0 + f).reshape(4, n, n, n)
    np.testing.assert_allclose(u[1:], b[1:], rtol=1e-10, atol=1e-14)


def test_forward_scattering_solution_residual():
    """sigma_hat_l = g^l (Henyey-Greenstein, g = 0.6), L = 2: the dense solve
    satisfies u = K u + b to rounding, and forward scattering carries the
    first moment further from a source than sigma_hat_1 = 0 does."""
    n, h, mu_t, mu_s, L = 4, 0.25, 6.0, 5.4, 2
    sig = [0.6 ** l for l in range(L + 1)]
    f = np.zeros((n, n, n))
    f[1, 1, 1] = 1.0
    u = A.solve_dense(n, h, mu_t, mu_s, sig, f)
    r = u.reshape(9, -1) - A.apply_K(n, h, mu_t, mu_s, sig, u) - A.rhs(n, h, mu_t, L, f)
    assert np.abs(r).max() < 1e-12 * np.abs(u).max()
    u_iso1 = A.solve_dense(n, h, mu_t, mu_s, [1.0, 0.0, 0.0], f)
    far = (3, 3, 3)  # [z, y, x], diagonal from the source: flux along +x
    assert u[(3,) + far] > u_iso1[(3,) + far] > 0


def test_transport_step_from_the_angular_form():
    """Independent route through the angular density: a source cell j with
    moments u_b gives Phi(v') = sqrt(4 pi) sum_b u_b Y_b(v'); the scattered
    source S(v) = mu_s int sigma_HG(v.v') Phi(v') dv' by brute-force quadrature
    with the Henyey-Greenstein function itself (not its moments); transporting
    S along v = (x_i - x_j)/r gives the moments at cell i,
    u_a(i) = (4 pi)^{-1/2} h^3 e^{-mu_t r} / r^2 Y_a(v) S(v)  (Sec. 3.1.2 with
    y = x - s v, dy = s^2 ds dv).  The oracle's K with sigma_hat_l = g^l must
    agree: this fixes the normalisation of sigma_hat, the 4 pi of W_ab and the
    direction of v."""
    n, h, mu_t, mu_s, g, L = 4, 0.25, 3.0, 2.5, 0.5, 2
    M = A.n_channels(L)
    rng = np.random.default_rng(11)
    ub = rng.standard_normal(M)
    j = (0, 1, 3)  # [z, y, x]
    x = np.zeros((M, n, n, n))
    x[(slice(None),) + j] = ub
    y = A.apply_K(n, h, mu_t, mu_s, [g ** l for l in range(L + 1)], x).reshape(M, n, n, n)
    # sphere quadrature: Gauss-Legendre in cos(theta) x uniform in psi
    t, w = np.polynomial.legendre.leggauss(400)
    npsi = 800
    psi = 2 * math.pi * np.arange(npsi) / npsi
    T, P = np.meshgrid(t, psi, indexing="ij")
    s = np.sqrt(1 - T * T)
    vq = np.stack([s * np.cos(P), s * np.sin(P), T], -1).reshape(-1, 3)
    wq = np.repeat(w, npsi) * (2 * math.pi / npsi)
    phi = math.sqrt(4 * math.pi) * A.real_sh(L, vq) @ ub
    for i in [(3, 2, 0), (1, 1, 1), (2, 3, 2)]:
        off = np.array([i[2] - j[2], i[1] - j[1], i[0] - j[0]], float) * h
        r = np.linalg.norm(off)
        v = off / r
        cosg = vq @ v
        sig = (1 - g * g) / (4 * math.pi * (1 + g * g - 2 * g * cosg) ** 1.5)
        S = mu_s * np.sum(wq * sig * phi)
        want = h ** 3 * math.exp(-mu_t * r) / r ** 2 * A.real_sh(L, v[None])[0] * S / math.sqrt(4 * math.pi)
        np.testing.assert_allclose(y[(slice(None),) + i], want, rtol=1e-9, atol=1e-12 * np.abs(want).max())
