"""Oracle: plain FP64 restatement of the homogeneous-medium method's operators.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Everything here follows the paper's definitions directly, with no FFT and no
symmetry tricks.  Field layout used throughout the oracle: a complex array of
shape ``(2L+1, n, n)`` (2D) holding modes k = -L..L in order, cell (i2, i1) at
``[k+L, i2, i1]`` (x index fastest); 3D isotropic fields are real ``(n, n, n)``
arrays indexed ``[i3, i2, i1]``.

Functions and what pins them (tests/test_oracle_pins.py):

* ``cell_weights_2d`` / ``cell_weight_3d`` -- the cell integral of the kernel
  (Sec. 2.3, the diagonal entry after Eq. iso_discretization).  Pinned by the
  closed forms at mu_t = 0 and by a 3x3 self-similar subdivision with
  tensor Gauss-Legendre on the non-singular sub-cells.
* ``ktilde_2d`` / ``ktilde_3d`` -- direct Nystrom sums (Eq. iso_discretization,
  Eq. ani_discretization).  Pinned by the point-source phase (Eq.
  ani_Fouriermode), by ray integration of the uncollided flux (Eq. def_cTinv),
  by reciprocity (P K~ Hermitian), by rotation equivariance and by the
  lattice sum tending to 1/mu_t.
* ``apply_K_2d``, ``rhs_2d``, ``solve_dense_2d``, ``gmres``, ``neumann``,
  ``sampled_residual_2d`` (and 3D analogues) -- the equation of Sec. 3.3
  (Eq. ani_AU) and of Sec. 2.3 for L = 0.  Pinned by mu_s = 0 (u = b),
  Neumann series versus LU, positivity, rotation equivariance, the Lemma
  Linfcontraction bound and grid refinement.  The sampled residuals are
  pinned by their vanishing at the dense LU solution (all cells, L = 0, 3, 4
  in 2D, and 3D) and by the identity r(u_LU + d) = -(I - K) d with (I - K)
  taken from the assembled dense matrix.
"""
import ctypes
import math
import warnings

import numpy as np
from scipy import integrate

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_Ktilde_2d.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int, ctypes.c_int, dp, dp, dp, ip, ctypes.c_int]
        lib.oracle_assemble_2d.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_int, ctypes.c_int, dp, dp]
        lib.oracle_Ktilde_3d.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, dp, dp, ip, ctypes.c_int]
        lib.oracle_assemble_3d.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, dp]
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def num_threads() -> int:
    """OpenMP threads the direct sums use."""
    return int(_load().oracle_num_threads())


# --------------------------------------------------------------------------
# Singular-cell weights (Sec. 2.3: "the integral of K~ at the i-th cell").
# --------------------------------------------------------------------------

def _radial_factor(mu_t, R):
    """int_0^R exp(-mu_t r) dr = (1 - exp(-mu_t R)) / mu_t (R when mu_t = 0)."""
    if mu_t == 0.0:
        return R
    return -math.expm1(-mu_t * R) / mu_t


def cell_weights_2d(mu_t: float, h: float, mmax: int) -> np.ndarray:
    """D_m = int_{cell} kappa(r) e^{i m theta_r} dr for m = -mmax..mmax (d = 2).

    kappa(r) = exp(-mu_t |r|) / (2 pi |r|) (Sec. 2.3.1).  In polar coordinates
    about the cell centre, r dr cancels the 1/|r|, leaving
    D_m = (1/2pi) int_0^{2pi} e^{i m phi} (1 - e^{-mu_t R(phi)})/mu_t dphi with
    R(phi) = (h/2) / max(|cos phi|, |sin phi|) the distance to the cell edge.
    The imaginary part vanishes by the reflection symmetry of the square, so
    the real part (a cosine integral) is returned.  Adaptive QUADPACK over the
    eight pieces between the kinks of R.
    """
    half = 0.5 * h
    out = np.zeros(2 * mmax + 1)

    def R(phi):
        return half / max(abs(math.cos(phi)), abs(math.sin(phi)))

    for m in range(0, mmax + 1):
        total = 0.0
        for q in range(8):
            a, b = q * math.pi / 4, (q + 1) * math.pi / 4
            with warnings.catch_warnings():
                # pieces that cancel (m not a multiple of 4) hit QUADPACK's
                # roundoff detector at the absolute floor; the sum is ~1e-19 h
                warnings.simplefilter("ignore", integrate.IntegrationWarning)
                val, _ = integrate.quad(lambda p: math.cos(m * p) * _radial_factor(mu_t, R(p)),
                                        a, b, epsabs=1e-17 * h, epsrel=2e-14, limit=200)
            total += val
        out[mmax + m] = out[mmax - m] = total / (2 * math.pi)
    return out


def cell_weight_3d(mu_t: float, h: float) -> float:
    """D = int_{cube} exp(-mu_t|r|)/(4 pi |r|^2) dr over one cell (d = 3).

    In spherical coordinates the r^2 of the volume element cancels, leaving
    (1/4pi) int_{S^2} (1 - e^{-mu_t R})/mu_t dOmega, R the distance from the
    centre to the cube surface.  By the 48-fold symmetry of the cube this is
    48 times the part over the cone that leaves through the +z face with
    0 <= phi <= pi/4, where R = (h/2)/cos(theta) and theta runs up to
    atan(1/cos phi).  Adaptive QUADPACK in (theta, phi).
    """
    a = 0.5 * h

    def inner(phi):
        tmax = math.atan(1.0 / math.cos(phi))
        val, _ = integrate.quad(lambda t: _radial_factor(mu_t, a / math.cos(t)) * math.sin(t),
                                0.0, tmax, epsabs=0.0, epsrel=2e-14, limit=200)
        return val

    val, _ = integrate.quad(inner, 0.0, math.pi / 4, epsabs=0.0, epsrel=2e-14, limit=200)
    return 48.0 * val / (4.0 * math.pi)


# --------------------------------------------------------------------------
# Direct Nystrom sums.
# --------------------------------------------------------------------------

def ktilde_2d(n, h, mu_t, phi, Lo, rows=None, D=None):
    """out[k, i] = sum_j sum_k' K~[(i,k),(j,k')] phi[k', j], k = -Lo..Lo.

    ``phi`` has shape (2Li+1, n, n) complex.  With ``rows`` (flat cell indices
    i = i2*n + i1) only those cells are evaluated; the result then has shape
    (2Lo+1, len(rows)).  Otherwise (2Lo+1, n, n).
    """
    lib = _load()
    phi = np.ascontiguousarray(phi, dtype=np.complex128)
    Mi = phi.shape[0]
    Li = (Mi - 1) // 2
    assert phi.shape == (Mi, n, n)
    if D is None:
        D = cell_weights_2d(mu_t, h, Lo + Li)
    D = np.ascontiguousarray(D, dtype=np.float64)
    assert D.shape == (2 * (Lo + Li) + 1,)
    pin = phi.view(np.float64)
    if rows is None:
        out = np.zeros((2 * Lo + 1, n, n), dtype=np.complex128)
        lib.oracle_Ktilde_2d(n, h, mu_t, Lo, Li, _dp(D), _dp(pin), _dp(out.view(np.float64)), None, 0)
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        out = np.zeros((2 * Lo + 1, rows.size), dtype=np.complex128)
        lib.oracle_Ktilde_2d(n, h, mu_t, Lo, Li, _dp(D), _dp(pin), _dp(out.view(np.float64)),
                             rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), int(rows.size))
    return out


def assemble_ktilde_2d(n, h, mu_t, L, D=None):
    """Dense K~ of size (2L+1)N x (2L+1)N, mode-major ordering (k, i)."""
    lib = _load()
    N = n * n
    M = 2 * L + 1
    if D is None:
        D = cell_weights_2d(mu_t, h, 2 * L)
    D = np.ascontiguousarray(D, dtype=np.float64)
    A = np.zeros((M * N, M * N), dtype=np.complex128)
    lib.oracle_assemble_2d(n, h, mu_t, L, L, _dp(D), _dp(A.view(np.float64)))
    return A


def ktilde_3d(n, h, mu_t, phi, rows=None, D=None):
    """out[i] = sum_j K~[i,j] phi[j] for the 3D isotropic kernel."""
    lib = _load()
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    assert phi.shape == (n, n, n)
    if D is None:
        D = cell_weight_3d(mu_t, h)
    if rows is None:
        out = np.zeros((n, n, n))
        lib.oracle_Ktilde_3d(n, h, mu_t, float(D), _dp(phi), _dp(out), None, 0)
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        out = np.zeros(rows.size)
        lib.oracle_Ktilde_3d(n, h, mu_t, float(D), _dp(phi), _dp(out),
                             rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), int(rows.size))
    return out


def assemble_ktilde_3d(n, h, mu_t, D=None):
    lib = _load()
    N = n ** 3
    if D is None:
        D = cell_weight_3d(mu_t, h)
    A = np.zeros((N, N))
    lib.oracle_assemble_3d(n, h, mu_t, float(D), _dp(A))
    return A


# --------------------------------------------------------------------------
# The equation (Sec. 3.3, Eq. ani_discretization / ani_AU; Sec. 2.3 for L=0).
#   K u = mu_s K~ (sigma_hat * u)     (sigma_hat weights the SOURCE mode k')
#   b   = K~ g,  g = f in mode 0       (T.1)
#   (I - K) u = b                      (T.2)
# --------------------------------------------------------------------------

def _sigma_full(sigma_hat):
    """sigma_hat given for |k| = 0..L  ->  array over k = -L..L."""
    s = np.asarray(sigma_hat, dtype=np.float64)
    return np.concatenate([s[:0:-1], s])


def apply_K_2d(n, h, mu_t, mu_s, sigma_hat, u, rows=None, D=None):
    L = (u.shape[0] - 1) // 2
    w = mu_s * _sigma_full(sigma_hat)[:, None, None] * u
    return ktilde_2d(n, h, mu_t, w, L, rows=rows, D=D)


def rhs_2d(n, h, mu_t, L, f, rows=None, D=None):
    g = np.asarray(f, dtype=np.complex128).reshape(1, n, n)
    return ktilde_2d(n, h, mu_t, g, L, rows=rows, D=D)


def apply_A_2d(n, h, mu_t, mu_s, sigma_hat, u, D=None):
    return u - apply_K_2d(n, h, mu_t, mu_s, sigma_hat, u, D=D)


def solve_dense_2d(n, h, mu_t, mu_s, sigma_hat, f):
    """Direct solve of (I - K) u = K~ g with LU (numpy.linalg.solve)."""
    L = len(sigma_hat) - 1
    Kt = assemble_ktilde_2d(n, h, mu_t, L)
    N = n * n
    sig = np.repeat(_sigma_full(sigma_hat), N)
    A = np.eye(Kt.shape[0], dtype=np.complex128) - mu_s * Kt * sig[None, :]
    g = np.zeros(Kt.shape[0], dtype=np.complex128)
    g[L * N:(L + 1) * N] = np.asarray(f).reshape(-1)
    b = Kt @ g
    u = np.linalg.solve(A, b)
    return u.reshape(2 * L + 1, n, n), b.reshape(2 * L + 1, n, n)


def apply_K_3d(n, h, mu_t, mu_s, u, rows=None, D=None):
    return mu_s * ktilde_3d(n, h, mu_t, u, rows=rows, D=D)


def rhs_3d(n, h, mu_t, f, rows=None, D=None):
    return ktilde_3d(n, h, mu_t, np.asarray(f, dtype=np.float64), rows=rows, D=D)


def solve_dense_3d(n, h, mu_t, mu_s, f):
    Kt = assemble_ktilde_3d(n, h, mu_t)
    b = Kt @ np.asarray(f, dtype=np.float64).reshape(-1)
    A = np.eye(Kt.shape[0]) - mu_s * Kt
    return np.linalg.solve(A, b).reshape(n, n, n), b.reshape(n, n, n)


def gmres(apply_A, b, tol=1e-10, restart=100, maxit=2000, x0=None):
    """Textbook restarted GMRES (Saad & Schultz), modified Gram-Schmidt Arnoldi,
    least squares by numpy.linalg.lstsq.  Stops when ||b - A x|| <= tol ||b||
    (true residual recomputed at each restart).  Returns (x, iterations, relres).
    """
    shape = b.shape
    bv = b.reshape(-1)
    x = np.zeros_like(bv) if x0 is None else x0.reshape(-1).astype(bv.dtype).copy()
    bnorm = np.linalg.norm(bv)
    if bnorm == 0.0:
        return x.reshape(shape), 0, 0.0
    its = 0
    while True:
        r = bv - apply_A(x.reshape(shape)).reshape(-1)
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm or its >= maxit:
            return x.reshape(shape), its, beta / bnorm
        V = [r / beta]
        H = np.zeros((restart + 1, restart), dtype=bv.dtype)
        y = None
        for j in range(restart):
            w = apply_A(V[j].reshape(shape)).reshape(-1)
            its += 1
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            e1 = np.zeros(j + 2, dtype=bv.dtype)
            e1[0] = beta
            y = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)[0]
            res = np.linalg.norm(e1 - H[:j + 2, :j + 1] @ y)
            if res <= tol * bnorm * 0.5 or H[j + 1, j] == 0.0 or its >= maxit:
                break
            V.append(w / H[j + 1, j])
        x = x + sum(y[i] * V[i] for i in range(len(y)))


def neumann(apply_K, b, terms):
    """u = sum_{j=0}^{terms-1} K^j b  (the contraction of Lemma Linfcontraction)."""
    u = b.copy()
    t = b.copy()
    for _ in range(terms - 1):
        t = apply_K(t)
        u = u + t
    return u


def sampled_residual_2d(n, h, mu_t, mu_s, sigma_hat, f, u, rows):
    """r = b - u + K u at the listed cells, all modes; FP64 direct sums."""
    L = (u.shape[0] - 1) // 2
    D = cell_weights_2d(mu_t, h, 2 * L)
    Ku = apply_K_2d(n, h, mu_t, mu_s, sigma_hat, u, rows=rows, D=D)
    # the right-hand side couples only the source mode k' = 0: m = -L..L
    b = rhs_2d(n, h, mu_t, L, f, rows=rows, D=D[L:3 * L + 1])
    ur = u.reshape(u.shape[0], -1)[:, rows]
    return b - ur + Ku, b


def sampled_residual_3d(n, h, mu_t, mu_s, f, u, rows):
    D = cell_weight_3d(mu_t, h)
    Ku = apply_K_3d(n, h, mu_t, mu_s, u, rows=rows, D=D)
    b = rhs_3d(n, h, mu_t, f, rows=rows, D=D)
    return b - u.reshape(-1)[rows] + Ku, b


def rel_l2(a, b):
    """Relative L2 error ||a - b|| / ||b|| (the paper's error measure, Sec. 2.4)."""
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))
