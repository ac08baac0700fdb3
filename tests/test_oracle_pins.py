"""Pins of the oracle against what the paper and the mathematics fix.

None of these retypes an oracle formula: each compares the oracle with an
independent route (a closed form, a different quadrature, a self-similar
subdivision, ray integration of the transport equation, a symmetry or bound
stated in the paper, or a second solver).
"""
import json
import math
import os

import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss

import oracle
import rte_synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# Singular-cell weights
# ---------------------------------------------------------------------------

def test_cell_weights_massless_closed_forms():
    """mu_t = 0: D_0 = (2h/pi) ln(1+sqrt2) and D_4 = (2h/pi)(ln(1+sqrt2) - 2sqrt2/3).

    With mu_t = 0 the cell integral of 1/(2 pi r) e^{i m phi} reduces to
    (1/2pi) int cos(m phi) R(phi) dphi, eight copies of an elementary integral
    of cos(m phi)/cos(phi) over [0, pi/4]."""
    with open(os.path.join(GOLDEN, "cell_weights.json")) as fh:
        gold = json.load(fh)
    for h in (1.0 / 64, 0.3, 1.0):
        D = oracle.cell_weights_2d(0.0, h, 4)
        lg = math.log(1 + math.sqrt(2))
        assert D[4] == pytest.approx(2 * h / math.pi * lg, rel=1e-13)
        assert D[8] == pytest.approx(2 * h / math.pi * (lg - 2 * math.sqrt(2) / 3), rel=1e-12)
        assert D[0] == D[8]
    assert oracle.cell_weights_2d(0.0, 1.0 / 64, 0)[0] == pytest.approx(gold["D0_massless_h1_64"], rel=1e-14)


def test_cell_weights_vanish_unless_multiple_of_four():
    """The square cell is invariant under 90-degree rotation: D_m = 0 unless 4 | m."""
    for mu in (0.0, 1.0, 37.0):
        D = oracle.cell_weights_2d(mu, 1.0 / 32, 8)
        for m in range(-8, 9):
            if m % 4:
                assert abs(D[m + 8]) < 1e-14 * D[8]


def _ring_2d(mu, h, m, npts=40):
    """Integral of kappa e^{i m theta} over the 8 outer sub-cells of a 3x3
    split of the cell of side h (none contains the singularity): tensor
    Gauss-Legendre in Cartesian coordinates."""
    x, w = leggauss(npts)
    a = h / 3.0
    tot = 0.0
    for cx in (-1, 0, 1):
        for cy in (-1, 0, 1):
            if cx == 0 and cy == 0:
                continue
            X = cx * a + 0.5 * a * x[None, :]
            Y = cy * a + 0.5 * a * x[:, None]
            r = np.hypot(X, Y)
            k = np.exp(-mu * r) / (2 * math.pi * r) * np.cos(m * np.arctan2(Y, X))
            tot += (0.25 * a * a) * float(np.sum(w[:, None] * w[None, :] * k))
    return tot


def _self_similar_2d(mu, h, m, depth, npts=40):
    """D_m(h) = D_m(h/3) + ring(h), recursed `depth` times; the remaining
    D_m(h/3^depth) is taken from the massless scaling D_m(h) = 1.5 ring_0(h)
    (D is linear in h at mu = 0), whose mass correction is O(mu h 3^-depth)."""
    tot = 0.0
    hh = h
    for _ in range(depth):
        tot += _ring_2d(mu, hh, m, npts)
        hh /= 3.0
    return tot + 1.5 * _ring_2d(0.0, hh, m, npts)


@pytest.mark.parametrize("mu,h,m", [(0.0, 1.0, 0), (0.0, 1.0, 4), (10.0, 1.0 / 64, 0),
                                    (10.0, 1.0 / 64, 4), (3.0, 0.5, 8), (100.0, 1.0 / 16, 0)])
def test_cell_weights_self_similar_subdivision(mu, h, m):
    depth = 0 if mu == 0.0 else 16
    ref = 1.5 * _ring_2d(0.0, h, m) if mu == 0.0 else _self_similar_2d(mu, h, m, depth)
    D = oracle.cell_weights_2d(mu, h, m)
    assert D[2 * m] == pytest.approx(ref, rel=1e-11, abs=1e-16)


@pytest.mark.parametrize("m,rel", [(32, 1e-11), (64, 2e-11), (128, 2e-10)])
def test_cell_weights_high_orders(m, rel):
    """The weights of the large truncations (2L up to 128): the self-similar
    subdivision with 160-point tensor rules per sub-cell (cos(m theta) runs
    through m/4 periods on a sub-cell next to the centre)."""
    ref = _self_similar_2d(10.0, 1.0 / 64, m, 16, npts=160)
    D = oracle.cell_weights_2d(10.0, 1.0 / 64, m)
    assert D[2 * m] == pytest.approx(ref, rel=rel)


def _ring_3d(mu, h, npts=24):
    x, w = leggauss(npts)
    a = h / 3.0
    W = w[:, None, None] * w[None, :, None] * w[None, None, :]
    tot = 0.0
    for cx in (-1, 0, 1):
        for cy in (-1, 0, 1):
            for cz in (-1, 0, 1):
                if cx == cy == cz == 0:
                    continue
                X = cx * a + 0.5 * a * x[None, None, :]
                Y = cy * a + 0.5 * a * x[None, :, None]
                Z = cz * a + 0.5 * a * x[:, None, None]
                r2 = X * X + Y * Y + Z * Z
                k = np.exp(-mu * np.sqrt(r2)) / (4 * math.pi * r2)
                tot += (0.125 * a ** 3) * float(np.sum(W * k))
    return tot


def test_cell_weight_3d_massless():
    """mu_t = 0: D = 1.5 x (integral over the 26 outer sub-cells), and D = 0.6106874 h
    (=(3/(4 pi)) int_{[-1,1]^2} du dv/(1+u^2+v^2) h)."""
    for h in (1.0, 1.0 / 128):
        ref = 1.5 * _ring_3d(0.0, h)
        assert oracle.cell_weight_3d(0.0, h) == pytest.approx(ref, rel=1e-11)
    assert oracle.cell_weight_3d(0.0, 1.0) == pytest.approx(0.6106874, rel=1e-7)


@pytest.mark.parametrize("mu,h", [(100.0, 1.0 / 128), (1.0, 0.5)])
def test_cell_weight_3d_self_similar(mu, h):
    tot, hh = 0.0, h
    for _ in range(14):
        tot += _ring_3d(mu, hh)
        hh /= 3.0
    tot += 1.5 * _ring_3d(0.0, hh)
    assert oracle.cell_weight_3d(mu, h) == pytest.approx(tot, rel=1e-10)


# ---------------------------------------------------------------------------
# Direct Nystrom sums
# ---------------------------------------------------------------------------

def test_point_source_phase():
    """Eq. ani_Fouriermode: Phi_hat(x,k) = avg Phi(x,theta) e^{-ik theta}.  With
    no scattering, flux from a point source at y reaches x travelling along
    x - y, so at a cell to the right of the source every mode has the same
    phase, directly above the phase is (-i)^k, to the left (-1)^k, below i^k."""
    n, L = 9, 3
    f = np.zeros((n, n))
    f[4, 4] = 1.0
    b = oracle.rhs_2d(n, 1.0 / n, 2.0, L, f)
    for d in (1, 3):
        cases = [((4, 4 + d), 1), ((4 + d, 4), -1j), ((4, 4 - d), -1), ((4 - d, 4), 1j)]
        for (i2, i1), phase in cases:
            b0 = b[L, i2, i1]
            assert b0.real > 0 and abs(b0.imag) < 1e-18
            for k in range(-L, L + 1):
                assert b[k + L, i2, i1] == pytest.approx(phase ** k * b0, rel=1e-12, abs=1e-18)


def _uncollided_modes(xy, mu, L, centre, width, ntheta=192, ns=160):
    """Phi_hat(x,k) for mu_s = 0 by the method of characteristics (Eq. def_cTinv):
    Phi(x, theta) = int_0^{tau} e^{-mu s} f(x - s v) ds, f the Gaussian restricted
    to the unit square, then the average over theta of Phi e^{-ik theta}.  The
    s-integral is split at the Gaussian's centre line with Gauss-Legendre on
    each piece; the theta average is the periodic trapezoid rule."""
    x, w = leggauss(ns)
    th = 2 * math.pi * np.arange(ntheta) / ntheta
    phi = np.zeros(ntheta)
    for t_i, t in enumerate(th):
        v = np.array([math.cos(t), math.sin(t)])
        # distance to leave the unit square going backwards (x - s v)
        taus = []
        for d in range(2):
            if v[d] > 0:
                taus.append(xy[d] / v[d])
            elif v[d] < 0:
                taus.append((xy[d] - 1.0) / v[d])
        tau = min(taus)
        s_star = float(np.clip(np.dot(np.asarray(xy) - centre, v), 0.0, tau))
        tot = 0.0
        for a, bnd in ((0.0, s_star), (s_star, tau)):
            if bnd <= a:
                continue
            s = a + (bnd - a) * 0.5 * (x + 1)
            px = xy[0] - s * v[0]
            py = xy[1] - s * v[1]
            fv = np.exp(-((px - centre[0]) ** 2 + (py - centre[1]) ** 2) / (2 * width * width))
            tot += 0.5 * (bnd - a) * float(np.sum(w * np.exp(-mu * s) * fv))
        phi[t_i] = tot
    return np.array([np.mean(phi * np.exp(-1j * k * th)) for k in range(-L, L + 1)])


def test_uncollided_flux_matches_ray_integration():
    """The Nystrom b = K~ g is the discretised uncollided angular-mode flux;
    compare with ray tracing of the transport equation, at two resolutions."""
    mu, L, centre, width = 2.0, 2, np.array([0.45, 0.55]), 0.12
    errs = []
    for n in (16, 32):
        f = rte_synth.gaussian_mixture_2d(n, [centre], [width])
        b = oracle.rhs_2d(n, 1.0 / n, mu, L, f)
        cells = [(n // 2, n // 2), (n // 4, 3 * n // 4), (n - 1, 1)]
        num, den = 0.0, 0.0
        for (i2, i1) in cells:
            xy = ((i1 + 0.5) / n, (i2 + 0.5) / n)
            ref = _uncollided_modes(xy, mu, L, centre, width)
            num += np.sum(np.abs(b[:, i2, i1] - ref) ** 2)
            den += np.sum(np.abs(ref) ** 2)
        errs.append(math.sqrt(num / den))
    # first order in h at cells inside the source (measured 2.5e-2 -> 1.35e-2)
    assert errs[1] < 2e-2
    assert errs[1] < 0.6 * errs[0]


def test_reciprocity_P_hermitian():
    """kappa(-r) = kappa(r), theta(-r) = theta(r) + pi: P K~ is Hermitian with
    P = diag((-1)^k), while K~ itself is not; and K = mu_s K~ diag(sigma_hat)
    puts sigma_hat on the source mode, so P K diag(1/sigma_hat) is Hermitian."""
    n, L, h, mu = 4, 2, 0.25, 1.7
    A = oracle.assemble_ktilde_2d(n, h, mu, L)
    N = n * n
    P = np.repeat([(-1.0) ** k for k in range(-L, L + 1)], N)
    PA = P[:, None] * A
    assert np.abs(PA - PA.conj().T).max() < 1e-16 * 1e3 * np.abs(A).max()
    assert np.abs(A - A.conj().T).max() > 1e-3 * np.abs(A).max()
    sig = np.array([1.0, 0.6, 0.3])
    u = np.zeros((2 * L + 1, n, n), complex)
    cols = []
    for c in range((2 * L + 1) * N):
        u.reshape(-1)[:] = 0
        u.reshape(-1)[c] = 1
        cols.append(oracle.apply_K_2d(n, h, mu, 0.8, sig, u).reshape(-1))
    K = np.array(cols).T
    sfull = np.repeat(np.concatenate([sig[:0:-1], sig]), N)
    B = P[:, None] * K / sfull[None, :]
    assert np.abs(B - B.conj().T).max() < 1e-13 * np.abs(B).max()


def _rot90(u):
    """Rotate mode fields by +90 degrees about the square's centre:
    u'_k(R x) = e^{-i k pi/2} u_k(x)  (Eq. ani_Fouriermode with theta -> theta + pi/2).
    Cell (i2, i1) moves to (i1, n-1-i2)."""
    M = u.shape[0]
    L = (M - 1) // 2
    out = np.empty_like(u)
    for kk in range(M):
        k = kk - L
        out[kk] = np.exp(-1j * k * math.pi / 2) * _rot_cells(u[kk])
    return out


def _rot_cells(a):
    n = a.shape[0]
    out = np.empty_like(a)
    for i2 in range(n):
        for i1 in range(n):
            out[i1, n - 1 - i2] = a[i2, i1]
    return out


def test_rotation_equivariance_matvec():
    n, L, h, mu = 6, 2, 1.0 / 6, 3.0
    rng = np.random.default_rng(5)
    u = rng.standard_normal((2 * L + 1, n, n)) + 1j * rng.standard_normal((2 * L + 1, n, n))
    sig = np.array([1.0, 0.5, 0.25])
    a = oracle.apply_K_2d(n, h, mu, 0.9 * mu, sig, _rot90(u))
    b = _rot90(oracle.apply_K_2d(n, h, mu, 0.9 * mu, sig, u))
    assert np.abs(a - b).max() < 1e-14 * np.abs(b).max()
    # the opposite phase convention must fail
    bad = np.array([np.exp(1j * k * math.pi) for k in range(-L, L + 1)])[:, None, None] * b
    assert np.abs(a - bad).max() > 1e-2 * np.abs(b).max()


def test_lattice_sum_tends_to_inverse_mu():
    """int_{R^2} kappa = 1/mu_t: the row sum at the centre of a large grid
    (whose edge is many mean free paths away) tends to 1/mu_t as h -> 0."""
    mu = 20.0
    errs = []
    for n in (64, 128, 256):
        ones = np.ones((1, n, n), complex)
        i = (n // 2) * n + n // 2
        s = oracle.ktilde_2d(n, 1.0 / n, mu, ones, 0, rows=[i])[0, 0].real
        errs.append(abs(s * mu - 1.0))
    # first order in h (measured 1.8e-2, 9.3e-3, 4.7e-3)
    assert errs[-1] < 6e-3
    assert errs[2] < 0.6 * errs[1] < 0.36 * errs[0]


def test_lattice_sum_3d():
    mu = 30.0
    errs = []
    for n in (32, 64):
        ones = np.ones((n, n, n))
        i = ((n // 2) * n + n // 2) * n + n // 2
        s = oracle.ktilde_3d(n, 1.0 / n, mu, ones, rows=[i])[0]
        errs.append(abs(s * mu - 1.0))
    # measured 6.2e-2 (n = 32), 3.8e-2 (n = 64)
    assert errs[-1] < 5e-2
    assert errs[1] < 0.7 * errs[0]


def test_3d_symmetric_and_ray_pin():
    """3D isotropic K~ is symmetric (Eq. iso_Fredholm2'), and b = K~ f agrees
    with the uncollided mean density from ray integration."""
    n = 4
    A = oracle.assemble_ktilde_3d(n, 0.25, 2.0)
    assert np.abs(A - A.T).max() == 0.0
    mu, centre, width = 3.0, np.array([0.5, 0.45, 0.55]), 0.15
    errs = []
    for n in (12, 24):
        f = rte_synth.gaussian_3d(n, centre, width)
        c = n // 2
        b = oracle.rhs_3d(n, 1.0 / n, mu, f, rows=[(c * n + c) * n + c])[0]
        xyz = np.array([(c + 0.5) / n] * 3)
        # ray integration over the sphere (product Gauss-Legendre in cos(theta), trapezoid in phi)
        ct, wt = leggauss(24)
        ph = 2 * math.pi * np.arange(48) / 48
        xs, ws = leggauss(80)
        tot = 0.0
        for c_t, w_t in zip(ct, wt):
            st = math.sqrt(1 - c_t * c_t)
            for p in ph:
                v = np.array([st * math.cos(p), st * math.sin(p), c_t])
                taus = [(xyz[d] / v[d]) if v[d] > 0 else ((xyz[d] - 1) / v[d]) for d in range(3) if v[d] != 0]
                tau = min(taus)
                s = 0.5 * tau * (xs + 1)
                pts = xyz[None, :] - s[:, None] * v[None, :]
                fv = np.exp(-np.sum((pts - centre) ** 2, axis=1) / (2 * width * width))
                tot += w_t * (2 * math.pi / 48) * 0.5 * tau * float(np.sum(ws * np.exp(-mu * s) * fv))
        ref = tot / (4 * math.pi)
        errs.append(abs(b - ref) / ref)
    # first order in h (measured 4.6e-2 at n = 12, 2.7e-2 at n = 24, 1.4e-2 at n = 48)
    assert errs[1] < 3.5e-2 and errs[1] < 0.7 * errs[0]


# ---------------------------------------------------------------------------
# Solves
# ---------------------------------------------------------------------------

def test_mu_s_zero_gives_rhs():
    """mu_s = 0 removes K: the solution is b = K~ g with no iteration (Eq. ani_2d_Fredholm)."""
    n, L = 6, 2
    f = rte_synth.gaussian_mixture_2d(n, [(0.4, 0.6)], [0.2])
    u, b = oracle.solve_dense_2d(n, 1.0 / n, 2.0, 0.0, rte_synth.hg_sigma_hat(0.5, L), f)
    assert np.abs(u - b).max() <= 1e-15 * np.abs(b).max()


def test_neumann_series_equals_dense_solve():
    """Lemma Linfcontraction: K is a contraction, so sum_j K^j b converges to the
    LU solution; at mu_s/mu_t = 0.1 thirty terms reach rounding."""
    n, L, h, mu = 6, 2, 1.0 / 6, 4.0
    sig = rte_synth.hg_sigma_hat(0.6, L)
    f = rte_synth.gaussian_mixture_2d(n, [(0.4, 0.6)], [0.2])
    u, b = oracle.solve_dense_2d(n, h, mu, 0.1 * mu, sig, f)
    D = oracle.cell_weights_2d(mu, h, 2 * L)
    un = oracle.neumann(lambda t: oracle.apply_K_2d(n, h, mu, 0.1 * mu, sig, t, D=D), b, 30)
    assert oracle.rel_l2(un, u) < 1e-14


def test_gmres_matches_dense_solve():
    n, L, h, mu = 6, 3, 1.0 / 6, 10.0
    sig = rte_synth.hg_sigma_hat(0.5, L)
    f = rte_synth.gaussian_mixture_2d(n, [(0.4, 0.6), (0.7, 0.2)], [0.2, 0.1])
    u, b = oracle.solve_dense_2d(n, h, mu, 0.95 * mu, sig, f)
    D = oracle.cell_weights_2d(mu, h, 2 * L)
    ug, its, rr = oracle.gmres(lambda t: t - oracle.apply_K_2d(n, h, mu, 0.95 * mu, sig, t, D=D),
                               b, tol=1e-13)
    assert rr <= 1e-13
    assert oracle.rel_l2(ug, u) < 1e-11


def test_solution_rotation_equivariance_and_symmetry():
    n, L, h, mu = 6, 2, 1.0 / 6, 5.0
    sig = rte_synth.hg_sigma_hat(0.7, L)
    f = rte_synth.gaussian_mixture_2d(n, [(0.3, 0.6)], [0.15])
    u, _ = oracle.solve_dense_2d(n, h, mu, 0.9 * mu, sig, f)
    fr = _rot_cells(f)
    ur, _ = oracle.solve_dense_2d(n, h, mu, 0.9 * mu, sig, fr)
    assert np.abs(ur - _rot90(u)).max() < 1e-13 * np.abs(u).max()
    # J-symmetry u_{-k} = conj(u_k) for a real source and real even sigma_hat
    assert np.abs(u[::-1] - u.conj()).max() < 1e-14 * np.abs(u).max()


def test_positivity_isotropic():
    """L = 0, f >= 0: every term of the Neumann series is >= 0, so u >= 0."""
    n = 8
    f = rte_synth.gaussian_mixture_2d(n, [(0.2, 0.3)], [0.05])
    u, _ = oracle.solve_dense_2d(n, 1.0 / n, 3.0, 2.9, np.array([1.0]), f)
    assert u.real.min() >= 0.0 and np.abs(u.imag).max() == 0.0


def test_contraction_and_a_priori_bounds():
    """Lemma Linfcontraction / Theorem existence with tau = sqrt(2) (unit square):
    ||K||_inf <= 1 - exp(-tau ||mu_s||) and ||u||_inf <= tau e^{tau mu_s} ||f||_inf."""
    n = 12
    tau = math.sqrt(2.0)
    for mu_t, mu_s in ((1.0, 1.0), (5.0, 4.0), (0.5, 0.1)):
        A = oracle.assemble_ktilde_2d(n, 1.0 / n, mu_t, 0).real
        assert mu_s * np.abs(A).sum(axis=1).max() <= 1 - math.exp(-tau * mu_s)
        f = rte_synth.gaussian_mixture_2d(n, [(0.5, 0.5)], [0.2])
        u, _ = oracle.solve_dense_2d(n, 1.0 / n, mu_t, mu_s, np.array([1.0]), f)
        assert np.abs(u).max() <= tau * math.exp(tau * mu_s) * np.abs(f).max()


def test_grid_refinement_converges():
    """Solutions on n and 2n grids (the 2n one averaged over 2x2 blocks) get
    closer as n doubles.  The rate is not stated in the paper: parity unpinned
    for the rate, only monotone decrease is required."""
    mu, mus = 1.0, 0.5
    sols = {}
    for n in (8, 16, 32):
        f = rte_synth.gaussian_mixture_2d(n, [(0.5, 0.5)], [0.1])
        sols[n], _ = oracle.solve_dense_2d(n, 1.0 / n, mu, mus, np.array([1.0]), f)
    d = []
    for n in (8, 16):
        fine = sols[2 * n][0].real
        coarse = fine.reshape(n, 2, n, 2).mean(axis=(1, 3))
        d.append(oracle.rel_l2(coarse, sols[n][0].real))
    assert d[1] < 0.5 * d[0]


def test_paper_table_error_order_of_magnitude():
    """Table iso_con_err: f1, mu_s = 1, mu_t = 1.2, n = 32; the error of the
    iterative solution at tolerance eps against the direct solve.  The paper
    used MATLAB's MINRES on the symmetric form, so only the order of magnitude
    can agree."""
    with open(os.path.join(GOLDEN, "paper_tables.json")) as fh:
        gold = json.load(fh)["iso_con_err_f1_n32"]
    n = 32
    f1, _, _ = rte_synth.paper_sources(n)
    h = 1.0 / n
    u, b = oracle.solve_dense_2d(n, h, 1.2, 1.0, np.array([1.0]), f1)
    D = oracle.cell_weights_2d(1.2, h, 0)
    for eps_s, err_paper in gold["values"].items():
        eps = float(eps_s)
        ug, _, _ = oracle.gmres(lambda t: t - oracle.apply_K_2d(n, h, 1.2, 1.0, [1.0], t, D=D), b, tol=eps)
        err = oracle.rel_l2(ug, u)
        assert abs(math.log10(err) - math.log10(err_paper)) <= 2.0, (eps, err, err_paper)


def test_neumann_3d_equals_dense():
    n, h, mu = 4, 0.25, 3.0
    f = rte_synth.gaussian_3d(n, (0.5, 0.5, 0.5), 0.2)
    u, b = oracle.solve_dense_3d(n, h, mu, 0.1 * mu, f)
    D = oracle.cell_weight_3d(mu, h)
    un = oracle.neumann(lambda t: oracle.apply_K_3d(n, h, mu, 0.1 * mu, t, D=D), b, 30)
    assert oracle.rel_l2(un, u) < 1e-14
    u0, b0 = oracle.solve_dense_3d(n, h, mu, 0.0, f)
    assert np.abs(u0 - b0).max() == 0.0


def test_paper_anisotropic_table_error_order_of_magnitude():
    """Table ani_con_err: sigma of Eq. sigma (L = 1), f1, mu_s = 1, mu_t = 1.2,
    n = 32, GMRES at tolerance eps against the direct solve."""
    with open(os.path.join(GOLDEN, "paper_tables.json")) as fh:
        gold = json.load(fh)["ani_con_err_f1_n32"]
    n = 32
    f1, _, _ = rte_synth.paper_sources(n)
    h = 1.0 / n
    sig = rte_synth.paper_sigma_hat()
    u, b = oracle.solve_dense_2d(n, h, 1.2, 1.0, sig, f1)
    D = oracle.cell_weights_2d(1.2, h, 2)
    for eps_s, err_paper in gold["values"].items():
        eps = float(eps_s)
        ug, _, _ = oracle.gmres(lambda t: t - oracle.apply_K_2d(n, h, 1.2, 1.0, sig, t, D=D), b, tol=eps)
        err = oracle.rel_l2(ug, u)
        assert abs(math.log10(err) - math.log10(err_paper)) <= 2.0, (eps, err, err_paper)


# ---------------------------------------------------------------------------
# The sampled residual: the checker of every full-size GPU solve
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("L", [0, 3, 4])
def test_sampled_residual_2d_vanishes_at_the_dense_solution(L):
    """Eq. ani_AU: at the LU solution of (I - K) u = K~ g the residual
    b - u + K u is zero at every cell and every mode -L..L.  L = 3 and 4 put
    the right-hand side's cell weights D_{-L..L} off the centre of the
    D_{-2L..2L} table (a shifted window would bring in D_{+-4} at the wrong
    modes), and all cells are sampled, in a scrambled order."""
    n, h, mu = 6, 1.0 / 6, 7.0
    sig = rte_synth.hg_sigma_hat(0.6, L)
    f = rte_synth.gaussian_mixture_2d(n, [(0.35, 0.6), (0.7, 0.3)], [0.15, 0.1])
    u, b = oracle.solve_dense_2d(n, h, mu, 0.9 * mu, sig, f)
    rows = np.random.default_rng(5).permutation(n * n)
    r, bs = oracle.sampled_residual_2d(n, h, mu, 0.9 * mu, sig, f, u, rows)
    assert r.shape == (2 * L + 1, n * n)
    assert np.abs(bs - b.reshape(2 * L + 1, -1)[:, rows]).max() <= 1e-14 * np.abs(b).max()
    assert np.linalg.norm(r) <= 1e-13 * np.linalg.norm(bs)


@pytest.mark.parametrize("L", [1, 3])
def test_sampled_residual_2d_of_a_perturbation(L):
    """For u = u_LU + d the residual is -(I - K) d, with (I - K) taken from the
    assembled dense matrix (the C assembly, not the row sums the residual
    uses): a wrong mode placement, sign or sigma weight fails here."""
    n, h, mu = 6, 1.0 / 6, 4.0
    mus = 0.8 * mu
    sig = rte_synth.hg_sigma_hat(0.5, L)
    f = rte_synth.gaussian_mixture_2d(n, [(0.4, 0.55)], [0.2])
    u, _ = oracle.solve_dense_2d(n, h, mu, mus, sig, f)
    rng = np.random.default_rng(11)
    d = rng.standard_normal(u.shape) + 1j * rng.standard_normal(u.shape)
    d = 0.5 * (d + d[::-1].conj())  # a J-symmetric perturbation, like every solver field
    Kt = oracle.assemble_ktilde_2d(n, h, mu, L)
    N = n * n
    sig_full = np.repeat(np.concatenate([sig[:0:-1], sig]), N)
    Ad = (d.reshape(-1) - mus * (Kt @ (sig_full * d.reshape(-1)))).reshape(2 * L + 1, N)
    rows = rng.choice(N, size=17, replace=False)
    r, _ = oracle.sampled_residual_2d(n, h, mu, mus, sig, f, u + d, rows)
    assert np.abs(r + Ad[:, rows]).max() <= 1e-13 * np.abs(Ad).max()


def test_sampled_residual_3d():
    """3D: zero residual at the LU solution, and -(I - K) d for a perturbation
    d, (I - K) from the assembled dense matrix."""
    n, h, mu = 4, 0.25, 6.0
    mus = 0.9 * mu
    f = rte_synth.gaussian_3d(n, (0.4, 0.5, 0.6), 0.2)
    u, b = oracle.solve_dense_3d(n, h, mu, mus, f)
    rows = np.random.default_rng(3).permutation(n ** 3)
    r, bs = oracle.sampled_residual_3d(n, h, mu, mus, f, u, rows)
    assert np.abs(bs - b.reshape(-1)[rows]).max() <= 1e-14 * np.abs(b).max()
    assert np.linalg.norm(r) <= 1e-13 * np.linalg.norm(bs)
    d = np.random.default_rng(4).standard_normal(u.shape)
    Ad = d.reshape(-1) - mus * (oracle.assemble_ktilde_3d(n, h, mu) @ d.reshape(-1))
    r, _ = oracle.sampled_residual_3d(n, h, mu, mus, f, u + d, rows[:20])
    assert np.abs(r + Ad[rows[:20]]).max() <= 1e-13 * np.abs(Ad).max()
