"""GPU parity of the 3D anisotropic (spherical-harmonic) operator through the
C ABI against the oracle (oracle/aniso3d.py).  Two pass families: the
general-Q Stockham passes channel by channel (n <= 16 and n > 128) and the
warp-register passes over all channels per launch (17 <= n <= 128, Q = 64,
128, 256).  Tolerances: FP64 and float-float 1e-12 relative L2 (FFT
rounding over Q^3 points); FP32 1e-5 (FP32 spectra and FFTs); solves (FP64
GMRES or FP32 inner GMRES with FP64-accurate residuals) within 2 tol cond of
the dense LU solution, cond = (1 + r)/(1 - r)."""
import numpy as np
import pytest

import oracle
import rte_synth
from oracle import aniso3d as A
from _util import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_03061_gb300 import build
    build.build()


def _hg(g, L):
    return [g ** l for l in range(L + 1)]


@pytest.mark.parametrize("L,mu_t,n", [(2, 3.0, 10), (3, 0.0, 4), (4, 40.0, 16)])
def test_cell_weights_match_oracle(L, mu_t, n):
    from paper_1802_03061_gb300 import Aniso3D
    op = Aniso3D(n, mu_t, 0.5 * mu_t, _hg(0.5, L))
    np.testing.assert_allclose(op.cell_weights(), A.cell_weights(L, mu_t, 1.0 / n), rtol=1e-12,
                               atol=1e-14 * oracle.cell_weight_3d(mu_t, 1.0 / n))
    op.close()


@pytest.mark.parametrize("n,L", [(1, 1), (3, 2), (5, 1), (6, 3), (8, 2), (7, 4)])
def test_apply_matches_oracle(n, L):
    """Every Q (2, 6, 10 -> 12, 12, 16, 16) and L = 1..4, FP64 and FP32."""
    from paper_1802_03061_gb300 import Aniso3D
    mu_t, mu_s = 7.0, 6.3
    sig = _hg(0.7, L)
    op = Aniso3D(n, mu_t, mu_s, sig)
    M = op.M
    x = np.random.default_rng(10 * n + L).standard_normal((M, n, n, n))
    ref = A.apply_K(n, 1.0 / n, mu_t, mu_s, sig, x).reshape(M, n, n, n)
    assert rel(op.apply_K(x).cpu().numpy(), ref) < 1e-12
    assert rel(op.apply_K64e(x).cpu().numpy(), ref) < 1e-12
    assert rel(op.apply_K32(x).cpu().numpy(), ref) < 1e-5
    f = np.random.default_rng(n).random((n, n, n))
    assert rel(op.rhs(f).cpu().numpy(), A.rhs(n, 1.0 / n, mu_t, L, f).reshape(M, n, n, n)) < 1e-12
    op.close()


# warp passes: n = 17 (Q = 64, ragged against the 16-row tiles), 24 with L = 4
# (M = 25), 33 and 48 (Q = 128), 97 (Q = 256); Stockham: 12 (Q = 24, radix 3)
# and 130 (Q = 288 = 2^5 3^2)
@pytest.mark.parametrize("n,L,Q", [(17, 2, 64), (24, 4, 64), (33, 2, 128), (48, 1, 128), (97, 1, 256), (12, 3, 24),
                                   (130, 1, 288)])
def test_sampled_rows_larger_grids(n, L, Q):
    """Sampled rows (all M channels) of K x, K x in float-float and in FP32,
    and of the right-hand side, against the direct sums."""
    from paper_1802_03061_gb300 import Aniso3D
    mu_t, mu_s = 10.0, 9.0
    sig = _hg(0.6, L)
    op = Aniso3D(n, mu_t, mu_s, sig)
    assert op.Q == Q
    M = op.M
    x = np.random.default_rng(n).standard_normal((M, n, n, n))
    y = op.apply_K(x).cpu().numpy().reshape(M, -1)
    ye = op.apply_K64e(x).cpu().numpy().reshape(M, -1)
    y32 = op.apply_K32(x).cpu().numpy().reshape(M, -1)
    rows = np.random.default_rng(1).choice(n ** 3, size=6 if n > 64 else 10, replace=False)
    D = A.cell_weights(L, mu_t, 1.0 / n)
    ref = A.apply_K(n, 1.0 / n, mu_t, mu_s, sig, x, rows=rows, D=D)
    assert rel(y[:, rows], ref) < 1e-12
    assert rel(ye[:, rows], ref) < 1e-12
    assert rel(y32[:, rows], ref) < 1e-5
    f = np.random.default_rng(n + 1).random((n, n, n))
    b = op.rhs(f).cpu().numpy().reshape(M, -1)
    assert rel(b[:, rows], A.rhs(n, 1.0 / n, mu_t, L, f, rows=rows, D=D)) < 1e-12
    op.close()


def test_isotropic_case_matches_the_plan():
    """L = 0 is the isotropic operator of rte_plan (d = 3)."""
    from paper_1802_03061_gb300 import Aniso3D, Plan
    n, mu_t, mu_s = 20, 6.0, 5.0
    x = np.random.default_rng(3).standard_normal((n, n, n))
    op = Aniso3D(n, mu_t, mu_s, [1.0])
    p = Plan(n, mu_t=mu_t, mu_s=mu_s, dim=3)
    y = op.apply_K(x[None]).cpu().numpy()[0]
    yp = p.apply_K(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, yp) < 1e-12
    op.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed_fp32"])
@pytest.mark.parametrize("n,L,g", [(4, 2, 0.6), (5, 1, -0.4)])
def test_solve_matches_dense(n, L, g, prec):
    from paper_1802_03061_gb300 import Aniso3D
    mu_t, mu_s = 8.0, 7.6
    sig = _hg(g, L)
    f = np.random.default_rng(n).random((n, n, n))
    op = Aniso3D(n, mu_t, mu_s, sig)
    u, st = op.solve(f, tol=1e-11, prec=prec)
    assert st["converged"] and st["relres_true"] <= 1e-11
    want = A.solve_dense(n, 1.0 / n, mu_t, mu_s, sig, f)
    # the bound of the other solve tests: 2 cond_est tol, cond_est = (1+r)/(1-r), r = mu_s/mu_t
    assert rel(u.cpu().numpy(), want) < 2 * 1e-11 * (1 + 0.95) / (1 - 0.95)
    op.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed_fp32"])
def test_solve_larger_grid_sampled_residual(prec):
    """n = 32, L = 2, Henyey-Greenstein g = 0.8, a Gaussian-mixture source:
    the residual u - K u - b at sampled cells from the direct sums; the mixed
    solve (FP32 inner GMRES) reaches the same FP64 residual."""
    from paper_1802_03061_gb300 import Aniso3D
    n, L, mu_t, mu_s = 32, 2, 20.0, 18.0
    sig = _hg(0.8, L)
    f = rte_synth.gaussian_3d(n, (0.4, 0.5, 0.5), 0.08) + rte_synth.gaussian_3d(n, (0.7, 0.3, 0.6), 0.05)
    op = Aniso3D(n, mu_t, mu_s, sig)
    u, st = op.solve(f, tol=1e-10, restart=40, prec=prec)
    assert st["converged"] and st["relres_true"] <= 1e-10, st
    if prec == "mixed_fp32":
        assert st["outer"] >= 2
    U = u.cpu().numpy().reshape(op.M, -1)
    rows = np.random.default_rng(2).choice(n ** 3, size=6, replace=False)
    D = A.cell_weights(L, mu_t, 1.0 / n)
    r = U[:, rows] - A.apply_K(n, 1.0 / n, mu_t, mu_s, sig, U, rows=rows, D=D) \
        - A.rhs(n, 1.0 / n, mu_t, L, f, rows=rows, D=D)
    assert np.abs(r).max() < 1e-8 * np.abs(U).max()
    # a second solve of the same handle (cached graph) with another source and
    # restart length, against a fresh handle's
    f2 = rte_synth.gaussian_3d(n, (0.5, 0.6, 0.3), 0.1)
    u2, st2 = op.solve(f2, tol=1e-10, restart=30, prec=prec)
    u3, st3 = op.solve(f2, tol=1e-10, restart=30, prec=prec)
    assert torch.equal(u2, u3) and st2["iters"] == st3["iters"]
    fresh = Aniso3D(n, mu_t, mu_s, sig)
    u4, _ = fresh.solve(f2, tol=1e-10, restart=30, prec=prec)
    assert torch.equal(u2, u4)
    fresh.close()
    op.close()


def test_solve_non_finite_source():
    from paper_1802_03061_gb300 import Aniso3D
    from paper_1802_03061_gb300 import _binding as B
    op = Aniso3D(20, 5.0, 4.0, _hg(0.5, 1))
    f = np.ones((20, 20, 20))
    f[3, 4, 5] = np.nan
    for prec in ("fp64", "mixed_fp32"):
        with pytest.raises(B.RteError) as ei:
            op.solve(f, prec=prec)
        assert ei.value.status == B.RTE_ENAN
    # the handle still solves afterwards
    u, st = op.solve(np.ones((20, 20, 20)), tol=1e-9, prec="mixed_fp32")
    assert st["converged"]
    op.close()


def test_invalid_arguments():
    from paper_1802_03061_gb300 import Aniso3D
    from paper_1802_03061_gb300 import _binding as B
    with pytest.raises(B.RteError):
        Aniso3D(8, 2.0, 1.0, [1.0] * 6)  # L = 5
    with pytest.raises(B.RteError):
        Aniso3D(8, 2.0, 1.0, [0.9, 0.5])  # sigma_hat_0 != 1
    with pytest.raises(B.RteError):
        Aniso3D(8, 2.0, 3.0, [1.0, 0.5])  # mu_s > mu_t
