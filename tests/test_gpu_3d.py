"""GPU parity of the 3D isotropic path (C ABI) against the oracle.

Tolerances as in the 2D tests: FP64 1e-12 relative L2, FP32 1e-5, solves
within cond_est * tol, cond_est = (1 + mu_s/mu_t)/(1 - mu_s/mu_t).
"""
import numpy as np
import pytest

import oracle
import rte_synth
from _util import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_03061_gb300 import build
    build.build()


def _plan(n, mu_t, mu_s, **kw):
    from paper_1802_03061_gb300 import Plan
    return Plan(n, mu_t=mu_t, mu_s=mu_s, sigma_hat=[1.0], dim=3, **kw)


CASES = [(1, 1.0, 0.5), (2, 2.0, 1.0), (3, 5.0, 4.0), (6, 3.0, 2.9), (9, 30.0, 29.0), (16, 100.0, 99.5)]


@pytest.mark.parametrize("n,mu_t,mu_s", CASES)
def test_cell_weight_3d(n, mu_t, mu_s):
    p = _plan(n, mu_t, mu_s)
    assert p.cell_weights()[0] == pytest.approx(oracle.cell_weight_3d(mu_t, 1.0 / n), rel=1e-13)
    p.close()


@pytest.mark.parametrize("n,mu_t,mu_s", CASES)
def test_apply_K_3d_fp64_matches_direct_sum(n, mu_t, mu_s):
    p = _plan(n, mu_t, mu_s)
    x = np.random.default_rng(n).standard_normal((n, n, n))
    y = p.apply_K(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle.apply_K_3d(n, 1.0 / n, mu_t, mu_s, x)
    assert rel(y, ref) < 1e-12
    ya = p.apply_A(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(ya, x - ref) < 1e-12
    b = p.rhs(torch.from_numpy(x)).cpu().numpy()
    assert rel(b, ref / mu_s) < 1e-12
    ye = p.apply_K64e(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(ye, ref) < 1e-12
    p.close()


# n = 32, 64: padded lengths 64, 128 take the warp-register FFT z pass;
# n = 6, 16: the shared-memory Stockham path
@pytest.mark.parametrize("n", [6, 16, 32, 64])
def test_apply_K32_3d(n):
    p = _plan(n, 10.0, 9.0, prec="mixed_fp32")
    x = np.random.default_rng(1).standard_normal((n, n, n)).astype(np.float32)
    y = p.apply_K32(torch.from_numpy(x).cuda()).cpu().numpy()
    if n <= 32:
        ref = oracle.apply_K_3d(n, 1.0 / n, 10.0, 9.0, x.astype(np.float64))
        assert rel(y, ref) < 1e-5
    else:
        rows = np.random.default_rng(3).choice(n ** 3, size=64, replace=False)
        ref = oracle.apply_K_3d(n, 1.0 / n, 10.0, 9.0, x.astype(np.float64), rows=rows)
        assert rel(y.reshape(-1)[rows], ref) < 1e-5
    p.close()


# q = 64, 128, 256, 512: the warp-register passes (FP32 and float-float) with
# 2, 4, 8, 16 registers per lane; n ragged against their 16-row / 16-z blocks
@pytest.mark.parametrize("n,q", [(12, 64), (20, 128), (24, 256), (9, 512)])
def test_apply_K_3d_warp_passes(n, q):
    mu_t, mu_s = 10.0, 9.0
    p = _plan(n, mu_t, mu_s, prec="mixed_fp32", q_policy=q)
    assert p.Q == q
    x = np.random.default_rng(n).standard_normal((n, n, n))
    x32 = x.astype(np.float32)
    y32 = p.apply_K32(torch.from_numpy(x32).cuda()).cpu().numpy()
    assert rel(y32, oracle.apply_K_3d(n, 1.0 / n, mu_t, mu_s, x32.astype(np.float64))) < 1e-5
    ref = oracle.apply_K_3d(n, 1.0 / n, mu_t, mu_s, x)
    ye = p.apply_K64e(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(ye, ref) < 1e-12
    # mixed solve: float-float RHS and residuals, FP32 inner passes
    f = rte_synth.gaussian_3d(n, (0.45, 0.5, 0.55), 0.15)
    u, st = p.solve(torch.from_numpy(f), tol=1e-10)
    assert st["converged"] and st["relres_true"] <= 1e-10
    rows = np.random.default_rng(7).choice(n ** 3, size=32, replace=False)
    r, b = oracle.sampled_residual_3d(n, 1.0 / n, mu_t, mu_s, f, u.cpu().numpy(), rows)
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-8
    p.close()


# FP32 warp passes for q = 64, 128, 256: odd n (a row pair with one row), n
# ragged against the 16-row and 16-z blocks, and the largest n of each length
@pytest.mark.parametrize("n,q", [(13, 64), (32, 64), (47, 128), (64, 128), (101, 256), (128, 256)])
def test_apply_K32_3d_warp_lengths(n, q):
    mu_t, mu_s = 10.0, 9.0
    p = _plan(n, mu_t, mu_s, prec="mixed_fp32", q_policy=q)
    assert p.Q == q
    x = np.random.default_rng(n + q).standard_normal((n, n, n)).astype(np.float32)
    y = p.apply_K32(torch.from_numpy(x).cuda()).cpu().numpy().reshape(-1)
    rows = np.random.default_rng(5).choice(n ** 3, size=48, replace=False)
    if n <= 13:
        rows = np.arange(n ** 3)
    ref = oracle.apply_K_3d(n, 1.0 / n, mu_t, mu_s, x.astype(np.float64), rows=rows)
    assert rel(y[rows], ref) < 1e-5
    p.close()


def test_apply_K_3d_full_size_sampled():
    """128^3 (zero padded to 256^3), mu_t = 100, mu_s = 99.5: FP64 K x against
    the oracle's direct sum at sampled cells."""
    n = 128
    p = _plan(n, 100.0, 99.5)
    x = rte_synth.iso3d_diffusion()["f"]
    y = p.apply_K(torch.from_numpy(x).cuda()).cpu().numpy()
    # cells where the field is significant: relative L2 at 1e-12; far cells
    # (values down to 1e-30 of the peak): absolute error at FP64 rounding of the peak
    rng = np.random.default_rng(2)
    support = np.flatnonzero(x.reshape(-1) > 1e-2 * x.max())
    near = rng.choice(support, size=24, replace=False)
    ref = oracle.apply_K_3d(n, 1.0 / n, 100.0, 99.5, x, rows=near)
    assert rel(y.reshape(-1)[near], ref) < 1e-12
    far = rng.choice(n ** 3, size=24, replace=False)
    ref_far = oracle.apply_K_3d(n, 1.0 / n, 100.0, 99.5, x, rows=far)
    assert np.abs(y.reshape(-1)[far] - ref_far).max() < 1e-14 * np.abs(ref).max()
    p.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed_fp32"])
def test_solve_3d_small_against_dense(prec):
    n, mu_t, mu_s = 8, 20.0, 19.0
    f = rte_synth.gaussian_3d(n, (0.45, 0.5, 0.55), 0.15)
    p = _plan(n, mu_t, mu_s, prec=prec)
    u_ref, _ = oracle.solve_dense_3d(n, 1.0 / n, mu_t, mu_s, f)
    u, st = p.solve(torch.from_numpy(f), tol=1e-10)
    assert st["converged"] and st["relres_true"] <= 1e-10
    cond = (1 + mu_s / mu_t) / (1 - mu_s / mu_t)
    assert rel(u.cpu().numpy(), u_ref) <= 2 * cond * 1e-10
    p.close()


def test_solve_3d_diffusion_full_size():
    """The 128^3 diffusion-regime workload (mu_t = 100, mu_s = 99.5) in the
    mixed mode: converged to 1e-8, and the oracle's FP64 direct-sum residual
    at sampled cells agrees."""
    prob = rte_synth.iso3d_diffusion()
    n = prob["n"]
    p = _plan(n, prob["mu_t"], prob["mu_s"], prec="mixed_fp32", restart=60, maxit=3000)
    u, st = p.solve(torch.from_numpy(prob["f"]), tol=1e-8)
    assert st["converged"] and st["relres_true"] <= 1e-8
    # Any set S of rows has ||r_S|| <= ||r|| <= tol ||b||: the oracle's
    # residual at sampled rows against that bound, ||b|| from the FP64 RHS.
    # Rows where the source is significant, and rows anywhere (far from the
    # source b is ~e^-30 of its peak, so an error there would hide in a
    # relative check against b_S)
    bnorm = float(torch.linalg.norm(p.rhs(torch.from_numpy(prob["f"]).cuda())).item())
    support = np.flatnonzero(prob["f"].reshape(-1) > 1e-2 * prob["f"].max())
    rng = np.random.default_rng(5)
    for rows in (rng.choice(support, size=16, replace=False), rng.choice(n ** 3, size=16, replace=False)):
        r, b = oracle.sampled_residual_3d(n, 1.0 / n, prob["mu_t"], prob["mu_s"], prob["f"], u.cpu().numpy(), rows)
        assert np.linalg.norm(r) <= 1.1e-8 * bnorm
    p.close()


@pytest.mark.parametrize("n,q", [(16, 0), (12, 48)])
def test_mixed_residual_equals_unfused_residual_3d(n, q):
    """3D: the fused float-float residual K~(mu_s u + f) - u of the mixed
    solve against b (FP64 rte_rhs) - u + rte_apply_K64e(u)."""
    mu_t, mu_s = 30.0, 29.0
    f = torch.from_numpy(rte_synth.gaussian_3d(n, (0.45, 0.5, 0.55), 0.15))
    p = _plan(n, mu_t, mu_s, prec="mixed_fp32", restart=60, q_policy=q)
    u, st = p.solve(f, tol=1e-9)
    assert st["converged"]
    b = p.rhs(f)
    r = (b - u + p.apply_K64e(u)).cpu().numpy()
    relres = float(np.linalg.norm(r) / np.linalg.norm(b.cpu().numpy()))
    assert relres <= 1e-9 * (1 + 1e-6)
    assert abs(relres - st["relres_true"]) <= 1e-6 * relres + 1e-12
    p.close()
