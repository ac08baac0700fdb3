"""MINRES inner solves (symmetric L = 0 operators, inner_solver="minres")
against the oracle's dense LU, against the GMRES inner solves, and its
iteration limit.  Bounds: cond_est * tol with cond_est =
(1 + mu_s/mu_t) / (1 - mu_s/mu_t)."""
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


def _plan(n, mu_t, mu_s, dim=2, **kw):
    from paper_1802_03061_gb300 import Plan
    return Plan(n, mu_t=mu_t, mu_s=mu_s, sigma_hat=[1.0], dim=dim, **kw)


def test_minres_2d_isotropic_bump_against_dense():
    """The 64 x 64 isotropic workload (mu_t = 1, mu_s = 0.5) in the mixed mode:
    MINRES inner solves, FP64-accurate refinement to 1e-10."""
    prob = rte_synth.iso2d_bump(64)
    p = _plan(64, prob["mu_t"], prob["mu_s"], prec="mixed_fp32", inner_solver="minres")
    u_ref, _ = oracle.solve_dense_2d(64, 1 / 64, prob["mu_t"], prob["mu_s"], [1.0], prob["f"])
    u, st = p.solve(torch.from_numpy(prob["f"]), tol=1e-10)
    assert st["converged"] and st["relres_true"] <= 1e-10
    assert rel(u.cpu().numpy(), u_ref) <= 2 * 3 * 1e-10  # 2 cond_est tol, cond_est = 3
    p.close()


@pytest.mark.parametrize("n,q", [(12, 0), (16, 64), (20, 128)])
def test_minres_matches_gmres_3d(n, q):
    """3D diffusion-like coefficients (cond_est 59): MINRES and GMRES inner
    solves reach the same solution; MINRES needs no more than 1.5x the inner
    iterations of GMRES(60); the oracle's sampled residual agrees."""
    mu_t, mu_s = 30.0, 29.0
    f = rte_synth.gaussian_3d(n, (0.45, 0.5, 0.55), 0.15)
    p = _plan(n, mu_t, mu_s, dim=3, prec="mixed_fp32", restart=60, maxit=3000, q_policy=q,
              inner_solver="minres")
    u_m, st_m = p.solve(torch.from_numpy(f), tol=1e-10)
    u_g, st_g = p.solve(torch.from_numpy(f), tol=1e-10, inner_solver="gmres")
    assert st_m["converged"] and st_g["converged"]
    cond = (1 + mu_s / mu_t) / (1 - mu_s / mu_t)
    assert rel(u_m.cpu().numpy(), u_g.cpu().numpy()) <= 2 * cond * 1e-10
    assert st_m["iters"] <= 1.5 * st_g["iters"] + 2
    rows = np.random.default_rng(n).choice(n ** 3, size=32, replace=False)
    r, b = oracle.sampled_residual_3d(n, 1.0 / n, mu_t, mu_s, f, u_m.cpu().numpy(), rows)
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-8
    p.close()


def test_minres_small_against_dense_3d():
    n, mu_t, mu_s = 8, 20.0, 19.0
    f = rte_synth.gaussian_3d(n, (0.45, 0.5, 0.55), 0.15)
    p = _plan(n, mu_t, mu_s, dim=3, prec="mixed_fp32", inner_solver="minres")
    u_ref, _ = oracle.solve_dense_3d(n, 1.0 / n, mu_t, mu_s, f)
    u, st = p.solve(torch.from_numpy(f), tol=1e-10)
    assert st["converged"] and st["relres_true"] <= 1e-10
    cond = (1 + mu_s / mu_t) / (1 - mu_s / mu_t)
    assert rel(u.cpu().numpy(), u_ref) <= 2 * cond * 1e-10
    p.close()


def test_minres_iteration_limit_gives_noconv():
    prob = rte_synth.iso2d_bump(32)
    p = _plan(32, 10.0, 9.9, prec="mixed_fp32", inner_solver="minres")
    u, st = p.solve(torch.from_numpy(prob["f"]), tol=1e-12, maxit=3)
    assert st["status"] == 5 and not st["converged"]
    assert 0 < st["relres_true"] < 1.0
    p.close()
