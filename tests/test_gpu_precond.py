"""The periodic preconditioner of the inner solves (rte_opts.precond).

Its application M x = crop((I - C)^{-1} pad(x)) is checked against a
reference built here from the oracle's dense Nystrom matrix: the matrix
entries give the kernel samples on the periodic padded grid, numpy's FFT
diagonalises C, and (I - C(xi))^{-1} is formed per frequency.  Tolerances:
2D 2e-2 (the inverse matrices are stored in BF16, 2^-9 per entry), 3D 1e-5
(FP32 inverse spectrum).  Preconditioned solves must reach the same solution
as the dense LU (cond_est * tol) in fewer inner iterations."""
import numpy as np
import pytest

import oracle
import rte_synth
from oracle import core
from _util import packed_to_full, random_packed, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_03061_gb300 import build
    build.build()


def _plan(n, mu_t, mu_s, sig, dim=2, **kw):
    from paper_1802_03061_gb300 import Plan
    return Plan(n, mu_t=mu_t, mu_s=mu_s, sigma_hat=sig, dim=dim, **kw)


def _ref_precond_2d(n, Q, mu_t, mu_s, sig, x_full, lmax=None):
    """Reference M x for the full mode field x_full [2L+1][n][n] (modes -L..L):
    M x = x + crop(P pad(x_low)), P = C[:, low] (I - C[low, low])^{-1} per
    frequency, low = the modes |k| <= lmax (all modes: M = crop (I - C)^{-1} pad)."""
    L = len(sig) - 1
    lmax = L if lmax is None else min(lmax, L)
    M = 2 * L + 1
    N = n * n
    Kt = core.assemble_ktilde_2d(n, 1.0 / n, mu_t, L)
    s_full = core._sigma_full(sig)
    G = np.zeros((M, M, Q, Q), complex)
    for k in range(M):
        for kp in range(M):
            blk = Kt[k * N:(k + 1) * N, kp * N:(kp + 1) * N]
            for o1 in range(-(n - 1), n):
                for o2 in range(-(n - 1), n):
                    i1, i2 = max(o1, 0), max(o2, 0)
                    G[k, kp, o2 % Q, o1 % Q] = blk[i2 * n + i1, (i2 - o2) * n + (i1 - o1)]
    C = np.moveaxis(mu_s * np.fft.fft2(G, axes=(2, 3)) * s_full[None, :, None, None], (2, 3), (0, 1))
    lo = np.arange(L - lmax, L + lmax + 1)
    inv = np.linalg.inv(np.eye(len(lo))[None, None] - C[:, :, lo][:, :, :, lo])
    Pm = np.einsum("abkl,ablm->abkm", C[:, :, :, lo], inv)
    V = np.zeros((len(lo), Q, Q), complex)
    V[:, :n, :n] = x_full[lo]
    F = np.moveaxis(np.fft.fft2(V, axes=(1, 2)), 0, -1)
    Y = np.einsum("abkl,abl->abk", Pm, F)
    return x_full + np.fft.ifft2(np.moveaxis(Y, -1, 0), axes=(1, 2))[:, :n, :n]


@pytest.mark.parametrize("n,L,q", [(12, 2, 64), (20, 1, 128), (9, 3, 64), (12, 8, 64), (16, 4, 256),
                                   (10, 2, 512), (7, 0, 512),
                                   # shared-memory (Stockham) passes: Q not 32 * 2^j, up to 1024
                                   (12, 2, 72), (20, 1, 96), (10, 8, 48), (12, 4, 216), (9, 1, 768),
                                   (7, 0, 1024)])
def test_precond_apply_2d_matches_reference(n, L, q):
    mu_t, mu_s = 10.0, 9.0
    sig = rte_synth.hg_sigma_hat(0.5, L)
    x = random_packed(np.random.default_rng(n), L, n).astype(np.complex64)
    # every mode inverted, and (L >= 3) only |k| <= 1 with the block-lower-triangular rest
    for lmax in ([L, 1] if L >= 3 else [L]):
        p = _plan(n, mu_t, mu_s, sig, prec="mixed_fp32", q_policy=q, precond_lmax=max(lmax, 1) if lmax < L else 99)
        y = p.apply_precond32(torch.from_numpy(x).cuda()).cpu().numpy()
        ref = _ref_precond_2d(n, q, mu_t, mu_s, sig, packed_to_full(x.astype(complex)), lmax)
        assert rel(y, ref[L:]) < 2e-2, lmax
        p.close()


def test_precond_apply_3d_matches_reference():
    n, mu_t, mu_s = 8, 20.0, 19.0
    p = _plan(n, mu_t, mu_s, [1.0], dim=3, prec="mixed_fp32")
    Q = p.Q
    Kt = core.assemble_ktilde_3d(n, 1.0 / n, mu_t)
    G = np.zeros((Q, Q, Q))
    idx = lambda a, b, c: (a * n + b) * n + c  # [z][y][x]
    for o0 in range(-(n - 1), n):
        for o1 in range(-(n - 1), n):
            for o2 in range(-(n - 1), n):
                i0, i1, i2 = max(o0, 0), max(o1, 0), max(o2, 0)
                G[o0 % Q, o1 % Q, o2 % Q] = Kt[idx(i0, i1, i2), idx(i0 - o0, i1 - o1, i2 - o2)]
    Minv = 1.0 / (1.0 - mu_s * np.fft.fftn(G))
    x = np.random.default_rng(3).standard_normal((n, n, n)).astype(np.float32)
    V = np.zeros((Q, Q, Q))
    V[:n, :n, :n] = x
    ref = np.fft.ifftn(Minv * np.fft.fftn(V)).real[:n, :n, :n]
    y = p.apply_precond32(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, ref) < 1e-5
    p.close()


@pytest.mark.parametrize("q", [64, 72])
def test_preconditioned_solve_2d_against_dense(q):
    n, L = 32, 2
    prob = rte_synth.hg2d_transport(n=n, L=L, seed=5)
    sig = prob["sigma_hat"]
    p = _plan(n, prob["mu_t"], prob["mu_s"], sig, prec="mixed_fp32", q_policy=q)
    f = torch.from_numpy(prob["f"])
    u_ref, _ = oracle.solve_dense_2d(n, 1.0 / n, prob["mu_t"], prob["mu_s"], sig, prob["f"])
    u0, st0 = p.solve(f, tol=1e-10)
    u1, st1 = p.solve(f, tol=1e-10, precond=1)
    assert st0["converged"] and st1["converged"] and st1["relres_true"] <= 1e-10
    rho = prob["mu_s"] / prob["mu_t"]
    cond = (1 + rho) / (1 - rho)
    assert rel(u1.cpu().numpy(), u_ref[L:]) <= 2 * cond * 1e-10
    assert st1["iters"] < st0["iters"]
    p.close()


@pytest.mark.parametrize("n,q", [(16, 0), (12, 64)])
def test_preconditioned_solve_3d(n, q):
    mu_t, mu_s = 30.0, 29.0
    f = rte_synth.gaussian_3d(n, (0.45, 0.5, 0.55), 0.15)
    p = _plan(n, mu_t, mu_s, [1.0], dim=3, prec="mixed_fp32", restart=60, q_policy=q)
    u0, st0 = p.solve(torch.from_numpy(f), tol=1e-10)
    u1, st1 = p.solve(torch.from_numpy(f), tol=1e-10, precond=1)
    assert st0["converged"] and st1["converged"]
    cond = (1 + mu_s / mu_t) / (1 - mu_s / mu_t)
    assert rel(u1.cpu().numpy(), u0.cpu().numpy()) <= 2 * cond * 1e-10
    assert st1["iters"] < st0["iters"]
    rows = np.random.default_rng(n).choice(n ** 3, size=32, replace=False)
    r, b = oracle.sampled_residual_3d(n, 1.0 / n, mu_t, mu_s, f, u1.cpu().numpy(), rows)
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-8
    p.close()


def test_preconditioned_full_size_transport_sampled_residual():
    """256^2, L = 8 (the transport workload): preconditioned mixed solve to
    1e-8; the oracle's FP64 direct-sum residual at sampled cells agrees."""
    prob = rte_synth.hg2d_transport()
    n, sig = prob["n"], prob["sigma_hat"]
    p = _plan(n, prob["mu_t"], prob["mu_s"], sig, prec="mixed_fp32", precond=1)
    u, st = p.solve(torch.from_numpy(prob["f"]), tol=1e-8)
    assert st["converged"] and st["relres_true"] <= 1e-8
    rows = np.random.default_rng(11).choice(n * n, size=24, replace=False)
    r, b = oracle.sampled_residual_2d(n, 1.0 / n, prob["mu_t"], prob["mu_s"], sig, prob["f"],
                                      packed_to_full(u.cpu().numpy()), rows)
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-7
    p.close()


def test_preconditioned_solve_q1024_sampled_residual():
    """n = 512, L = 8 (Q = 1024, the shared-memory passes; the heaviest
    instances of the batched workload): preconditioned and plain mixed solves
    to 1e-8 agree within cond_est * tol, the preconditioned one in fewer
    iterations, and the oracle's FP64 direct-sum residual at sampled cells
    agrees."""
    rng = np.random.default_rng(21)
    d = rte_synth.random_instance_2d(rng, 512, 8)
    n, sig = d["n"], d["sigma_hat"]
    p = _plan(n, d["mu_t"], d["mu_s"], sig, prec="mixed_fp32", restart=30, maxit=4000)
    assert p.Q == 1024
    f = torch.from_numpy(d["f"])
    u0, st0 = p.solve(f, tol=1e-8)
    u1, st1 = p.solve(f, tol=1e-8, precond=1)
    assert st0["converged"] and st1["converged"] and st1["relres_true"] <= 1e-8
    assert st1["iters"] < st0["iters"]
    rho = d["mu_s"] / d["mu_t"]
    assert rel(u1.cpu().numpy(), u0.cpu().numpy()) <= 2 * (1 + rho) / (1 - rho) * 1e-8
    rows = np.random.default_rng(12).choice(n * n, size=8, replace=False)
    r, b = oracle.sampled_residual_2d(n, 1.0 / n, d["mu_t"], d["mu_s"], sig, d["f"],
                                      packed_to_full(u1.cpu().numpy()), rows)
    assert np.linalg.norm(r) / np.linalg.norm(b) < 1e-7
    p.close()


def test_automatic_mode_truncation():
    """The default lmax: the smallest with (mu_s/mu_t) max_{k>lmax} |sigma_hat_k|
    <= 0.03 -- 4 for g = 0.5, mu_s/mu_t = 0.9 (0.9 * 0.5^5 = 0.028), all
    modes for g = 0.8 at L = 8 (0.9 * 0.8^8 = 0.15), 0 without anisotropy."""
    from paper_1802_03061_gb300 import _binding as B
    x = None
    for g, L, want in [(0.5, 8, 4), (0.8, 8, 8), (0.0, 4, 0), (0.5, 2, 2)]:
        sig = rte_synth.hg_sigma_hat(g, L)
        p = _plan(16, 10.0, 9.0, sig, prec="mixed_fp32")
        x = torch.zeros(p.shape(), dtype=torch.complex64, device="cuda")
        p.apply_precond32(x)
        assert B.rte_precond_info(p.handle) == want, (g, L)
        p.close()
