"""GPU parity of the 2D path (C ABI) against the oracle.

Tolerances: FP64 operator and FP64 solves 1e-12 relative L2; FP32 spectra
1e-5 (FP32 FFT convolution, error ~ log2(Q^2) * 2^-24 relative); BF16
spectra 1e-2 (each spectrum value carries a 2^-9 relative rounding);
mixed solves cond_est * tol with cond_est = (1 + mu_s/mu_t)/(1 - mu_s/mu_t).
"""
import numpy as np
import pytest

import oracle
import rte_synth
from _util import packed_to_full, random_packed, rel

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_03061_gb300 import build
    build.build()


def _plan(n, mu_t, mu_s, sig, **kw):
    from paper_1802_03061_gb300 import Plan
    return Plan(n, mu_t=mu_t, mu_s=mu_s, sigma_hat=sig, **kw)


# (n, L, mu_t, mu_s, g): tiny, ragged (n not a multiple of the row block),
# odd n (Q = 72 = 8*3*3), several tiles, largest L
CASES = [(1, 0, 1.0, 0.5, 0.0), (2, 1, 2.0, 1.0, 0.5), (3, 2, 5.0, 4.0, 0.3), (8, 0, 1.0, 0.5, 0.0),
         (12, 3, 10.0, 9.0, 0.5), (33, 2, 3.0, 2.5, 0.7), (20, 8, 10.0, 9.0, 0.5), (40, 4, 25.0, 20.0, 0.6)]


@pytest.mark.parametrize("n,L,mu_t,mu_s,g", CASES)
def test_cell_weights(n, L, mu_t, mu_s, g):
    p = _plan(n, mu_t, mu_s, rte_synth.hg_sigma_hat(g, L))
    D = np.array(p.cell_weights())
    ref = oracle.cell_weights_2d(mu_t, 1.0 / n, 2 * L)[2 * L:]
    # D_m with 4 not dividing m vanish by symmetry: compare them at roundoff of D_0
    assert np.allclose(D, ref, rtol=1e-13, atol=1e-14 * abs(ref[0]))
    p.close()


@pytest.mark.parametrize("n,L,mu_t,mu_s,g", CASES)
def test_apply_K_fp64_matches_direct_sum(n, L, mu_t, mu_s, g):
    sig = rte_synth.hg_sigma_hat(g, L)
    p = _plan(n, mu_t, mu_s, sig)
    rng = np.random.default_rng(100 + n)
    x = random_packed(rng, L, n)
    y = p.apply_K(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = oracle.apply_K_2d(n, 1.0 / n, mu_t, mu_s, sig, packed_to_full(x))
    assert rel(y, ref[L:]) < 1e-12
    ya = p.apply_A(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(ya, x - ref[L:]) < 1e-12
    # the same operator in float-float arithmetic on the FP32 units
    ye = p.apply_K64e(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(ye, ref[L:]) < 1e-12
    p.close()


@pytest.mark.parametrize("q", [512, 1024])
@pytest.mark.parametrize("n,L", [(20, 8), (33, 2), (7, 0), (40, 4)])
def test_float_float_and_fp64_operators_at_residue_lengths(n, L, q):
    """Q = 512 and 1024, where the float-float row and column passes run as
    two half-length warp FFTs (residues xi mod 2; the forward row pass only at
    512):
    K64e, the float-float right-hand side and the native FP64 K to 1e-12
    against the direct sum (K32 at these Q is covered by test_apply_K32)."""
    sig = rte_synth.hg_sigma_hat(0.5, L)
    p = _plan(n, 10.0, 9.0, sig, q_policy=q)
    assert p.Q == q
    rng = np.random.default_rng(300 + n)
    x = random_packed(rng, L, n)
    ref = oracle.apply_K_2d(n, 1.0 / n, 10.0, 9.0, sig, packed_to_full(x))
    ye = p.apply_K64e(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(ye, ref[L:]) < 1e-12
    y = p.apply_K(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, ref[L:]) < 1e-12
    f = rte_synth.gaussian_mixture_2d(n, [(0.4, 0.6), (0.7, 0.3)], [0.1, 0.05])
    b = p.rhs(torch.from_numpy(f)).cpu().numpy()
    assert rel(b, oracle.rhs_2d(n, 1.0 / n, 10.0, L, f)[L:]) < 1e-12
    p.close()


@pytest.mark.parametrize("n,L,mu_t,mu_s,g", CASES)
def test_rhs_matches_direct_sum(n, L, mu_t, mu_s, g):
    p = _plan(n, mu_t, mu_s, rte_synth.hg_sigma_hat(g, L))
    f = rte_synth.gaussian_mixture_2d(n, [(0.4, 0.6), (0.7, 0.3)], [0.1, 0.05])
    b = p.rhs(torch.from_numpy(f)).cpu().numpy()
    ref = oracle.rhs_2d(n, 1.0 / n, mu_t, L, f)
    assert rel(b, ref[L:]) < 1e-12
    p.close()


# q = 0: the default padded length (24, 48, 72 here: shared-memory FFT
# passes); q = 32 * 2^j: the warp-register row and column passes with
# R = 2, 4, 8, 16 registers per lane, n ragged against their 8/16-row blocks
@pytest.mark.parametrize("prec,tol", [("mixed_fp32", 1e-5), ("mixed_bf16", 1e-2)])
@pytest.mark.parametrize("n,L,q", [(12, 3, 0), (20, 8, 0), (33, 2, 0), (12, 3, 64), (20, 8, 128), (33, 2, 256),
                                   (33, 5, 512), (64, 1, 128),
                                   # Q = 1024: two 512-point residues per column
                                   (20, 8, 1024), (33, 2, 1024), (7, 0, 1024), (64, 4, 1024)])
def test_apply_K32(prec, tol, n, L, q):
    sig = rte_synth.hg_sigma_hat(0.5, L)
    p = _plan(n, 10.0, 9.0, sig, prec=prec, q_policy=q)
    assert q == 0 or p.Q == q
    rng = np.random.default_rng(7)
    x = random_packed(rng, L, n)
    y = p.apply_K32(torch.from_numpy(x.astype(np.complex64)).cuda()).cpu().numpy()
    ref = oracle.apply_K_2d(n, 1.0 / n, 10.0, 9.0, sig, packed_to_full(x.astype(np.complex64).astype(complex)))
    e = rel(y, ref[L:])
    assert e < tol
    if prec == "mixed_bf16":
        assert e > 1e-6  # really the BF16 spectra
    p.close()


def test_padding_length_does_not_change_the_result():
    """Q >= 2n-1 only; the result must not depend on Q (circulant embedding)."""
    n, L = 12, 2
    sig = rte_synth.hg_sigma_hat(0.4, L)
    x = random_packed(np.random.default_rng(3), L, n)
    ys = []
    for q in (0, 32, 36, 48):
        p = _plan(n, 4.0, 3.0, sig, q_policy=q)
        ys.append(p.apply_K(torch.from_numpy(x).cuda()).cpu().numpy())
        p.close()
    for y in ys[1:]:
        assert rel(y, ys[0]) < 1e-13


def test_solve_fp64_isotropic_bump_64():
    """64x64, mu_t = 1, mu_s = 0.5, L = 0, Gaussian bump: GMRES to 1e-10, and
    to 1e-13 against the oracle's dense LU (cond <= 3)."""
    prob = rte_synth.iso2d_bump(64)
    p = _plan(64, prob["mu_t"], prob["mu_s"], [1.0])
    f = torch.from_numpy(prob["f"])
    u_ref, _ = oracle.solve_dense_2d(64, 1 / 64, prob["mu_t"], prob["mu_s"], [1.0], prob["f"])
    u, st = p.solve(f, tol=1e-10)
    assert st["converged"] and st["relres_true"] <= 1e-10
    assert rel(u.cpu().numpy(), u_ref) <= 3e-10
    u, st = p.solve(f, tol=1e-13)
    assert st["relres_true"] <= 1e-13
    assert rel(u.cpu().numpy(), u_ref) <= 1e-12
    p.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed_fp32", "mixed_bf16"])
def test_solve_transport_regime_small(prec):
    """Down-scaled copy of the 256^2 HG transport workload (L = 8, mu_t = 10,
    mu_s = 9): error vs dense LU within cond_est * tol (cond_est = 19)."""
    n, L = 16, 8
    prob = rte_synth.hg2d_transport(n=n, L=L, seed=2)
    p = _plan(n, prob["mu_t"], prob["mu_s"], prob["sigma_hat"], prec=prec)
    u_ref, _ = oracle.solve_dense_2d(n, 1 / n, prob["mu_t"], prob["mu_s"], prob["sigma_hat"], prob["f"])
    u, st = p.solve(torch.from_numpy(prob["f"]), tol=1e-8)
    assert st["converged"] and st["relres_true"] <= 1e-8
    assert rel(u.cpu().numpy(), u_ref[L:]) <= 19 * 1e-8 * 2
    if prec != "fp64":
        assert st["outer"] >= 1
    p.close()


def test_mu_s_zero_solution_is_rhs():
    n, L = 10, 2
    p = _plan(n, 3.0, 0.0, rte_synth.hg_sigma_hat(0.5, L))
    f = rte_synth.gaussian_mixture_2d(n, [(0.5, 0.5)], [0.2])
    b = p.rhs(torch.from_numpy(f)).cpu().numpy()
    u, st = p.solve(torch.from_numpy(f), tol=1e-12)
    assert rel(u.cpu().numpy(), b) < 1e-14
    p.close()


def test_solve_host_buffers_match_device_solve():
    n, L = 24, 3
    prob = rte_synth.hg2d_transport(n=n, L=L, seed=5)
    p = _plan(n, prob["mu_t"], prob["mu_s"], prob["sigma_hat"], prec="mixed_fp32")
    u_d, _ = p.solve(torch.from_numpy(prob["f"]), tol=1e-9)
    u_h, st = p.solve_host(prob["f"], tol=1e-9)
    assert st["converged"]
    assert rel(u_h, u_d.cpu().numpy()) < 1e-8
    p.close()


def test_nonfinite_source_is_reported():
    from paper_1802_03061_gb300 import RteError
    n = 8
    p = _plan(n, 2.0, 1.0, [1.0])
    f = np.ones((n, n))
    f[3, 3] = np.nan
    with pytest.raises(RteError) as ei:
        p.solve(torch.from_numpy(f))
    assert ei.value.status == 7
    p.close()


def test_maxit_gives_noconv_with_best_iterate():
    n, L = 16, 2
    prob = rte_synth.hg2d_transport(n=n, L=L, seed=9)
    p = _plan(n, prob["mu_t"], prob["mu_s"], prob["sigma_hat"])
    u, st = p.solve(torch.from_numpy(prob["f"]), tol=1e-12, maxit=3, restart=3)
    assert st["status"] == 5 and not st["converged"]
    assert 0 < st["relres_true"] < 1.0
    p.close()


def test_full_size_transport_256_sampled_residual():
    """The 256^2, L = 8 workload at full size in the mixed BF16 mode: the
    oracle's FP64 direct-sum residual at sampled cells (all modes)."""
    prob = rte_synth.hg2d_transport()
    n, L = prob["n"], 8
    p = _plan(n, prob["mu_t"], prob["mu_s"], prob["sigma_hat"], prec="mixed_bf16")
    u, st = p.solve(torch.from_numpy(prob["f"]), tol=1e-8)
    assert st["converged"] and st["relres_true"] <= 1e-8
    rows = np.random.default_rng(11).choice(n * n, size=24, replace=False)
    uf = packed_to_full(u.cpu().numpy())
    r, b = oracle.sampled_residual_2d(n, 1 / n, prob["mu_t"], prob["mu_s"], prob["sigma_hat"], prob["f"], uf, rows)
    # rows S anywhere: ||r_S|| <= ||r|| <= tol ||b||, ||b|| (all modes) from the FP64 RHS
    bnorm = _wnorm(p.rhs(torch.from_numpy(prob["f"])).cpu().numpy())
    assert np.linalg.norm(r) <= 1.1e-8 * bnorm
    p.close()


def _wnorm(v):
    """The solver's norm of a packed field: mode 0 once, modes k >= 1 twice
    (their conjugates), i.e. the norm of the full 2L+1 mode vector."""
    w = np.ones(v.shape[0])
    w[1:] = 2.0
    return float(np.sqrt(np.sum(w * np.sum(np.abs(v.reshape(v.shape[0], -1)) ** 2, axis=1))))


@pytest.mark.parametrize("prec,q", [("mixed_fp32", 0), ("mixed_bf16", 0), ("mixed_fp32", 72), ("mixed_fp32", 512),
                                    ("mixed_fp32", 1024), ("mixed_bf16", 1024)])
def test_mixed_residual_equals_unfused_residual(prec, q):
    """The mixed solve forms every residual as K~(mu_s sigma_hat u + g) - u in
    one float-float application and b in FP32 only.  The residual rebuilt from
    the FP64 right-hand side (rte_rhs) and rte_apply_K64e must give the same
    relative residual: to 1e-12 absolute (an FP32-accurate residual would be
    off by ~1e-7), the solver's ||b|| carrying an FP32 relative error."""
    n, L = 24, 4
    prob = rte_synth.hg2d_transport(n=n, L=L, seed=7)
    p = _plan(n, prob["mu_t"], prob["mu_s"], prob["sigma_hat"], prec=prec, q_policy=q)
    f = torch.from_numpy(prob["f"])
    u, st = p.solve(f, tol=1e-9)
    assert st["converged"]
    b = p.rhs(f)
    r = (b - u + p.apply_K64e(u)).cpu().numpy()
    relres = _wnorm(r) / _wnorm(b.cpu().numpy())
    assert relres <= 1e-9 * (1 + 1e-6)
    assert abs(relres - st["relres_true"]) <= 1e-6 * relres + 1e-12
    p.close()
