"""The mode coupling by FFTs along the mode axis (the kernel of the pair
(k, k') depends only on k - k', Sec. 3.3.1): the operator for truncations
beyond the direct mix (L = 12..64) and, forced, at small L, against the
oracle's direct Nystrom sum and against the direct (2L+1)^2 mix.  FP64 and
float-float to 1e-12, FP32 to 1e-5 (relative L2)."""
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


def _plan(n, L, mode_mix=0, prec="mixed_fp32", q=0, g=0.6, mu_t=10.0, mu_s=9.0):
    from paper_1802_03061_gb300 import Plan
    return Plan(n, mu_t=mu_t, mu_s=mu_s, sigma_hat=rte_synth.hg_sigma_hat(g, L), prec=prec, q_policy=q,
                mode_mix=mode_mix)


# n ragged against the 16-frequency blocks; P = 72 (L = 16), 144 (L = 32),
# 288 (L = 64); q = 64: the warp row passes
@pytest.mark.parametrize("n,L,q", [(8, 12, 0), (11, 16, 0), (12, 32, 0), (7, 64, 0), (20, 16, 64)])
def test_large_L_operator_matches_direct_sum(n, L, q):
    p = _plan(n, L, q=q)
    assert p.Q == (q or p.Q)
    sig = p.sigma_hat
    x = random_packed(np.random.default_rng(n + L), L, n)
    ref = oracle.apply_K_2d(n, 1.0 / n, 10.0, 9.0, sig, packed_to_full(x))[L:]
    xd = torch.from_numpy(x).cuda()
    assert rel(p.apply_K(xd).cpu().numpy(), ref) < 1e-12
    assert rel(p.apply_K64e(xd).cpu().numpy(), ref) < 1e-12
    x32 = x.astype(np.complex64)
    ref32 = oracle.apply_K_2d(n, 1.0 / n, 10.0, 9.0, sig, packed_to_full(x32.astype(complex)))[L:]
    assert rel(p.apply_K32(torch.from_numpy(x32).cuda()).cpu().numpy(), ref32) < 1e-5
    p.close()


@pytest.mark.parametrize("L", [0, 1, 3, 8])
def test_mode_fft_equals_direct_mix_at_small_L(L):
    """mode_mix = 2 forces the mode-axis FFT where the direct mix also runs:
    the two agree to rounding and both match the direct sum."""
    n = 20
    pf, pd = _plan(n, L, mode_mix="fft"), _plan(n, L, mode_mix="direct")
    x = random_packed(np.random.default_rng(3 + L), L, n)
    ref = oracle.apply_K_2d(n, 1.0 / n, 10.0, 9.0, pf.sigma_hat, packed_to_full(x))[L:]
    xd = torch.from_numpy(x).cuda()
    yf, yd = pf.apply_K(xd).cpu().numpy(), pd.apply_K(xd).cpu().numpy()
    assert rel(yf, ref) < 1e-12 and rel(yd, ref) < 1e-12 and rel(yf, yd) < 1e-12
    yf32 = pf.apply_K32(xd.to(torch.complex64)).cpu().numpy()
    yd32 = pd.apply_K32(xd.to(torch.complex64)).cpu().numpy()
    assert rel(yf32, yd32) < 1e-5
    pf.close()
    pd.close()


@pytest.mark.parametrize("n,L", [(9, 16), (6, 40)])
def test_large_L_rhs_matches_direct_sum(n, L):
    p = _plan(n, L)
    f = rte_synth.gaussian_mixture_2d(n, [(0.4, 0.6), (0.7, 0.3)], [0.1, 0.05])
    b = p.rhs(torch.from_numpy(f)).cpu().numpy()
    assert rel(b, oracle.rhs_2d(n, 1.0 / n, 10.0, L, f)[L:]) < 1e-12
    p.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed_fp32"])
def test_large_L_solve_matches_dense(prec):
    """n = 6, L = 16 (1188 complex unknowns): the solve against dense LU
    within 2 cond_est tol."""
    n, L, mu_t, mu_s = 6, 16, 8.0, 7.2
    p = _plan(n, L, prec=prec, mu_t=mu_t, mu_s=mu_s, g=0.7)
    f = rte_synth.gaussian_mixture_2d(n, [(0.4, 0.55)], [0.2])
    u, st = p.solve(torch.from_numpy(f), tol=1e-11)
    assert st["converged"] and st["relres_true"] <= 1e-11
    u_ref, _ = oracle.solve_dense_2d(n, 1.0 / n, mu_t, mu_s, p.sigma_hat, f)
    rho = mu_s / mu_t
    assert rel(u.cpu().numpy(), u_ref[L:]) < 2 * (1 + rho) / (1 - rho) * 1e-11
    p.close()


def test_large_L_full_size_sampled():
    """256^2 cells, L = 32 (65 real channels, P = 144): K32 and K64e at
    sampled cells (all 65 modes) against the direct sum."""
    n, L = 256, 32
    p = _plan(n, L, g=0.8)
    x = random_packed(np.random.default_rng(9), L, n).astype(np.complex64)
    rows = np.random.default_rng(10).choice(n * n, size=3, replace=False)
    ref = oracle.apply_K_2d(n, 1.0 / n, 10.0, 9.0, p.sigma_hat, packed_to_full(x.astype(complex)), rows=rows)[L:]
    y32 = p.apply_K32(torch.from_numpy(x).cuda()).cpu().numpy().reshape(L + 1, -1)[:, rows]
    ye = p.apply_K64e(torch.from_numpy(x.astype(complex)).cuda()).cpu().numpy().reshape(L + 1, -1)[:, rows]
    assert rel(ye, ref) < 1e-12
    assert rel(y32, ref) < 1e-5
    p.close()


def test_direct_mix_beyond_its_range_is_refused():
    from paper_1802_03061_gb300 import _binding as B
    with pytest.raises(B.RteError) as ei:
        _plan(8, 9, mode_mix="direct")
    assert ei.value.status == B.RTE_EINVAL
