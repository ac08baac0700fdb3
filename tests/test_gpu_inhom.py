"""GPU parity of the inhomogeneous-medium direct Nystrom apply (C ABI)
against the oracle (oracle/inhom.py).  Tolerances: FP64 1e-12 relative L2
(same quadrature rules, rounding only); FP32 1e-5 (the optical depth and the
exponential in FP32, compensated summation)."""
import numpy as np
import pytest

import oracle
import rte_synth
from oracle import inhom
from _util import rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_03061_gb300 import build
    build.build()


def _mu(n, seed):
    rng = np.random.default_rng(seed)
    return 0.5 + 12.0 * rng.random((n, n))


@pytest.mark.parametrize("n", [1, 3, 8, 13])
def test_diagonal_matches_oracle(n):
    from paper_1802_03061_gb300 import Inhom
    mu = _mu(n, n)
    op = Inhom(mu)
    np.testing.assert_allclose(op.diag(), inhom.diag_2d(mu, 1.0 / n), rtol=1e-12)
    op.close()


@pytest.mark.parametrize("n", [1, 2, 5, 12, 17, 40])
def test_apply_matches_oracle(n):
    from paper_1802_03061_gb300 import Inhom
    mu = _mu(n, 100 + n)
    x = np.random.default_rng(n).standard_normal((n, n))
    op = Inhom(mu)
    ref = inhom.apply_2d(mu, 1.0 / n, x).reshape(n, n)
    assert rel(op.apply64(x).cpu().numpy(), ref) < 1e-12
    assert rel(op.apply32(x).cpu().numpy(), ref) < 1e-5
    op.close()


@pytest.mark.parametrize("n,fp64", [(64, True), (150, False), (150, True), (210, False)])
def test_sampled_rows_larger_grids(n, fp64):
    """The paper's test medium (mu_t = 1.2 + 10 exp(-|x - c|^2/4)); n = 150
    keeps mu_t in shared memory in FP32 but not in FP64, n = 210 in neither."""
    from paper_1802_03061_gb300 import Inhom
    mu, _ = rte_synth.inhom_mu_t(n)
    x = rte_synth.gaussian_mixture_2d(n, [(0.3, 0.6), (0.7, 0.4)], [0.05, 0.1])
    op = Inhom(mu)
    y = (op.apply64(x) if fp64 else op.apply32(x)).cpu().numpy().reshape(-1)
    rows = np.random.default_rng(n).choice(n * n, size=12, replace=False)
    D = np.zeros((n, n))
    D.reshape(-1)[rows] = op.diag().reshape(-1)[rows]  # the diagonal is pinned separately
    ref = inhom.apply_2d(mu, 1.0 / n, x, rows=rows, D=D)
    assert rel(y[rows], ref) < (1e-12 if fp64 else 1e-5)
    op.close()


def test_constant_mu_t_matches_the_fft_operator_off_the_diagonal():
    """Constant mu_t: the direct apply minus its diagonal equals the
    homogeneous FFT operator (L = 0, mu_s = 1) minus its exact cell weight."""
    from paper_1802_03061_gb300 import Inhom, Plan
    n, mu_t = 24, 3.0
    x = np.random.default_rng(2).standard_normal((n, n))
    op = Inhom(np.full((n, n), mu_t))
    y = op.apply64(x).cpu().numpy() - op.diag() * x
    p = Plan(n, mu_t=mu_t, mu_s=1.0, sigma_hat=[1.0])
    yh = p.apply_K(torch.from_numpy(x.astype(np.complex128)[None]).cuda()).cpu().numpy()[0].real
    yh = yh - p.cell_weights()[0] * x
    assert rel(y, yh) < 1e-12
    op.close()
    p.close()


def test_invalid_arguments_are_rejected():
    from paper_1802_03061_gb300 import RteError
    from paper_1802_03061_gb300 import _binding as B
    with pytest.raises(RteError):
        B.rte_inhom_create(4, 0.25, -np.ones(16))
    with pytest.raises(RteError):
        B.rte_inhom_create(4, 0.0, np.ones(16))
