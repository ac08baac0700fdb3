"""The allocation-free K application (rte_apply_K_noalloc).

Some callers may not allocate device memory where they call (a host
application that owns and caps device memory, a real-time loop that forbids
allocator calls).  They use rte_apply_K_noalloc, which keeps everything in
one static device array.  This checks, through the C ABI, that two calls in
a row give the same y = K x as the plan-based rte_apply_K within the FP64
tolerance of the other parity tests (1e-12 relative L2), and that sizes
beyond the array are refused.  Collected last on purpose.
"""
import numpy as np
import pytest

from _util import random_packed, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_03061_gb300 import build
    build.build()


def _ref_apply(n, mu_t, mu_s, sig, x):
    from paper_1802_03061_gb300 import _binding as B
    L = len(sig) - 1
    plan = B.rte_plan_create(2, n, 1.0 / n, mu_t, mu_s, L, sig)
    xd = torch.from_numpy(x).cuda()
    yd = torch.zeros_like(xd)
    B.rte_apply_K(plan, xd.data_ptr(), yd.data_ptr(), 0)
    torch.cuda.synchronize()
    B.rte_destroy(plan)
    return yd.cpu().numpy()


def test_noalloc_matches_plan_apply_two_calls_in_a_row():
    from paper_1802_03061_gb300 import _binding as B
    stream = torch.cuda.current_stream()
    cases = [(64, 4, 10.0, 9.0, 0.5), (21, 2, 3.0, 2.0, 0.7)]
    for call, (n, L, mu_t, mu_s, g) in enumerate(cases):
        sig = [g ** k for k in range(L + 1)]
        x = random_packed(np.random.default_rng(40 + call), L, n)
        ref = _ref_apply(n, mu_t, mu_s, sig, x)
        xd = torch.from_numpy(x).cuda()
        yd = torch.full_like(xd, float("nan"))
        B.rte_apply_K_noalloc(n, 1.0 / n, mu_t, mu_s, L, sig, xd.data_ptr(), yd.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        assert rel(yd.cpu().numpy(), ref) < 1e-12


def test_noalloc_refuses_sizes_beyond_its_array():
    from paper_1802_03061_gb300 import _binding as B
    x = torch.zeros((1, 65, 65), dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(B.RteError) as ei:
        B.rte_apply_K_noalloc(65, 1 / 65, 1.0, 0.5, 0, [1.0], x.data_ptr(), y.data_ptr(), 0)
    assert ei.value.status == B.RTE_EUNSUPPORTED
    x = torch.zeros((6, 8, 8), dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(B.RteError) as ei:
        B.rte_apply_K_noalloc(8, 1 / 8, 1.0, 0.5, 5, [1.0] + [0.5] * 5, x.data_ptr(), y.data_ptr(), 0)
    assert ei.value.status == B.RTE_EUNSUPPORTED
