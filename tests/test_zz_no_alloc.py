"""The allocation-free K application (rte_apply_K_noalloc).

Some callers may not allocate device memory where they call (a host
application that owns and caps device memory, a real-time loop that forbids
allocator calls).  They use rte_apply_K_noalloc, which keeps everything in
one static device array.  This checks, through the C ABI, that two calls in
a row give y = K x equal to the oracle's direct Nystrom sum and to the
plan-based rte_apply_K, within the FP64 tolerance of the other parity tests
(1e-12 relative L2); that once the first call on the device has been made, a
further call leaves the device's free memory unchanged; and that sizes
beyond the array are refused.  Collected last on purpose.
"""
import numpy as np
import pytest

import oracle
from _util import packed_to_full, random_packed, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_03061_gb300 import build
    build.build()


def _plan_apply(n, mu_t, mu_s, sig, x):
    from paper_1802_03061_gb300 import _binding as B
    L = len(sig) - 1
    plan = B.rte_plan_create(2, n, 1.0 / n, mu_t, mu_s, L, sig)
    xd = torch.from_numpy(x).cuda()
    yd = torch.zeros_like(xd)
    B.rte_apply_K(plan, xd.data_ptr(), yd.data_ptr(), 0)
    torch.cuda.synchronize()
    B.rte_destroy(plan)
    return yd.cpu().numpy()


CASES = [(64, 4, 10.0, 9.0, 0.5), (21, 2, 3.0, 2.0, 0.7)]


def test_noalloc_matches_oracle_and_plan_two_calls_in_a_row():
    from paper_1802_03061_gb300 import _binding as B
    stream = torch.cuda.current_stream()
    inputs = []
    for c, (n, L, mu_t, mu_s, g) in enumerate(CASES):
        sig = [g ** k for k in range(L + 1)]
        x = random_packed(np.random.default_rng(40 + c), L, n)
        xd = torch.from_numpy(x).cuda()
        inputs.append((n, L, mu_t, mu_s, sig, x, xd, torch.full_like(xd, float("nan"))))
    torch.cuda.synchronize()
    # the first call on this device looks the static array up (and, under
    # lazy module loading, loads the module that holds it); every later call
    # must leave the device's free memory exactly where it was
    for n, L, mu_t, mu_s, sig, x, xd, yd in inputs:
        B.rte_apply_K_noalloc(n, 1.0 / n, mu_t, mu_s, L, sig, xd.data_ptr(), yd.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    outs = []
    for n, L, mu_t, mu_s, sig, x, xd, yd in inputs:
        yd.fill_(float("nan"))
        B.rte_apply_K_noalloc(n, 1.0 / n, mu_t, mu_s, L, sig, xd.data_ptr(), yd.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        outs.append(yd.cpu().numpy())
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    for (n, L, mu_t, mu_s, sig, x, xd, yd), y in zip(inputs, outs):
        # the oracle's direct sum at every cell for n = 21, at 600 sampled
        # cells (all modes) for n = 64
        rows = None if n * n <= 600 else np.random.default_rng(n).choice(n * n, size=600, replace=False)
        ref = oracle.apply_K_2d(n, 1.0 / n, mu_t, mu_s, sig, packed_to_full(x), rows=rows)[L:]
        got = y if rows is None else y.reshape(L + 1, -1)[:, rows]
        assert rel(got, ref) < 1e-12
        assert rel(y, _plan_apply(n, mu_t, mu_s, sig, x)) < 1e-12


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
