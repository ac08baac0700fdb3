"""Allocation failure, injected on the host: every create call (and the
first solve, which allocates the Krylov workspace) must return RTE_ENOMEM
when any one of its device or pinned-host allocations fails, and leave no
allocation behind.  The failure is simulated by the library's allocation
wrapper (rte_debug_fail_alloc): no real out-of-memory condition and no GPU
fault is caused.  For each create call the test counts its allocations in a
successful run, then fails each of them in turn and checks the library's
live-allocation counts and the device's free memory."""
import numpy as np
import pytest

import rte_synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_03061_gb300 import build
    build.build()
    yield
    from paper_1802_03061_gb300 import _binding as B
    B.rte_debug_fail_alloc(0)


def _every_failure(create, destroy):
    from paper_1802_03061_gb300 import _binding as B
    B.rte_debug_fail_alloc(0)
    h = create()
    torch.cuda.synchronize()
    seen, _, _ = B.rte_debug_fail_alloc(0)
    destroy(h)
    torch.cuda.synchronize()
    _, dev0, host0 = B.rte_debug_fail_alloc(0)
    free0 = torch.cuda.mem_get_info()[0]
    assert seen >= 3
    for k in range(1, seen + 1):
        B.rte_debug_fail_alloc(k)
        with pytest.raises(B.RteError) as ei:
            h = create()
        assert ei.value.status == B.RTE_ENOMEM, (k, seen)
        _, dev, host = B.rte_debug_fail_alloc(0)
        assert (dev, host) == (dev0, host0), (k, seen)
    torch.cuda.synchronize()
    # the stream-ordered pool returns its memory at the synchronisation
    assert torch.cuda.mem_get_info()[0] >= free0 - (4 << 20)
    # and the call still works afterwards
    destroy(create())
    return seen


@pytest.mark.parametrize("dim,n,L,q", [(2, 24, 3, 64), (2, 20, 2, 0), (3, 10, 0, 0)])
def test_plan_create_fails_cleanly(dim, n, L, q):
    from paper_1802_03061_gb300 import _binding as B
    sig = list(rte_synth.hg_sigma_hat(0.5, L))
    opts = B.make_opts("mixed_fp32", q_policy=q)
    _every_failure(lambda: B.rte_plan_create(dim, n, 1.0 / n, 5.0, 4.0, L, sig, opts), B.rte_destroy)


def test_first_solve_workspace_failure_leaves_the_plan_usable():
    """The first solve allocates the Krylov workspace (and, when asked for,
    the preconditioner): a failure there returns RTE_ENOMEM and a later
    solve of the same plan succeeds."""
    from paper_1802_03061_gb300 import Plan
    from paper_1802_03061_gb300 import _binding as B
    d = rte_synth.hg2d_transport(n=24, L=2, seed=5)
    f = torch.from_numpy(d["f"]).cuda()
    ref = Plan(24, mu_t=d["mu_t"], mu_s=d["mu_s"], sigma_hat=d["sigma_hat"], prec="mixed_fp32", precond=1)
    B.rte_debug_fail_alloc(0)
    want, st = ref.solve(f)
    seen, _, _ = B.rte_debug_fail_alloc(0)
    ref.close()
    assert st["converged"] and seen >= 1
    for k in range(1, seen + 1):
        p = Plan(24, mu_t=d["mu_t"], mu_s=d["mu_s"], sigma_hat=d["sigma_hat"], prec="mixed_fp32", precond=1)
        B.rte_debug_fail_alloc(k)
        with pytest.raises(B.RteError) as ei:
            p.solve(f)
        assert ei.value.status == B.RTE_ENOMEM
        B.rte_debug_fail_alloc(0)
        u, st = p.solve(f)
        assert st["converged"] and torch.equal(u, want)
        p.close()


def test_batch_create_fails_cleanly():
    from paper_1802_03061_gb300 import _binding as B
    rng = np.random.default_rng(3)
    inst = [rte_synth.random_instance_2d(rng, n, L) for n, L in ((8, 1), (12, 2), (6, 0))]
    opts = B.make_opts("mixed_fp32", 1e-8, 20)
    _every_failure(lambda: B.rte_batch_create(inst, opts), B.rte_batch_destroy)


def test_inhom_create_fails_cleanly():
    from paper_1802_03061_gb300 import _binding as B
    mu, _ = rte_synth.inhom_mu_t(12)
    _every_failure(lambda: B.rte_inhom_create(12, 1.0 / 12, np.ascontiguousarray(mu)), B.rte_inhom_destroy)


@pytest.mark.parametrize("n", [6, 20])  # the Stockham and the warp passes (float-float copies)
def test_aniso3d_create_fails_cleanly(n):
    from paper_1802_03061_gb300 import _binding as B
    _every_failure(lambda: B.rte_aniso3d_create(n, 1.0 / n, 4.0, 3.0, 1, [1.0, 0.5]), B.rte_aniso3d_destroy)


@pytest.mark.parametrize("prec", ["fp64", "mixed_fp32"])
def test_aniso3d_first_solve_failure_leaves_the_handle_usable(prec):
    """The first solve allocates its vectors and the Krylov workspace: a
    failure there returns RTE_ENOMEM, and a later solve of the same handle
    gives the result of an undisturbed one."""
    from paper_1802_03061_gb300 import Aniso3D
    from paper_1802_03061_gb300 import _binding as B
    n = 20
    f = rte_synth.gaussian_3d(n, (0.4, 0.5, 0.5), 0.1)
    ref = Aniso3D(n, 6.0, 5.0, [1.0, 0.5])
    B.rte_debug_fail_alloc(0)
    want, st = ref.solve(f, tol=1e-9, prec=prec)
    seen, _, _ = B.rte_debug_fail_alloc(0)
    ref.close()
    assert st["converged"] and seen >= 3
    for k in range(1, seen + 1):
        op = Aniso3D(n, 6.0, 5.0, [1.0, 0.5])
        B.rte_debug_fail_alloc(k)
        with pytest.raises(B.RteError) as ei:
            op.solve(f, tol=1e-9, prec=prec)
        assert ei.value.status == B.RTE_ENOMEM
        B.rte_debug_fail_alloc(0)
        u, st = op.solve(f, tol=1e-9, prec=prec)
        assert st["converged"] and torch.equal(u, want)
        op.close()


def test_cnn_create_fails_cleanly():
    from paper_1802_03061_gb300 import _binding as B
    _every_failure(lambda: B.rte_cnn_create(16, 64, 3, 16, 1), B.rte_cnn_destroy)
