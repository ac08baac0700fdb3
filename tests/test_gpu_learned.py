"""The learned initial guess: trained on solver-generated solutions (small
grids here), it must lower the initial residual on held-out seeds and cost at
most one extra GMRES iteration, and the solve must reach the same FP64
residual (and the same solution within cond_est * tol) as the zero start.
The iteration and time differences against the zero start are printed, so
the measured gain or loss is stated, not implied.
The iteration gain of a guess with initial relative residual r0 is only
about log(1/r0) / log(1e8) of the iterations, so a 3x3 network whose
receptive field (13 cells) is far below the transport Green's function's
decay length gains little; the test records the numbers."""
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


def _instances(seeds, n=64, L=4):
    return [rte_synth.learned_guess_instance(s, n=n, L=L) for s in seeds]


def test_learned_guess_lowers_initial_residual_without_iteration_regression():
    from paper_1802_03061_gb300 import learned
    train = _instances(range(10**6, 10**6 + 192))
    held = _instances(range(0, 12))
    net = learned.GuessNet(L=4, depth=6, seed=1)
    X, T, st = learned.generate(train, net.cin, net.cout, chunk=96)
    assert all(s["converged"] for s in st)
    before = net.loss(X[:64], T[:64])
    net.train(X, T, epochs=6, batch=8, lr=2e-3)
    after = net.loss(X[:64], T[:64])
    assert after < 0.5 * before
    rows = learned.evaluate(net, held, flush=False)
    s = learned.summarize(rows)
    assert s["all_converged"]
    assert s["guess_relres0_median"] < 0.5          # the guess is much closer than u0 = 0 (relres 1)
    assert s["guess_iters"] <= s["zero_iters"] + 1  # no iteration penalty beyond one
    print("learned guess vs zero start: iterations %+.2f, ms %+.3f (%s)"
          % (s["guess_iters"] - s["zero_iters"], s["guess_ms"] - s["zero_ms"], s))
    for r in rows:
        assert r["diff"] < 2e-6                      # cond_est (<= 199) * 1e-8
    net.close()


def test_bad_guess_falls_back_to_zero_start():
    from paper_1802_03061_gb300 import Plan
    d = rte_synth.learned_guess_instance(5, n=32, L=2)
    p = Plan(32, mu_t=d["mu_t"], mu_s=d["mu_s"], sigma_hat=d["sigma_hat"], prec="mixed_fp32")
    f = torch.from_numpy(d["f"]).cuda()
    u, st = p.solve(f)
    bad = torch.full_like(u, 1e6)
    u2, st2 = p.solve(f, u=bad)
    assert st2["converged"] and st2["iters"] == st["iters"]
    assert torch.allclose(u, u2, rtol=0, atol=1e-12 * float(u.abs().max()))
    p.close()


def test_guess_handle_load_and_apply(tmp_path):
    """The boundary's rte_guess handle: a network saved by rte_cnn_save,
    loaded by rte_guess_load (shape from the file), gives through
    rte_guess_apply the same initial guess as the network it was saved from,
    and the solve started from it reaches the zero start's solution."""
    from paper_1802_03061_gb300 import Plan, learned
    from paper_1802_03061_gb300 import _binding as B
    d = rte_synth.learned_guess_instance(7, n=48, L=2)
    net = learned.GuessNet(L=2, depth=3, seed=4)
    path = str(tmp_path / "guess.bin")
    net.save(path)
    g = B.rte_guess_load(path)
    p = Plan(48, mu_t=d["mu_t"], mu_s=d["mu_s"], sigma_hat=d["sigma_hat"], prec="mixed_fp32")
    f = torch.from_numpy(d["f"]).cuda()
    want, _ = net.guess(p, f)
    u0 = p.empty()
    B.rte_guess_apply(g, p.handle, f.data_ptr(), u0.data_ptr())
    torch.cuda.synchronize()
    assert torch.equal(u0, want)
    u, st = p.solve(f, u=u0.clone())
    uz, stz = p.solve(f)
    assert st["converged"] and stz["converged"]
    rho = d["mu_s"] / d["mu_t"]
    assert float((u - uz).abs().max()) <= 2 * (1 + rho) / (1 - rho) * 1e-8 * float(uz.abs().max())
    B.rte_guess_destroy(g)
    with pytest.raises(B.RteError) as ei:
        B.rte_guess_load(str(tmp_path / "missing.bin"))
    assert ei.value.status == B.RTE_EINVAL
    p.close()
    net.close()


def test_multiscale_features_are_tile_means_of_b():
    """The network input of a multi-scale net (32 channels at L = 2): channels
    2L+5.. hold the 8 x 8 and 32 x 32 tile means of the scaled b channels
    (n = 48: partial 32-tiles at the border average their own cells)."""
    from paper_1802_03061_gb300 import Plan
    from paper_1802_03061_gb300 import _binding as B
    n, L = 48, 2
    nch = 2 * L + 1
    d = rte_synth.learned_guess_instance(3, n=n, L=L)
    p = Plan(n, mu_t=d["mu_t"], mu_s=d["mu_s"], sigma_hat=d["sigma_hat"], prec="mixed_fp32")
    f = torch.from_numpy(d["f"]).cuda()
    b = p.rhs(f)
    X = torch.empty((n, n, 32), dtype=torch.bfloat16, device="cuda")
    B.rte_guess_features(p.handle, 32, f.data_ptr(), b.data_ptr(), X.data_ptr())
    Xh = X.float().cpu().numpy()
    bh = b.cpu().numpy()
    chans = [bh[0].real] + [v for k in range(1, L + 1) for v in (bh[k].real, bh[k].imag)]
    s_b = np.sqrt(sum((c ** 2).sum() for c in chans) / (nch * n * n))
    for c, ch in enumerate(chans):
        sc = ch / s_b
        assert np.abs(Xh[..., c] - sc).max() <= 1e-2 * np.abs(sc).max() + 1e-6
        for t, off in ((8, nch + 4), (32, 2 * nch + 4)):
            want = np.zeros_like(sc)
            for y0 in range(0, n, t):
                for x0 in range(0, n, t):
                    want[y0:y0 + t, x0:x0 + t] = sc[y0:y0 + t, x0:x0 + t].mean()
            assert np.abs(Xh[..., off + c] - want).max() <= 1e-2 * np.abs(sc).max() + 1e-6
    p.close()
