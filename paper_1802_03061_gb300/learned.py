"""Learned initial guess for the solve (task extension; no counterpart in the paper).

Training data are solutions produced by the solver itself: for each seeded
instance, the library computes b = K~ g (step T.1), the network input
(b scaled by its RMS, the source, the coefficients) and the target
(u - b) / s_b.  The network (library kernels, BF16 tensor cores) is trained
with Adam on the GPU; the guess u0 = b + s_b * net(input) starts the solve,
which always runs to the same FP64 residual tolerance and falls back to the
zero start when the guess does not reduce the residual.
"""
import time

import numpy as np
import torch

from . import _binding as B
from .plan import Batch, Plan, _stream_ptr


class _Dev:
    def __init__(self, ptr, shape, typestr="<f4"):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3}


def _view(ptr, shape):
    return torch.as_tensor(_Dev(ptr, shape), device="cuda")


class GuessNet:
    """The 3x3 network of the learned guess (library object rte_cnn)."""

    def __init__(self, L, depth=6, seed=0, multiscale=True):
        """multiscale: 32 input channels, the last 2 (2L+1) holding b averaged
        over the 8 x 8 and 32 x 32 tiles around each pixel (where 3 (2L+1) + 4
        channels fit, L <= 4); else 16 (or 32) channels of b, f, coefficients."""
        self.L = L
        if multiscale and 3 * (2 * L + 1) + 4 <= 32:
            self.cin = 32
        else:
            self.cin = 16 if 2 * L + 5 <= 16 else 32
        self.cout = 16 if 2 * L + 1 <= 16 else 32
        self.depth = depth
        self.used = 2 * L + 1
        self.handle = B.rte_cnn_create(self.cin, 64, depth, self.cout, seed)
        self.steps = 0

    def train(self, X, T, epochs=4, batch=8, lr=1e-3, seed=0, log_every=0):
        """X, T: bf16 CUDA tensors [N, n, n, cin|cout]."""
        N, n = X.shape[0], X.shape[1]
        g = torch.Generator(device="cpu").manual_seed(seed)
        losses = []
        total = epochs * ((N + batch - 1) // batch)
        k = 0
        for ep in range(epochs):
            perm = torch.randperm(N, generator=g)
            for i in range(0, N - batch + 1, batch):
                idx = perm[i:i + batch].cuda()
                xb = X.index_select(0, idx).contiguous()
                tb = T.index_select(0, idx).contiguous()
                # cosine decay of the step size
                lr_k = lr * 0.5 * (1.0 + np.cos(np.pi * k / max(1, total)))
                want = log_every and (k % log_every == 0)
                loss = B.rte_cnn_train_step(self.handle, xb.data_ptr(), tb.data_ptr(), batch, n, n, self.used,
                                            lr_k, want_loss=bool(want))
                if want:
                    losses.append((k, loss))
                k += 1
                self.steps += 1
        return losses

    def loss(self, X, T, batch=8):
        N, n = X.shape[0], X.shape[1]
        tot, cnt = 0.0, 0
        for i in range(0, N - batch + 1, batch):
            xb = X[i:i + batch].contiguous()
            tb = T[i:i + batch].contiguous()
            tot += B.rte_cnn_train_step(self.handle, xb.data_ptr(), tb.data_ptr(), batch, n, n, self.used, 0.0)
            cnt += 1
        return tot / max(1, cnt)

    def guess(self, plan, f_dev, stream=None):
        """u0 (FP64 mode field) and b for a plan and a source on the device."""
        n = plan.n
        b = plan.empty()
        u0 = plan.empty()
        Xs = torch.empty((n, n, self.cin), dtype=torch.bfloat16, device="cuda")
        B.rte_cnn_guess_apply(self.handle, plan.handle, f_dev.data_ptr(), b.data_ptr(), Xs.data_ptr(),
                              u0.data_ptr(), _stream_ptr(stream))
        return u0, b

    def state(self):
        out = {}
        for l in range(self.depth):
            d = B.rte_cnn_layer(self.handle, l)
            out["w%d" % l] = _view(d["w"], (9, d["cin"], d["cout"])).cpu().numpy().copy()
            out["b%d" % l] = _view(d["b"], (d["cout"],)).cpu().numpy().copy()
        return out

    def load_state(self, st):
        for l in range(self.depth):
            d = B.rte_cnn_layer(self.handle, l)
            _view(d["w"], (9, d["cin"], d["cout"])).copy_(torch.from_numpy(np.asarray(st["w%d" % l], np.float32)))
            _view(d["b"], (d["cout"],)).copy_(torch.from_numpy(np.asarray(st["b%d" % l], np.float32)))
        B.rte_cnn_sync_weights(self.handle)

    def save(self, path):
        """Weights to a file (library format, rte_cnn_save)."""
        B.rte_cnn_save(self.handle, path)

    def load(self, path, stream=None):
        """Weights from a file written by save() for a network of this shape."""
        B.rte_cnn_load(self.handle, path, _stream_ptr(stream))

    def save_checkpoint(self, path):
        """Training checkpoint: weights, Adam moments and step count (rte_cnn_save_state)."""
        B.rte_cnn_save_state(self.handle, path)

    def load_checkpoint(self, path, stream=None):
        """Resume from save_checkpoint(): later training steps repeat the saving run's."""
        B.rte_cnn_load_state(self.handle, path, _stream_ptr(stream))

    def close(self):
        if getattr(self, "handle", None):
            B.rte_cnn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def generate(instances, cin, cout, chunk=128, prec="mixed_fp32", restart=30):
    """Solve every instance (batched, one graph launch per chunk) and build the
    network inputs X and targets T (bf16, on the GPU)."""
    N = len(instances)
    n = int(instances[0]["n"])
    X = torch.empty((N, n, n, cin), dtype=torch.bfloat16, device="cuda")
    T = torch.empty((N, n, n, cout), dtype=torch.bfloat16, device="cuda")
    stats_all = []
    for c0 in range(0, N, chunk):
        part = instances[c0:c0 + chunk]
        bt = Batch(part, prec=prec, tol=1e-8, restart=restart, maxit=4000)
        f = bt.pack_sources([d["f"] for d in part])
        u, stats, _ = bt.solve(f)
        stats_all.extend(stats)
        for i, d in enumerate(part):
            plan = B.rte_batch_plan(bt.handle, i)
            L = len(d["sigma_hat"]) - 1
            fi = f[bt.f_off[i]:bt.f_off[i + 1]]
            ui = u[bt.u_off[i]:bt.u_off[i + 1]]
            bi = torch.empty(2 * (L + 1) * n * n, dtype=torch.float64, device="cuda")
            B.rte_rhs(plan, fi.data_ptr(), bi.data_ptr())
            B.rte_guess_features(plan, cin, fi.data_ptr(), bi.data_ptr(), X[c0 + i].data_ptr())
            B.rte_guess_targets(plan, cout, fi.data_ptr(), ui.data_ptr(), bi.data_ptr(), T[c0 + i].data_ptr())
        torch.cuda.synchronize()
        bt.close()
    return X, T, stats_all


def evaluate(net, instances, prec="mixed_fp32", restart=30, flush=True, preconds=(0,)):
    """Per instance: zero-start solve vs learned-guess solve (guess time
    included), both to the same FP64 relative residual 1e-8 with the same
    solver settings, for each setting of the periodic preconditioner in
    `preconds` (keys "zero"/"guess" without it, "zero_pc"/"guess_pc" with it),
    and the guess's initial relative residual."""
    rows = []
    fl = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda") if flush else None
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    for d in instances:
        plan = Plan(int(d["n"]), h=d["h"], mu_t=d["mu_t"], mu_s=d["mu_s"], sigma_hat=d["sigma_hat"], prec=prec,
                    restart=restart, maxit=4000)
        f = torch.from_numpy(d["f"]).cuda()
        res = {}
        for pc in preconds:
            sfx = "_pc" if pc else ""
            # warm both paths once (graph capture, workspaces)
            plan.solve(f, precond=pc)
            u0, _ = net.guess(plan, f)
            plan.solve(f, u=u0.clone(), precond=pc)
            for mode in ("zero", "guess"):
                if fl is not None:
                    fl.zero_()
                torch.cuda.synchronize()
                e0.record(stream)
                if mode == "zero":
                    u, st = plan.solve(f, precond=pc)
                else:
                    u0, _ = net.guess(plan, f)
                    u, st = plan.solve(f, u=u0, precond=pc)
                e1.record(stream)
                e1.synchronize()
                res[mode + sfx] = dict(ms=e0.elapsed_time(e1), iters=st["iters"], outer=st["outer"],
                                       relres=st["relres_true"], converged=st["converged"], u=u)
            res["diff" + sfx] = float(
                torch.linalg.vector_norm(torch.view_as_real(res["zero" + sfx]["u"] - res["guess" + sfx]["u"])) /
                torch.linalg.vector_norm(torch.view_as_real(res["zero" + sfx]["u"])))
            del res["zero" + sfx]["u"], res["guess" + sfx]["u"]
        # initial residual of the guess
        u0, b = net.guess(plan, f)
        r = plan.apply_A(u0) - b
        res["guess_relres0"] = float(torch.linalg.vector_norm(torch.view_as_real(r)) /
                                     torch.linalg.vector_norm(torch.view_as_real(b)))
        rows.append(res)
        plan.close()
    return rows


def summarize(rows, sfx=""):
    """Means over the instances of one preconditioner setting (sfx "" or "_pc")."""
    z_ms = np.array([r["zero" + sfx]["ms"] for r in rows])
    g_ms = np.array([r["guess" + sfx]["ms"] for r in rows])
    z_it = np.array([r["zero" + sfx]["iters"] for r in rows])
    g_it = np.array([r["guess" + sfx]["iters"] for r in rows])
    r0 = np.array([r["guess_relres0"] for r in rows])
    return dict(count=len(rows), zero_ms=float(z_ms.mean()), guess_ms=float(g_ms.mean()),
                zero_iters=float(z_it.mean()), guess_iters=float(g_it.mean()),
                guess_relres0_median=float(np.median(r0)), guess_relres0_p10=float(np.percentile(r0, 10)),
                guess_relres0_p90=float(np.percentile(r0, 90)), time_ratio=float(g_ms.mean() / z_ms.mean()),
                fewer_iters_frac=float(np.mean(g_it < z_it)), more_iters_frac=float(np.mean(g_it > z_it)),
                all_converged=bool(all(r["zero" + sfx]["converged"] and r["guess" + sfx]["converged"] for r in rows)),
                max_solution_diff=float(max(r["diff" + sfx] for r in rows)))
