"""Torch-tensor convenience wrapper over the C ABI (allocation and streams only)."""
import numpy as np
import torch

from . import _binding as B


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Plan:
    """A plan for one grid and one set of coefficients.

    dim = 2: fields are complex tensors of shape (L+1, n, n) (modes 0..L);
    dim = 3: real tensors of shape (n, n, n).  FP64 for apply_K / apply_A /
    rhs / solve; FP32 (complex64 / float32) for apply_K32.
    """

    def __init__(self, n, h=None, mu_t=1.0, mu_s=0.5, sigma_hat=(1.0,), dim=2, prec="fp64", tol=1e-8,
                 restart=40, maxit=2000, inner_tol=1e-4, q_policy=0, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.dim, self.n = dim, int(n)
        self.h = 1.0 / n if h is None else float(h)
        self.mu_t, self.mu_s = float(mu_t), float(mu_s)
        self.sigma_hat = [float(v) for v in sigma_hat]
        self.L = len(self.sigma_hat) - 1
        self.opts = B.make_opts(prec, tol, restart, maxit, inner_tol, 0, q_policy)
        self.handle = B.rte_plan_create(dim, self.n, self.h, self.mu_t, self.mu_s, self.L, self.sigma_hat,
                                        self.opts, _stream_ptr(stream))
        self.info = B.rte_plan_info(self.handle)
        self.Q = self.info["Q"]

    # -- buffers ------------------------------------------------------------
    def shape(self):
        return (self.L + 1, self.n, self.n) if self.dim == 2 else (self.n, self.n, self.n)

    def empty(self, fp32=False):
        if self.dim == 2:
            dt = torch.complex64 if fp32 else torch.complex128
        else:
            dt = torch.float32 if fp32 else torch.float64
        return torch.zeros(self.shape(), dtype=dt, device="cuda")

    def _check(self, t, fp32=False):
        want = self.empty(fp32).dtype
        if t.dtype != want or tuple(t.shape) != self.shape() or not t.is_cuda or not t.is_contiguous():
            raise ValueError("expected a contiguous CUDA tensor %s of shape %s" % (want, self.shape()))

    # -- operators ----------------------------------------------------------
    def apply_K(self, x, y=None, stream=None):
        self._check(x)
        y = self.empty() if y is None else y
        B.rte_apply_K(self.handle, x.data_ptr(), y.data_ptr(), _stream_ptr(stream))
        return y

    def apply_A(self, x, y=None, stream=None):
        self._check(x)
        y = self.empty() if y is None else y
        B.rte_apply_A(self.handle, x.data_ptr(), y.data_ptr(), _stream_ptr(stream))
        return y

    def apply_K32(self, x, y=None, stream=None):
        self._check(x, fp32=True)
        y = self.empty(fp32=True) if y is None else y
        B.rte_apply_K32(self.handle, x.data_ptr(), y.data_ptr(), _stream_ptr(stream))
        return y

    def rhs(self, f, b=None, stream=None):
        f = f.to(device="cuda", dtype=torch.float64).contiguous()
        b = self.empty() if b is None else b
        B.rte_rhs(self.handle, f.data_ptr(), b.data_ptr(), _stream_ptr(stream))
        return b

    def solve(self, f, u=None, prec=None, tol=None, restart=None, maxit=None, inner_tol=None, stream=None):
        f = f.to(device="cuda", dtype=torch.float64).contiguous()
        use_guess = u is not None
        u = self.empty() if u is None else u
        o = self.opts
        opts = B.make_opts(prec if prec is not None else o.prec, tol or o.tol, restart or o.restart,
                           maxit or o.maxit, inner_tol or o.inner_tol, use_guess, o.q_policy)
        stats = B.rte_solve(self.handle, f.data_ptr(), u.data_ptr(), opts, _stream_ptr(stream))
        return u, stats

    def solve_host(self, f_host, u_host=None, prec=None, tol=None, stream=None):
        """f_host: numpy float64 array; u_host: numpy complex128 (2D) / float64 (3D) output."""
        f_host = np.ascontiguousarray(f_host, dtype=np.float64)
        if u_host is None:
            u_host = np.zeros(self.shape(), dtype=np.complex128 if self.dim == 2 else np.float64)
        o = self.opts
        opts = B.make_opts(prec if prec is not None else o.prec, tol or o.tol, o.restart, o.maxit, o.inner_tol, 0,
                           o.q_policy)
        stats = B.rte_solve_host(self.handle, f_host.ctypes.data, u_host.ctypes.data, opts, _stream_ptr(stream))
        return u_host, stats

    def cell_weights(self):
        return B.rte_plan_cell_weights(self.handle, 2 * self.L + 1 if self.dim == 2 else 1)

    def close(self):
        if getattr(self, "handle", None):
            B.rte_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
