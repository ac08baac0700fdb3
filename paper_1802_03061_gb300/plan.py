"""Torch-tensor convenience wrapper over the C ABI (allocation and streams only)."""
import json
import os

import numpy as np
import torch

from . import _binding as B

TUNE_CACHE = os.environ.get("RTE_TUNE_CACHE",
                            os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tune_cache.json"))


def autotune(shapes, prec="mixed_fp32", reps=10, cache_path=TUNE_CACHE, stream=None):
    """Pick (Q, rows per block) for each (n, L) by measurement (rte_autotune),
    persisting results in a JSON cache keyed by device name, n, L and prec."""
    dev = torch.cuda.get_device_name()
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as fh:
                cache = json.load(fh)
        except (OSError, ValueError):
            cache = {}
    out = {}
    changed = False
    for (n, L) in sorted(set(shapes)):
        key = "%s|%d|%d|%s" % (dev, n, L, prec)
        if key not in cache:
            q, rb, ms = B.rte_autotune(n, L, prec, reps, _stream_ptr(stream))
            cache[key] = {"q": q, "rows_per_block": rb, "ms": ms}
            changed = True
        out[(n, L)] = cache[key]
    if changed and cache_path:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1)
        os.replace(tmp, cache_path)
    return out


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
                 restart=40, maxit=2000, inner_tol=1e-4, q_policy=0, stream=None, inner_solver="gmres", precond=0,
                 precond_lmax=0, mode_mix=0):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.dim, self.n = dim, int(n)
        self.h = 1.0 / n if h is None else float(h)
        self.mu_t, self.mu_s = float(mu_t), float(mu_s)
        self.sigma_hat = [float(v) for v in sigma_hat]
        self.L = len(self.sigma_hat) - 1
        self.opts = B.make_opts(prec, tol, restart, maxit, inner_tol, 0, q_policy, inner_solver, precond,
                                precond_lmax, mode_mix)
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

    def apply_K64e(self, x, y=None, stream=None):
        """FP64-accurate K x in float-float arithmetic on the FP32 units."""
        self._check(x)
        y = self.empty() if y is None else y
        B.rte_apply_K64e(self.handle, x.data_ptr(), y.data_ptr(), _stream_ptr(stream))
        return y

    def apply_precond32(self, x, y=None, stream=None):
        """The periodic preconditioner on an FP32 field (see rte_apply_precond32)."""
        self._check(x, fp32=True)
        y = self.empty(fp32=True) if y is None else y
        B.rte_apply_precond32(self.handle, x.data_ptr(), y.data_ptr(), _stream_ptr(stream))
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

    def solve(self, f, u=None, prec=None, tol=None, restart=None, maxit=None, inner_tol=None, stream=None,
              inner_solver=None, precond=None):
        f = f.to(device="cuda", dtype=torch.float64).contiguous()
        use_guess = u is not None
        u = self.empty() if u is None else u
        o = self.opts
        opts = B.make_opts(prec if prec is not None else o.prec, tol or o.tol, restart or o.restart,
                           maxit or o.maxit, inner_tol or o.inner_tol, use_guess, o.q_policy,
                           inner_solver if inner_solver is not None else o.inner_solver,
                           precond if precond is not None else o.precond, o.precond_lmax, o.mode_mix)
        stats = B.rte_solve(self.handle, f.data_ptr(), u.data_ptr(), opts, _stream_ptr(stream))
        return u, stats

    def solve_host(self, f_host, u_host=None, prec=None, tol=None, stream=None):
        """f_host: numpy float64 array; u_host: numpy complex128 (2D) / float64 (3D) output."""
        f_host = np.ascontiguousarray(f_host, dtype=np.float64)
        if u_host is None:
            u_host = np.zeros(self.shape(), dtype=np.complex128 if self.dim == 2 else np.float64)
        o = self.opts
        opts = B.make_opts(prec if prec is not None else o.prec, tol or o.tol, o.restart, o.maxit, o.inner_tol, 0,
                           o.q_policy, o.inner_solver, o.precond, o.precond_lmax, o.mode_mix)
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


class Batch:
    """Many independent 2D instances solved by one graph launch.

    instances: list of dicts (n, h, mu_t, mu_s, sigma_hat[, q, rows_per_block]).
    """

    def __init__(self, instances, prec="mixed_fp32", tol=1e-8, restart=30, maxit=2000, inner_tol=1e-4, stream=None,
                 tune=False, inner_solver="gmres", precond=0, precond_lmax=0):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.instances = [dict(d) for d in instances]
        if tune:
            shapes = [(int(d["n"]), len(d["sigma_hat"]) - 1) for d in self.instances]
            best = autotune(shapes, prec if prec != "fp64" else "mixed_fp32")
            for d in self.instances:
                t = best[(int(d["n"]), len(d["sigma_hat"]) - 1)]
                d["q"], d["rows_per_block"] = t["q"], t["rows_per_block"]
        self.count = len(self.instances)
        self.opts = B.make_opts(prec, tol, restart, maxit, inner_tol, 0, 0, inner_solver, precond, precond_lmax)
        self.handle = B.rte_batch_create(self.instances, self.opts, _stream_ptr(stream))
        self.f_off, self.u_off = B.rte_batch_layout(self.handle, self.count)

    def pack_sources(self, sources):
        f = torch.empty(self.f_off[-1], dtype=torch.float64, device="cuda")
        for i, src in enumerate(sources):
            f[self.f_off[i]:self.f_off[i + 1]] = torch.as_tensor(src, dtype=torch.float64).reshape(-1).to("cuda")
        return f

    def unpack(self, u_packed, i):
        d = self.instances[i]
        L = len(d["sigma_hat"]) - 1
        n = int(d["n"])
        seg = u_packed[self.u_off[i]:self.u_off[i + 1]]
        return torch.view_as_complex(seg.view(L + 1, n, n, 2))

    def solve(self, f_packed, u_packed=None, stream=None):
        if u_packed is None:
            u_packed = torch.zeros(self.u_off[-1], dtype=torch.float64, device="cuda")
        st, stats, ms = B.rte_batch_solve_packed(self.handle, self.count, f_packed.data_ptr(),
                                                 u_packed.data_ptr(), _stream_ptr(stream))
        return u_packed, stats, ms

    def solve_list(self, sources, solutions=None, stream=None):
        """One device tensor per instance: sources[i] (n_i, n_i) float64, the
        solutions complex128 (L_i+1, n_i, n_i) (allocated when None)."""
        fs = [torch.as_tensor(f).to(device="cuda", dtype=torch.float64).contiguous() for f in sources]
        if solutions is None:
            solutions = [torch.zeros((len(d["sigma_hat"]), int(d["n"]), int(d["n"])), dtype=torch.complex128,
                                     device="cuda") for d in self.instances]
        st, stats = B.rte_batch_solve(self.handle, [f.data_ptr() for f in fs], [u.data_ptr() for u in solutions],
                                      _stream_ptr(stream))
        return solutions, stats

    def close(self):
        if getattr(self, "handle", None):
            B.rte_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Inhom:
    """The inhomogeneous-medium isotropic Nystrom matrix K~ in 2D, applied
    directly (see rte_inhom_create): mu_t is an (n, n) array of cell values
    indexed [i2, i1]; fields are (n, n) tensors, float32 (apply32) or float64
    (apply64)."""

    def __init__(self, mu_t, h=None, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        mu_t = np.asarray(mu_t, dtype=np.float64)
        self.n = int(mu_t.shape[0])
        self.h = 1.0 / self.n if h is None else float(h)
        self.handle = B.rte_inhom_create(self.n, self.h, mu_t, _stream_ptr(stream))

    def _field(self, x, dt):
        x = torch.as_tensor(x).to(device="cuda", dtype=dt).contiguous()
        if tuple(x.shape) != (self.n, self.n):
            raise ValueError("field shape must be (%d, %d)" % (self.n, self.n))
        return x

    def apply32(self, x, stream=None):
        x = self._field(x, torch.float32)
        y = torch.empty_like(x)
        B.rte_inhom_apply32(self.handle, x.data_ptr(), y.data_ptr(), _stream_ptr(stream))
        return y

    def apply64(self, x, stream=None):
        x = self._field(x, torch.float64)
        y = torch.empty_like(x)
        B.rte_inhom_apply64(self.handle, x.data_ptr(), y.data_ptr(), _stream_ptr(stream))
        return y

    def diag(self):
        return np.array(B.rte_inhom_diag(self.handle, self.n * self.n)).reshape(self.n, self.n)

    def close(self):
        if self.handle:
            B.rte_inhom_destroy(self.handle)
            self.handle = None


class Aniso3D:
    """3D anisotropic scattering in real spherical harmonics (see
    rte_aniso3d_create): M = (L+1)^2 moment channels, fields (M, n, n, n)
    float64 tensors (float32 for apply_K32), the source (n, n, n)."""

    def __init__(self, n, mu_t, mu_s, sigma_hat, h=None, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.n = int(n)
        self.h = 1.0 / self.n if h is None else float(h)
        self.L = len(sigma_hat) - 1
        self.handle = B.rte_aniso3d_create(self.n, self.h, mu_t, mu_s, self.L, sigma_hat, _stream_ptr(stream))
        self.M, self.Q = B.rte_aniso3d_info(self.handle)

    def _field(self, x, dt, chans):
        x = torch.as_tensor(x).to(device="cuda", dtype=dt).contiguous()
        want = ((chans,) if chans else ()) + (self.n,) * 3
        if tuple(x.shape) != want:
            raise ValueError("field shape must be %s" % (want,))
        return x

    def apply_K(self, x, stream=None):
        x = self._field(x, torch.float64, self.M)
        y = torch.empty_like(x)
        B.rte_aniso3d_apply_K(self.handle, x.data_ptr(), y.data_ptr(), _stream_ptr(stream))
        return y

    def apply_K64e(self, x, stream=None):
        """K x to FP64 accuracy in float-float arithmetic (the residual's form)."""
        x = self._field(x, torch.float64, self.M)
        y = torch.empty_like(x)
        B.rte_aniso3d_apply_K64e(self.handle, x.data_ptr(), y.data_ptr(), _stream_ptr(stream))
        return y

    def apply_K32(self, x, stream=None):
        x = self._field(x, torch.float32, self.M)
        y = torch.empty_like(x)
        B.rte_aniso3d_apply_K32(self.handle, x.data_ptr(), y.data_ptr(), _stream_ptr(stream))
        return y

    def rhs(self, f, stream=None):
        f = self._field(f, torch.float64, 0)
        b = torch.empty((self.M,) + (self.n,) * 3, dtype=torch.float64, device="cuda")
        B.rte_aniso3d_rhs(self.handle, f.data_ptr(), b.data_ptr(), _stream_ptr(stream))
        return b

    def solve(self, f, tol=1e-10, restart=40, maxit=400, prec="fp64", stream=None):
        """prec: "fp64" or "mixed_fp32" (FP32 inner GMRES, FP64-accurate
        residuals); the device solve graph of rte_solve on this operator."""
        f = self._field(f, torch.float64, 0)
        u = torch.empty((self.M,) + (self.n,) * 3, dtype=torch.float64, device="cuda")
        stats = B.rte_aniso3d_solve(self.handle, f.data_ptr(), u.data_ptr(), tol, restart, maxit, prec,
                                    _stream_ptr(stream))
        return u, stats

    def cell_weights(self):
        return np.array(B.rte_aniso3d_cell_weights(self.handle, self.M)).reshape(self.M, self.M)

    def close(self):
        if self.handle:
            B.rte_aniso3d_destroy(self.handle)
            self.handle = None

