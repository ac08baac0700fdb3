"""CPU checks of the boundary: the library builds, loads and exports every
function that include/rte.h declares (no compute calls: no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(rte_\w+)\s*\(", text))
    return names


# the core calls of the boundary (plan, operators, solve, batch, learned guess)
BOUNDARY = ("rte_plan_create", "rte_apply_K", "rte_apply_A", "rte_rhs", "rte_solve", "rte_destroy", "rte_status_str",
            "rte_batch_create", "rte_batch_solve", "rte_guess_load", "rte_guess_apply")


def test_header_declares_the_boundary_calls():
    names = _declared()
    for must in BOUNDARY:
        assert must in names


def test_boundary_calls_are_exported():
    from paper_1802_03061_gb300 import build
    lib = ctypes.CDLL(build.build())
    assert all(hasattr(lib, n) for n in BOUNDARY)


def test_guess_load_rejects_a_missing_or_foreign_file_without_a_gpu(tmp_path):
    """rte_guess_load reads and checks the file header before any device call."""
    from paper_1802_03061_gb300 import _binding as B
    with pytest.raises(B.RteError) as ei:
        B.rte_guess_load(str(tmp_path / "missing.bin"))
    assert ei.value.status == B.RTE_EINVAL
    bad = tmp_path / "foreign.bin"
    bad.write_bytes(b"NOTAWEIGHTSFILE!" * 4)
    with pytest.raises(B.RteError) as ei:
        B.rte_guess_load(str(bad))
    assert ei.value.status == B.RTE_EINVAL


def test_library_loads_and_exports_all_symbols():
    from paper_1802_03061_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    from paper_1802_03061_gb300 import _binding as B
    assert B.rte_status_str(B.RTE_EINVAL) == "invalid argument"
    assert B.rte_status_str(B.RTE_ENOCONV).startswith("solver")


def test_binding_refuses_missing_library(tmp_path, monkeypatch):
    from paper_1802_03061_gb300 import _binding as B
    monkeypatch.setattr(B, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(B, "_lib", None)
    with pytest.raises(RuntimeError):
        B.lib()


@pytest.mark.parametrize("args", [
    dict(n=8, mu_t=1.0, mu_s=2.0, L=0, sig=[1.0]),          # mu_s > mu_t (C2)
    dict(n=8, mu_t=1.0, mu_s=0.5, L=1, sig=[0.9, 0.1]),     # sigma_hat_0 != 1
    dict(n=8, mu_t=1.0, mu_s=0.5, L=1, sig=[1.0, 1.5]),     # |sigma_hat_k| > 1
    dict(n=0, mu_t=1.0, mu_s=0.5, L=0, sig=[1.0]),          # empty grid
    dict(n=8, mu_t=-1.0, mu_s=0.0, L=0, sig=[1.0]),         # negative mu_t
    dict(n=8, mu_t=1.0, mu_s=0.5, L=65, sig=[1.0] * 66),    # L beyond the supported 64
])
def test_plan_create_rejects_invalid_arguments_before_any_device_call(args):
    from paper_1802_03061_gb300 import _binding as B
    with pytest.raises(B.RteError) as ei:
        B.rte_plan_create(2, args["n"], 0.125, args["mu_t"], args["mu_s"], args["L"], args["sig"])
    assert ei.value.status == B.RTE_EINVAL


@pytest.mark.parametrize("L,mix", [(9, "direct"), (3, 3), (2, -1)])
def test_plan_create_rejects_bad_mode_mix_before_any_device_call(L, mix):
    """The direct (2L+1)^2 mix runs to L = 8; larger L need the mode-axis FFT."""
    from paper_1802_03061_gb300 import _binding as B
    opts = B.make_opts("mixed_fp32", mode_mix=mix)
    with pytest.raises(B.RteError) as ei:
        B.rte_plan_create(2, 8, 0.125, 1.0, 0.5, L, [1.0] + [0.5] * L, opts)
    assert ei.value.status == B.RTE_EINVAL


def test_plan_create_3d_anisotropic_unsupported():
    from paper_1802_03061_gb300 import _binding as B
    with pytest.raises(B.RteError) as ei:
        B.rte_plan_create(3, 8, 0.125, 1.0, 0.5, 1, [1.0, 0.5])
    assert ei.value.status == B.RTE_EUNSUPPORTED


@pytest.mark.parametrize("args,status", [
    (dict(n=8, mu_t=1.0, mu_s=2.0, L=1, sig=[1.0, 0.5]), "RTE_EINVAL"),        # mu_s > mu_t
    (dict(n=8, mu_t=1.0, mu_s=0.5, L=1, sig=[0.9, 0.5]), "RTE_EINVAL"),        # sigma_hat_0 != 1
    (dict(n=8, mu_t=1.0, mu_s=0.5, L=2, sig=[1.0, 0.5, -1.2]), "RTE_EINVAL"),  # |sigma_hat_l| > 1
    (dict(n=0, mu_t=1.0, mu_s=0.5, L=0, sig=[1.0]), "RTE_EINVAL"),             # empty grid
    (dict(n=8, mu_t=1.0, mu_s=0.5, L=5, sig=[1.0] * 6), "RTE_EINVAL"),         # degree beyond 4
    (dict(n=600, mu_t=1.0, mu_s=0.5, L=4, sig=[1.0] * 5), "RTE_EUNSUPPORTED"),  # 25 channels x Q = 1296
])
def test_aniso3d_create_rejects_before_any_device_call(args, status):
    """The spherical-harmonic operator checks its arguments and its shared
    memory limit (all M channels of one z line in one block) on the host."""
    from paper_1802_03061_gb300 import _binding as B
    with pytest.raises(B.RteError) as ei:
        B.rte_aniso3d_create(args["n"], 1.0 / max(args["n"], 1), args["mu_t"], args["mu_s"], args["L"], args["sig"])
    assert ei.value.status == getattr(B, status)


def test_aniso3d_null_handles_without_gpu():
    from paper_1802_03061_gb300 import _binding as B
    L = B.lib()
    assert L.rte_aniso3d_destroy(None) == B.RTE_OK
    assert L.rte_aniso3d_apply_K(None, None, None, None) == B.RTE_EINVAL
    assert L.rte_aniso3d_info(None, None, None) == B.RTE_EINVAL


@pytest.mark.parametrize("L", [0, 1, 2, 4])
def test_aniso3d_pair_table_matches_harmonic_parities(L):
    """The host table the spectra are stored by (rte_aniso3d_pair_table, no
    device call): symmetric, one index per unordered pair, and the flags equal
    the parities of Y_a Y_b measured from the oracle's harmonics at mirrored
    directions (imaginary spectrum iff W_ab is odd under v -> -v)."""
    import numpy as np
    from oracle import aniso3d as A
    from paper_1802_03061_gb300 import _binding as B
    M = A.n_channels(L)
    t = np.array(B.rte_aniso3d_pair_table(L)).reshape(M, M)
    assert (t == t.T).all()
    iu = np.triu_indices(M)
    idx = t[iu] & 0xFFFF
    assert sorted(idx.tolist()) == list(range(M * (M + 1) // 2))
    v = np.array([[0.31, -0.52, 0.79]])
    v /= np.linalg.norm(v)
    Y = A.real_sh(L, v)[0]
    par = []
    for k in range(3):
        m = v.copy()
        m[:, k] *= -1
        par.append(np.sign(np.round(A.real_sh(L, m)[0] / Y, 9)).astype(int))
    px, py, pz = (np.outer(p, p) for p in par)
    np.testing.assert_array_equal((t >> 16) & 1, (px * py * pz < 0).astype(int))
    np.testing.assert_array_equal((t >> 17) & 1, (py < 0).astype(int))
    np.testing.assert_array_equal((t >> 18) & 1, (pz < 0).astype(int))


def test_aniso3d_octant_storage_rebuilds_the_spectra():
    """Each pair's spectrum is stored as the real octant xi in [0, Q/2]^3 of its
    real or imaginary part; the pair table's flags (imaginary, odd in y, odd in
    z) must rebuild the half spectrum xi_x in [0, Q/2], all xi_y, xi_z of the
    sampled kernel h^3 e^{-mu r}/(4 pi r^2) 4 pi Y_a Y_b exactly (numpy FFT of
    the oracle's harmonics; no device call)."""
    import math

    import numpy as np
    from oracle import aniso3d as A
    from paper_1802_03061_gb300 import _binding as B
    L, n, Q, h, mu = 2, 5, 12, 0.2, 3.0
    M, H = A.n_channels(L), Q // 2 + 1
    t = np.array(B.rte_aniso3d_pair_table(L)).reshape(M, M)
    o = np.arange(Q)
    s = np.where(o < Q // 2, o, o - Q)
    SZ, SY, SX = np.meshgrid(s, s, s, indexing="ij")
    d = np.sqrt(SX ** 2 + SY ** 2 + SZ ** 2).astype(float)
    valid = (abs(SX) < n) & (abs(SY) < n) & (abs(SZ) < n) & (d > 0)
    ds = np.where(d > 0, d, 1.0)
    v = np.stack([SX / ds, SY / ds, SZ / ds], -1)
    Y = A.real_sh(L, v)
    kap = np.where(valid, h ** 3 * np.exp(-mu * h * ds) / (4 * math.pi * (h * ds) ** 2), 0.0)
    ky = np.arange(Q)[:, None]
    kz = np.arange(Q)[None, :]
    fy, fz = np.minimum(ky, Q - ky), np.minimum(kz, Q - kz)
    for a in range(M):
        for b in range(a, M):
            g = 4 * math.pi * kap * Y[..., a] * Y[..., b]  # [oz, oy, ox]
            G = np.fft.fftn(g).transpose(2, 1, 0)          # [kx, ky, kz]
            info = t[a, b]
            imag, oy, oz = (info >> 16) & 1, (info >> 17) & 1, (info >> 18) & 1
            part = G.imag if imag else G.real
            np.testing.assert_allclose(G.real if imag else G.imag, 0, atol=1e-13 * np.abs(G).max())
            oct_ = part[:H, :H, :H]
            sgn = np.where((ky > Q // 2) & bool(oy), -1.0, 1.0) * np.where((kz > Q // 2) & bool(oz), -1.0, 1.0)
            rebuilt = sgn[None] * oct_[:, fy, fz]
            np.testing.assert_allclose(rebuilt, part[:H], atol=1e-13 * np.abs(G).max())


def test_training_checkpoint_calls_reject_null_arguments_without_a_gpu(tmp_path):
    """rte_cnn_save_state / rte_cnn_load_state check their handle and path
    before any device call."""
    from paper_1802_03061_gb300 import _binding as B
    for fn, args in ((B.rte_cnn_save_state, (None, tmp_path / "c.bin")),
                     (B.rte_cnn_load_state, (None, tmp_path / "c.bin"))):
        with pytest.raises(B.RteError) as ei:
            fn(*args)
        assert ei.value.status == B.RTE_EINVAL
