"""Test helpers: layout conversion between the library's packed mode fields
(modes 0..L) and the oracle's full fields (modes -L..L)."""
import numpy as np


def packed_to_full(u):
    """(L+1, n, n) modes 0..L -> (2L+1, n, n) modes -L..L using u_{-k} = conj(u_k)."""
    u = np.asarray(u)
    L = u.shape[0] - 1
    return np.concatenate([np.conj(u[:0:-1]), u], axis=0) if L > 0 else u.copy()


def random_packed(rng, L, n):
    u = rng.standard_normal((L + 1, n, n)) + 1j * rng.standard_normal((L + 1, n, n))
    u[0] = u[0].real
    return u


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def bf16_round(a):
    """Round to bfloat16 (round to nearest even on the upper 16 bits of FP32)."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rnd = ((u >> 16) & 1) + 0x7FFF
    u = ((u + rnd) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def to_bf16_bits(a):
    """float array -> uint16 bfloat16 bit patterns (round to nearest even)."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rnd = ((u >> 16) & 1) + 0x7FFF
    return ((u + rnd) >> 16).astype(np.uint16)
