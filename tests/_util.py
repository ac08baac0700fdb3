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
