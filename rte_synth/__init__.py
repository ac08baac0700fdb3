"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the method: it only draws problem
parameters and evaluates analytic source functions at cell centres
x_i = ((i1 + 1/2) h, (i2 + 1/2) h [, (i3 + 1/2) h]).  Both the CUDA path and
the oracle receive the arrays it returns.

Workloads (shapes follow the paper's 2D/3D test problems, Sec. 2.4 and 3.4):

* ``iso2d_bump``          -- 64x64, mu_t = 1, mu_s = 0.5, L = 0, one Gaussian
                             bump of standard deviation 0.1 at (0.5, 0.5).
* ``hg2d_transport``      -- 256x256, L = 8, Henyey-Greenstein g = 0.5
                             (sigma_hat_k = g^|k|), mu_t = 10, mu_s = 9, four
                             Gaussians, centres U[0.2,0.8]^2, widths U[0.03,0.1].
* ``iso3d_diffusion``     -- 128^3, mu_t = 100, mu_s = 99.5, one Gaussian of
                             width 0.05, centre U[0.3,0.7]^3.
* ``batch_instances``     -- uneven 2D instances (sides, L, mu_t, mu_s/mu_t, g,
                             1-6 Gaussians) for batched solves.
* ``paper_sources``       -- the paper's f1, f2, f3 (Eq. source).
"""
import math

import numpy as np


def cell_centres(n, dim=2):
    h = 1.0 / n
    c = (np.arange(n) + 0.5) * h
    if dim == 2:
        Y, X = np.meshgrid(c, c, indexing="ij")
        return X, Y
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    return X, Y, Z


def gaussian_mixture_2d(n, centres, widths, amps=None):
    """f(x) = sum_a amp_a exp(-|x - c_a|^2 / (2 s_a^2)) at the n x n cell centres."""
    X, Y = cell_centres(n, 2)
    f = np.zeros((n, n))
    amps = np.ones(len(centres)) if amps is None else amps
    for (cx, cy), s, a in zip(centres, widths, amps):
        f += a * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2.0 * s * s))
    return f


def gaussian_3d(n, centre, width):
    X, Y, Z = cell_centres(n, 3)
    cx, cy, cz = centre
    return np.exp(-((X - cx) ** 2 + (Y - cy) ** 2 + (Z - cz) ** 2) / (2.0 * width * width))


def hg_sigma_hat(g, L):
    """Fourier coefficients of the 2D Henyey-Greenstein phase function,
    sigma(theta) = (1 - g^2) / (1 + g^2 - 2 g cos theta): sigma_hat_k = g^|k|,
    truncated to |k| <= L.  Returned for k = 0..L."""
    return np.array([g ** k for k in range(L + 1)], dtype=np.float64)


def paper_sigma_hat():
    """sigma(theta) = 1 + (e^{i theta} + e^{-i theta})/5 (Eq. sigma): L = 1."""
    return np.array([1.0, 0.2])


def paper_sources(n):
    """f1, f2, f3 of Eq. source at the n x n cell centres."""
    T = 4e-3
    c1, c2, c3 = (0.3, 0.7), (0.7, 0.3), (0.6, 0.4)
    X, Y = cell_centres(n, 2)
    pref = 1.0 / math.sqrt(2 * math.pi * T)
    f1 = (pref * np.exp(-((X - c1[0]) ** 2 + (Y - c1[1]) ** 2) / (2 * T))
          + pref * np.exp(-((X - c2[0]) ** 2 + (Y - c2[1]) ** 2) / (2 * T)))
    d3 = np.sqrt((X - c3[0]) ** 2 + (Y - c3[1]) ** 2)
    f2 = ((d3 >= 3 / 20) & (d3 <= 1 / 4)).astype(np.float64)
    f3 = ((X >= 0.5) & (X <= 0.75) & (Y >= 0.5) & (Y <= 0.75)).astype(np.float64)
    return f1, f2, f3


def iso2d_bump(n=64):
    f = gaussian_mixture_2d(n, [(0.5, 0.5)], [0.1])
    return dict(n=n, h=1.0 / n, mu_t=1.0, mu_s=0.5, sigma_hat=np.array([1.0]), f=f)


def hg2d_transport(n=256, L=8, g=0.5, mu_t=10.0, mu_s=9.0, seed=2, ngauss=4):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.2, 0.8, size=(ngauss, 2))
    widths = rng.uniform(0.03, 0.1, size=ngauss)
    f = gaussian_mixture_2d(n, centres, widths)
    return dict(n=n, h=1.0 / n, mu_t=mu_t, mu_s=mu_s, sigma_hat=hg_sigma_hat(g, L), f=f)


def iso3d_diffusion(n=128, mu_t=100.0, mu_s=99.5, width=0.05, seed=3):
    rng = np.random.default_rng(seed)
    centre = rng.uniform(0.3, 0.7, size=3)
    f = gaussian_3d(n, centre, width)
    return dict(n=n, h=1.0 / n, mu_t=mu_t, mu_s=mu_s, f=f)


def random_instance_2d(rng, n, L, mu_t_range=(1.0, 50.0), ratio_range=(0.5, 0.99),
                       g_range=(0.0, 0.8), ngauss_range=(1, 6)):
    mu_t = float(math.exp(rng.uniform(math.log(mu_t_range[0]), math.log(mu_t_range[1]))))
    mu_s = mu_t * float(rng.uniform(*ratio_range))
    g = float(rng.uniform(*g_range))
    k = int(rng.integers(ngauss_range[0], ngauss_range[1] + 1))
    centres = rng.uniform(0.2, 0.8, size=(k, 2))
    widths = rng.uniform(0.03, 0.1, size=k)
    f = gaussian_mixture_2d(n, centres, widths)
    return dict(n=n, h=1.0 / n, mu_t=mu_t, mu_s=mu_s, g=g, sigma_hat=hg_sigma_hat(g, L), f=f)


def batch_instances(count=512, seed=4, sides=(64, 96, 128, 192, 256, 384, 512), Ls=(0, 2, 4, 8)):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.choice(sides))
        L = int(rng.choice(Ls))
        out.append(random_instance_2d(rng, n, L))
    return out


def learned_guess_instance(seed, n=256, L=4):
    """One problem of the learned-initial-guess workload: HG g in [0, 0.7],
    mu_t log-uniform in [1, 50], mu_s/mu_t in [0.5, 0.99], 1-6 Gaussians."""
    rng = np.random.default_rng(seed)
    return random_instance_2d(rng, n, L, g_range=(0.0, 0.7))


def inhom_mu_t(n, rho=10.0, gap=0.2):
    """Cell-centred mu_t of the inhomogeneous test medium: mu_s(x) = 1 + rho
    exp(-|x - c|^2 / 4), c = (1/2, 1/2), and mu_t = mu_s + gap (the paper's
    choice mu_t = mu_s + 0.2).  Returns (mu_t, mu_s), (n, n) arrays [i2, i1]."""
    xc = (np.arange(n) + 0.5) / n
    r2 = (xc[None, :] - 0.5) ** 2 + (xc[:, None] - 0.5) ** 2
    mu_s = 1.0 + rho * np.exp(-r2 / 4.0)
    return mu_s + gap, mu_s

