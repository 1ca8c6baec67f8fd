"""Seeded synthetic inputs shared by the tests, the bench and the oracle legs.

Holds no HOTRG arithmetic: only random numbers with fixed seeds, in the
interchange layout of a local tensor (axes x_1, x_1', ..., x_d, x_d', x_1
slowest), and random symmetric / orthogonal test matrices.
"""

from __future__ import annotations

import numpy as np


def gaussian_tensor(chis, seed: int) -> np.ndarray:
    """N(0, 1) local tensor with bond dims chis[k] on both legs of axis k."""
    rng = np.random.default_rng(seed)
    shape = []
    for c in chis:
        shape += [c, c]
    return rng.standard_normal(shape)


def reflection_symmetric_tensor(chis, seed: int) -> np.ndarray:
    """Gaussian tensor symmetrised under every leg swap x_k <-> x_k' (the
    lattice reflections the Ising tensor has)."""
    t = gaussian_tensor(chis, seed)
    d = len(chis)
    for k in range(d):
        perm = list(range(2 * d))
        perm[2 * k], perm[2 * k + 1] = perm[2 * k + 1], perm[2 * k]
        t = 0.5 * (t + np.transpose(t, perm))
    return t


def random_spd(n: int, seed: int, extra: int = 3) -> np.ndarray:
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, n + extra))
    return g @ g.T


def random_psd_with_spectrum(lam, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    n = len(lam)
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (q * np.asarray(lam, dtype=np.float64)[None, :]) @ q.T
