"""Exact and closed-form Ising results that pin the oracle from outside.

Independent of the HOTRG code: brute-force enumeration, transfer matrices,
Onsager's 2D free energy and the high-temperature series.  The lattice is the
one the tensor network builds: every site i has, for each direction k, one
bond to i + e_k mod L_k, so L_k = 1 gives a self bond and L_k = 2 a double
bond.  H = -sum_bonds s s' - h sum_i s, Z = sum exp(-beta H).
"""

from __future__ import annotations

import itertools
import math

import numpy as np
from scipy import integrate


def brute_force_ln_z(shape: tuple, beta: float, h: float) -> float:
    """ln Z of the periodic lattice `shape` by summing over all 2^N states."""
    n = int(np.prod(shape))
    if n > 24:
        raise ValueError("lattice too large for brute force")
    states = np.array(list(itertools.product([1.0, -1.0], repeat=n))).reshape((-1,) + tuple(shape))
    energy = np.zeros(states.shape[0])
    for k in range(len(shape)):
        energy += (states * np.roll(states, -1, axis=1 + k)).reshape(states.shape[0], -1).sum(1)
    mag = states.reshape(states.shape[0], -1).sum(1)
    expo = beta * energy + beta * h * mag
    top = expo.max()
    return float(top + math.log(np.exp(expo - top).sum()))


def _row_states(n: int) -> np.ndarray:
    return np.array(list(itertools.product([1.0, -1.0], repeat=n)))


def transfer_matrix_ln_z_2d(lx: int, ly: int, beta: float, h: float) -> float:
    """ln Z = ln Tr(T_row^ly), T_row over a periodic row of lx spins."""
    s = _row_states(lx)
    e_row = (s * np.roll(s, -1, axis=1)).sum(1)
    m = s.sum(1)
    inter = s @ s.T
    log_t = 0.5 * beta * (e_row[:, None] + e_row[None, :]) + beta * inter \
        + 0.5 * beta * h * (m[:, None] + m[None, :])
    t = np.exp(log_t)
    ev = np.linalg.eigvals(t)
    return float(math.log(np.real((ev ** ly).sum())))


def transfer_matrix_ln_z_3d(lx: int, ly: int, lz: int, beta: float, h: float) -> float:
    """ln Z = ln Tr(T_layer^lz), T_layer over a periodic lx x ly layer."""
    s = _row_states(lx * ly).reshape(-1, lx, ly)
    e_layer = (s * np.roll(s, -1, axis=1)).sum((1, 2)) + (s * np.roll(s, -1, axis=2)).sum((1, 2))
    m = s.sum((1, 2))
    flat = s.reshape(s.shape[0], -1)
    inter = flat @ flat.T
    log_t = 0.5 * beta * (e_layer[:, None] + e_layer[None, :]) + beta * inter \
        + 0.5 * beta * h * (m[:, None] + m[None, :])
    t = np.exp(log_t)
    ev = np.linalg.eigvals(t)
    return float(math.log(np.real((ev ** lz).sum())))


def onsager_ln_z_per_site(beta: float) -> float:
    """Onsager: ln Z/N = ln(2 cosh 2b) + (1/2pi) int_0^pi ln[(1 + sqrt(1 - k^2 sin^2 t))/2] dt,
    k = 2 sinh 2b / cosh^2 2b (infinite square lattice, J = 1, h = 0)."""
    k = 2.0 * math.sinh(2 * beta) / math.cosh(2 * beta) ** 2

    def f(t):
        return math.log(0.5 * (1.0 + math.sqrt(max(0.0, 1.0 - k * k * math.sin(t) ** 2))))

    val, _ = integrate.quad(f, 0.0, math.pi, limit=400, epsabs=1e-15, epsrel=1e-14,
                            points=[math.pi / 2])
    return math.log(2.0 * math.cosh(2 * beta)) + val / (2.0 * math.pi)


def onsager_double_integral(beta: float, n: int = 512) -> float:
    """ln 2 + (1/8pi^2) int int ln[cosh^2 2b - sinh 2b (cos t1 + cos t2)] by the periodic
    trapezoid rule (spectrally accurate away from the critical point)."""
    t = 2.0 * math.pi * np.arange(n) / n
    c1, c2 = np.meshgrid(np.cos(t), np.cos(t))
    integrand = np.log(math.cosh(2 * beta) ** 2 - math.sinh(2 * beta) * (c1 + c2))
    return math.log(2.0) + 0.5 * integrand.mean()


def high_t_series(d: int, beta: float) -> float:
    """ln Z/N = ln 2 + d ln cosh b + (d(d-1)/2) tanh^4 b + O(tanh^6 b)."""
    t = math.tanh(beta)
    return math.log(2.0) + d * math.log(math.cosh(beta)) + 0.5 * d * (d - 1) * t ** 4


def lattice_after(d: int, axes) -> tuple:
    """Periodic lattice extents after coarse-graining along `axes` (each doubles L)."""
    ext = [1] * d
    for a in axes:
        ext[a] *= 2
    return tuple(ext)


def brute_force_energy(shape: tuple, beta: float, h: float) -> float:
    """u = -d(ln Z / N)/d beta = <H> / N of the periodic lattice `shape`, by enumeration."""
    n = int(np.prod(shape))
    if n > 24:
        raise ValueError("lattice too large for brute force")
    states = np.array(list(itertools.product([1.0, -1.0], repeat=n))).reshape((-1,) + tuple(shape))
    bonds = np.zeros(states.shape[0])
    for k in range(len(shape)):
        bonds += (states * np.roll(states, -1, axis=1 + k)).reshape(states.shape[0], -1).sum(1)
    mag = states.reshape(states.shape[0], -1).sum(1)
    expo = beta * bonds + beta * h * mag
    w = np.exp(expo - expo.max())
    return float(-(w * (bonds + h * mag)).sum() / w.sum() / n)


def onsager_energy_per_site(beta: float) -> float:
    """Onsager: u = -coth(2b) [1 + (2/pi) (2 tanh^2 2b - 1) K(k)], k = 2 sinh 2b / cosh^2 2b,
    K the complete elliptic integral of the first kind (infinite square lattice, h = 0)."""
    from scipy import special

    k = 2.0 * math.sinh(2 * beta) / math.cosh(2 * beta) ** 2
    kk = special.ellipk(k * k)
    return -(1.0 / math.tanh(2 * beta)) * (1.0 + (2.0 / math.pi) * (2.0 * math.tanh(2 * beta) ** 2 - 1.0) * kk)


def brute_force_specific_heat(shape: tuple, beta: float, h: float) -> float:
    """c = beta^2 d^2(ln Z / N)/d beta^2 = beta^2 (<H^2> - <H>^2) / N by enumeration."""
    n = int(np.prod(shape))
    if n > 24:
        raise ValueError("lattice too large for brute force")
    states = np.array(list(itertools.product([1.0, -1.0], repeat=n))).reshape((-1,) + tuple(shape))
    bonds = np.zeros(states.shape[0])
    for k in range(len(shape)):
        bonds += (states * np.roll(states, -1, axis=1 + k)).reshape(states.shape[0], -1).sum(1)
    mag = states.reshape(states.shape[0], -1).sum(1)
    energy = -(bonds + h * mag)
    expo = -beta * energy
    w = np.exp(expo - expo.max())
    w /= w.sum()
    mean = (w * energy).sum()
    return float(beta * beta * ((w * (energy - mean) ** 2).sum()) / n)
