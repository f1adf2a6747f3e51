"""Quenched U(1) gauge fields on an N x N torus (Sec. 2, Eq. 2.3).

Layout: U[mu, y, x] complex128, mu = 0 (x) or 1 (y); U_mu(x, y) sits on the
edge from (x, y) to (x, y) + e_mu.  Gauge links are periodic in both
directions (the antiperiodic boundary belongs to the fermion operator).

Metropolis: cold start (all phases 0); a sweep visits the four link classes
(x-links on even rows, x-links on odd rows, y-links on even columns, y-links
on odd columns) in turn; links of one class share no plaquette, so a class is
updated at once.  Proposal theta' = theta + delta, delta ~ U(-1, 1) rad;
accept with probability min(1, exp(beta * (sum cos P' - sum cos P))) over the
two plaquettes that hold the link.  Random numbers come from the counter-based
generator in rng.py (stream = 8 * (4 * sweep + class) + {0: proposal,
1: accept} + 1024).
"""
import numpy as np

from .rng import uniform01


def unit_gauge(N: int) -> np.ndarray:
    return np.ones((2, N, N), dtype=np.complex128)


def metropolis_u1(N: int, beta: float, sweeps: int, seed: int, delta: float = 1.0) -> np.ndarray:
    if N % 2:
        raise ValueError("N must be even")
    th = np.zeros((2, N, N), dtype=np.float64)
    nlinks = N * N // 2
    idx = np.arange(nlinks, dtype=np.uint64)
    sel = [np.zeros((N, N), dtype=bool) for _ in range(4)]
    sel[0][0::2, :] = True   # x-links, even y
    sel[1][1::2, :] = True   # x-links, odd y
    sel[2][:, 0::2] = True   # y-links, even x
    sel[3][:, 1::2] = True   # y-links, odd x
    for sw in range(sweeps):
        for cls in range(4):
            base = 8 * (4 * sw + cls) + 1024
            dlt = delta * (2.0 * uniform01(seed, base + 0, idx) - 1.0)
            acc = uniform01(seed, base + 1, idx)
            tx, ty = th[0], th[1]
            if cls < 2:
                # P(x,y) = tx(x,y) + ty(x+1,y) - tx(x,y+1) - ty(x,y)
                a1 = np.roll(ty, -1, axis=1) - np.roll(tx, -1, axis=0) - ty
                # P(x,y-1) = tx(x,y-1) + ty(x+1,y-1) - tx(x,y) - ty(x,y-1)
                a2 = np.roll(tx, 1, axis=0) + np.roll(np.roll(ty, -1, axis=1), 1, axis=0) - np.roll(ty, 1, axis=0)
                t = tx[sel[cls]]
                b1, b2 = a1[sel[cls]], a2[sel[cls]]
                tn = t + dlt
                ds = beta * (np.cos(tn + b1) + np.cos(-tn + b2) - np.cos(t + b1) - np.cos(-t + b2))
                ok = acc < np.exp(np.minimum(ds, 0.0))
                t = np.where(ok, tn, t)
                tx[sel[cls]] = np.remainder(t + np.pi, 2 * np.pi) - np.pi
            else:
                # P(x,y) = tx(x,y) + ty(x+1,y) - tx(x,y+1) - ty(x,y)
                c1 = tx + np.roll(ty, -1, axis=1) - np.roll(tx, -1, axis=0)
                # P(x-1,y) = tx(x-1,y) + ty(x,y) - tx(x-1,y+1) - ty(x-1,y)
                c2 = np.roll(tx, 1, axis=1) - np.roll(np.roll(tx, 1, axis=1), -1, axis=0) - np.roll(ty, 1, axis=1)
                t = ty[sel[cls]]
                b1, b2 = c1[sel[cls]], c2[sel[cls]]
                tn = t + dlt
                ds = beta * (np.cos(-tn + b1) + np.cos(tn + b2) - np.cos(-t + b1) - np.cos(t + b2))
                ok = acc < np.exp(np.minimum(ds, 0.0))
                t = np.where(ok, tn, t)
                ty[sel[cls]] = np.remainder(t + np.pi, 2 * np.pi) - np.pi
    return np.exp(1j * th)


def random_gauge_transform(U: np.ndarray, seed: int):
    """Return (U', g) with U'_mu(z) = g(z) U_mu(z) conj(g(z + mu)), |g| = 1.
    Used only by tests of gauge covariance."""
    N = U.shape[1]
    g = np.exp(2j * np.pi * uniform01(seed, 7, np.arange(N * N, dtype=np.uint64))).reshape(N, N)
    Up = np.empty_like(U)
    Up[0] = g * U[0] * np.conj(np.roll(g, -1, axis=1))
    Up[1] = g * U[1] * np.conj(np.roll(g, -1, axis=0))
    return Up, g
