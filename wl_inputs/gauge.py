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
    tx = np.zeros((N, N), dtype=np.float64)   # theta_x[y, x]
    ty = np.zeros((N, N), dtype=np.float64)   # theta_y[y, x]
    idx = np.arange(N * N // 2, dtype=np.uint64)
    two_pi = 2 * np.pi

    def accept(t, b1, b2, sign, sw, cls):
        base = 8 * (4 * sw + cls) + 1024
        dlt = (delta * (2.0 * uniform01(seed, base + 0, idx) - 1.0)).reshape(t.shape)
        acc = uniform01(seed, base + 1, idx).reshape(t.shape)
        tn = t + dlt
        ds = beta * (np.cos(sign * tn + b1) + np.cos(-sign * tn + b2)
                     - np.cos(sign * t + b1) - np.cos(-sign * t + b2))
        ok = acc < np.exp(np.minimum(ds, 0.0))
        return np.remainder(np.where(ok, tn, t) + np.pi, two_pi) - np.pi

    for sw in range(sweeps):
        for p in (0, 1):   # x-links on rows y = p (mod 2)
            Y = np.arange(p, N, 2)
            Yp, Ym = (Y + 1) % N, (Y - 1) % N
            tyY = ty[Y]
            # P(x,y)   = tx(x,y) + ty(x+1,y) - tx(x,y+1) - ty(x,y)
            b1 = np.roll(tyY, -1, axis=1) - tx[Yp] - tyY
            # P(x,y-1) = tx(x,y-1) + ty(x+1,y-1) - tx(x,y) - ty(x,y-1)
            tyM = ty[Ym]
            b2 = tx[Ym] + np.roll(tyM, -1, axis=1) - tyM
            tx[Y] = accept(tx[Y], b1, b2, 1.0, sw, p)
        for p in (0, 1):   # y-links on columns x = p (mod 2)
            X = np.arange(p, N, 2)
            Xp, Xm = (X + 1) % N, (X - 1) % N
            # P(x,y)   = tx(x,y) + ty(x+1,y) - tx(x,y+1) - ty(x,y)   (ty enters with -)
            txX = tx[:, X]
            b1 = txX + ty[:, Xp] - np.roll(txX, -1, axis=0)
            # P(x-1,y) = tx(x-1,y) + ty(x,y) - tx(x-1,y+1) - ty(x-1,y)  (ty enters with +)
            txM = tx[:, Xm]
            b2 = txM - np.roll(txM, -1, axis=0) - ty[:, Xm]
            ty[:, X] = accept(ty[:, X], b1, b2, -1.0, sw, 2 + p)
    return np.exp(1j * np.stack([tx, ty]))


def random_gauge_transform(U: np.ndarray, seed: int):
    """Return (U', g) with U'_mu(z) = g(z) U_mu(z) conj(g(z + mu)), |g| = 1.
    Used only by tests of gauge covariance."""
    N = U.shape[1]
    g = np.exp(2j * np.pi * uniform01(seed, 7, np.arange(N * N, dtype=np.uint64))).reshape(N, N)
    Up = np.empty_like(U)
    Up[0] = g * U[0] * np.conj(np.roll(g, -1, axis=1))
    Up[1] = g * U[1] * np.conj(np.roll(g, -1, axis=0))
    return Up, g
