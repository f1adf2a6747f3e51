"""Pins of the seeded input generators (not of the solver)."""
import numpy as np
import pytest
from scipy.special import iv

from wl_inputs import metropolis_u1, cgauss, rhs_batch, WORKLOADS


@pytest.mark.parametrize("beta", [3.0, 6.0])
def test_metropolis_plaquette_expectation(beta):
    """Eq. 2.3 in two dimensions factorises over plaquettes, so in infinite
    volume <cos P> = I_1(beta) / I_0(beta) (modified Bessel functions)."""
    N = 64
    U = metropolis_u1(N, beta, 300, 42)
    th = np.angle(U)
    P = th[0] + np.roll(th[1], -1, axis=1) - np.roll(th[0], -1, axis=0) - th[1]
    exact = iv(1, beta) / iv(0, beta)
    sd = np.sqrt((1 - np.cos(P) ** 2).mean() / P.size)
    assert abs(np.cos(P).mean() - exact) <= 6 * sd + 2.0 / P.size
    assert np.allclose(np.abs(U), 1.0, atol=1e-15)


def test_gaussian_moments():
    """Complex Gaussian: Re and Im independent N(0, 1)."""
    g = cgauss(9, 1, 200000)
    assert abs(g.real.mean()) < 0.01 and abs(g.imag.mean()) < 0.01
    assert abs(g.real.var() - 1) < 0.02 and abs(g.imag.var() - 1) < 0.02
    assert abs(np.mean(g.real * g.imag)) < 0.01


def test_determinism_and_shapes():
    a = rhs_batch(16, 3, 5)
    b = rhs_batch(16, 3, 5)
    assert a.shape == (3, 16, 16, 2) and np.array_equal(a, b)
    assert not np.array_equal(a[0], a[1])
    assert np.array_equal(rhs_batch(16, 2, 5, first=1)[0], a[1])
    assert set(WORKLOADS) >= {"C1", "C2", "C3", "C4"}
