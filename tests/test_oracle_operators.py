"""Pins of the oracle's operators against facts the paper and the mathematics
fix (Sec. 2, Eqs. 2.1-2.2; Sec. 3.2, Eqs. 3.2-3.3), independent of the
oracle's own code paths."""
import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

from wl_inputs import metropolis_u1, unit_gauge, random_gauge_transform, cgauss


def _rand_gauge(N, seed):
    th = 2 * np.pi * np.random.default_rng(seed).random((2, N, N))
    return np.exp(1j * th)


def _g5(n_sites):
    return np.diag(np.tile([1.0, -1.0], n_sites)).astype(complex)


def _match(a, b):
    r, c = linear_sum_assignment(np.abs(a[:, None] - b[None, :]))
    return np.abs(a[r] - b[c]).max()


@pytest.mark.parametrize("N,kind", [(4, "rand"), (8, "rand"), (8, "metro"), (16, "metro")])
def test_gamma5_hermiticity(O, N, kind):
    """Sec. 2.2: Gamma5 D = D^H Gamma5; Eq. 3.3: Dhat^H Gamma_e = Gamma_e Dhat."""
    U = _rand_gauge(N, 1) if kind == "rand" else metropolis_u1(N, 3.0, 30, 3)
    m = -0.07
    D = O.wilson_csr(N, U, m).toarray()
    G = _g5(N * N)
    assert np.abs(G @ D - D.conj().T @ G).max() <= 1e-14 * np.abs(D).max()
    Dh = O.dhat_csr(N, U, m).toarray()
    Ge = _g5(N * N // 2)
    assert np.abs(Ge @ Dh - Dh.conj().T @ Ge).max() <= 1e-14 * np.abs(Dh).max()


@pytest.mark.parametrize("N,kind", [(4, "rand"), (8, "metro")])
def test_z_is_hermitian(O, N, kind):
    """Thm. 3.1: Z = Gamma5 D is Hermitian (a consequence of the
    gamma5-hermiticity of D).  Z is assembled column by column from z_apply,
    so a wrong spin sign or layout in z_apply breaks the symmetry."""
    U = _rand_gauge(N, 2) if kind == "rand" else metropolis_u1(N, 3.0, 30, 5)
    m = 0.11
    n = 2 * N * N
    Z = np.empty((n, n), complex)
    for j in range(n):
        e = np.zeros(n, complex)
        e[j] = 1.0
        Z[:, j] = O.z_apply(N, U, m, e.reshape(N, N, 2)).reshape(-1)
    assert np.abs(Z - Z.conj().T).max() <= 1e-14 * np.abs(Z).max()
    assert np.abs(np.diag(Z)[1::2] + (m + 2)).max() <= 1e-14  # Gamma5 flips the spin-1 diagonal


def test_block_form(O):
    """Eq. 2.2: in spin-permuted order D = 1/2 [[A, B], [-B^H, A]] with the
    gauge Laplacian A and the gauge gradient B of Sec. 2.  Readings: the
    paper's A and B carry conj(U^z) on the forward neighbour while Eq. 2.1
    carries U^z, so the oracle's D is built from conj(U); and the Pauli
    sigma_2 = -gamma_2 flips the sign of the y part of B."""
    N, m = 8, 0.13
    U = _rand_gauge(N, 4)
    D = O.wilson_csr(N, np.conj(U), m).toarray()
    n = N * N
    perm = np.concatenate([np.arange(0, 2 * n, 2), np.arange(1, 2 * n, 2)])
    Dp = D[np.ix_(perm, perm)]
    A = np.zeros((n, n), complex)
    B = np.zeros((n, n), complex)
    z = lambda x, y: (y % N) * N + (x % N)  # noqa: E731
    for y in range(N):
        for x in range(N):
            i = z(x, y)
            sy_f = -1.0 if y == N - 1 else 1.0   # antiperiodic y
            sy_b = -1.0 if y == 0 else 1.0
            A[i, i] += 4 + 2 * m
            A[i, z(x - 1, y)] -= U[0, y, (x - 1) % N]
            A[i, z(x, y - 1)] -= U[1, (y - 1) % N, x] * sy_b
            A[i, z(x + 1, y)] -= np.conj(U[0, y, x])
            A[i, z(x, y + 1)] -= np.conj(U[1, y, x]) * sy_f
            B[i, z(x + 1, y)] += np.conj(U[0, y, x])
            B[i, z(x - 1, y)] -= U[0, y, (x - 1) % N]
            B[i, z(x, y + 1)] -= 1j * np.conj(U[1, y, x]) * sy_f   # sigma_2 = -gamma_2
            B[i, z(x, y - 1)] += 1j * U[1, (y - 1) % N, x] * sy_b
    ref = 0.5 * np.block([[A, B], [-B.conj().T, A]])
    assert np.abs(Dp - ref).max() <= 1e-14


@pytest.mark.parametrize("N", [4, 8, 16])
def test_free_field_spectrum(O, N):
    """U = 1 (Sec. 2: A is the 5-point Laplacian, B a central difference).
    Plane waves with p1 = 2 pi k / N, p2 = (2k+1) pi / N (antiperiodic) give
    lambda = m + sum_mu (1 - cos p_mu) +- i sqrt(sum_mu sin^2 p_mu); the
    even-site Schur complement has eigenvalues 1 - (1 - lambda/c)^2."""
    m = 0.21
    U = unit_gauge(N)
    ks = []
    for k1 in range(N):
        for k2 in range(N):
            p1, p2 = 2 * np.pi * k1 / N, (2 * k2 + 1) * np.pi / N
            re = m + (1 - np.cos(p1)) + (1 - np.cos(p2))
            im = np.sqrt(np.sin(p1) ** 2 + np.sin(p2) ** 2)
            ks += [re + 1j * im, re - 1j * im]
    ks = np.array(ks)
    ev = np.linalg.eigvals(O.wilson_csr(N, U, m).toarray())
    assert _match(ev, ks) <= 1e-12
    c = m + 2
    evh = np.linalg.eigvals(O.dhat_csr(N, U, m).toarray())
    pred = 1 - (1 - ks / c) ** 2
    # every Dhat eigenvalue is predicted, and each prediction occurs (twice)
    assert np.abs(evh[:, None] - pred[None, :]).min(axis=1).max() <= 1e-12
    assert np.abs(pred[:, None] - evh[None, :]).min(axis=1).max() <= 1e-12


def test_gauge_covariance(O):
    """U_mu(z) -> g(z) U_mu(z) conj(g(z+mu)) and psi -> g psi give
    D' = G D G^H exactly."""
    N, m = 8, -0.05
    U = metropolis_u1(N, 6.0, 20, 9)
    Up, g = random_gauge_transform(U, 17)
    D = O.wilson_csr(N, U, m).toarray()
    Dp = O.wilson_csr(N, Up, m).toarray()
    G = np.diag(np.repeat(g.reshape(-1), 2))
    assert np.abs(Dp - G @ D @ G.conj().T).max() <= 1e-14


@pytest.mark.parametrize("N", [4, 8])
def test_schur_solve_equals_full_solve(O, N):
    """Sec. 3.2: two-step solve with Dhat equals the full dense solve."""
    U = _rand_gauge(N, 5)
    m = 0.3
    D = O.wilson_csr(N, U, m).toarray()
    b = cgauss(3, 0, 2 * N * N).reshape(N, N, 2)
    psi = np.linalg.solve(D, b.reshape(-1)).reshape(N, N, 2)
    bh = O.eo_reduce(N, U, m, b)
    Dh = O.dhat_csr(N, U, m).toarray()
    xe = np.linalg.solve(Dh, bh)
    psi2 = O.eo_reconstruct(N, U, m, b, xe)
    assert np.abs(psi2 - psi).max() <= 1e-12 * np.abs(psi).max()
    # the oracle's own dense LU (textbook partial pivoting) agrees too
    xe2 = O.dense_lu_solve(Dh, bh)
    assert np.abs(xe2 - xe).max() <= 1e-12 * np.abs(xe).max()


def test_dhat_product_vs_successive(O):
    """Dhat formed as a sparse product equals x - (D_eo/c)((D_oe/c) x)."""
    N, m = 16, -0.02
    U = metropolis_u1(N, 3.0, 20, 2)
    x = cgauss(1, 1, N * N)
    assert np.abs(O.dhat_apply(N, U, m, x) - O.dhat_csr(N, U, m) @ x).max() <= 1e-14 * np.abs(x).max()


def test_dhat_stencil_structure(O):
    """Sec. 3.2 / Fig. 3.1 (b): Dhat couples an even site to itself and the
    eight even sites (+-1, +-1), (+-2, 0), (0, +-2); the diagonal block is I
    (the two hops out and back through one odd site cancel: (1-s)(1+s) = 0)."""
    N, m = 16, 0.1
    U = _rand_gauge(N, 8)
    Dh = O.dhat_csr(N, U, m)
    n = N * N // 2
    for h in range(n):
        y, x = h // (N // 2), 2 * (h % (N // 2)) + ((h // (N // 2)) & 1)
        allowed = {((x + dx) % N, (y + dy) % N) for dx, dy in
                   [(0, 0), (1, 1), (-1, -1), (1, -1), (-1, 1), (2, 0), (-2, 0), (0, 2), (0, -2)]}
        cols = set()
        for s in range(2):
            row = Dh.getrow(2 * h + s)
            for j, v in zip(row.indices, row.data):
                if abs(v) > 0:
                    hj = j // 2
                    yj = hj // (N // 2)
                    xj = 2 * (hj % (N // 2)) + (yj & 1)
                    cols.add((xj, yj))
            # centre block is the identity
            d = Dh[2 * h + s, 2 * h:2 * h + 2].toarray().ravel()
            assert np.abs(d - np.eye(2)[s]).max() <= 1e-15
        assert cols <= allowed and len(cols) == 9
    # the oracle's stencil neighbour map enumerates exactly these offsets
    for h in range(0, n, 7):
        nb = {O.neighbour(N, h, d) for d in range(9)}
        assert len(nb) == 9 and h in nb


def test_colour_classes_independent(O):
    """Reading of Sec. 3.1: 16 colours (a mod 4, b mod 4); two variables of
    one colour have disjoint column supports (3x3 boxes in (a, b))."""
    for N in (8, 16, 32):
        n = N * N // 2
        supp = [{O.neighbour(N, h, d) for d in range(9)} for h in range(n)]
        col = [O.colour(N, h) for h in range(n)]
        assert sorted(set(col)) == list(range(16))
        assert all(col.count(k) == n // 16 for k in range(16))
        for k in range(16):
            seen = set()
            for h in range(n):
                if col[h] == k:
                    assert not (supp[h] & seen)
                    seen |= supp[h]
