"""Pins of the oracle's aggregation coarse space (Sec. 4's unexplored
alternative of more interpolation variables per coarse point, read as
spin-split aggregation over the B x B cells of Sec. 3.2's full coarsening,
with the gamma5-compatible Galerkin coarsening of Sec. 3.5).

Everything the pins compare against is assembled here from definitions:
the cell membership of a site from the rotated coordinates a = (x+y)/2,
b = (x-y)/2, dense P from the per-(aggregate, spin) columns, dense P^H A P,
and the 9-point block stencil turned back into a dense matrix."""
import numpy as np
import pytest

from wl_inputs import metropolis_u1, cgauss


def site_xy(N, h):
    y = h // (N // 2)
    return 2 * (h % (N // 2)) + (y & 1), y


def site_of(N, x, y):
    x, y = x % N, y % N
    return y * (N // 2) + x // 2


def member(N, B, h):
    """(coarse site, member index ia B + ib) of fine site h"""
    x, y = site_xy(N, h)
    a, b = (x + y) // 2, (x - y) // 2
    a0, b0 = B * (a // B), B * (b // B)
    return site_of(N // B, ((a0 + b0) % N) // B, ((a0 - b0) % N) // B), (a - a0) * B + (b - b0)


def dense_P(N, B, k, Q):
    nf, nc = N * N // 2, (N // B) ** 2 // 2
    P = np.zeros((2 * nf, 2 * k * nc), complex)
    for h in range(nf):
        hc, m = member(N, B, h)
        for s in range(2):
            P[2 * h + s, 2 * k * hc + k * s:2 * k * hc + k * s + k] = Q[hc, s, m]
    return P


def dense_stencil(Nc, Ac):
    nc, K2 = Ac.shape[0], Ac.shape[2]
    A = np.zeros((nc * K2, nc * K2), complex)
    for h in range(nc):
        x, y = site_xy(Nc, h)
        for d in range(9):
            da, db = d // 3 - 1, d % 3 - 1
            j = site_of(Nc, x + da + db, y + da - db)
            A[h * K2:(h + 1) * K2, j * K2:(j + 1) * K2] += Ac[h, d]
    return A


@pytest.fixture(scope="module")
def h32(O):
    U = metropolis_u1(32, 6.0, 100, 21)
    return O.Hierarchy.setup(32, U, -0.05, O.setup_params([2], k_r=6, k_e=6, mu1=6, mu2=3, seed=5))


def _vectors(n, k, seed):
    return np.stack([cgauss(seed, j, n) for j in range(k)])


@pytest.mark.parametrize("B,k", [(2, 4), (4, 8)])
def test_interp_is_orthonormal_spin_split_gram_schmidt(O, B, k):
    """Columns of each (aggregate, spin) block are orthonormal, P is block
    diagonal in spin (Gamma5 P = P Gamma5c), and Q^H V of each block is upper
    triangular with a positive diagonal: the columns are the test vectors
    orthonormalised in their given order (modified Gram-Schmidt)."""
    N = 32
    V = _vectors(N * N, k, 71)
    Q = O.agg_interp(N, B, k, V)
    P = dense_P(N, B, k, Q)
    assert np.abs(P.conj().T @ P - np.eye(P.shape[1])).max() <= 1e-13
    g5f = np.tile([1.0, -1.0], P.shape[0] // 2)
    g5c = np.tile(np.repeat([1.0, -1.0], k), P.shape[1] // (2 * k))
    assert np.abs(g5f[:, None] * P - P * g5c[None, :]).max() == 0.0
    nf = N * N // 2
    for hc in (0, 7, Q.shape[0] - 1):
        rows = [h for h in range(nf) if member(N, B, h)[0] == hc]
        assert len(rows) == B * B
        rows.sort(key=lambda h: member(N, B, h)[1])
        for s in range(2):
            Vb = V[:, [2 * h + s for h in rows]].T          # (B*B) x k, test vectors as columns
            R = Q[hc, s].conj().T @ Vb
            assert np.abs(np.tril(R, -1)).max() <= 1e-12 * np.abs(R).max()
            assert np.all(np.abs(np.diag(R).imag) <= 1e-12) and np.all(np.diag(R).real > 0)
            assert np.abs(Q[hc, s] @ R - Vb).max() <= 1e-12 * np.abs(Vb).max()


def test_interp_recovers_a_planted_space(O):
    """Test vectors that lie in the range of a planted block-diagonal P_true
    give the same coarse space: P P^H v = v for every test vector, and the
    projector P P^H equals the orthogonal projector onto range(P_true)."""
    N, B, k = 32, 4, 6
    rng = np.random.default_rng(5)
    nc = (N // B) ** 2 // 2
    Qt = rng.standard_normal((nc, 2, B * B, k)) + 1j * rng.standard_normal((nc, 2, B * B, k))
    Pt = dense_P(N, B, k, Qt)
    C = rng.standard_normal((Pt.shape[1], k)) + 1j * rng.standard_normal((Pt.shape[1], k))
    V = (Pt @ C).T
    P = dense_P(N, B, k, O.agg_interp(N, B, k, V))
    for v in V:
        assert np.abs(P @ (P.conj().T @ v) - v).max() <= 1e-12 * np.abs(v).max()
    proj_t = Pt @ np.linalg.solve(Pt.conj().T @ Pt, Pt.conj().T)
    assert np.abs(P @ P.conj().T - proj_t).max() <= 1e-11


def test_interp_rejects_rank_deficient_blocks(O):
    """Two equal test vectors leave a zero column: refused."""
    V = _vectors(32 * 32, 3, 72)
    V[2] = V[1]
    with pytest.raises(RuntimeError):
        O.agg_interp(32, 4, 3, V)


@pytest.mark.parametrize("B,k", [(2, 4), (4, 8)])
def test_galerkin_block_stencil(O, h32, B, k):
    """Sec. 3.5 with the aggregation P: the block stencil, assembled back into
    a dense matrix, equals the dense product P^H A P; it is Gamma5c-Hermitian;
    each coarse row couples to its 9 stencil neighbours only (by
    construction of the dense assembly, every entry of P^H A P is covered)."""
    N = 32
    A = h32.dense(0)
    V = _vectors(N * N, k, 73)
    Q = O.agg_interp(N, B, k, V)
    P = dense_P(N, B, k, Q)
    Ac = h32.agg_galerkin(0, B, k, Q)
    ref = P.conj().T @ A @ P
    Ad = dense_stencil(N // B, Ac)
    assert np.abs(Ad - ref).max() <= 1e-13 * np.abs(ref).max()
    g5c = np.tile(np.repeat([1.0, -1.0], k), Ad.shape[0] // (2 * k))
    Z = g5c[:, None] * Ad
    assert np.abs(Z - Z.conj().T).max() <= 1e-13 * np.abs(Z).max()


def test_galerkin_on_a_coarse_level(O):
    """The same construction on a coarse LS level (level 1 of a three-grid
    hierarchy, a 2x2-block stencil of side 32) gives dense P^H A_1 P."""
    U = metropolis_u1(64, 6.0, 50, 23)
    h = O.Hierarchy.setup(64, U, 0.02, O.setup_params([2, 2], k_r=4, k_e=4, mu1=3, mu2=2, seed=9))
    B, k = 4, 4
    V = _vectors(32 * 32, k, 74)
    Q = O.agg_interp(32, B, k, V)
    P = dense_P(32, B, k, Q)
    ref = P.conj().T @ h.dense(1) @ P
    Ad = dense_stencil(8, h.agg_galerkin(1, B, k, Q))
    assert np.abs(Ad - ref).max() <= 1e-13 * np.abs(ref).max()


def test_apply_restrict_prolong(O, h32):
    """The block-stencil apply, restriction P^H r and prolongation x + P e
    against dense products."""
    N, B, k = 32, 4, 8
    Q = O.agg_interp(N, B, k, _vectors(N * N, k, 75))
    Ac = h32.agg_galerkin(0, B, k, Q)
    P = dense_P(N, B, k, Q)
    Ad = dense_stencil(N // B, Ac)
    xc = cgauss(76, 1, Ad.shape[0])
    y = O.agg_apply(N // B, k, Ac, xc)
    assert np.abs(y - Ad @ xc).max() <= 1e-13 * np.abs(y).max()
    r = cgauss(76, 2, N * N)
    fc = O.agg_restrict(N, B, k, Q, r)
    assert np.abs(fc - P.conj().T @ r).max() <= 1e-13 * np.abs(fc).max()
    x0 = cgauss(76, 3, N * N)
    x = O.agg_prolong(N, B, k, Q, xc, x0)
    assert np.abs(x - (x0 + P @ xc)).max() <= 1e-13 * np.abs(x).max()
