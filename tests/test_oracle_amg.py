"""Pins of the oracle's multigrid pieces (Secs. 1, 3.1, 3.3-3.5, 4) against
definitions and theorems: line-minimiser property of Kaczmarz, Thm. 3.1,
exact recovery of a planted interpolation, dense Galerkin products, the
two-grid error propagation formula, the GMRES minimal-residual property and
dense solves."""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from wl_inputs import metropolis_u1, cgauss, workload, rhs_batch

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def h32(O):
    U = metropolis_u1(32, 6.0, 100, 21)
    m = -0.05
    p = O.setup_params([2], k_r=6, k_e=6, mu1=6, mu2=3, seed=5)
    return O.Hierarchy.setup(32, U, m, p)


@pytest.fixture(scope="module")
def h64(O):
    w = workload("T64")
    p = O.setup_params(w["blocks"], k_r=w["k"], k_e=w["k"], seed=w["seed"])
    return O.Hierarchy.setup(w["N"], w["U"], w["m"], p), w


def _dense_kaczmarz(A, b, x, order):
    x = x.copy()
    r = b - A @ x
    for i in order:
        c = A[:, i]
        s = np.vdot(c, r) / np.vdot(c, c).real
        x[i] += s
        r -= s * c
    return x, r


def test_kaczmarz_residual_and_line_minimiser(O, h32):
    """Sec. 3.1: r is kept equal to f - A x, ||r|| does not grow, and after
    the update of variable i the residual is orthogonal to A e_i (s_i is the
    exact minimiser along e_i)."""
    A = h32.dense(0)
    n = A.shape[0]
    f = cgauss(2, 3, n)
    x0 = cgauss(2, 4, n) * 0.1
    r0 = f - A @ x0
    for order in (O.ORDER_LEX, O.ORDER_COLOUR):
        x, r = h32.kaczmarz(0, x0, r0, order=order, sweeps=1)
        assert np.abs(r - (f - A @ x)).max() <= 1e-12 * np.abs(f).max()
        assert np.linalg.norm(r) < np.linalg.norm(r0)
    x, r = h32.kaczmarz(0, x0, r0, order=O.ORDER_LEX, sweeps=1)
    last = n - 1
    assert abs(np.vdot(A[:, last], r)) <= 1e-12 * np.linalg.norm(A[:, last]) * np.linalg.norm(r0)


def test_kaczmarz_colour_order_is_a_forward_sweep(O, h32):
    """The multicolour sweep is the forward Kaczmarz sweep taken in colour
    order (colour 0..15, sites ascending, spin 0 then 1); compared with a
    dense textbook sweep in that order."""
    A = h32.dense(0)
    n = A.shape[0] // 2
    f = cgauss(5, 1, 2 * n)
    order = []
    for k in range(16):
        for h in range(n):
            if O.colour(32, h) == k:
                order += [2 * h, 2 * h + 1]
    xr, rr = _dense_kaczmarz(A, f, np.zeros(2 * n, complex), order)
    x, r = h32.kaczmarz(0, np.zeros(2 * n), f, order=O.ORDER_COLOUR)
    assert np.abs(x - xr).max() <= 1e-13 * np.abs(xr).max()


def test_kaczmarz_within_colour_permutation(O, h32):
    """Updates inside one colour commute (disjoint supports): any site order
    within the colours gives the same sweep up to rounding."""
    n = 32 * 32 // 2
    f = cgauss(6, 1, 2 * n)
    x1, _ = h32.kaczmarz(0, np.zeros(2 * n), f, order=O.ORDER_COLOUR, sweeps=2)
    perm = np.random.default_rng(3).permutation(n)
    x2, _ = h32.kaczmarz(0, np.zeros(2 * n), f, order=O.ORDER_COLOUR, sweeps=2, perm=perm)
    assert np.abs(x1 - x2).max() <= 1e-15 * np.abs(x1).max() * 10


def test_theorem_kaczmarz_on_Z(O, h32):
    """Thm. 3.1 (ii): Kaczmarz on D x = b and on Z x = Gamma5 b (Z = Gamma5 D)
    produce the same iterates."""
    A = h32.dense(0)
    n = A.shape[0]
    g5 = np.tile([1.0, -1.0], n // 2)
    Z = g5[:, None] * A
    f = cgauss(7, 1, n)
    xz, _ = _dense_kaczmarz(Z, g5 * f, np.zeros(n, complex), range(n))
    x, _ = h32.kaczmarz(0, np.zeros(n), f, order=O.ORDER_LEX)
    assert np.abs(x - xz).max() <= 1e-12 * np.abs(x).max()


def test_interpolation_structure(O, h32):
    """Eqs. 3.13-3.15: P is block diagonal in spin (Gamma5 P = P Gamma5c), a
    fine variable interpolates from <= 4 coarse variables and, for 2x2 cells,
    exactly from the same-spin coarse neighbours in the graph of Dhat; C rows
    are the identity."""
    gold = json.load(open(os.path.join(GOLDEN, "paper_structure.json")))
    P = h32.dense(0, which=1)
    A = h32.dense(0)
    nf, nc = P.shape
    g5f, g5c = np.tile([1.0, -1.0], nf // 2), np.tile([1.0, -1.0], nc // 2)
    assert np.abs(g5f[:, None] * P - P * g5c[None, :]).max() == 0.0
    nnz = (np.abs(P) > 0).sum(axis=1)
    assert nnz.max() <= gold["max_interpolation_points"]
    # coarse points: fine unknowns that are identity rows
    crow = {}
    for i in range(nf):
        js = np.nonzero(np.abs(P[i]) > 0)[0]
        if len(js) == 1 and abs(P[i, js[0]] - 1) < 1e-14:
            crow[js[0]] = i
    assert len(crow) == nc
    for i in range(nf):
        if i in crow.values():
            continue
        graph = {j for j in range(nc) if j % 2 == i % 2 and abs(A[i, crow[j]]) > 0}
        assert set(np.nonzero(np.abs(P[i]) > 0)[0]) == graph


def test_galerkin_dense(O, h64):
    """Sec. 3.5: D_{l+1} = P^H D_l P; the coarse operator is gamma5-Hermitian
    and keeps the 9-point pattern with at most 18 non-zeros per row."""
    h, _ = h64
    gold = json.load(open(os.path.join(GOLDEN, "paper_structure.json")))
    for l in range(h.L - 1):
        A, P, Ac = h.dense(l), h.dense(l, 1), h.dense(l + 1)
        ref = P.conj().T @ A @ P
        assert np.abs(Ac - ref).max() <= 1e-13 * np.abs(ref).max()
        g5 = np.tile([1.0, -1.0], Ac.shape[0] // 2)
        assert np.abs(g5[:, None] * Ac - (g5[:, None] * Ac).conj().T).max() == 0.0
        assert (np.abs(Ac) > 0).sum(axis=1).max() <= gold["max_coarse_nnz_per_row"]


def test_petrov_galerkin_equals_galerkin(O, h32):
    """Sec. 3.5: with R = (Gamma5 P)^H, P (R D P)^-1 R = P (P^H D P)^-1 P^H."""
    A, P = h32.dense(0), h32.dense(0, 1)
    g5 = np.tile([1.0, -1.0], A.shape[0] // 2)
    R = (g5[:, None] * P).conj().T
    lhs = P @ np.linalg.solve(R @ A @ P, R)
    rhs = P @ np.linalg.solve(P.conj().T @ A @ P, P.conj().T)
    assert np.abs(lhs - rhs).max() <= 1e-10 * np.abs(rhs).max()


def test_ls_fit_exact_recovery_and_optimality(O, h32):
    """Eq. 3.4: test vectors that lie in range(P_true) are fitted exactly
    (P_true is recovered); perturbing a fitted row increases the functional."""
    N, B = 32, 2
    nf = N * N // 2
    rng = np.random.default_rng(11)
    Pw_true = h32.export()[0][0].copy()
    mask = np.abs(Pw_true) > 0
    Pw_true[mask] = rng.standard_normal(mask.sum()) + 1j * rng.standard_normal(mask.sum())
    # C rows stay the identity
    for hf in range(nf):
        for s in range(2):
            if mask[hf, s].sum() == 1:
                Pw_true[hf, s] = 0
                Pw_true[hf, s, 0] = 1.0
    _, As = h32.export()
    hp = O.Hierarchy.from_arrays(N, h32.U, h32.m, h32.Nl, h32.Bl, [Pw_true], As)
    P = hp.dense(0, 1)
    k = 7
    Vc = rng.standard_normal((k, P.shape[1])) + 1j * rng.standard_normal((k, P.shape[1]))
    V = Vc @ P.T
    w = rng.random(k) + 0.5
    Pw = O.ls_fit(N, B, V, w)
    assert np.abs(Pw - Pw_true).max() <= 1e-10
    # optimality of a fit of noisy vectors
    Vn = V + 0.3 * (rng.standard_normal(V.shape) + 1j * rng.standard_normal(V.shape))
    Pn = O.ls_fit(N, B, Vn, w)
    hn = O.Hierarchy.from_arrays(N, h32.U, h32.m, h32.Nl, h32.Bl, [Pn], As)
    Pd = hn.dense(0, 1)
    cidx = [np.nonzero(np.abs(Pd[:, j]) == 1)[0] for j in range(Pd.shape[1])]
    cpos = np.array([c[0] for c in cidx])
    for i in rng.choice(Pd.shape[0], 20, replace=False):
        js = np.nonzero(np.abs(Pd[i]) > 0)[0]
        if len(js) < 2:
            continue
        def L(p):
            resid = Vn[:, i] - Vn[:, cpos[js]] @ p
            return float(np.sum(w * np.abs(resid) ** 2))
        p0 = Pd[i, js]
        for _ in range(5):
            dp = 1e-3 * (rng.standard_normal(len(js)) + 1j * rng.standard_normal(len(js)))
            assert L(p0 + dp) >= L(p0)


def test_generalised_eigensolver(O):
    """Thm. 3.1 (i): Z V = T V Lambda against LAPACK's generalised Hermitian
    solver (scipy.linalg.eigh)."""
    rng = np.random.default_rng(2)
    n = 40
    Zr = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Z = Zr + Zr.conj().T
    Tr = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    T = Tr @ Tr.conj().T + n * np.eye(n)
    lam, V = O.gen_eig(Z, T)
    ref = sla.eigh(Z, T, eigvals_only=True)
    assert np.abs(lam - ref).max() <= 1e-12 * np.abs(ref).max()
    for k in range(n):
        v = V[k]
        assert np.linalg.norm(Z @ v - lam[k] * (T @ v)) <= 1e-11 * np.linalg.norm(Z)
        assert abs(np.vdot(v, T @ v) - 1) <= 1e-12


def test_theorem_singular_triplets(O, h64):
    """Thm. 3.1 (i), (iii): an eigenpair Z_L v = lambda T_L v gives the
    generalised singular triplet D_L v = |lambda| T_L u, D_L^H u = |lambda|
    T_L v with u = sign(lambda) Gamma5 v (Q_L = T_L)."""
    h, w = h64
    O_ = O
    p = O_.setup_params(w["blocks"], k_r=4, k_e=4, mu1=3, mu2=2, seed=3)
    hh = O_.Hierarchy.setup(w["N"], w["U"], w["m"], p)
    L = hh.L - 1
    A = hh.dense(L)
    T = hh.dense(L, which=2)
    g5 = np.tile([1.0, -1.0], A.shape[0] // 2)
    lam, V = O_.gen_eig(g5[:, None] * A, T)
    for k in range(0, A.shape[0], 17):
        v = V[k]
        u = np.sign(lam[k]) * g5 * v
        sig = abs(lam[k])
        assert np.linalg.norm(A @ v - sig * (T @ u)) <= 1e-10 * np.linalg.norm(A)
        assert np.linalg.norm(A.conj().T @ u - sig * (T @ v)) <= 1e-10 * np.linalg.norm(A)


def test_two_grid_error_propagation(O, h32):
    """Sec. 1: one pre-smoothing step and the Galerkin correction give
    x = x_s + P A_c^-1 P^H (f - A x_s), x_s the smoothed iterate from 0."""
    A, P = h32.dense(0), h32.dense(0, 1)
    n = A.shape[0]
    f = cgauss(9, 2, n)
    xs, _ = h32.kaczmarz(0, np.zeros(n), f, order=O.ORDER_COLOUR, sweeps=1)
    Ac = P.conj().T @ A @ P
    ref = xs + P @ np.linalg.solve(Ac, P.conj().T @ (f - A @ xs))
    x = h32.cycle(f, nu1=1, nu2=0)
    assert np.abs(x - ref).max() <= 1e-11 * np.abs(ref).max()


def test_cycle_linear(O, h64):
    """The V- and W-cycles are linear maps of f."""
    h, _ = h64
    n = h.n(0)
    f, g = cgauss(1, 5, n), cgauss(1, 6, n)
    a = 0.7 - 0.3j
    for gamma in (1, 2):
        lhs = h.cycle(a * f + g, gamma=gamma)
        rhs = a * h.cycle(f, gamma=gamma) + h.cycle(g, gamma=gamma)
        assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(lhs).max()


@pytest.mark.parametrize("gs_passes", [1, 2])
def test_gmres_minimal_residual(O, h32, gs_passes):
    """Unpreconditioned GMRES after k steps minimises ||b - A x|| over the
    Krylov space span{b, Ab, ..., A^{k-1} b} (dense least squares), with
    classical Gram-Schmidt (one pass) and with one reorthogonalisation (two
    passes): in exact arithmetic both give the same Arnoldi basis."""
    A = h32.dense(0)
    n = A.shape[0]
    b = cgauss(4, 4, n)
    k = 6
    x, info = h32.fgmres(b, tol=0.0, m=k, max_restarts=1, precond=0, gs_passes=gs_passes)
    K = np.empty((n, k), complex)
    v = b.copy()
    for j in range(k):
        K[:, j] = v
        v = A @ v
    Q, _ = np.linalg.qr(K)
    y = np.linalg.lstsq(A @ Q, b, rcond=None)[0]
    ref = Q @ y
    assert info["iters"] == k
    assert np.abs(x - ref).max() <= 1e-9 * np.abs(ref).max()


def test_fgmres_one_pass_cycle_solve(O, h64):
    """The benchmark's Krylov variant (one Gram-Schmidt pass, tile-coloured
    V(4,4) cycle) converges to the same solution as the default (two passes,
    16-colour V(2,2)), and to the sparse-direct solution; the lexicographic
    cycle too."""
    h, w = h64
    N = w["N"]
    b = rhs_batch(N, 1, 5)[0]
    D = O.wilson_csr(N, w["U"], w["m"]).tocsc()
    ref = spla.spsolve(D, b.reshape(-1)).reshape(N, N, 2)
    for kw in (dict(gs_passes=1, nu1=4, nu2=4, order=O.ORDER_TILE), dict(gs_passes=2, order=O.ORDER_LEX)):
        psi, info = h.solve(b, tol=1e-13, **kw)
        assert info["status"] == 0, kw
        assert np.linalg.norm(psi - ref) <= 1e-10 * np.linalg.norm(ref), kw


def test_solve_dense_8x8(O):
    """Whole solve (reduce, FGMRES + V-cycle, reconstruct) against the dense
    solution of D psi = b on an 8x8 lattice."""
    N, m = 8, 0.05
    U = metropolis_u1(N, 3.0, 30, 77)
    p = O.setup_params([2], k_r=4, k_e=4, mu1=4, mu2=2, seed=1)
    h = O.Hierarchy.setup(N, U, m, p)
    b = cgauss(8, 8, 2 * N * N).reshape(N, N, 2)
    psi, info = h.solve(b, tol=1e-13)
    D = O.wilson_csr(N, U, m).toarray()
    ref = np.linalg.solve(D, b.reshape(-1)).reshape(N, N, 2)
    assert info["status"] == 0
    assert np.linalg.norm(psi - ref) <= 1e-11 * np.linalg.norm(ref)


def test_solve_sparse_direct_64(O, h64):
    """Whole solve on the 64x64 workload against SciPy's sparse LU of D."""
    h, w = h64
    N = w["N"]
    b = rhs_batch(N, 1, 5)[0]
    psi, info = h.solve(b, tol=1e-13)
    D = O.wilson_csr(N, w["U"], w["m"]).tocsc()
    ref = spla.spsolve(D, b.reshape(-1)).reshape(N, N, 2)
    assert info["status"] == 0
    assert np.linalg.norm(psi - ref) <= 1e-10 * np.linalg.norm(ref)


def test_setup_quality_band(O, h64):
    """Sec. 4.1 (quality, not parity): the preconditioned Krylov solve needs
    far fewer iterations than plain GMRES and the stand-alone W(4,4) cycle
    converges with rate rho well below 1."""
    h, w = h64
    bh = O.eo_reduce(w["N"], w["U"], w["m"], rhs_batch(w["N"], 1, 6)[0])
    _, info = h.fgmres(bh, tol=1e-10, m=20, max_restarts=20)
    assert info["status"] == 0 and info["iters"] <= 40
    A = h.dense(0)
    x = cgauss(3, 9, h.n(0))
    e_prev = np.linalg.norm(x)
    for _ in range(12):
        x = x - h.cycle(A @ x, nu1=4, nu2=4, gamma=2)  # error iteration on A x = 0
        e = np.linalg.norm(x)
        rho, e_prev = e / e_prev, e
    assert rho <= 0.8


def test_hierarchy_roundtrip(O, h64):
    """Export to (P weights, coarse stencils) and import gives the same
    operators and the same cycle."""
    h, w = h64
    Pw, As = h.export()
    h2 = O.Hierarchy.from_arrays(w["N"], w["U"], w["m"], h.Nl, h.Bl[:-1], Pw, As)
    f = cgauss(12, 1, h.n(0))
    assert np.abs(h.cycle(f) - h2.cycle(f)).max() == 0.0
    for l in range(h.L):
        assert np.abs(h.dense(l) - h2.dense(l)).max() == 0.0


def test_rng_reference_values(O):
    """SplitMix64 published test vector: state 0 -> 0xE220A8397B1DCDAF,
    0x6E789E6AA1B965F4 (first two outputs); u64(seed,stream,i) composes it."""
    from wl_inputs import rng as R
    assert R._sm_scalar(0) == 0xE220A8397B1DCDAF
    assert R._sm_scalar(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4
    for s, st, i in [(0, 0, 0), (123, 7, 99), (2**63 + 5, 3, 2**40)]:
        assert int(R.rng_u64(s, st, [i])[0]) == O.rng_u64(s, st, i)


def _tile_order(O, N):
    """the tile-coloured permutation written out from its definition"""
    T = O.tile_size(N)
    order = []
    for tc in range(4):
        for ta in range(N // T):
            for tb in range(N // (2 * T)):
                if (ta & 1) + 2 * (tb & 1) != tc:
                    continue
                # site colours 4 (a mod 4) + (b mod 4), the 4 x 4 colour grid taken
                # row by row, even rows left to right, odd rows right to left
                for row in range(4):
                    for col in (range(4) if row % 2 == 0 else range(3, -1, -1)):
                        c = 4 * row + col
                        order += _tile_colour_sites(N, T, ta, tb, c)
    return order


def _tile_colour_sites(N, T, ta, tb, c):
    """sites of colour c in tile (ta, tb), increasing (a, b)"""
    out = []
    for i in range(T):
        for j in range(T):
            a, b = ta * T + i, tb * T + j
            if 4 * (a % 4) + (b % 4) != c:
                continue
            x, y = (a + b) % N, (a - b) % N
            out.append(y * (N // 2) + x // 2)
    return out


def test_tile_order_covers_every_site_and_tiles_are_independent(O):
    """The tile-coloured ordering (a reading of Sec. 3.1's parallel
    ordering): each site once per sweep, and tiles of one tile colour touch
    disjoint 3x3 column supports, so they can be relaxed at the same time."""
    for N in (64, 128):
        T = O.tile_size(N)
        assert T == 8
        order = _tile_order(O, N)
        assert sorted(order) == list(range(N * N // 2))
        supp = {h: {O.neighbour(N, h, d) for d in range(9)} for h in range(N * N // 2)}
        per_tile = N * N // 2 // ((N // T) * (N // (2 * T)))
        tiles = [order[k:k + per_tile] for k in range(0, len(order), per_tile)]
        ntc = len(tiles) // 4
        for tc in range(4):
            seen = set()
            for t in tiles[tc * ntc:(tc + 1) * ntc]:
                region = set().union(*(supp[h] for h in t))
                assert not (region & seen)
                seen |= region
    assert O.tile_size(32) == 0  # small grids keep the 16-colour order


def test_tile_sweep_is_a_forward_sweep(O, h64):
    """One tile-coloured sweep equals the dense textbook forward sweep over
    the variables in the tile order (spin 0 then 1 per site)."""
    h, w = h64
    A = h.dense(0)
    n = A.shape[0] // 2
    f = cgauss(15, 1, 2 * n)
    order = []
    for s_ in _tile_order(O, w["N"]):
        order += [2 * s_, 2 * s_ + 1]
    xr, _ = _dense_kaczmarz(A, f, np.zeros(2 * n, complex), order)
    x, r = h.kaczmarz(0, np.zeros(2 * n), f, order=O.ORDER_TILE)
    assert np.abs(x - xr).max() <= 1e-13 * np.abs(xr).max()
    assert np.abs(r - (f - A @ x)).max() <= 1e-12 * np.abs(f).max()


def test_rho_two_grid_projector(O, h32):
    """Sec. 4's rho with no smoothing on two grids: the error propagator
    I - P A_c^-1 P^H A of a Galerkin coarse correction is a projector
    (its square is itself), so after one iteration the error stays put and
    rho = 1 exactly, while the first step reduces the error."""
    x0 = cgauss(4, 1, h32.n(0))
    rho, nu, hist, met = h32.rho(x0, tol=1e-300, maxit=6, nu1=0, nu2=0, gamma=1)
    assert nu == 6 and not met
    assert hist[1] < hist[0]
    assert abs(rho - 1.0) <= 1e-12
    assert np.abs(hist[1:] / hist[1] - 1.0).max() <= 1e-12


def test_rho_is_the_spectral_radius(O, h32):
    """After 100 iterations the ratio |e^nu| / |e^(nu-1)| of Sec. 4 equals
    the spectral radius of the error propagator I - M A_0, assembled column
    by column from the cycle and handed to a dense eigensolver."""
    A = h32.dense(0)
    n = A.shape[0]
    E = np.eye(n, dtype=complex)
    for j in range(n):
        E[:, j] -= h32.cycle(A[:, j], nu1=1, nu2=1, gamma=1)
    sr = np.abs(np.linalg.eigvals(E)).max()
    rho, nu, hist, met = h32.rho(cgauss(4, 1, n), tol=1e-300, maxit=100, nu1=1, nu2=1, gamma=1)
    assert nu == 100 and not met
    assert abs(rho - sr) <= 1e-6 * sr, (rho, sr)


def test_rho_stops_at_tolerance(O, h64):
    """The estimate is taken at the first iteration whose error norm is
    below tol times the initial one (W(4,4), Sec. 4)."""
    h, _ = h64
    rho, nu, hist, met = h.rho(cgauss(4, 2, h.n(0)), tol=1e-8, maxit=100, nu1=4, nu2=4, gamma=2)
    assert met and nu < 100
    assert hist[-1] <= 1e-8 * hist[0] < hist[-2]
    assert abs(rho - hist[-1] / hist[-2]) <= 1e-15
    assert rho < 0.6


def test_super_v_setup(O, h64):
    """Sec. 4.2's super-V setup (each grid visited once): on two grids it is
    the W setup (the only coarse visit is the coarsest eigensolve); on three
    grids it yields a convergent stand-alone W(4,4) solver and a
    preconditioner within the quality band of the W setup."""
    U = metropolis_u1(32, 6.0, 100, 21)
    pw = O.setup_params([2], k_r=6, k_e=6, mu1=6, mu2=3, seed=5)
    pv = O.setup_params([2], k_r=6, k_e=6, mu1=6, mu2=3, seed=5, super_v=True)
    hw, hv = O.Hierarchy.setup(32, U, -0.05, pw), O.Hierarchy.setup(32, U, -0.05, pv)
    assert np.array_equal(hw.dense(0, 1), hv.dense(0, 1))
    h, w = h64
    p = O.setup_params(w["blocks"], k_r=w["k"], k_e=w["k"], seed=w["seed"], super_v=True)
    hs = O.Hierarchy.setup(w["N"], w["U"], w["m"], p)
    assert not np.array_equal(hs.dense(1, 1), h.dense(1, 1))
    x0 = cgauss(4, 3, h.n(0))
    rho_v, nu_v, _, met_v = hs.rho(x0, tol=1e-8, maxit=100, nu1=4, nu2=4, gamma=2)
    rho_w, nu_w, _, _ = h.rho(x0, tol=1e-8, maxit=100, nu1=4, nu2=4, gamma=2)
    assert met_v and rho_v < 0.9
    bh = O.eo_reduce(w["N"], w["U"], w["m"], rhs_batch(w["N"], 1, 6)[0])
    _, iv = hs.fgmres(bh, tol=1e-8, m=32, max_restarts=5, nu1=4, nu2=4, gamma=2)
    _, iw = h.fgmres(bh, tol=1e-8, m=32, max_restarts=5, nu1=4, nu2=4, gamma=2)
    assert iv["status"] == 0 and iv["iters"] <= 2 * iw["iters"] + 5, (iv, iw, rho_v, rho_w)


def test_rho_divergent_cycle_stops_at_overflow(O, h32):
    """A cycle whose coarse correction is scaled up diverges; the estimate
    stops at the last finite error norm and reports the ratio of the last two
    (the definition in Sec. 4 presumes convergence)."""
    Pw, As = h32.export()
    hb = O.Hierarchy.from_arrays(h32.N, h32.U, h32.m, h32.Nl, h32.Bl[:-1], Pw, [a * 1e-6 for a in As])
    x0 = cgauss(4, 1, h32.n(0))
    rho, nu, hist, met = hb.rho(x0, tol=1e-8, maxit=100, nu1=1, nu2=1, gamma=1)
    assert not met and 2 <= nu < 100
    assert np.all(np.isfinite(hist)) and hist[-1] > 1e100
    assert rho > 1e4 and rho == hist[-1] / hist[-2]


def test_hierarchy_complexities(O, h64):
    """Sec. 4's structure: with 2x2 cells down to the N = 16 coarsest grid,
    N = 128 gives 4 grids and N = 256 gives 5 (the Sec. 4 workloads), and the
    grid and operator complexities stay below the stated 1.4."""
    from wl_inputs.workloads import WORKLOADS
    gold = json.load(open(os.path.join(GOLDEN, "paper_structure.json")))
    assert len(WORKLOADS["P128_b6_c0"]["blocks"]) + 1 == gold["grids_N128"]
    assert len(WORKLOADS["P256_b6_c0"]["blocks"]) + 1 == gold["grids_N256"]
    h, _ = h64
    rows = [h.dense(l).shape[0] for l in range(h.L)]
    nnz = [int((np.abs(h.dense(l)) > 0).sum()) for l in range(h.L)]
    assert h.Nl[-1] == gold["coarsest_N"]
    assert sum(rows) / rows[0] <= gold["max_complexity"]
    assert sum(nnz) / nnz[0] <= gold["max_complexity"]
