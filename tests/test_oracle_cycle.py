"""Pin of the oracle's multigrid cycle (Sec. 1: the two-grid correction
E = (I - P A_c^-1 P^H A)(I - M A) with pre- and post-smoothing, applied
recursively; Sec. 4: V- and W-cycles) against an independent restatement.

The reference below assembles every operator itself from the hierarchy's raw
arrays (the random interpolation weights and coarse stencils it feeds the
oracle), with the level geometry written out from its definition: sites of
the even sublattice, rotated coordinates a = (x+y)/2, b = (x-y)/2, the
9-point box stencil in (a, b), B x B cells whose <= 4 corners carry the
coarse points.  Kaczmarz is the column form of Sec. 3.1 taken variable by
variable in the 16-colour, tile-coloured or lexicographic order.  The
recursion is the textbook one: smooth from x = 0, restrict the residual with
P^H, visit the coarse level gamma times (recomputing the coarse residual
before each later visit), prolongate, recompute the residual, smooth again.
A dropped term, a stale residual, a wrong second W visit or a lost coarse
correction on an inner level changes the result by O(1), far above the
1e-12 tolerance."""
import numpy as np
import pytest
import scipy.sparse as sp

from wl_inputs import metropolis_u1, cgauss


# ------------------------------------------------------------ geometry
def site_xy(N, h):
    y = h // (N // 2)
    x = 2 * (h % (N // 2)) + (y & 1)
    return x, y


def site_of(N, x, y):
    x, y = x % N, y % N
    return y * (N // 2) + x // 2


def rot(N, h):
    x, y = site_xy(N, h)
    return (x + y) // 2, (x - y) // 2  # floor division keeps b = (x - y) / 2 exact (x - y is even)


def stencil_dense(N, As):
    """A[2h+s, 2j+u] = sum over offsets d with neighbour j of As[h, d, s, u];
    offset d = 3 (da+1) + (db+1) moves (a, b) by (da, db), i.e. (x, y) by
    (da+db, da-db)."""
    n = N * N // 2
    A = np.zeros((2 * n, 2 * n), complex)
    for h in range(n):
        x, y = site_xy(N, h)
        for d in range(9):
            da, db = d // 3 - 1, d % 3 - 1
            j = site_of(N, x + da + db, y + da - db)
            A[2 * h:2 * h + 2, 2 * j:2 * j + 2] += As[h, d]
    return A


def interp_dense(Nf, B, Pw):
    """P[2h+s, 2c+s] = Pw[h, s, k] for the existing corners k = ka + 2 kb of
    the B x B cell of fine site h (corner (a0 + ka B, b0 + kb B), present
    unless the fine site lies on that cell edge)."""
    nf, Nc = Nf * Nf // 2, Nf // B
    P = np.zeros((2 * nf, 2 * (Nc * Nc // 2)), complex)
    for h in range(nf):
        a, b = rot(Nf, h)
        a0, b0 = B * (a // B), B * (b // B)
        ra, rb = a - a0, b - b0
        for k in range(4):
            ka, kb = k & 1, k >> 1
            if (ka and not ra) or (kb and not rb):
                continue
            ac, bc = a0 + ka * B, b0 + kb * B
            xc, yc = (ac + bc) % Nf, (ac - bc) % Nf
            c = site_of(Nc, xc // B, yc // B)
            for s in range(2):
                P[2 * h + s, 2 * c + s] += Pw[h, s, k]
    return P


def colour_order(N):
    n = N * N // 2
    col = [4 * (rot(N, h)[0] % 4) + (rot(N, h)[1] % 4) for h in range(n)]
    return [h for k in range(16) for h in range(n) if col[h] == k]


def tile_order(N, T=8):
    out = []
    for tc in range(4):
        for ta in range(N // T):
            for tb in range(N // (2 * T)):
                if (ta & 1) + 2 * (tb & 1) != tc:
                    continue
                # the 4 x 4 colour grid row by row, odd rows right to left
                for c in (0, 1, 2, 3, 7, 6, 5, 4, 8, 9, 10, 11, 15, 14, 13, 12):
                    for i in range(T):
                        for j in range(T):
                            a, b = ta * T + i, tb * T + j
                            if 4 * (a % 4) + (b % 4) == c:
                                out.append(site_of(N, a + b, a - b))
    return out


LEX, COLOUR, TILE = 0, 1, 2


def variable_order(N, order):
    if order == LEX or N % 8:
        sites = list(range(N * N // 2))
    elif order == TILE and N >= 64 and N % 32 == 0:
        sites = tile_order(N)
    else:
        sites = colour_order(N)
    return [2 * h + s for h in sites for s in (0, 1)]


# ------------------------------------------------------------ reference
class RefHierarchy:
    def __init__(self, A, P, Ns):
        self.A = [sp.csc_matrix(a) for a in A]
        self.Ad = A[-1]
        self.P = P
        self.Ns = Ns

    def kaczmarz(self, l, x, r, order, sweeps):
        A = self.A[l]
        seq = variable_order(self.Ns[l], order)
        for _ in range(sweeps):
            for i in seq:
                idx = A.indices[A.indptr[i]:A.indptr[i + 1]]
                col = A.data[A.indptr[i]:A.indptr[i + 1]]
                s = np.vdot(col, r[idx]) / np.vdot(col, col).real
                x[i] += s
                r[idx] -= s * col

    def cycle(self, l, f, nu1, nu2, gamma, order):
        if l == len(self.A) - 1:
            return np.linalg.solve(self.Ad, f)
        A, P = self.A[l], self.P[l]
        x = np.zeros_like(f)
        r = f.copy()
        self.kaczmarz(l, x, r, order, nu1)
        fc = P.conj().T @ r
        e = np.zeros_like(fc)
        for g in range(gamma):
            rc = fc - self.A[l + 1] @ e
            e = e + self.cycle(l + 1, rc, nu1, nu2, gamma, order)
        x += P @ e
        r = f - A @ x
        self.kaczmarz(l, x, r, order, nu2)
        return x


def random_hierarchy(O, N, blocks, seed):
    """An oracle hierarchy whose interpolation weights and coarse stencils are
    random (the cycle's algebra holds for any operators), and the same
    operators assembled by the reference."""
    rng = np.random.default_rng(seed)
    U = metropolis_u1(N, 3.0, 20, seed)
    m = 0.2
    Ns = [N]
    for b in blocks:
        Ns.append(Ns[-1] // b)
    Pw = [rng.standard_normal((n * n // 2, 2, 4)) + 1j * rng.standard_normal((n * n // 2, 2, 4))
          for n in Ns[:-1]]
    Pw = [0.5 * p for p in Pw]
    As = []
    for n in Ns[1:]:
        a = 0.15 * (rng.standard_normal((n * n // 2, 9, 2, 2)) + 1j * rng.standard_normal((n * n // 2, 9, 2, 2)))
        a[:, 4] += 2.0 * np.eye(2)
        As.append(a)
    h = O.Hierarchy.from_arrays(N, U, m, Ns, blocks, Pw, As)
    A = [O.dhat_csr(N, U, m).toarray()] + [stencil_dense(n, a) for n, a in zip(Ns[1:], As)]
    P = [interp_dense(n, b, p) for n, b, p in zip(Ns[:-1], blocks, Pw)]
    return h, RefHierarchy(A, P, Ns), A, P


@pytest.fixture(scope="module")
def three_grid(O):
    return random_hierarchy(O, 32, [2, 2], 41)


@pytest.fixture(scope="module")
def four_grid(O):
    return random_hierarchy(O, 64, [2, 2, 2], 43)


def test_reference_operators_match_the_oracle(three_grid):
    """The reference's own assembly of the coarse stencils and of P equals the
    oracle's CSR matrices (the cycle pin below then compares cycles on the
    same operators)."""
    h, ref, A, P = three_grid
    for l in range(1, h.L):
        assert np.array_equal(h.dense(l), A[l])
    for l in range(h.L - 1):
        assert np.array_equal(h.dense(l, 1), P[l])


def _inputs(n):
    f = [cgauss(61, k, n) for k in range(2)]
    e0 = np.zeros(n, complex)
    e0[0] = 1.0
    el = np.zeros(n, complex)
    el[n - 1] = 1.0
    return f + [e0, el]


@pytest.mark.parametrize("nu1,nu2,gamma", [(1, 1, 1), (2, 2, 1), (4, 4, 1), (1, 1, 2), (2, 2, 2), (4, 4, 2),
                                           (3, 1, 2), (0, 2, 1), (2, 0, 2)])
def test_cycle_three_grids(O, three_grid, nu1, nu2, gamma):
    """Three grids (32 -> 16 -> 8), 16-colour Kaczmarz: V- and W-cycles with
    unequal and one-sided smoothing, on random and unit vectors."""
    h, ref, A, _ = three_grid
    for f in _inputs(A[0].shape[0]):
        got = h.cycle(f, nu1=nu1, nu2=nu2, gamma=gamma, order=O.ORDER_COLOUR)
        want = ref.cycle(0, f, nu1, nu2, gamma, COLOUR)
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max(), (nu1, nu2, gamma)


@pytest.mark.parametrize("order", ["lex", "tile"])
@pytest.mark.parametrize("gamma", [1, 2])
def test_cycle_four_grids(O, four_grid, order, gamma):
    """Four grids (64 -> 32 -> 16 -> 8): the W-cycle recurses twice per
    visit through two inner levels; the tile-coloured ordering on the 64 grid
    (the 16-colour one below it) and the lexicographic ordering."""
    h, ref, A, _ = four_grid
    oo = {"lex": (O.ORDER_LEX, LEX), "tile": (O.ORDER_TILE, TILE)}[order]
    f = cgauss(62, gamma, A[0].shape[0])
    got = h.cycle(f, nu1=2, nu2=1, gamma=gamma, order=oo[0])
    want = ref.cycle(0, f, 2, 1, gamma, oo[1])
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_cycle_pin_detects_a_planted_mistake(three_grid):
    """The comparison is sensitive to the mistakes it guards against: the
    reference with the coarse correction of the inner level dropped, or with
    the post-smoothing run on a stale residual, differs from the correct
    cycle by far more than the tolerance."""
    h, ref, A, P = three_grid
    f = cgauss(61, 0, A[0].shape[0])
    good = ref.cycle(0, f, 2, 2, 2, COLOUR)

    class NoInnerCorrection(RefHierarchy):
        def cycle(self, l, f, nu1, nu2, gamma, order):
            if l == 1:
                x = np.zeros_like(f)
                r = f.copy()
                self.kaczmarz(l, x, r, order, nu1 + nu2)
                return x
            return super().cycle(l, f, nu1, nu2, gamma, order)

    class StaleResidual(RefHierarchy):
        def cycle(self, l, f, nu1, nu2, gamma, order):
            if l == len(self.A) - 1:
                return np.linalg.solve(self.Ad, f)
            x = np.zeros_like(f)
            r = f.copy()
            self.kaczmarz(l, x, r, order, nu1)
            fc = self.P[l].conj().T @ r
            e = np.zeros_like(fc)
            for g in range(gamma):
                e = e + self.cycle(l + 1, fc - self.A[l + 1] @ e, nu1, nu2, gamma, order)
            x += self.P[l] @ e
            self.kaczmarz(l, x, r, order, nu2)   # r not recomputed after the correction
            return x

    for bad in (NoInnerCorrection, StaleResidual):
        b = bad([a for a in A], P, ref.Ns).cycle(0, f, 2, 2, 2, COLOUR)
        assert np.abs(b - good).max() > 1e-6 * np.abs(good).max()
