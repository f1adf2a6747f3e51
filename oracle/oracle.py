"""ctypes front end of the FP64 CPU oracle (wilson_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU-baseline leg.  The product (the CUDA library and its binding)
never imports this module.

Array conventions (complex128 throughout):
  gauge U[2][N][N] (mu, y, x); full fields [N][N][2] (y, x, spin);
  level vectors [n_l * 2] with unknown 2*h + s on the even sublattice;
  interpolation weights Pw[l] [n_l][2][4]; coarse stencils As[l] [n_l][9][2][2].
"""
import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wilson_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
# the same source built with -fopenmp: timed as the all-cores CPU baseline only
_LIB_OMP_PATH = os.path.join(_HERE, "liboracle_omp.so")
_lib = None
_variant = "plain"

ORDER_LEX = 0
ORDER_COLOUR = 1
ORDER_TILE = 2


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no architecture flags); with
    omp, the all-cores variant of the same source (-fopenmp)."""
    path = _LIB_OMP_PATH if omp else _LIB_PATH
    if force or not os.path.exists(path) or os.path.getmtime(path) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "wilson_oracle.h"))):
        tmp = path + ".%d.tmp" % os.getpid()
        flags = ["-fopenmp"] if omp else []
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", *flags,
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, path)
    return path


def use_variant(name: str) -> None:
    """Select, before the first call, which build this process loads:
    "plain" (the oracle the tests check against) or "omp" (the same source
    built with OpenMP, for the timed all-cores CPU baseline)."""
    global _variant
    if _lib is not None and name != _variant:
        raise RuntimeError("oracle library already loaded as %s" % _variant)
    if name not in ("plain", "omp"):
        raise ValueError(name)
    _variant = name


def threads() -> int:
    """Host threads the loaded build runs its loops on."""
    return lib().or_threads()


def lib():
    global _lib
    if _lib is None:
        path = build(omp=_variant == "omp")
        L = C.CDLL(path)
        P = C.c_void_p
        i, d = C.c_int, C.c_double
        sig = {
            "or_wilson_nnz": (i, [i]),
            "or_wilson_csr": (i, [i, P, d, P, P, P]),
            "or_wilson_apply": (i, [i, P, d, P, P]),
            "or_dhat_nnz": (i, [i, P, d]),
            "or_dhat_csr": (i, [i, P, d, P, P, P]),
            "or_dhat_apply": (i, [i, P, d, P, P]),
            "or_eo_reduce": (i, [i, P, d, P, P]),
            "or_eo_reconstruct": (i, [i, P, d, P, P, P]),
            "or_colour": (i, [i, i]),
            "or_stencil_neighbour": (i, [i, i, i]),
            "or_hier_import": (P, [i, P, d, i, P, P, P, P]),
            "or_hier_export": (i, [P, P, P]),
            "or_setup": (P, [i, P, d, P, P]),
            "or_hier_free": (None, [P]),
            "or_hier_levels": (i, [P, P, P]),
            "or_level_apply": (i, [P, i, P, P]),
            "or_kaczmarz": (i, [P, i, P, P, i, i, d, P]),
            "or_restrict": (i, [P, i, P, P]),
            "or_prolong": (i, [P, i, P, P]),
            "or_coarsest_solve": (i, [P, P, P]),
            "or_cycle": (i, [P, i, P, P, i, i, i, i]),
            "or_fgmres": (i, [P, P, P, d, i, i, i, i, i, i, i, P, P, P]),
            "or_solve": (i, [i, P, d, P, P, P, d, i, i, i, i, i, i, i, P, P]),
            "or_threads": (i, []),
            "or_agg_interp": (i, [i, i, i, P, P]),
            "or_agg_galerkin": (i, [P, i, i, i, P, P]),
            "or_agg_apply": (i, [i, i, P, P, P]),
            "or_agg_restrict": (i, [i, i, i, P, P, P]),
            "or_agg_prolong": (i, [i, i, i, P, P, P]),
            "or_rho": (i, [P, P, d, i, i, i, i, i, P, P, P]),
            "or_tile_size": (i, [i]),
            "or_ls_fit": (i, [i, i, i, P, P, P]),
            "or_galerkin": (i, [P, i, P]),
            "or_gen_eig": (i, [i, P, P, P, P]),
            "or_dense_lu_solve": (i, [i, P, P, P]),
            "or_hier_level_dense": (i, [P, i, i, P]),
            "or_rng_u64": (C.c_uint64, [C.c_uint64, C.c_uint64, C.c_uint64]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        L.or_rng_cgauss.restype = None  # returns a C complex; not called through ctypes
        _lib = L
    return _lib


def _c(a, dtype=np.complex128):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _chk(rc, what):
    if rc < 0:
        raise RuntimeError("oracle %s failed (%d)" % (what, rc))
    return rc


# ---------------------------------------------------------------- operators
def wilson_csr(N, U, m):
    import scipy.sparse as sp
    U = _c(U)
    nnz = lib().or_wilson_nnz(N)
    rp = np.zeros(2 * N * N + 1, np.int32)
    col = np.zeros(nnz, np.int32)
    val = np.zeros(nnz, np.complex128)
    got = _chk(lib().or_wilson_csr(N, _p(U), m, _p(rp), _p(col), _p(val)), "wilson_csr")
    return sp.csr_matrix((val[:got], col[:got], rp), shape=(2 * N * N, 2 * N * N))


def wilson_apply(N, U, m, psi):
    U, psi = _c(U), _c(psi)
    out = np.zeros_like(psi)
    _chk(lib().or_wilson_apply(N, _p(U), m, _p(psi), _p(out)), "wilson_apply")
    return out


def z_apply(N, U, m, psi):
    """Z psi = Gamma5 D psi (Thm. 3.1), Gamma5 = diag(1, -1) on each site's
    two spins; psi and the result in the full-field layout [N][N][2]."""
    out = wilson_apply(N, U, m, psi).reshape(N, N, 2)
    out[..., 1] *= -1
    return out.reshape(np.shape(psi))


def dhat_csr(N, U, m):
    import scipy.sparse as sp
    U = _c(U)
    nnz = _chk(lib().or_dhat_nnz(N, _p(U), m), "dhat_nnz")
    rp = np.zeros(N * N + 1, np.int32)
    col = np.zeros(nnz, np.int32)
    val = np.zeros(nnz, np.complex128)
    _chk(lib().or_dhat_csr(N, _p(U), m, _p(rp), _p(col), _p(val)), "dhat_csr")
    return sp.csr_matrix((val, col, rp), shape=(N * N, N * N))


def dhat_apply(N, U, m, xe):
    U, xe = _c(U), _c(xe)
    out = np.zeros_like(xe)
    _chk(lib().or_dhat_apply(N, _p(U), m, _p(xe), _p(out)), "dhat_apply")
    return out


def eo_reduce(N, U, m, b):
    U, b = _c(U), _c(b)
    out = np.zeros(N * N, np.complex128)
    _chk(lib().or_eo_reduce(N, _p(U), m, _p(b), _p(out)), "eo_reduce")
    return out


def eo_reconstruct(N, U, m, b, xe):
    U, b, xe = _c(U), _c(b), _c(xe)
    out = np.zeros((N, N, 2), np.complex128)
    _chk(lib().or_eo_reconstruct(N, _p(U), m, _p(b), _p(xe), _p(out)), "eo_reconstruct")
    return out


def colour(N, h):
    return lib().or_colour(N, h)


def neighbour(N, h, d):
    return lib().or_stencil_neighbour(N, h, d)


def tile_size(N):
    return lib().or_tile_size(N)


def rng_u64(seed, stream, i):
    return lib().or_rng_u64(seed, stream, i)


# ------------------------------------------------------------- setup pieces
def ls_fit(Nf, B, V, w):
    V = _c(V)
    w = _c(w, np.float64)
    k = V.shape[0]
    out = np.zeros((Nf * Nf // 2, 2, 4), np.complex128)
    _chk(lib().or_ls_fit(Nf, B, k, _p(V), _p(w), _p(out)), "ls_fit")
    return out


def gen_eig(Z, T):
    Z, T = _c(Z), _c(T)
    n = Z.shape[0]
    lam = np.zeros(n)
    V = np.zeros((n, n), np.complex128)
    _chk(lib().or_gen_eig(n, _p(Z), _p(T), _p(lam), _p(V)), "gen_eig")
    return lam, V  # V[k] = eigenvector k


def dense_lu_solve(A, b):
    A, b = _c(A), _c(b)
    x = np.zeros_like(b)
    _chk(lib().or_dense_lu_solve(A.shape[0], _p(A), _p(b), _p(x)), "dense_lu_solve")
    return x


# ------------------------------------------------- aggregation coarse space
def agg_interp(N, B, k, V):
    """Q [nc][2][B*B][k]: per aggregate (B x B cell) and spin, the k test
    vectors V [k][N*N] restricted there, orthonormalised in order."""
    V = _c(V)
    nc = (N // B) ** 2 // 2
    Q = np.zeros((nc, 2, B * B, k), np.complex128)
    _chk(lib().or_agg_interp(N, B, k, _p(V), _p(Q)), "agg_interp")
    return Q


def agg_apply(Nc, k, Ac, x):
    Ac, x = _c(Ac), _c(x)
    y = np.zeros_like(x)
    _chk(lib().or_agg_apply(Nc, k, _p(Ac), _p(x), _p(y)), "agg_apply")
    return y


def agg_restrict(N, B, k, Q, r):
    Q, r = _c(Q), _c(r)
    fc = np.zeros((N // B) ** 2 // 2 * 2 * k, np.complex128)
    _chk(lib().or_agg_restrict(N, B, k, _p(Q), _p(r), _p(fc)), "agg_restrict")
    return fc


def agg_prolong(N, B, k, Q, e, x):
    Q, e, x = _c(Q), _c(e), _c(x).copy()
    _chk(lib().or_agg_prolong(N, B, k, _p(Q), _p(e), _p(x)), "agg_prolong")
    return x


class SetupParams(C.Structure):
    _fields_ = [("levels", C.c_int), ("block", C.c_int * 8), ("k_r", C.c_int), ("k_e", C.c_int),
                ("mu1", C.c_int), ("mu2", C.c_int), ("nu_pre", C.c_int), ("nu_post", C.c_int),
                ("gamma", C.c_int), ("setup_cycle", C.c_int), ("seed", C.c_uint64)]


def setup_params(blocks, k_r=8, k_e=8, mu1=10, mu2=5, nu_pre=4, nu_post=4, gamma=2, seed=1, super_v=False):
    p = SetupParams()
    p.levels = len(blocks) + 1
    for i, b in enumerate(blocks):
        p.block[i] = b
    p.k_r, p.k_e, p.mu1, p.mu2 = k_r, k_e, mu1, mu2
    p.nu_pre, p.nu_post, p.gamma, p.setup_cycle, p.seed = nu_pre, nu_post, gamma, 1 if super_v else 2, seed
    return p


# ---------------------------------------------------------------- hierarchy
class Hierarchy:
    """Owns an or_hier*.  Level 0 is Dhat; levels 1.. are Galerkin stencils."""

    def __init__(self, ptr, N, U, m):
        if not ptr:
            raise RuntimeError("oracle hierarchy construction failed")
        self._h = C.c_void_p(ptr)
        self.N, self.U, self.m = N, _c(U), m
        Nl = np.zeros(8, np.int32)
        Bl = np.zeros(8, np.int32)
        self.L = lib().or_hier_levels(self._h, _p(Nl), _p(Bl))
        self.Nl = [int(v) for v in Nl[: self.L]]
        self.Bl = [int(v) for v in Bl[: self.L]]

    @classmethod
    def setup(cls, N, U, m, params, ritz=None):
        U = _c(U)
        rz = np.zeros(64)
        ptr = lib().or_setup(N, _p(U), m, C.byref(params), _p(rz))
        h = cls(ptr, N, U, m)
        h.ritz = rz[: params.k_e].copy()
        return h

    @classmethod
    def from_arrays(cls, N, U, m, Nl, Bl, Pw, As):
        U = _c(U)
        L = len(Nl)
        Nl_a = np.asarray(Nl, np.int32)
        Bl_a = np.asarray(list(Bl) + [0] * (L - len(Bl)), np.int32)
        Pw = [_c(p) for p in Pw] + [np.zeros(1, np.complex128)]
        As = [np.zeros(1, np.complex128)] + [_c(a) for a in As]
        pw_ptrs = (C.c_void_p * L)(*[p.ctypes.data for p in Pw[:L]])
        as_ptrs = (C.c_void_p * L)(*[a.ctypes.data for a in As[:L]])
        ptr = lib().or_hier_import(N, _p(U), m, L, _p(Nl_a), _p(Bl_a), pw_ptrs, as_ptrs)
        return cls(ptr, N, U, m)

    def export(self):
        Pw = [np.zeros((self.Nl[l] ** 2 // 2, 2, 4), np.complex128) for l in range(self.L - 1)]
        As = [np.zeros((self.Nl[l] ** 2 // 2, 9, 2, 2), np.complex128) for l in range(1, self.L)]
        pw_ptrs = (C.c_void_p * self.L)(*([p.ctypes.data for p in Pw] + [0]))
        as_ptrs = (C.c_void_p * self.L)(*([0] + [a.ctypes.data for a in As]))
        _chk(lib().or_hier_export(self._h, pw_ptrs, as_ptrs), "hier_export")
        return Pw, As

    def close(self):
        if self._h:
            lib().or_hier_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def n(self, l):
        return self.Nl[l] ** 2 // 2 * 2

    def dense(self, l, which=0):
        rows = self.n(l)
        cols = self.n(l + 1) if which == 1 else rows
        out = np.zeros((rows, cols), np.complex128)
        _chk(lib().or_hier_level_dense(self._h, l, which, _p(out)), "level_dense")
        return out

    def agg_galerkin(self, l, B, k, Q):
        """Ac [nc][9][2k][2k]: P^H A_l P for the aggregation P of Q, as a
        9-point stencil of dense 2k x 2k blocks on the N_l / B lattice."""
        Q = _c(Q)
        nc = (self.Nl[l] // B) ** 2 // 2
        Ac = np.zeros((nc, 9, 2 * k, 2 * k), np.complex128)
        _chk(lib().or_agg_galerkin(self._h, l, B, k, _p(Q), _p(Ac)), "agg_galerkin")
        return Ac

    def apply(self, l, x):
        x = _c(x)
        y = np.zeros_like(x)
        _chk(lib().or_level_apply(self._h, l, _p(x), _p(y)), "apply")
        return y

    def kaczmarz(self, l, x, r, order=ORDER_COLOUR, sweeps=1, omega=1.0, perm=None):
        x, r = _c(x).copy(), _c(r).copy()
        pp = None if perm is None else _c(perm, np.int32)
        _chk(lib().or_kaczmarz(self._h, l, _p(x), _p(r), order, sweeps, omega,
                               None if pp is None else _p(pp)), "kaczmarz")
        return x, r

    def restrict(self, l, r):
        r = _c(r)
        out = np.zeros(self.n(l + 1), np.complex128)
        _chk(lib().or_restrict(self._h, l, _p(r), _p(out)), "restrict")
        return out

    def prolong(self, l, e, x):
        e, x = _c(e), _c(x).copy()
        _chk(lib().or_prolong(self._h, l, _p(e), _p(x)), "prolong")
        return x

    def coarsest_solve(self, f):
        f = _c(f)
        x = np.zeros_like(f)
        _chk(lib().or_coarsest_solve(self._h, _p(f), _p(x)), "coarsest")
        return x

    def cycle(self, f, l=0, nu1=2, nu2=2, gamma=1, order=ORDER_COLOUR):
        f = _c(f)
        x = np.zeros_like(f)
        _chk(lib().or_cycle(self._h, l, _p(f), _p(x), nu1, nu2, gamma, order), "cycle")
        return x

    def fgmres(self, b, x0=None, tol=1e-10, m=20, max_restarts=50, nu1=2, nu2=2, gamma=1,
               precond=1, gs_passes=2):
        """precond: 0 none, 1 / 2 / 3 the cycle with the 16-colour / tile /
        lexicographic Kaczmarz ordering; gs_passes: 1 = classical
        Gram-Schmidt, 2 = with one reorthogonalisation."""
        b = _c(b)
        x = np.zeros_like(b) if x0 is None else _c(x0).copy()
        it, rs, rr = C.c_int(), C.c_int(), C.c_double()
        st = _chk(lib().or_fgmres(self._h, _p(b), _p(x), tol, m, max_restarts, nu1, nu2, gamma,
                                  precond, gs_passes, C.byref(it), C.byref(rs), C.byref(rr)), "fgmres")
        return x, dict(status=st, iters=it.value, restarts=rs.value, relres=rr.value)

    def rho(self, x0, tol=1e-8, maxit=100, nu1=4, nu2=4, gamma=2, order=ORDER_COLOUR):
        """Sec. 4's estimate rho = |e^nu| / |e^(nu-1)| of the stand-alone
        cycle on A_0 x = 0 from x0; returns (rho, nu, [|e^0|, .., |e^nu|],
        met) where met says whether |e^nu| <= tol |e^0| was reached."""
        x0 = _c(x0)
        r, it = C.c_double(), C.c_int()
        hist = np.zeros(maxit + 1)
        st = _chk(lib().or_rho(self._h, _p(x0), tol, maxit, nu1, nu2, gamma, order, C.byref(r),
                               C.byref(it), _p(hist)), "rho")
        return r.value, it.value, hist[:it.value + 1], st == 0

    def solve(self, b, tol=1e-10, m=20, max_restarts=50, nu1=2, nu2=2, gamma=1, order=ORDER_COLOUR,
              gs_passes=2):
        b = _c(b)
        psi = np.zeros_like(b)
        it, rr = C.c_int(), C.c_double()
        st = _chk(lib().or_solve(self.N, _p(self.U), self.m, self._h, _p(b), _p(psi), tol, m,
                                 max_restarts, nu1, nu2, gamma, order, gs_passes, C.byref(it), C.byref(rr)),
                  "solve")
        return psi, dict(status=st, iters=it.value, relres=rr.value)
