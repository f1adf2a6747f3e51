"""The aggregation coarse space on the GPU (Sec. 4's "more interpolation
variables per coarse point", spin-split aggregation over the B x B cells of
the full coarsening, Galerkin operator of Sec. 3.5) against the oracle,
through the C ABI: construction of P and of the 2k x 2k block stencil from
test vectors, the block-stencil apply on CUDA cores (FP64 and FP32) and on
the tensor cores (tcgen05, TF32 operands split into high and low parts,
FP32 accumulation), restriction and prolongation.  Tolerances: FP64 1e-13
(construction) and 1e-14 (apply, transfers); FP32 and tensor cores 1e-6,
relative to the largest output."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected only on GPU machines
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1308_5992_gb300 import wilson_amg as W  # noqa: E402
from wl_inputs import workload, cgauss, rhs_batch  # noqa: E402

DEV = torch.device("cuda:0")


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).to(DEV)


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module")
def t64(O, tmp_path_factory):
    from oracle.hierfile import write_hierarchy
    w = workload("T64")
    h = O.Hierarchy.setup(w["N"], w["U"], w["m"], O.setup_params(w["blocks"], k_r=w["k"], k_e=w["k"],
                                                                  seed=w["seed"]))
    path = str(tmp_path_factory.mktemp("agg") / "t64.wlh")
    write_hierarchy(path, h)
    op = W.wilson_create(T(w["U"]), w["N"], w["m"])
    amg = W.amg_import(op, path, W.amg_params_default())
    return w, h, amg


def _vectors(n, k, seed):
    return np.stack([cgauss(seed, j, n) for j in range(k)])


@pytest.mark.parametrize("level,B,k", [(0, 4, 8), (0, 2, 4), (1, 2, 4)])
def test_construction_matches_oracle(O, t64, level, B, k):
    """agg_create from k test vectors: the orthonormal columns Q and the
    Galerkin block stencil P^H A_l P equal the oracle's."""
    w, h, amg = t64
    N = h.Nl[level]
    V = _vectors(N * N, k, 80 + level)
    g = W.agg_create(amg, level, B, k, T(V))
    nc = (N // B) ** 2 // 2
    Qg = torch.zeros(nc * 2 * B * B * k, dtype=torch.complex128, device=DEV)
    Ag = torch.zeros(nc * 9 * 4 * k * k, dtype=torch.complex128, device=DEV)
    W.agg_export(g, Qg, Ag)
    Qr = O.agg_interp(N, B, k, V)
    Ar = h.agg_galerkin(level, B, k, Qr)
    assert np.abs(Qg.cpu().numpy().reshape(Qr.shape) - Qr).max() <= 1e-12
    assert rel(Ag.cpu().numpy().reshape(Ar.shape), Ar) <= 1e-13


def test_rank_deficient_test_vectors_are_refused(t64):
    w, h, amg = t64
    V = _vectors(64 * 64, 4, 85)
    V[3] = V[0]
    with pytest.raises(W.WilsonAMGError) as e:
        W.agg_create(amg, 0, 4, 4, T(V))
    assert e.value.code == W.WL_EINVAL and "rank" in str(e.value)


@pytest.fixture(scope="module")
def imported(O, t64):
    """the oracle's aggregation operators on level 0 (B = 4, k = 8), imported"""
    w, h, amg = t64
    B, k = 4, 8
    Q = O.agg_interp(64, B, k, _vectors(64 * 64, k, 86))
    Ac = h.agg_galerkin(0, B, k, Q)
    g = W.agg_import(amg, 0, B, k, T(Q), T(Ac))
    return Q, Ac, g


@pytest.mark.parametrize("nrhs", [1, 5, 64, 70])
def test_apply_matches_oracle(O, imported, nrhs):
    """y = Ac x on every kernel, against the oracle's block-stencil apply;
    70 right-hand sides take a full and a ragged chunk of 64."""
    Q, Ac, g = imported
    Nc, K2 = 16, 16
    x = np.stack([cgauss(87, r, g.nc * K2) for r in range(nrhs)])
    ref = np.stack([O.agg_apply(Nc, 8, Ac, x[r]) for r in range(nrhs)])
    for kernel, tol in ((W.WL_AGG_FP64, 1e-14), (W.WL_AGG_FP32, 1e-6), (W.WL_AGG_TC, 1e-6)):
        y = torch.full((nrhs, g.nc * K2), float("nan"), dtype=torch.complex128, device=DEV)
        W.agg_apply(g, T(x), y, nrhs, kernel)
        err = rel(y.cpu().numpy(), ref)
        assert err <= tol, (kernel, nrhs, err)


def _round_tf32(a):
    """complex128 -> nearest float32 -> nearest TF32 (10 explicit mantissa
    bits, ties away from zero), as complex128"""
    def r(v):
        u = np.ascontiguousarray(v.astype(np.float32)).view(np.uint32).astype(np.uint64)
        u = (u + 0x1000) & 0xFFFFE000
        return u.astype(np.uint32).view(np.float32).astype(np.float64)
    return r(a.real) + 1j * r(a.imag)


def test_single_term_tf32_apply(O, t64, imported):
    """WL_AGG_TC1 multiplies the TF32-rounded operands once: on an operator
    and vectors whose entries are TF32 numbers every product is exact, so it
    matches the oracle to FP32 accumulation (1e-6); on general operands it
    stays within TF32 rounding (5e-3)."""
    w, h, amg = t64
    Q, Ac, g = imported
    nrhs = 64
    x = np.stack([cgauss(94, r, g.nc * 16) for r in range(nrhs)])
    y = torch.zeros((nrhs, g.nc * 16), dtype=torch.complex128, device=DEV)
    W.agg_apply(g, T(x), y, nrhs, W.WL_AGG_TC1)
    ref = np.stack([O.agg_apply(16, 8, Ac, x[r]) for r in range(nrhs)])
    assert rel(y.cpu().numpy(), ref) <= 5e-3
    Ar, xr = _round_tf32(Ac), _round_tf32(x)
    gr = W.agg_import(amg, 0, 4, 8, T(Q), T(Ar))
    W.agg_apply(gr, T(xr), y, nrhs, W.WL_AGG_TC1)
    ref = np.stack([O.agg_apply(16, 8, Ar, xr[r]) for r in range(nrhs)])
    assert rel(y.cpu().numpy(), ref) <= 1e-6


def test_tensor_core_apply_twice_in_a_row(imported):
    """Two launches in a row (tensor memory allocated, freed and allocated
    again; the pipeline's barriers start from their initial phase) give the
    same bits."""
    Q, Ac, g = imported
    x = T(np.stack([cgauss(88, r, g.nc * 16) for r in range(64)]))
    y1, y2 = torch.zeros_like(x), torch.zeros_like(x)
    W.agg_apply(g, x, y1, 64, W.WL_AGG_TC)
    W.agg_apply(g, x, y2, 64, W.WL_AGG_TC)
    assert torch.equal(y1, y2)


def test_restrict_prolong_match_oracle(O, imported):
    Q, Ac, g = imported
    nrhs = 3
    r = np.stack([cgauss(89, j, 64 * 64) for j in range(nrhs)])
    fc = torch.zeros((nrhs, g.nc * 16), dtype=torch.complex128, device=DEV)
    W.agg_restrict(g, T(r), fc, nrhs)
    ref = np.stack([O.agg_restrict(64, 4, 8, Q, r[j]) for j in range(nrhs)])
    assert rel(fc.cpu().numpy(), ref) <= 1e-14
    e = np.stack([cgauss(90, j, g.nc * 16) for j in range(nrhs)])
    x0 = np.stack([cgauss(91, j, 64 * 64) for j in range(nrhs)])
    x = T(x0)
    W.agg_prolong(g, T(e), x, nrhs)
    ref = np.stack([O.agg_prolong(64, 4, 8, Q, e[j], x0[j]) for j in range(nrhs)])
    assert rel(x.cpu().numpy(), ref) <= 1e-14


def test_full_size_tensor_core_apply(O):
    """The benchmark's size: the 512 x 512 lattice of the batched workload,
    4 x 4 aggregates with k = 8 (8192 coarse sites, 16 x 16 blocks), 64
    right-hand sides.  The GPU builds the operator from relaxed-free random
    test vectors; the tensor-core apply matches the oracle's apply of the
    exported operator on four sampled right-hand sides (1e-6) and the GPU's
    FP64 apply on all of them."""
    w = workload("C4")
    N = w["N"]
    op = W.wilson_create(T(w["U"]), N, w["m"])
    p = W.amg_params_default(k_r=4, k_e=4, seed=1, setup_mu=(2, 1))
    p.levels = len(w["blocks"]) + 1
    for l, b in enumerate(w["blocks"]):
        p.block[l] = b
    amg = W.amg_setup(op, p)
    k, B = 8, 4
    g = W.agg_create(amg, 0, B, k, T(_vectors(N * N, k, 92)))
    assert g.nc == 8192
    Ag = torch.zeros(g.nc * 9 * 256, dtype=torch.complex128, device=DEV)
    Qg = torch.zeros(g.nc * 2 * 16 * k, dtype=torch.complex128, device=DEV)
    W.agg_export(g, Qg, Ag)
    Ac = Ag.cpu().numpy().reshape(g.nc, 9, 16, 16)
    nrhs = 64
    x = T(np.stack([cgauss(93, r, g.nc * 16) for r in range(nrhs)]))
    y_tc, y64 = torch.zeros_like(x), torch.zeros_like(x)
    W.agg_apply(g, x, y_tc, nrhs, W.WL_AGG_TC)
    W.agg_apply(g, x, y64, nrhs, W.WL_AGG_FP64)
    yt, yd = y_tc.cpu().numpy(), y64.cpu().numpy()
    assert rel(yt, yd) <= 1e-6
    xh = x.cpu().numpy()
    for r in (0, 17, 40, 63):
        ref = O.agg_apply(N // B, k, Ac, xh[r])
        assert rel(yt[r], ref) <= 1e-6, r
        assert rel(yd[r], ref) <= 1e-13, r
