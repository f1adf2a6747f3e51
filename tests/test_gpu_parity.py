"""GPU-versus-oracle parity of every solve-phase step, called through the C
ABI (binding paper_1308_5992_gb300.wilson_amg).  Tolerances: FP64 matvec
1e-14 relative, FP32 1e-6; one Kaczmarz sweep 1e-13 (FP64) and 1e-6 (FP32,
from the FP32 values of the inputs); one FP64 cycle on a shared
(oracle-built) hierarchy 1e-12; final solutions 1e-10 relative error
against the oracle."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected only on GPU machines
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1308_5992_gb300 import wilson_amg as W  # noqa: E402
from wl_inputs import workload, rhs_batch, cgauss  # noqa: E402

DEV = torch.device("cuda:0")


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).to(DEV)


def H(t):
    return t.cpu().numpy()


def _round32(a):
    """complex128 -> the nearest complex64 -> complex128"""
    return np.asarray(a).astype(np.complex64).astype(np.complex128)


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module")
def ops():
    cache = {}

    def get(name):
        if name not in cache:
            w = workload(name)
            cache[name] = (w, W.wilson_create(T(w["U"]), w["N"], w["m"]))
        return cache[name]
    return get


@pytest.fixture(scope="module")
def shared(O, ops, tmp_path_factory):
    """GPU hierarchies imported from oracle-built hierarchy files."""
    from oracle.hierfile import write_hierarchy
    cache = {}

    def get(name):
        if name not in cache:
            w, op = ops(name)
            p = O.setup_params(w["blocks"], k_r=w["k"], k_e=w["k"], seed=w["seed"])
            h = O.Hierarchy.setup(w["N"], w["U"], w["m"], p)
            path = str(tmp_path_factory.mktemp("h") / ("%s.wlh" % name))
            write_hierarchy(path, h)
            amg = W.amg_import(op, path, W.amg_params_default(zero_guess=1))
            cache[name] = (w, op, h, amg, path)
        return cache[name]
    return get


# ------------------------------------------------------------- operators
@pytest.mark.parametrize("name,nrhs", [("T16", 1), ("T32", 3), ("T64", 5), ("C2", 2)])
def test_dhat_and_d_apply(O, ops, name, nrhs):
    w, op = ops(name)
    N, U, m = w["N"], w["U"], w["m"]
    x = np.stack([cgauss(10 + r, 1, N * N) for r in range(nrhs)])
    ref = np.stack([O.dhat_apply(N, U, m, x[r]) for r in range(nrhs)])
    for prec, tol in ((W.WL_FP64, 1e-14), (W.WL_FP32, 1e-6)):
        y = torch.zeros_like(T(x))
        W.wl_apply(op, W.WL_OP_DHAT, T(x), y, nrhs, prec)
        assert rel(H(y), ref) <= tol, (prec, rel(H(y), ref))
    psi = np.stack([cgauss(20 + r, 1, 2 * N * N).reshape(N, N, 2) for r in range(nrhs)])
    refD = np.stack([O.wilson_apply(N, U, m, psi[r].reshape(-1)).reshape(N, N, 2) for r in range(nrhs)])
    refZ = np.stack([O.z_apply(N, U, m, psi[r]) for r in range(nrhs)])
    for prec, tol in ((W.WL_FP64, 1e-14), (W.WL_FP32, 1e-6)):
        y = torch.zeros_like(T(psi))
        W.wl_apply(op, W.WL_OP_D, T(psi), y, nrhs, prec)
        assert rel(H(y), refD) <= tol
        z = torch.zeros_like(T(psi))
        W.wl_apply(op, W.WL_OP_Z, T(psi), z, nrhs, prec)  # Z = Gamma5 D (Thm. 3.1)
        assert rel(H(z), refZ) <= tol
        g5y = H(y)
        g5y[..., 1] *= -1
        assert np.array_equal(H(z), g5y)  # an exact sign flip of the D result


@pytest.mark.parametrize("name,nrhs", [("T32", 1), ("T64", 3)])
def test_eo_reduce_reconstruct(O, ops, name, nrhs):
    w, op = ops(name)
    N, U, m = w["N"], w["U"], w["m"]
    b = rhs_batch(N, nrhs, 7)
    bh = torch.zeros((nrhs, N * N), dtype=torch.complex128, device=DEV)
    W.wl_eo_reduce(op, T(b), bh, nrhs)
    ref = np.stack([O.eo_reduce(N, U, m, b[r]) for r in range(nrhs)])
    assert rel(H(bh), ref) <= 1e-14
    xe = np.stack([cgauss(30 + r, 2, N * N) for r in range(nrhs)])
    psi = torch.zeros_like(T(b))
    W.wl_eo_reconstruct(op, T(b), T(xe), psi, nrhs)
    refp = np.stack([O.eo_reconstruct(N, U, m, b[r], xe[r]) for r in range(nrhs)])
    assert rel(H(psi), refp) <= 1e-14


# ------------------------------------------------- per-level cycle steps
@pytest.mark.parametrize("name,nrhs", [("T64", 2), ("C1", 2), ("T64", 16), ("C2", 8), ("C2", 37)])
def test_level_apply(shared, name, nrhs):
    """Level operators against the oracle; batches of 8 or more on grids of
    64 and up take the shared-memory tiled stencil (chunks of 8 / 16 / 32,
    ragged and odd counts), which must equal the one-site-per-thread kernel
    bit for bit (checked against single right-hand-side applies)."""
    w, op, h, amg, _ = shared(name)
    for l in range(h.L):
        n = h.n(l)
        x = np.stack([cgauss(40 + l, r, n) for r in range(nrhs)])
        ref = np.stack([h.apply(l, x[r]) for r in range(nrhs)])
        for prec, tol in ((W.WL_FP64, 1e-14), (W.WL_FP32, 1e-6)):
            y = torch.zeros_like(T(x))
            W.amg_level_apply(amg, l, T(x), y, nrhs, prec)
            assert rel(H(y), ref) <= tol, (l, prec, rel(H(y), ref))
            if nrhs >= 8:
                for r in (0, nrhs - 1):
                    y1 = torch.zeros_like(T(x[r:r + 1]))
                    W.amg_level_apply(amg, l, T(x[r:r + 1]), y1, 1, prec)
                    assert np.array_equal(H(y1)[0], H(y)[r]), (l, prec, r)


@pytest.mark.parametrize("name,nrhs,form", [("T64", 3, 1), ("T64", 3, 2), ("T64", 1, 1), ("T64", 1, 2),
                                            ("C1", 3, 0), ("C2", 1, 1), ("C2", 5, 2)])
def test_kaczmarz_sweep(O, shared, name, nrhs, form):
    """One multicolour sweep: GPU (row/gamma5 form) vs oracle (true columns),
    per-colour launches (form 1) and the cooperative single launch (form 2),
    thread-per-item (nrhs > 1) and warp-per-site (nrhs = 1) kernels."""
    w, op, h, _, path = shared(name)
    amg = W.amg_import(op, path, W.amg_params_default(zero_guess=1, sweep_kernel=form))
    for l in range(h.L - 1):
        n = h.n(l)
        f = np.stack([cgauss(50 + l, r, n) for r in range(nrhs)])
        x0 = 0.1 * np.stack([cgauss(60 + l, r, n) for r in range(nrhs)])
        r0 = np.stack([f[r] - h.apply(l, x0[r]) for r in range(nrhs)])
        for prec, tol in ((W.WL_FP64, 1e-13), (W.WL_FP32, 1e-6)):
            # FP32: the oracle starts from the FP32 values the kernel reads
            xi, ri = (x0, r0) if prec == W.WL_FP64 else (_round32(x0), _round32(r0))
            ref = [h.kaczmarz(l, xi[r], ri[r], order=O.ORDER_COLOUR, sweeps=1) for r in range(nrhs)]
            xr, rr = np.stack([a for a, _ in ref]), np.stack([b for _, b in ref])
            xg, rg = T(xi), T(ri)
            W.amg_kaczmarz(amg, l, xg, rg, nrhs, 1, prec)
            assert rel(H(xg), xr) <= tol, (l, prec, rel(H(xg), xr))
            assert rel(H(rg), rr) <= tol, (l, prec, rel(H(rg), rr))


@pytest.mark.parametrize("name,nrhs", [("T64", 1), ("T64", 3), ("T64", 16), ("C2", 40), ("C2", 19), ("C2", 1)])
def test_kaczmarz_tile_sweep(O, shared, name, nrhs):
    """Tile-coloured sweep (8x8 tiles, shared-memory kernel) against the
    oracle's tile order; grids below 64 keep the 16-colour order."""
    w, op, h, _, path = shared(name)
    amg = W.amg_import(op, path, W.amg_params_default(zero_guess=1, kacz_order=1))
    for l in range(h.L - 1):
        n = h.n(l)
        f = np.stack([cgauss(150 + l, r, n) for r in range(nrhs)])
        x0 = 0.1 * np.stack([cgauss(160 + l, r, n) for r in range(nrhs)])
        r0 = np.stack([f[r] - h.apply(l, x0[r]) for r in range(nrhs)])
        for prec, tol in ((W.WL_FP64, 1e-13), (W.WL_FP32, 1e-6)):
            xi, ri = (x0, r0) if prec == W.WL_FP64 else (_round32(x0), _round32(r0))
            ref = [h.kaczmarz(l, xi[r], ri[r], order=O.ORDER_TILE, sweeps=2) for r in range(nrhs)]
            xr, rr = np.stack([a for a, _ in ref]), np.stack([b for _, b in ref])
            xg, rg = T(xi), T(ri)
            W.amg_kaczmarz(amg, l, xg, rg, nrhs, 2, prec)
            assert rel(H(xg), xr) <= tol, (l, prec, rel(H(xg), xr))
            assert rel(H(rg), rr) <= tol, (l, prec, rel(H(rg), rr))


@pytest.mark.parametrize("order", [0, 1])
def test_sweep_forms_agree_and_autotuner(O, shared, order):
    """Every launch form of a Kaczmarz sweep computes the same numbers in the
    same order: per-colour launches, the cooperative launch and the
    autotuner's choice give bitwise-equal x and r; after the first cycle of a
    batch width every non-coarsest level has a measured form."""
    w, op, h, _, path = shared("C2")
    nrhs, prec = 4, W.WL_FP32
    outs = {}
    for sk in (1, 2, 0):
        amg = W.amg_import(op, path, W.amg_params_default(zero_guess=1, sweep_kernel=sk, kacz_order=order,
                                                          precision=prec))
        if sk == 0:
            f = T(np.stack([cgauss(180, r, h.n(0)) for r in range(nrhs)]))
            W.amg_cycle(amg, f, torch.zeros_like(f), nrhs, prec)
            for l in range(h.L - 1):
                form, param, us = W.amg_sweep_form(amg, l, nrhs, prec)
                assert us > 0 and form in (0, 1, 2, 3), (l, form, param, us)
                assert (form == 2) == (order == 1 and h.Nl[l] >= 64)
        res = []
        for l in range(h.L - 1):
            n = h.n(l)
            x0 = 0.1 * np.stack([cgauss(190 + l, r, n) for r in range(nrhs)])
            r0 = np.stack([cgauss(200 + l, r, n) for r in range(nrhs)])
            xg, rg = T(x0), T(r0)
            W.amg_kaczmarz(amg, l, xg, rg, nrhs, 2, prec)
            res.append((H(xg), H(rg)))
        outs[sk] = res
        amg.close()
    for sk in (2, 0):
        for l, ((xa, ra), (xb, rb)) in enumerate(zip(outs[1], outs[sk])):
            assert np.array_equal(xa, xb) and np.array_equal(ra, rb), (sk, l)


def test_pin_sweep_form(shared):
    """A pinned launch form survives the autotuner (the other levels are
    still tuned); forms of the other ordering and the coarsest level are
    refused."""
    w, op, h, _, path = shared("C2")
    nrhs, prec = 4, W.WL_FP32
    amg = W.amg_import(op, path, W.amg_params_default(zero_guess=1, kacz_order=1, precision=prec))
    W.amg_pin_sweep_form(amg, 0, nrhs, prec, 2, 16 | 8 << 8)
    f = T(np.stack([cgauss(185, r, h.n(0)) for r in range(nrhs)]))
    W.amg_cycle(amg, f, torch.zeros_like(f), nrhs, prec)
    assert W.amg_sweep_form(amg, 0, nrhs, prec)[:2] == (2, 16 | 8 << 8)
    assert W.amg_sweep_form(amg, 1, nrhs, prec)[2] > 0
    for level, form, param in ((0, 0, 0), (1, 2, 32), (h.L - 1, 0, 0)):
        with pytest.raises(W.WilsonAMGError):
            W.amg_pin_sweep_form(amg, level, nrhs, prec, form, param)
    amg.close()


@pytest.mark.parametrize("order,nrhs", [(0, 5), (1, 5), (1, 40)])
def test_every_launch_form_agrees_bitwise(shared, order, nrhs):
    """Each launch form of the sweep (per-colour, cooperative with several
    block counts, block-resident on small levels; tile kernel with
    right-hand-side chunks 8 / 16 / 32 and one or two right-hand sides per
    thread, with scalar or paired FP32 FMAs, one tile per block or
    persistent, or each item split over a pair of lanes) gives
    bit-identical x and r."""
    w, op, h, _, path = shared("C2")
    prec = W.WL_FP32
    amg = W.amg_import(op, path, W.amg_params_default(zero_guess=1, kacz_order=order, precision=prec))
    for l in range(h.L - 1):
        if order == 1 and h.Nl[l] < 64:
            continue
        n = h.n(l)
        if order == 0:
            forms = [(0, 0), (1, 1), (1, 7), (1, 64)]
            # block-resident sweeps where x and r of the chunk fit 200 KB of shared memory
            forms += [(3, rc) for rc in (1, 2, 4) if rc <= nrhs and n * 2 * 8 * rc <= 200 * 1024]
            # and with the stencil rows and denominators staged in shared memory as well
            forms += [(3, rc | 1 << 8) for rc in (1, 2, 4)
                      if rc <= nrhs and n * 2 * 8 * rc * 2 + n * 36 * 8 + n * 2 * 4 <= 227 * 1024]
        else:
            forms = [(2, 8), (2, 16), (2, 16 | 2 << 8), (2, 32), (2, 32 | 2 << 8), (2, 8 | 8 << 8),
                     (2, 16 | 8 << 8), (2, 32 | 8 << 8),
                     # the persistent form (double-buffered r by bulk copies) where chunks are full,
                     # else the one-tile-per-block form
                     (2, 8 | 1 << 12), (2, 16 | 8 << 8 | 1 << 12), (2, 32 | 1 << 12), (2, 32 | 8 << 8 | 1 << 12),
                     # each item split over a pair of lanes
                     (2, 8 | 8 << 8 | 1 << 13), (2, 16 | 8 << 8 | 1 << 13), (2, 32 | 8 << 8 | 1 << 13)]
        x0 = 0.1 * np.stack([cgauss(210 + l, r, n) for r in range(nrhs)])
        r0 = np.stack([cgauss(220 + l, r, n) for r in range(nrhs)])
        outs = []
        for form, param in forms:
            xg, rg = T(x0), T(r0)
            W.amg_kaczmarz_form(amg, l, xg, rg, nrhs, 2, prec, form, param)
            outs.append((H(xg), H(rg)))
        for f, (xa, ra) in zip(forms[1:], outs[1:]):
            assert np.array_equal(xa, outs[0][0]) and np.array_equal(ra, outs[0][1]), (l, f)
    z = np.zeros((nrhs, h.n(0)))
    with pytest.raises(W.WilsonAMGError):  # a form of the other ordering
        W.amg_kaczmarz_form(amg, 0, T(z), T(z), nrhs, 1, prec, 2 if order == 0 else 0, 8)


def test_tile_ordered_solve(O, shared):
    w, op, h, _, path = shared("C2")
    amg = W.amg_import(op, path, W.amg_params_default(zero_guess=1, kacz_order=1))
    b = rhs_batch(w["N"], 2, 17)
    psi = torch.zeros_like(T(b))
    rc, info = W.amg_solve(amg, T(b), psi, 2, 1e-13)
    assert rc == W.WL_OK
    for q in range(2):
        ref, oi = h.solve(b[q], tol=1e-13, order=O.ORDER_TILE)
        assert np.linalg.norm(H(psi[q]) - ref) / np.linalg.norm(ref) <= 1e-10
        assert abs(info[q]["iters"] - oi["iters"]) <= 2, (info[q], oi)


@pytest.mark.parametrize("cycle", [W.WL_CYCLE_V, W.WL_CYCLE_W])
def test_rho_protocol(O, shared, cycle):
    """Sec. 4's convergence estimate rho = |e^nu| / |e^(nu-1)| of the
    stand-alone cycle on Dhat x = 0, stopped at |e^nu| <= 1e-8 |e^0|:
    GPU FP64 cycle against the oracle's on a shared hierarchy (error norms
    1e-9 relative, same stopping iteration); the FP32 cycle inside the FP64
    iteration gives the same rate and stopping point within rounding."""
    w, op, h, _, path = shared("C2")
    n, R = h.n(0), 3
    x0 = np.stack([cgauss(170, r, n) for r in range(R)])
    refs = [h.rho(x0[r], tol=1e-8, maxit=100, nu1=4, nu2=4, gamma=cycle + 1) for r in range(R)]
    for prec in (W.WL_FP64, W.WL_FP32):
        amg = W.amg_import(op, path, W.amg_params_default(cycle=cycle, nu_pre=4, nu_post=4, precision=prec))
        x = torch.zeros_like(T(x0))
        rc, rho, it, hist = W.amg_rho(amg, T(x0), x, R, 1e-8, 100, hist=True)
        assert rc == W.WL_OK
        for r in range(R):
            rr, ir, hr, met = refs[r]
            assert met
            if prec == W.WL_FP64:
                assert it[r] == ir, (r, it[r], ir)
                assert np.abs(hist[r, :ir + 1] / hr - 1).max() <= 1e-9
                assert abs(rho[r] - rr) <= 1e-9 * rr
            else:
                k = min(it[r], ir)
                assert abs(int(it[r]) - ir) <= 1, (r, it[r], ir)
                assert np.abs(hist[r, :k + 1] / hr[:k + 1] - 1).max() <= 1e-3
                assert abs(rho[r] - rr) <= 0.05 * rr
        amg.close()


def test_rho_divergent_cycle(O, ops, tmp_path):
    """A cycle whose coarse correction is scaled up diverges: GPU and oracle
    stop at the last finite error norm with the same ratio (the definition in
    Sec. 4 presumes convergence); the GPU call reports WL_NOT_CONVERGED."""
    from oracle.hierfile import write
    w, op = ops("C1")
    h = O.Hierarchy.setup(w["N"], w["U"], w["m"], O.setup_params(w["blocks"], k_r=w["k"], k_e=w["k"],
                                                                  seed=w["seed"]))
    Pw, As = h.export()
    As = [a * 1e-6 for a in As]
    hb = O.Hierarchy.from_arrays(h.N, h.U, h.m, h.Nl, h.Bl[:-1], Pw, As)
    path = str(tmp_path / "scaled.wlh")
    write(path, h.U, h.m, h.Nl, h.Bl, Pw, As)
    amg = W.amg_import(op, path, W.amg_params_default(nu_pre=1, nu_post=1))
    x0 = cgauss(4, 1, h.n(0))
    rr, ir, hr, met = hb.rho(x0, tol=1e-8, maxit=100, nu1=1, nu2=1, gamma=1)
    assert not met and rr > 1e4
    rc, rho, it, hist = W.amg_rho(amg, T(x0[None]), T(np.zeros((1, h.n(0)))), 1, 1e-8, 100, hist=True)
    assert rc == W.WL_NOT_CONVERGED
    assert abs(int(it[0]) - ir) <= 1 and np.isfinite(rho[0])
    k = min(int(it[0]), ir)
    assert np.abs(hist[0, :k + 1] / hr[:k + 1] - 1).max() <= 1e-6
    assert abs(rho[0] - rr) <= 1e-3 * rr


@pytest.mark.parametrize("name", ["T64", "C1"])
def test_transfers_and_coarsest(shared, name):
    w, op, h, amg, _ = shared(name)
    for l in range(h.L - 1):
        nf, nc = h.n(l), h.n(l + 1)
        r = np.stack([cgauss(70 + l, q, nf) for q in range(2)])
        ref = np.stack([h.restrict(l, r[q]) for q in range(2)])
        fc = torch.zeros((2, nc), dtype=torch.complex128, device=DEV)
        W.amg_restrict(amg, l, T(r), fc, 2, W.WL_FP64)
        assert rel(H(fc), ref) <= 1e-14
        e = np.stack([cgauss(80 + l, q, nc) for q in range(2)])
        x = np.stack([cgauss(90 + l, q, nf) for q in range(2)])
        refp = np.stack([h.prolong(l, e[q], x[q]) for q in range(2)])
        xg = T(x)
        W.amg_prolong(amg, l, T(e), xg, 2, W.WL_FP64)
        assert rel(H(xg), refp) <= 1e-14
    nc = h.n(h.L - 1)
    f = np.stack([cgauss(99, q, nc) for q in range(3)])
    ref = np.stack([h.coarsest_solve(f[q]) for q in range(3)])
    xg = torch.zeros_like(T(f))
    W.amg_coarsest(amg, T(f), xg, 3)
    assert rel(H(xg), ref) <= 1e-11


@pytest.mark.parametrize("name", ["T64", "C1", "C2"])
def test_cycle(O, shared, name):
    """One V(2,2) cycle on the shared hierarchy, FP64 1e-12 (FP32 1e-5)."""
    w, op, h, amg, _ = shared(name)
    n = h.n(0)
    f = np.stack([cgauss(123, q, n) for q in range(2)])
    ref = np.stack([h.cycle(f[q], nu1=2, nu2=2, gamma=1) for q in range(2)])
    for prec, tol in ((W.WL_FP64, 1e-12), (W.WL_FP32, 1e-5)):
        xg = torch.zeros_like(T(f))
        W.amg_cycle(amg, T(f), xg, 2, prec)
        assert rel(H(xg), ref) <= tol, (prec, rel(H(xg), ref))


@pytest.mark.parametrize("name", ["T64", "C2"])
def test_w_cycle(O, shared, name):
    """The W(4,4) cycle of Sec. 4 (gamma = 2 recursion), FP64 1e-12."""
    w, op, h, _, path = shared(name)
    amg = W.amg_import(op, path, W.amg_params_default(zero_guess=1, cycle=W.WL_CYCLE_W, nu_pre=4, nu_post=4))
    n = h.n(0)
    f = np.stack([cgauss(321, q, n) for q in range(2)])
    ref = np.stack([h.cycle(f[q], nu1=4, nu2=4, gamma=2) for q in range(2)])
    xg = torch.zeros_like(T(f))
    W.amg_cycle(amg, T(f), xg, 2, W.WL_FP64)
    assert rel(H(xg), ref) <= 1e-12, rel(H(xg), ref)


@pytest.mark.parametrize("cycle,nrhs", [(W.WL_CYCLE_V, 3), (W.WL_CYCLE_W, 3), (W.WL_CYCLE_V, 24)])
def test_tile_ordered_cycle(O, shared, cycle, nrhs):
    """Whole cycles with the tile-coloured ordering (tile kernel on the 128x128
    grid, 16 colours below) against the oracle's tile-ordered cycle: FP64
    1e-12, FP32 1e-5; 24 right-hand sides take the tiled stencil and the
    autotuned launch forms."""
    w, op, h, _, path = shared("C2")
    amg = W.amg_import(op, path, W.amg_params_default(zero_guess=1, cycle=cycle, nu_pre=4, nu_post=4,
                                                      kacz_order=1))
    n = h.n(0)
    f = np.stack([cgauss(331, q, n) for q in range(nrhs)])
    ref = np.stack([h.cycle(f[q], nu1=4, nu2=4, gamma=cycle + 1, order=O.ORDER_TILE) for q in range(nrhs)])
    for prec, tol in ((W.WL_FP64, 1e-12), (W.WL_FP32, 1e-5)):
        xg = torch.zeros_like(T(f))
        W.amg_cycle(amg, T(f), xg, nrhs, prec)
        assert rel(H(xg), ref) <= tol, (prec, rel(H(xg), ref))


# ---------------------------------------------------------- full solves
@pytest.mark.parametrize("name", ["T64", "C1", "C2"])
def test_fgmres_and_solve_match_oracle(shared, name):
    w, op, h, amg, _ = shared(name)
    N = w["N"]
    b = rhs_batch(N, 2, 11)
    psi = torch.zeros_like(T(b))
    rc, info = W.amg_solve(amg, T(b), psi, 2, 1e-13)
    assert rc == W.WL_OK, info
    for q in range(2):
        ref, oi = h.solve(b[q], tol=1e-13)
        err = np.linalg.norm(H(psi[q]) - ref) / np.linalg.norm(ref)
        assert err <= 1e-10, (q, err)
        assert abs(info[q]["iters"] - oi["iters"]) <= 2, (info[q], oi)


@pytest.mark.parametrize("prec", [W.WL_FP32, W.WL_FP32_BF16])
@pytest.mark.parametrize("order,matvec", [(0, 0), (1, 1)])
def test_mixed_precision_solve(O, ops, shared, prec, order, matvec):
    """FP32 (or BF16-stored) cycle inside FP64 FGMRES with iterative
    refinement reaches the FP64 accuracy, with the 16-colour or the
    tile-coloured ordering and the FP64 or FP32 Arnoldi matvec."""
    w, op, h, _, path = shared("C2")
    amg = W.amg_import(op, path, W.amg_params_default(zero_guess=1, precision=prec, kacz_order=order,
                                                      arnoldi_matvec=matvec))
    b = rhs_batch(w["N"], 1, 12)
    psi = torch.zeros_like(T(b))
    rc, info = W.amg_solve(amg, T(b), psi, 1, 1e-13)
    assert rc == W.WL_OK and info[0]["true_relres"] <= 1e-13
    ref, _ = h.solve(b[0], tol=1e-13)
    assert np.linalg.norm(H(psi[0]) - ref) / np.linalg.norm(ref) <= 1e-10


@pytest.mark.parametrize("name,nrhs,order,passes", [("T64", 3, 0, 2), ("C2", 40, 1, 1), ("C2", 9, 1, 2)])
def test_double_float_gram_schmidt(O, shared, name, nrhs, order, passes):
    """gs_arith = 1 (Krylov basis, dots, updates and norms in double-float on
    the FP32 pipes): every right-hand side reaches the FP64 true residual
    1e-13 and the oracle's solution to 1e-10, with iteration counts within 2
    of the FP64 Gram-Schmidt on the same cycle.  40 right-hand sides take
    mdot launches of up to 8 dots and the tiled Arnoldi matvec; 3 and 9 the
    per-site one, one and two Gram-Schmidt passes."""
    w, op, h, _, path = shared(name)
    kw = dict(zero_guess=1, precision=W.WL_FP32, kacz_order=order, arnoldi_matvec=1, gs_passes=passes)
    a64 = W.amg_import(op, path, W.amg_params_default(gs_arith=0, **kw))
    adf = W.amg_import(op, path, W.amg_params_default(gs_arith=1, **kw))
    b = rhs_batch(w["N"], nrhs, 31)
    x64, xdf = torch.zeros_like(T(b)), torch.zeros_like(T(b))
    rc64, i64 = W.amg_solve(a64, T(b), x64, nrhs, 1e-13)
    rcdf, idf = W.amg_solve(adf, T(b), xdf, nrhs, 1e-13)
    assert rc64 == W.WL_OK and rcdf == W.WL_OK
    assert all(i["true_relres"] <= 1e-13 for i in idf)
    for q in range(nrhs):
        assert abs(idf[q]["iters"] - i64[q]["iters"]) <= 2, (q, idf[q], i64[q])
    for q in sorted({0, nrhs // 2, nrhs - 1}):
        ref, _ = h.solve(b[q], tol=1e-13, order=O.ORDER_TILE if order else O.ORDER_COLOUR)
        assert np.linalg.norm(H(xdf[q]) - ref) / np.linalg.norm(ref) <= 1e-10, q


def test_double_float_gram_schmidt_needs_an_fp32_matvec(ops):
    """gs_arith = 1 is refused with an FP64 cycle or an FP64 Arnoldi matvec."""
    w, op = ops("T64")
    for kw in (dict(precision=W.WL_FP64, arnoldi_matvec=1), dict(precision=W.WL_FP32, arnoldi_matvec=0)):
        with pytest.raises(W.WilsonAMGError) as e:
            W.amg_setup(op, W.amg_params_default(gs_arith=1, **kw))
        assert e.value.code == W.WL_EINVAL


def test_batch_equals_alone(shared):
    """Each right-hand side gives the same result alone and in a batch."""
    w, op, h, amg, _ = shared("T64")
    N = w["N"]
    b = rhs_batch(N, 7, 13)
    psi = torch.zeros_like(T(b))
    rc, info = W.amg_solve(amg, T(b), psi, 7, 1e-12)
    assert rc == W.WL_OK
    for q in (0, 3, 6):
        one = torch.zeros_like(T(b[q:q + 1]))
        W.amg_solve(amg, T(b[q:q + 1]), one, 1, 1e-12)
        assert np.linalg.norm(H(one[0]) - H(psi[q])) / np.linalg.norm(H(one[0])) <= 1e-10


@pytest.mark.parametrize("name,nb,order", [("T64", 40, 0), ("C2", 33, 1)])
def test_two_lane_solve(O, shared, name, nb, order):
    """amg_params.overlap: a batch of 40 (33) is solved as two halves of 20
    and 20 (17 and 16) on two streams at the same time (a second workspace
    viewing the same operators; with 33 the second lane's width has launch
    forms of its own, tuned on the first lane and handed over); every
    right-hand side matches the one-lane solve and the oracle's solve to
    1e-10, twice in a row (the second call reuses the second lane and its
    graphs).  The 33-wide case runs the tile-coloured sweeps."""
    w, op, h, _, path = shared(name)
    N = w["N"]
    p1 = W.amg_params_default(zero_guess=1, precision=W.WL_FP32, overlap=1, kacz_order=order)
    p0 = W.amg_params_default(zero_guess=1, precision=W.WL_FP32, overlap=0, kacz_order=order)
    a1, a0 = W.amg_import(op, path, p1), W.amg_import(op, path, p0)
    b = rhs_batch(N, nb, 15)
    x0 = torch.zeros_like(T(b))
    rc0, i0 = W.amg_solve(a0, T(b), x0, nb, 1e-13)
    assert rc0 == W.WL_OK
    h0 = (nb + 1) // 2
    for _ in range(2):
        x1 = torch.zeros_like(T(b))
        rc1, i1 = W.amg_solve(a1, T(b), x1, nb, 1e-13)
        assert rc1 == W.WL_OK and all(i["true_relres"] <= 1e-13 for i in i1)
        assert float((x1 - x0).abs().max() / x0.abs().max()) <= 1e-10
    for q in (0, h0 - 1, h0, nb - 1):
        ref, _ = h.solve(b[q], tol=1e-13, order=O.ORDER_TILE if order else O.ORDER_COLOUR)
        assert np.linalg.norm(H(x1[q]) - ref) / np.linalg.norm(ref) <= 1e-10, q


@pytest.mark.parametrize("overlap,nb,pinned,zero", [(0, 3, True, 1), (1, 40, True, 1), (1, 33, False, 0)])
def test_solve_with_host_buffers(shared, overlap, nb, pinned, zero):
    """amg_solve_host (b and x in host memory, copied by the library, one
    lane's copies beside the other lane's solve) gives the device call's
    solution bit for bit, from pinned or pageable memory, with a zero or a
    given initial guess."""
    w, op, h, _, path = shared("T64")
    N = w["N"]
    p = W.amg_params_default(zero_guess=zero, precision=W.WL_FP32, overlap=overlap, arnoldi_matvec=1, gs_arith=1)
    amg = W.amg_import(op, path, p)
    b = rhs_batch(N, nb, 41)
    x0 = 0.01 * rhs_batch(N, nb, 42)
    xd = T(x0)
    rcd, infd = W.amg_solve(amg, T(b), xd, nb, 1e-12)
    bh = torch.from_numpy(np.ascontiguousarray(b))
    xh = torch.from_numpy(np.ascontiguousarray(x0))
    if pinned:
        bh, xh = bh.pin_memory(), xh.pin_memory()
    rch, infh = W.amg_solve_host(amg, bh, xh, nb, 1e-12)
    assert rcd == rch == W.WL_OK
    assert [i["iters"] for i in infh] == [i["iters"] for i in infd]
    assert np.array_equal(xh.numpy(), H(xd))
    with pytest.raises(TypeError):
        W.amg_solve_host(amg, T(b), xh, nb, 1e-12)  # a device tensor


def test_fp64_fma_probe(shared):
    """wl_time_kernel's FP64 FMA probe (the check on the derived FP64 peak
    that the Gram-Schmidt roofline uses) runs and reports a rate below the
    unit-count bound at the top clock (152 SMs x 2 FMA x 2 flop x 2070 MHz,
    which a probe whose chains were optimised away would exceed) and above a
    tenth of it."""
    w, op, h, amg, path = shared("T64")
    ms = W.wl_time_kernel(amg, W.WL_K_FP64_FMA, 0, 1, W.WL_FP64, 3)
    nsm = torch.cuda.get_device_properties(DEV).multi_processor_count
    gflops = nsm * 8 * 256 * 8 * 4096 * 2 / (ms * 1e-3) / 1e9
    bound = nsm * 2 * 2 * 2.07
    assert 0.1 * bound <= gflops <= 1.02 * bound, (gflops, bound)


def test_gpu_setup_quality(O, ops):
    """The GPU bootstrap setup gives a preconditioner of the same quality as
    the oracle's (iterations within a band) and solutions to 1e-10."""
    w, op = ops("T64")
    p = W.amg_params_default(k_r=w["k"], k_e=w["k"], seed=w["seed"], zero_guess=1)
    for l, b in enumerate(w["blocks"]):
        p.block[l] = b
    p.levels = len(w["blocks"]) + 1
    amg = W.amg_setup(op, p)
    b = rhs_batch(w["N"], 1, 14)
    psi = torch.zeros_like(T(b))
    rc, info = W.amg_solve(amg, T(b), psi, 1, 1e-12)
    assert rc == W.WL_OK
    ho = O.Hierarchy.setup(w["N"], w["U"], w["m"],
                           O.setup_params(w["blocks"], k_r=w["k"], k_e=w["k"], seed=w["seed"]))
    ref, oi = ho.solve(b[0], tol=1e-13)
    assert np.linalg.norm(H(psi[0]) - ref) / np.linalg.norm(ref) <= 1e-9
    assert info[0]["iters"] <= 2 * oi["iters"] + 5, (info, oi)


def test_setup_independent_of_solve_options(ops, tmp_path):
    """The setup relaxes with the 16-colour ordering whatever the solve
    phase uses: hierarchies built with either Kaczmarz ordering, launch form
    or Arnoldi matvec precision are byte-identical files."""
    w, op = ops("T64")
    files = []
    for kw in (dict(), dict(kacz_order=1, arnoldi_matvec=1, sweep_kernel=1)):
        p = W.amg_params_default(k_r=w["k"], k_e=w["k"], seed=w["seed"], **kw)
        for l, b in enumerate(w["blocks"]):
            p.block[l] = b
        p.levels = len(w["blocks"]) + 1
        amg = W.amg_setup(op, p)
        path = str(tmp_path / ("h%d.wlh" % len(files)))
        W.amg_export(amg, path)
        files.append(open(path, "rb").read())
        amg.close()
    assert files[0] == files[1]


def test_gpu_super_v_setup_quality(O, ops):
    """Sec. 4.2's super-V setup on the GPU: the stand-alone W(4,4) cycle
    converges and GMRES(32) needs iterations within the band of the oracle's
    super-V setup of the same configuration; solutions match to 1e-9."""
    w, op = ops("C2")
    p = W.amg_params_default(k_r=w["k"], k_e=w["k"], seed=w["seed"], zero_guess=1, setup_cycle=1,
                             cycle=W.WL_CYCLE_W, nu_pre=4, nu_post=4, fgmres_m=32)
    for l, b in enumerate(w["blocks"]):
        p.block[l] = b
    p.levels = len(w["blocks"]) + 1
    amg = W.amg_setup(op, p)
    x0 = T(cgauss(4, 3, w["N"] ** 2)[None, :])
    rc, rho, nu, _ = W.amg_rho(amg, x0, torch.zeros_like(x0), 1, 1e-8, 100)
    assert rc == W.WL_OK and rho[0] < 0.9, (rho, nu)
    b = rhs_batch(w["N"], 1, 14)
    psi = torch.zeros_like(T(b))
    rc, info = W.amg_solve(amg, T(b), psi, 1, 1e-12)
    assert rc == W.WL_OK
    ho = O.Hierarchy.setup(w["N"], w["U"], w["m"], O.setup_params(w["blocks"], k_r=w["k"], k_e=w["k"],
                                                                  seed=w["seed"], super_v=True))
    ref, oi = ho.solve(b[0], tol=1e-13, m=32, nu1=4, nu2=4, gamma=2)
    assert np.linalg.norm(H(psi[0]) - ref) / np.linalg.norm(ref) <= 1e-9
    assert info[0]["iters"] <= 2 * oi["iters"] + 5, (info, oi)


def test_hierarchy_roundtrip_and_errors(shared, ops, tmp_path):
    w, op, h, amg, path = shared("T64")
    out = str(tmp_path / "x.wlh")
    W.amg_export(amg, out)
    amg2 = W.amg_import(op, out)
    assert W.amg_levels(amg2) == h.Nl
    data = bytearray(open(out, "rb").read())
    data[100] ^= 1
    bad = str(tmp_path / "bad.wlh")
    open(bad, "wb").write(bytes(data))
    with pytest.raises(W.WilsonAMGError) as e:
        W.amg_import(op, bad)
    assert e.value.code == W.WL_BAD_HIERARCHY
    w2, op2 = ops("C1")
    with pytest.raises(W.WilsonAMGError) as e:
        W.amg_import(op2, out)  # another operator
    assert e.value.code == W.WL_BAD_HIERARCHY
    nc = h.n(len(h.Nl) - 1)   # the coarsest level has no Kaczmarz sweep: the library refuses it
    with pytest.raises(W.WilsonAMGError) as e:
        W.amg_kaczmarz(amg, len(h.Nl) - 1, T(np.zeros(nc)), T(np.zeros(nc)), 1)
    assert e.value.code == W.WL_EINVAL


def test_degenerate_inputs(O, shared, ops):
    """Degenerate cases: a zero right-hand side in a batch converges at once
    to x = 0 without disturbing its batch mates; an initial guess that is
    already the solution stops with no iteration; empty or oversized
    batches and a vanishing diagonal c = m + 2 are rejected."""
    w, op, h, amg, path = shared("T64")
    N = w["N"]
    b = rhs_batch(N, 3, 31)
    b[1] = 0
    psi = torch.zeros_like(T(b))
    rc, info = W.amg_solve(amg, T(b), psi, 3, 1e-12)
    assert rc == W.WL_OK
    assert np.all(H(psi[1]) == 0) and info[1]["iters"] == 0 and info[1]["true_relres"] == 0
    for q in (0, 2):
        ref, _ = h.solve(b[q], tol=1e-13)
        assert np.linalg.norm(H(psi[q]) - ref) / np.linalg.norm(ref) <= 1e-10
    # the solution as initial guess: no iteration
    amg_g = W.amg_import(op, path, W.amg_params_default(zero_guess=0))
    ref, _ = h.solve(b[0], tol=1e-14)
    x0 = T(ref[None])
    rc, info = W.amg_solve(amg_g, T(b[:1]), x0, 1, 1e-10)
    assert rc == W.WL_OK and info[0]["iters"] == 0
    with pytest.raises(W.WilsonAMGError) as e:
        W.amg_solve(amg, T(b[:1]), psi[:1], 0, 1e-10)
    assert e.value.code == W.WL_EINVAL
    with pytest.raises(W.WilsonAMGError) as e:
        W.amg_rho(amg, T(np.zeros((257, h.n(0)))), T(np.zeros((257, h.n(0)))), 257, 1e-8, 10)
    assert e.value.code == W.WL_EINVAL
    with pytest.raises(W.WilsonAMGError) as e:
        W.wilson_create(T(w["U"]), N, -2.0)
    assert e.value.code == W.WL_EINVAL


def test_batch_above_the_launch_limit(shared):
    """amg_solve splits a call with more right-hand sides than one batched
    launch takes (256) into chunks; every right-hand side converges and
    matches its own single solve."""
    w, op, h, amg, _ = shared("T32")
    N, nrhs = w["N"], 300
    b = rhs_batch(N, nrhs, 41)
    psi = torch.zeros_like(T(b))
    rc, info = W.amg_solve(amg, T(b), psi, nrhs, 1e-11)
    assert rc == W.WL_OK and len(info) == nrhs
    assert max(i["true_relres"] for i in info) <= 1e-11
    for q in (0, 255, 256, 299):
        one = torch.zeros_like(T(b[q:q + 1]))
        W.amg_solve(amg, T(b[q:q + 1]), one, 1, 1e-11)
        assert np.linalg.norm(H(one[0]) - H(psi[q])) / np.linalg.norm(H(one[0])) <= 1e-8, q


def _round_bf16(a):
    """complex128 -> nearest float32 -> nearest bfloat16 (ties to even),
    returned as complex128: the rounding the library applies to stencils"""
    def r(x):
        u = np.ascontiguousarray(x.astype(np.float32)).view(np.uint32).astype(np.uint64)
        u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
        return u.astype(np.uint32).view(np.float32).astype(np.float64)
    return r(a.real) + 1j * r(a.imag)


def test_bf16_stencil_sweeps(O, ops, tmp_path):
    """BF16 storage: on a hierarchy whose coarse stencils and interpolation
    weights are already BF16 numbers (so every stored copy is exact), the
    BF16 coarse stencil apply, restriction, prolongation and the Kaczmarz
    sweeps of both orderings (the tile kernel on the 64x64 level) match the
    oracle's FP64 steps on the same operators to FP32 rounding."""
    from oracle.hierfile import write
    w, op = ops("T128")
    h = O.Hierarchy.setup(w["N"], w["U"], w["m"], O.setup_params(w["blocks"], k_r=w["k"], k_e=w["k"],
                                                                  seed=w["seed"]))
    Pw, As = h.export()
    Pw = [_round_bf16(p) for p in Pw]
    As = [_round_bf16(a) for a in As]
    hb = O.Hierarchy.from_arrays(h.N, h.U, h.m, h.Nl, h.Bl[:-1], Pw, As)
    path = str(tmp_path / "bf16.wlh")
    write(path, h.U, h.m, h.Nl, h.Bl, Pw, As)
    nrhs = 6
    # BF16-stored coarse stencil apply and BF16-stored transfers
    amg = W.amg_import(op, path, W.amg_params_default(zero_guess=1))
    for l in range(h.L):
        n = h.n(l)
        x = np.stack([cgauss(250 + l, r, n) for r in range(nrhs)])
        if l >= 1:
            y = torch.zeros_like(T(x))
            W.amg_level_apply(amg, l, T(x), y, nrhs, W.WL_FP32_BF16)
            ref = np.stack([hb.apply(l, x[r]) for r in range(nrhs)])
            assert rel(H(y), ref) <= 1e-6, ("apply", l, rel(H(y), ref))
        if l + 1 < h.L:
            nc = h.n(l + 1)
            fc = torch.zeros((nrhs, nc), dtype=torch.complex128, device=DEV)
            W.amg_restrict(amg, l, T(x), fc, nrhs, W.WL_FP32_BF16)
            ref = np.stack([hb.restrict(l, x[r]) for r in range(nrhs)])
            assert rel(H(fc), ref) <= 1e-6, ("restrict", l, rel(H(fc), ref))
            e = np.stack([cgauss(260 + l, r, nc) for r in range(nrhs)])
            xg = torch.zeros_like(T(x))
            W.amg_prolong(amg, l, T(e), xg, nrhs, W.WL_FP32_BF16)
            ref = np.stack([hb.prolong(l, e[r], np.zeros(n)) for r in range(nrhs)])
            assert rel(H(xg), ref) <= 1e-6, ("prolong", l, rel(H(xg), ref))
    amg.close()
    for order, oorder in ((0, O.ORDER_COLOUR), (1, O.ORDER_TILE)):
        amg = W.amg_import(op, path, W.amg_params_default(zero_guess=1, kacz_order=order))
        for l in range(1, h.L - 1):
            n = h.n(l)
            x0 = 0.1 * np.stack([cgauss(230 + l, r, n) for r in range(nrhs)])
            r0 = np.stack([cgauss(240 + l, r, n) for r in range(nrhs)])
            ref = [hb.kaczmarz(l, x0[r], r0[r], order=oorder, sweeps=2) for r in range(nrhs)]
            xr, rr = np.stack([a for a, _ in ref]), np.stack([b for _, b in ref])
            xg, rg = T(x0), T(r0)
            W.amg_kaczmarz(amg, l, xg, rg, nrhs, 2, W.WL_FP32_BF16)
            assert rel(H(xg), xr) <= 1e-5 and rel(H(rg), rr) <= 1e-5, (order, l, rel(H(xg), xr))
        amg.close()
