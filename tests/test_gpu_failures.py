"""Failure paths made on the host (no GPU fault is provoked): a right-hand
side poisoned with NaN before the call, a restart budget too small for the
tolerance, a buffer shorter than the call needs, and a poisoned request
inside a running server.  Each failure stays with its own right-hand side:
the rest of the batch, and the server, carry on."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - collected only on GPU machines
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1308_5992_gb300 import wilson_amg as W  # noqa: E402
from wl_inputs import workload, rhs_batch  # noqa: E402

DEV = torch.device("cuda:0")


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).to(DEV)


def even_part(N, psi):
    """level-0 vector [N^2/2][2] of the even sites of a full field [N][N][2]"""
    out = np.empty((N * N // 2, 2), complex)
    for h in range(N * N // 2):
        y = h // (N // 2)
        x = 2 * (h % (N // 2)) + (y & 1)
        out[h] = psi[y, x]
    return out.reshape(-1)


@pytest.fixture(scope="module")
def t64(O, tmp_path_factory):
    from oracle.hierfile import write_hierarchy
    w = workload("T64")
    h = O.Hierarchy.setup(w["N"], w["U"], w["m"], O.setup_params(w["blocks"], k_r=w["k"], k_e=w["k"],
                                                                  seed=w["seed"]))
    path = str(tmp_path_factory.mktemp("f") / "t64.wlh")
    write_hierarchy(path, h)
    op = W.wilson_create(T(w["U"]), w["N"], w["m"])
    return w, h, op, path


@pytest.mark.parametrize("prec", [W.WL_FP64, W.WL_FP32])
def test_nan_rhs_is_retired_alone(t64, prec):
    """One right-hand side with a NaN entry: the call returns WL_NAN, that
    right-hand side reports WL_NAN, and its batch mates converge to the
    oracle's solutions as if it were not there."""
    w, h, op, path = t64
    N = w["N"]
    amg = W.amg_import(op, path, W.amg_params_default(zero_guess=1, precision=prec))
    b = rhs_batch(N, 3, 51)
    b[1, 5, 7, 0] = np.nan
    psi = torch.zeros_like(T(b))
    rc, info = W.amg_solve(amg, T(b), psi, 3, 1e-13)
    assert rc == W.WL_NAN
    assert info[1]["status"] == W.WL_NAN
    assert "non-finite" in W.last_error()
    x = psi.cpu().numpy()
    for q in (0, 2):
        assert info[q]["status"] == W.WL_OK and info[q]["true_relres"] <= 1e-13
        ref, _ = h.solve(b[q], tol=1e-13)
        assert np.linalg.norm(x[q] - ref) / np.linalg.norm(ref) <= 1e-10, q
    # the same batch mates alone: the same iterations (up to the rounding of
    # the batch-width-dependent reduction trees) and the same solutions
    good = b[[0, 2]]
    psi2 = torch.zeros_like(T(good))
    rc2, info2 = W.amg_solve(amg, T(good), psi2, 2, 1e-13)
    assert rc2 == W.WL_OK
    for q, q2 in ((0, 0), (2, 1)):
        assert abs(info[q]["iters"] - info2[q2]["iters"]) <= 1
        x2 = psi2[q2].cpu().numpy()
        assert np.linalg.norm(x[q] - x2) / np.linalg.norm(x2) <= 1e-10


def test_restart_budget_returns_best_iterate(O, t64):
    """max_restarts = 1 at a tolerance one cycle cannot reach: WL_NOT_CONVERGED
    with x the iterate after that cycle, whose true reduced residual (the
    oracle's Dhat) is the one reported and is below the starting one."""
    w, h, op, path = t64
    N, U, m = w["N"], w["U"], w["m"]
    p = W.amg_params_default(zero_guess=1, max_restarts=1, fgmres_m=4)
    amg = W.amg_import(op, path, p)
    b = rhs_batch(N, 2, 52)
    psi = torch.zeros_like(T(b))
    rc, info = W.amg_solve(amg, T(b), psi, 2, 1e-14)
    assert rc == W.WL_NOT_CONVERGED
    x = psi.cpu().numpy()
    for q in range(2):
        assert info[q]["status"] == W.WL_NOT_CONVERGED and info[q]["restarts"] == 1
        assert info[q]["iters"] == 4
        bh = O.eo_reduce(N, U, m, b[q])
        res = np.linalg.norm(bh - O.dhat_apply(N, U, m, even_part(N, x[q]))) / np.linalg.norm(bh)
        assert 1e-14 < res < 1.0
        assert abs(res - info[q]["true_relres"]) <= 1e-6 * res


def test_short_buffer_is_refused_before_the_call(t64):
    """The C ABI sees bare pointers; the binding refuses a tensor that holds
    fewer values than the call would touch, or one on another device."""
    w, h, op, path = t64
    N = w["N"]
    x = torch.zeros((2, N * N), dtype=torch.complex128, device=DEV)
    y = torch.zeros((1, N * N), dtype=torch.complex128, device=DEV)
    n0 = W.wl_launch_count()
    with pytest.raises(ValueError, match="holds"):
        W.wl_apply(op, W.WL_OP_DHAT, x, y, 2, W.WL_FP64)
    with pytest.raises(ValueError, match="holds"):
        W.wl_dhat_apply_noalloc(op, x, y, 2)
    with pytest.raises(TypeError):
        W.wl_apply(op, W.WL_OP_DHAT, x.cpu(), x, 1, W.WL_FP64)
    assert W.wl_launch_count() == n0


def test_nan_request_in_a_running_server(t64):
    """A request whose right-hand side is poisoned is retired with WL_NAN;
    a request submitted with it is solved, and the server keeps serving."""
    w, h, op, path = t64
    N = w["N"]
    amg = W.amg_import(op, path, W.amg_params_default(precision=W.WL_FP32))
    srv = W.srv_create(8 << 30, 4)
    cfg = W.srv_add(srv, amg)
    W.srv_start(srv)
    b = rhs_batch(N, 3, 53)
    bad = b[:1].copy()
    bad[0, 0, 0, 1] = np.inf
    bb, xb = T(bad), torch.zeros((1, N, N, 2), dtype=torch.complex128, device=DEV)
    bg, xg = T(b[1:]), torch.zeros((2, N, N, 2), dtype=torch.complex128, device=DEV)
    torch.cuda.synchronize()
    r_bad = W.srv_submit(srv, cfg, bb, xb, 1, 1e-12)
    r_good = W.srv_submit(srv, cfg, bg, xg, 2, 1e-12)
    W.srv_drain(srv)
    done, info, _ = W.srv_poll(srv, r_bad, 1)
    assert done and info[0]["status"] == W.WL_NAN
    done, info, _ = W.srv_poll(srv, r_good, 2)
    assert done and all(i["status"] == W.WL_OK and i["true_relres"] <= 1e-12 for i in info)
    # still serving
    x2 = torch.zeros_like(bg[:1])
    rid = W.srv_submit(srv, cfg, bg[:1].contiguous(), x2, 1, 1e-12)
    W.srv_drain(srv)
    done, info, _ = W.srv_poll(srv, rid, 1)
    assert done and info[0]["status"] == W.WL_OK
    assert float(torch.linalg.norm(x2[0] - xg[0]) / torch.linalg.norm(xg[0])) <= 1e-9
    srv.close()
