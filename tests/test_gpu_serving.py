"""Serving runtime (continuous batching over resident hierarchies) through
the C ABI: results equal alone and in a mix, requests of several lattice
sizes overlap, device-memory admission."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1308_5992_gb300 import wilson_amg as W  # noqa: E402
from wl_inputs import workload, rhs_batch  # noqa: E402

DEV = torch.device("cuda:0")
TOL = 1e-12


def _T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture(scope="module")
def resident():
    out = []
    for name in ("T32", "T64"):
        w = workload(name)
        op = W.wilson_create(_T(w["U"]), w["N"], w["m"])
        p = W.amg_params_default(k_r=w["k"], k_e=w["k"], seed=w["seed"], precision=W.WL_FP32)
        p.levels = len(w["blocks"]) + 1
        for l, b in enumerate(w["blocks"]):
            p.block[l] = b
        out.append((w, op, W.amg_setup(op, p)))
    return out


def _residual(op, w, b, x):
    """relative residual ||D x - b|| / ||b|| with the GPU's FP64 D apply"""
    y = torch.zeros_like(x)
    W.wl_apply(op, W.WL_OP_D, x, y, x.shape[0], W.WL_FP64)
    return [float(torch.linalg.norm(y[r] - b[r]) / torch.linalg.norm(b[r])) for r in range(x.shape[0])]


def test_alone_equals_mix(resident):
    (w0, op0, a0), (w1, op1, a1) = resident
    b0 = _T(rhs_batch(w0["N"], 5, 41))
    b1 = _T(rhs_batch(w1["N"], 7, 42))
    # alone: one request of one right-hand side
    srv = W.srv_create(8 << 30, 8)
    c0 = W.srv_add(srv, a0)
    W.srv_start(srv)
    x_alone = torch.zeros_like(b0[2:3])
    rid = W.srv_submit(srv, c0, b0[2:3].contiguous(), x_alone, 1, TOL)
    W.srv_drain(srv)
    done, info, lat = W.srv_poll(srv, rid, 1)
    assert done and info[0]["status"] == W.WL_OK and lat > 0
    srv.close()
    # mix: both lattices, several requests, more right-hand sides than slots
    srv = W.srv_create(8 << 30, 4)
    c0, c1 = W.srv_add(srv, a0), W.srv_add(srv, a1)
    W.srv_start(srv)
    xs, reqs = [], []
    for (cfg, b, lo, hi) in [(c1, b1, 0, 4), (c0, b0, 0, 5), (c1, b1, 4, 7), (c0, b0, 2, 3)]:
        x = torch.zeros_like(b[lo:hi])
        reqs.append((W.srv_submit(srv, cfg, b[lo:hi].contiguous(), x, hi - lo, TOL), hi - lo))
        xs.append(x)
    W.srv_drain(srv)
    for rid, n in reqs:
        done, info, lat = W.srv_poll(srv, rid, n)
        assert done and all(i["status"] == W.WL_OK and i["true_relres"] <= TOL for i in info)
    # the same right-hand side alone and in the mix (inside a 5-RHS request
    # and as its own request)
    for x in (xs[1][2], xs[3][0]):
        assert float(torch.linalg.norm(x - x_alone[0]) / torch.linalg.norm(x_alone[0])) <= 1e-9
    assert max(_residual(op0, w0, b0, xs[1])) <= 1e-9
    assert max(_residual(op1, w1, b1[0:4].contiguous(), xs[0])) <= 1e-9
    srv.close()


def test_admission_by_memory(resident):
    (w0, op0, a0), _ = resident
    srv = W.srv_create(1024, 8)  # far too small for one slot
    with pytest.raises(W.WilsonAMGError) as e:
        W.srv_add(srv, a0)
    assert e.value.code == W.WL_OOM
    srv.close()


def test_alone_equals_mix_benchmark_cycle():
    """The serving configuration the benchmark runs (FP32 tile-coloured
    V(4,4), FP32 Arnoldi matvec, one Gram-Schmidt pass): a right-hand side
    gives the same solution alone and inside a larger request that overflows
    the slots, so it is admitted while its batch mates are on the GPU."""
    w = workload("T64")
    op = W.wilson_create(_T(w["U"]), w["N"], w["m"])
    p = W.amg_params_default(k_r=w["k"], k_e=w["k"], seed=w["seed"], precision=W.WL_FP32, nu_pre=4, nu_post=4,
                             gs_passes=1, kacz_order=1, arnoldi_matvec=1)
    p.levels = len(w["blocks"]) + 1
    for l, b in enumerate(w["blocks"]):
        p.block[l] = b
    amg = W.amg_setup(op, p)
    b = _T(rhs_batch(w["N"], 9, 43))
    srv = W.srv_create(8 << 30, 4)
    cfg = W.srv_add(srv, amg)
    W.srv_start(srv)
    x_alone = torch.zeros_like(b[5:6])
    rid = W.srv_submit(srv, cfg, b[5:6].contiguous(), x_alone, 1, TOL)
    W.srv_drain(srv)
    assert W.srv_poll(srv, rid, 1)[0]
    x_mix = torch.zeros_like(b)
    rid = W.srv_submit(srv, cfg, b, x_mix, 9, TOL)
    W.srv_drain(srv)
    done, info, lat = W.srv_poll(srv, rid, 9)
    assert done and all(i["status"] == W.WL_OK and i["true_relres"] <= TOL for i in info)
    assert float(torch.linalg.norm(x_mix[5] - x_alone[0]) / torch.linalg.norm(x_alone[0])) <= 1e-9
    assert max(_residual(op, w, b, x_mix)) <= 1e-9
    srv.close()


def test_serving_matches_oracle(O, tmp_path):
    """Requests of two lattice sizes (32x32 and 128x128) served together with
    the benchmark's serving cycle, on hierarchies exported by the oracle: a
    sampled right-hand side of each request, solved in the mix, matches the
    oracle's own solve on the same hierarchy to 1e-10 relative error."""
    from oracle.hierfile import write_hierarchy
    p = W.amg_params_default(precision=W.WL_FP32, nu_pre=4, nu_post=4, gs_passes=1, kacz_order=1,
                             arnoldi_matvec=1)
    srv = W.srv_create(8 << 30, 4)
    cfgs = []
    for name in ("T32", "T128"):
        w = workload(name)
        h = O.Hierarchy.setup(w["N"], w["U"], w["m"], O.setup_params(w["blocks"], k_r=w["k"], k_e=w["k"],
                                                                      seed=w["seed"]))
        path = str(tmp_path / ("%s.wlh" % name))
        write_hierarchy(path, h)
        op = W.wilson_create(_T(w["U"]), w["N"], w["m"])
        cfgs.append((w, h, W.srv_add(srv, W.amg_import(op, path, p))))
    W.srv_start(srv)
    live = []
    for k, (w, h, cfg) in enumerate(cfgs * 2):   # two requests per lattice, interleaved
        b = rhs_batch(w["N"], 3 + k, 44 + k)
        x = torch.zeros((3 + k, w["N"], w["N"], 2), dtype=torch.complex128, device=DEV)
        bd = _T(b)
        torch.cuda.synchronize()
        live.append((w, h, b, x, bd, W.srv_submit(srv, cfg, bd, x, 3 + k, 1e-13)))
    W.srv_drain(srv)
    for k, (w, h, b, x, bd, rid) in enumerate(live):
        done, info, _ = W.srv_poll(srv, rid, 3 + k)
        assert done and all(i["status"] == W.WL_OK and i["true_relres"] <= 1e-13 for i in info)
        q = k % (3 + k)
        ref, _ = h.solve(b[q], tol=1e-13)
        got = x[q].cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-10, (w["name"], k)
    srv.close()

