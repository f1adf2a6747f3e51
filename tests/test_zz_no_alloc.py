"""The allocation-free Dhat entry point (for callers that cannot allocate
device memory when they apply the operator: their memory is held by their
own pool, or they cannot afford the synchronisation of cudaMalloc/cudaFree)
agrees with the regular entry point, on two calls in a row through the C
ABI, and refuses sizes beyond its fixed scratch array.  Collected last so a
stop-at-first-failure run has already run every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1308_5992_gb300 import wilson_amg as W  # noqa: E402
from wl_inputs import workload, cgauss  # noqa: E402

DEV = torch.device("cuda:0")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).to(DEV)


def test_noalloc_matches_wl_apply_twice():
    w = workload("T64")
    N = w["N"]
    op = W.wilson_create(_dev(w["U"]), N, w["m"])
    for call, nrhs in enumerate((3, 1)):
        x = _dev(np.stack([cgauss(500 + 10 * call + r, 1, N * N) for r in range(nrhs)]))
        ref = torch.zeros_like(x)
        W.wl_apply(op, W.WL_OP_DHAT, x, ref, nrhs, W.WL_FP64)
        y = torch.full_like(x, float("nan"))
        W.wl_dhat_apply_noalloc(op, x, y, nrhs)
        err = float((y - ref).abs().max() / ref.abs().max())
        assert err <= 1e-14, (call, err)


def test_noalloc_allocates_no_device_memory():
    """After the first call (which only looks up the array's address), a call
    changes neither the device's free memory nor torch's allocator."""
    w = workload("T64")
    N = w["N"]
    op = W.wilson_create(_dev(w["U"]), N, w["m"])
    x = _dev(np.stack([cgauss(600 + r, 1, N * N) for r in range(2)]))
    y = torch.zeros_like(x)
    W.wl_dhat_apply_noalloc(op, x, y, 2)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        W.wl_dhat_apply_noalloc(op, x, y, 2)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0


def test_noalloc_rejects_oversize():
    w = workload("T64")
    op = W.wilson_create(_dev(w["U"]), w["N"], w["m"])
    nrhs = (1 << 20) // (w["N"] * w["N"]) + 1
    x = torch.zeros((nrhs, w["N"] * w["N"]), dtype=torch.complex128, device=DEV)
    with pytest.raises(W.WilsonAMGError) as e:
        W.wl_dhat_apply_noalloc(op, x, torch.zeros_like(x), nrhs)
    assert e.value.code == W.WL_EINVAL and "holds" in str(e.value)
