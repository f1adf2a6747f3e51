"""CPU checks of the C ABI: the library builds for sm_103a, loads, and
exports every function that include/wilson_amg.h declares (no compute call
is made without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "wilson_amg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|char)\s*\**\s*(\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_1308_5992_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_abi():
    from paper_1308_5992_gb300 import wilson_amg as W
    for n in declared_functions():
        assert hasattr(W, n), n
    W.lib()


def test_params_defaults_and_errors():
    """Host-side argument checks need no device."""
    from paper_1308_5992_gb300 import wilson_amg as W
    p = W.amg_params_default()
    assert (p.k_r, p.k_e, p.nu_pre, p.nu_post, p.fgmres_m) == (8, 8, 2, 2, 20)
    assert (p.setup_mu[0], p.setup_mu[1], p.omega, p.precision) == (10, 5, 1.0, W.WL_FP64)
    out = ctypes.c_void_p()
    # L not a power of two -> WL_EINVAL before any device work
    rc = W.lib().wilson_create(ctypes.c_void_p(8), 24, 0.1, None, ctypes.byref(out))
    assert rc == W.WL_EINVAL and "power of two" in W.last_error()
    rc = W.lib().wilson_create(None, 32, 0.1, None, ctypes.byref(out))
    assert rc == W.WL_EINVAL


def test_float_widening_formula():
    """The kernels widen normal floats to doubles with integer operations
    (sign, exponent + 896, mantissa << 29); check the formula is exact for
    every normal exponent against numpy's conversion."""
    import numpy as np
    rng = np.random.default_rng(0)
    mant = rng.integers(0, 1 << 23, size=4096, dtype=np.uint32)
    for e in range(1, 255):
        for sign in (0, 1):
            u = (np.uint32(sign) << np.uint32(31)) | (np.uint32(e) << np.uint32(23)) | mant
            f = u.view(np.float32)
            d = ((u.astype(np.uint64) & np.uint64(0x80000000)) << np.uint64(32)) | \
                (np.uint64(e + 896) << np.uint64(52)) | ((u.astype(np.uint64) & np.uint64(0x7FFFFF)) << np.uint64(29))
            assert np.array_equal(d.view(np.float64), f.astype(np.float64))


def test_binding_constants_match_header_enums():
    """Every enumerator of include/wilson_amg.h has the same value in the binding."""
    from paper_1308_5992_gb300 import wilson_amg as W
    txt = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "wilson_amg.h")).read(), flags=re.S)
    pairs = []
    for body in re.findall(r"enum\s*\{([^}]*)\}", txt):
        for item in body.split(","):
            m = re.match(r"\s*(WL_\w+)\s*=\s*(-?\d+)\s*$", item)
            if m:
                pairs.append((m.group(1), int(m.group(2))))
    assert len(pairs) >= 15
    for name, value in pairs:
        assert getattr(W, name) == value, name


def test_no_host_fallback_without_a_device():
    """Without a CUDA device the library reports WL_ECUDA instead of
    computing anything on the host (there is no CPU path)."""
    torch = __import__("pytest").importorskip("torch")
    if torch.cuda.is_available():
        __import__("pytest").skip("a device is present")
    import numpy as np
    from paper_1308_5992_gb300 import wilson_amg as W
    U = np.ones((2, 32, 32), np.complex128)
    out = ctypes.c_void_p()
    rc = W.lib().wilson_create(ctypes.c_void_p(U.ctypes.data), 32, 0.1, None, ctypes.byref(out))
    assert rc == W.WL_ECUDA and not out.value
