"""Thin Python binding of libwilson_amg.so (C ABI in include/wilson_amg.h).

Argument marshalling only: every step runs in the CUDA library.  Arrays are
torch tensors on the GPU (complex128, contiguous); the binding passes their
device pointers and the current torch stream.  The C ABI receives bare
pointers and cannot see how large a buffer is, so before every call the
binding checks that each tensor lives on the operator's device and holds at
least the complex values the call reads or writes (ValueError otherwise):
a short buffer would make a kernel read or write past its end.  Importing
this module fails loudly if the library cannot be loaded: there is no CPU
path.
"""
import atexit
import ctypes as C
import os
import weakref

from . import _build

WL_OK, WL_NOT_CONVERGED = 0, 1
WL_EINVAL, WL_OOM, WL_ECUDA, WL_TIMEOUT, WL_NAN, WL_BAD_HIERARCHY = -1, -2, -3, -4, -5, -6
WL_FP64, WL_FP32, WL_FP32_BF16 = 0, 1, 2
WL_OP_D, WL_OP_DHAT, WL_OP_Z = 0, 1, 2
WL_CYCLE_V, WL_CYCLE_W = 0, 1
(WL_K_DHAT, WL_K_KACZ, WL_K_STENCIL, WL_K_RESTRICT, WL_K_PROLONG, WL_K_COARSEST, WL_K_GS_DOT,
 WL_K_GS_AXPY, WL_K_KACZ_TILE, WL_K_FP64_FMA) = range(10)
WL_AGG_FP64, WL_AGG_FP32, WL_AGG_TC, WL_AGG_TC1 = 0, 1, 2, 3


class amg_params(C.Structure):
    _fields_ = [("levels", C.c_int), ("block", C.c_int * 8), ("k_r", C.c_int), ("k_e", C.c_int),
                ("setup_mu", C.c_int * 2), ("nu_pre", C.c_int), ("nu_post", C.c_int),
                ("omega", C.c_double), ("cycle", C.c_int), ("fgmres_m", C.c_int),
                ("max_restarts", C.c_int), ("precision", C.c_int), ("seed", C.c_ulonglong),
                ("gs_passes", C.c_int), ("zero_guess", C.c_int), ("sweep_kernel", C.c_int),
                ("kacz_order", C.c_int), ("arnoldi_matvec", C.c_int),
                ("setup_cycle", C.c_int), ("overlap", C.c_int), ("gs_arith", C.c_int)]


class wl_info(C.Structure):
    _fields_ = [("status", C.c_int), ("restarts", C.c_int), ("iters", C.c_int),
                ("true_relres", C.c_double)]

    def as_dict(self):
        return dict(status=self.status, restarts=self.restarts, iters=self.iters,
                    true_relres=self.true_relres)


class WilsonAMGError(RuntimeError):
    def __init__(self, what, code):
        super().__init__("%s failed (%d): %s" % (what, code, last_error()))
        self.code = code


_lib = None


def library_path():
    return _build.LIB


def lib():
    """Load (building first if the sources are newer) the CUDA library."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libwilson_amg.so is missing; the CUDA build did not produce it")
        L = C.CDLL(path)
        P, i, d = C.c_void_p, C.c_int, C.c_double
        sig = {
            "amg_params_default": (None, [C.POINTER(amg_params)]),
            "wilson_create": (i, [P, i, d, P, C.POINTER(P)]),
            "wl_destroy": (None, [P]),
            "wl_apply": (i, [P, i, P, P, i, i]),
            "wl_eo_reduce": (i, [P, P, P, i]),
            "wl_eo_reconstruct": (i, [P, P, P, P, i]),
            "amg_setup": (i, [P, C.POINTER(amg_params), C.POINTER(P)]),
            "amg_solve": (i, [P, P, P, i, d, C.POINTER(wl_info)]),
            "amg_solve_host": (i, [P, P, P, i, d, C.POINTER(wl_info)]),
            "amg_export": (i, [P, C.c_char_p]),
            "amg_import": (i, [P, C.c_char_p, C.POINTER(amg_params), C.POINTER(P)]),
            "amg_destroy": (None, [P]),
            "amg_levels": (i, [P, P]),
            "amg_level_apply": (i, [P, i, P, P, i, i]),
            "amg_kaczmarz": (i, [P, i, P, P, i, i, i]),
            "amg_restrict": (i, [P, i, P, P, i, i]),
            "amg_prolong": (i, [P, i, P, P, i, i]),
            "amg_coarsest": (i, [P, P, P, i]),
            "amg_cycle": (i, [P, P, P, i, i]),
            "amg_fgmres": (i, [P, P, P, i, d, C.POINTER(wl_info)]),
            "amg_rho": (i, [P, P, P, i, d, i, P, P, P]),
            "amg_sweep_form": (i, [P, i, i, i, P, P, P]),
            "amg_pin_sweep_form": (i, [P, i, i, i, i, i]),
            "amg_kaczmarz_form": (i, [P, i, P, P, i, i, i, i, i]),
            "wl_last_error": (C.c_char_p, []),
            "wl_time_kernel": (i, [P, i, i, i, i, i, C.POINTER(d)]),
            "wl_dhat_apply_noalloc": (i, [P, P, P, i]),
            "srv_create": (i, [C.c_ulonglong, i, C.POINTER(P)]),
            "srv_add": (i, [P, P, C.POINTER(i)]),
            "srv_start": (i, [P]),
            "srv_info": (i, [P, i, C.POINTER(i), C.POINTER(C.c_ulonglong)]),
            "srv_submit": (i, [P, i, P, P, i, d, C.POINTER(C.c_longlong)]),
            "srv_poll": (i, [P, C.c_longlong, C.POINTER(i), C.POINTER(wl_info), C.POINTER(d)]),
            "srv_drain": (i, [P]),
            "srv_destroy": (None, [P]),
            "wl_launch_count": (C.c_longlong, []),
            "wl_hash_bytes": (C.c_ulonglong, [P, C.c_size_t]),
            "agg_create": (i, [P, i, i, i, P, C.POINTER(P)]),
            "agg_import": (i, [P, i, i, i, P, P, C.POINTER(P)]),
            "agg_export": (i, [P, P, P]),
            "agg_info": (i, [P, C.POINTER(i), C.POINTER(i), C.POINTER(i)]),
            "agg_destroy": (None, [P]),
            "agg_apply": (i, [P, P, P, i, i]),
            "agg_restrict": (i, [P, P, P, i]),
            "agg_prolong": (i, [P, P, P, i]),
            "agg_time_apply": (i, [P, i, i, i, C.POINTER(d)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def last_error():
    return lib().wl_last_error().decode()


def _ptr(t):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != torch.complex128 or not t.is_contiguous():
        raise TypeError("expected a contiguous complex128 tensor")
    return C.c_void_p(t.data_ptr())


def _nrhs(nrhs):
    """nrhs as a count of buffer rows; the library itself rejects nrhs < 1
    and counts above its limits (WL_EINVAL)"""
    if not isinstance(nrhs, int):
        raise TypeError("nrhs must be an int, got %r" % (nrhs,))
    return max(nrhs, 0)


def _buf(t, need, device, what):
    """Device pointer of t after checking that t is a contiguous complex128
    CUDA tensor on `device` with at least `need` elements."""
    p = _ptr(t)
    if device is not None and t.device != device:
        raise ValueError("%s is on %s, the operator on %s" % (what, t.device, device))
    if t.numel() < need:
        raise ValueError("%s holds %d complex values, the call needs %d" % (what, t.numel(), need))
    return p


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _chk(rc, what, ok=(WL_OK,)):
    if rc not in ok:
        raise WilsonAMGError(what, rc)
    return rc


def amg_params_default(**kw):
    p = amg_params()
    lib().amg_params_default(C.byref(p))
    for k, v in kw.items():
        if k == "block":
            for j, b in enumerate(v):
                p.block[j] = b
        elif k == "setup_mu":
            p.setup_mu[0], p.setup_mu[1] = v
        else:
            setattr(p, k, v)
    return p


# --------------------------------------------------------------- handles
# Live handles, destroyed in a fixed order (hierarchies before operators)
# when the interpreter exits, while the library and the CUDA runtime are
# still fully alive.
_live_amg = weakref.WeakSet()
_live_op = weakref.WeakSet()


_live_srv = weakref.WeakSet()


def _close_all():
    for v in list(_live_srv):
        v.close()
    for a in list(_live_amg):
        a.close()
    for o in list(_live_op):
        o.close()


atexit.register(_close_all)


class wl_op:
    """Owns a wl_op* (Wilson operator for one gauge field)."""

    def __init__(self, ptr, L, m, device=None):
        self._p = ptr
        self.L, self.m = L, m
        self.device = device
        self._amgs = weakref.WeakSet()
        _live_op.add(self)

    @property
    def handle(self):
        return self._p

    def close(self):
        if self._p:
            for a in list(self._amgs):   # a hierarchy never outlives its operator
                a.close()
            lib().wl_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class wl_amg:
    """Owns a wl_amg* (hierarchy); keeps its wl_op alive."""

    def __init__(self, ptr, op):
        self._p = ptr
        self.op = op
        op._amgs.add(self)
        _live_amg.add(self)
        buf = (C.c_int * 8)()
        nl = lib().amg_levels(ptr, C.cast(buf, C.c_void_p))
        self.Nl = [buf[i] for i in range(nl)]  # lattice side of every level

    def n(self, level):
        """complex values of one level vector (N_l^2 / 2 sites, 2 spins)"""
        if not 0 <= level < len(self.Nl):
            raise ValueError("level %d outside 0..%d" % (level, len(self.Nl) - 1))
        return self.Nl[level] ** 2

    @property
    def handle(self):
        return self._p

    def close(self):
        if self._p:
            lib().amg_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------- C ABI mirrors
def wilson_create(gauge, L, m):
    g = _buf(gauge, 2 * max(int(L), 0) ** 2, None, "gauge")   # the library checks L itself
    out = C.c_void_p()
    _chk(lib().wilson_create(g, L, m, _stream(), C.byref(out)), "wilson_create")
    return wl_op(out, L, m, gauge.device)


def _full(op, nrhs):   # full fields [nrhs][L][L][2]
    return _nrhs(nrhs) * op.L * op.L * 2


def _even(op, nrhs):   # level-0 vectors [nrhs][L^2/2][2]
    return _nrhs(nrhs) * op.L * op.L


def wl_apply(op, which, x, y, nrhs, prec=WL_FP64):
    need = _even(op, nrhs) if which == WL_OP_DHAT else _full(op, nrhs)
    return _chk(lib().wl_apply(op.handle, which, _buf(x, need, op.device, "x"), _buf(y, need, op.device, "y"),
                               nrhs, prec), "wl_apply")


def wl_eo_reduce(op, b, bhat, nrhs):
    return _chk(lib().wl_eo_reduce(op.handle, _buf(b, _full(op, nrhs), op.device, "b"),
                                   _buf(bhat, _even(op, nrhs), op.device, "bhat"), nrhs), "wl_eo_reduce")


def wl_eo_reconstruct(op, b, xe, psi, nrhs):
    return _chk(lib().wl_eo_reconstruct(op.handle, _buf(b, _full(op, nrhs), op.device, "b"),
                                        _buf(xe, _even(op, nrhs), op.device, "xe"),
                                        _buf(psi, _full(op, nrhs), op.device, "psi"), nrhs),
                "wl_eo_reconstruct")


def amg_setup(op, params=None):
    p = params or amg_params_default()
    out = C.c_void_p()
    _chk(lib().amg_setup(op.handle, C.byref(p), C.byref(out)), "amg_setup")
    return wl_amg(out, op)


def amg_import(op, path, params=None):
    out = C.c_void_p()
    pp = C.byref(params) if params is not None else None
    _chk(lib().amg_import(op.handle, os.fsencode(path), pp, C.byref(out)), "amg_import")
    return wl_amg(out, op)


def amg_export(amg, path):
    return _chk(lib().amg_export(amg.handle, os.fsencode(path)), "amg_export")


def amg_levels(amg):
    buf = (C.c_int * 8)()
    L = lib().amg_levels(amg.handle, C.cast(buf, C.c_void_p))
    return [buf[i] for i in range(L)]


def amg_solve(amg, b, x, nrhs, tol):
    """(rc, info per right-hand side); rc is WL_OK, WL_NOT_CONVERGED or WL_NAN
    (some right-hand side had a non-finite residual and was retired; info
    says which), other codes raise."""
    op = amg.op
    need = _full(op, nrhs)
    info = (wl_info * nrhs)()
    rc = _chk(lib().amg_solve(amg.handle, _buf(b, need, op.device, "b"), _buf(x, need, op.device, "x"), nrhs,
                              tol, info), "amg_solve", ok=(WL_OK, WL_NOT_CONVERGED, WL_NAN))
    return rc, [i.as_dict() for i in info]


def _host_buf(t, need, what):
    """Host pointer of t after checking that t is a contiguous complex128 CPU
    tensor with at least `need` elements (page-locked memory lets the
    library's copies run asynchronously)."""
    import torch
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError("%s: expected a CPU tensor" % what)
    if t.dtype != torch.complex128 or not t.is_contiguous():
        raise TypeError("%s: expected a contiguous complex128 tensor" % what)
    if t.numel() < need:
        raise ValueError("%s holds %d complex values, the call needs %d" % (what, t.numel(), need))
    return C.c_void_p(t.data_ptr())


def amg_solve_host(amg, b, x, nrhs, tol):
    """amg_solve with b and x in host memory (CPU tensors, ideally pinned):
    the library copies them in and out, overlapping one solve lane's copies
    with the other lane's solve."""
    need = _full(amg.op, nrhs)
    info = (wl_info * nrhs)()
    rc = _chk(lib().amg_solve_host(amg.handle, _host_buf(b, need, "b"), _host_buf(x, need, "x"), nrhs, tol, info),
              "amg_solve_host", ok=(WL_OK, WL_NOT_CONVERGED, WL_NAN))
    return rc, [i.as_dict() for i in info]


def amg_fgmres(amg, bhat, x, nrhs, tol):
    op = amg.op
    need = _even(op, nrhs)
    info = (wl_info * nrhs)()
    rc = _chk(lib().amg_fgmres(amg.handle, _buf(bhat, need, op.device, "bhat"), _buf(x, need, op.device, "x"),
                               nrhs, tol, info), "amg_fgmres", ok=(WL_OK, WL_NOT_CONVERGED, WL_NAN))
    return rc, [i.as_dict() for i in info]


def amg_rho(amg, x0, x, nrhs, tol=1e-8, maxit=100, hist=False):
    """Sec. 4's rho of the stand-alone cycle on Dhat x = 0 from x0; returns
    (rc, rho[nrhs], iters[nrhs], hist [nrhs][maxit + 1] or None)."""
    import numpy as np
    need = _even(amg.op, nrhs)
    dev = amg.op.device
    x0p, xp = _buf(x0, need, dev, "x0"), _buf(x, need, dev, "x")
    rho = np.zeros(nrhs)
    it = np.zeros(nrhs, dtype=np.int32)
    h = np.zeros((nrhs, maxit + 1)) if hist else None
    rc = _chk(lib().amg_rho(amg.handle, x0p, xp, nrhs, tol, maxit, rho.ctypes.data_as(C.c_void_p),
                            it.ctypes.data_as(C.c_void_p), h.ctypes.data_as(C.c_void_p) if hist else None),
              "amg_rho", ok=(WL_OK, WL_NOT_CONVERGED))
    return rc, rho, it, h


def amg_pin_sweep_form(amg, level, nrhs, prec, form, param):
    """Pin the Kaczmarz launch form of `level` for (nrhs, prec); cycles of
    that width captured afterwards use it (see amg_sweep_form for the codes)."""
    return _chk(lib().amg_pin_sweep_form(amg.handle, level, nrhs, prec, form, param), "amg_pin_sweep_form")


def amg_sweep_form(amg, level, nrhs, prec):
    """(form, param, us) of the Kaczmarz sweep on `level`: form 0 per-colour
    launches, 1 cooperative (param blocks), 2 tile kernel (param = RHS chunk | RHS per thread << 8,
    8 meaning one RHS per thread with paired FP32 FMAs), 3 block-resident (param RHS per block);
    us = measured time of one sweep (0 if not measured)."""
    f, p, u = C.c_int(), C.c_int(), C.c_float()
    _chk(lib().amg_sweep_form(amg.handle, level, nrhs, prec, C.byref(f), C.byref(p), C.byref(u)),
         "amg_sweep_form")
    return f.value, p.value, u.value


def _lev(amg, level, nrhs, *named):
    """device pointers of level-`level` vectors [nrhs][N_l^2/2][2]"""
    need = _nrhs(nrhs) * amg.n(level)
    return [_buf(t, need, amg.op.device, what) for what, t in named]


def amg_level_apply(amg, level, x, y, nrhs, prec=WL_FP64):
    xp, yp = _lev(amg, level, nrhs, ("x", x), ("y", y))
    return _chk(lib().amg_level_apply(amg.handle, level, xp, yp, nrhs, prec), "amg_level_apply")


def amg_kaczmarz(amg, level, x, r, nrhs, sweeps=1, prec=WL_FP64):
    xp, rp = _lev(amg, level, nrhs, ("x", x), ("r", r))
    return _chk(lib().amg_kaczmarz(amg.handle, level, xp, rp, nrhs, sweeps, prec), "amg_kaczmarz")


def amg_kaczmarz_form(amg, level, x, r, nrhs, sweeps, prec, form, param):
    xp, rp = _lev(amg, level, nrhs, ("x", x), ("r", r))
    return _chk(lib().amg_kaczmarz_form(amg.handle, level, xp, rp, nrhs, sweeps, prec, form, param),
                "amg_kaczmarz_form")


def amg_restrict(amg, level, r, fc, nrhs, prec=WL_FP64):
    (rp,) = _lev(amg, level, nrhs, ("r", r))
    (fp,) = _lev(amg, level + 1, nrhs, ("fc", fc))
    return _chk(lib().amg_restrict(amg.handle, level, rp, fp, nrhs, prec), "amg_restrict")


def amg_prolong(amg, level, e, x, nrhs, prec=WL_FP64):
    (ep,) = _lev(amg, level + 1, nrhs, ("e", e))
    (xp,) = _lev(amg, level, nrhs, ("x", x))
    return _chk(lib().amg_prolong(amg.handle, level, ep, xp, nrhs, prec), "amg_prolong")


def amg_coarsest(amg, f, x, nrhs):
    fp, xp = _lev(amg, len(amg.Nl) - 1, nrhs, ("f", f), ("x", x))
    return _chk(lib().amg_coarsest(amg.handle, fp, xp, nrhs), "amg_coarsest")


def amg_cycle(amg, f, x, nrhs, prec=WL_FP64):
    fp, xp = _lev(amg, 0, nrhs, ("f", f), ("x", x))
    return _chk(lib().amg_cycle(amg.handle, fp, xp, nrhs, prec), "amg_cycle")


def wl_last_error():
    return last_error()


def wl_destroy(op):
    op.close()


def amg_destroy(amg):
    amg.close()


def wl_time_kernel(amg, kind, level, nrhs, prec, reps):
    ms = C.c_double()
    _chk(lib().wl_time_kernel(amg.handle, kind, level, nrhs, prec, reps, C.byref(ms)), "wl_time_kernel")
    return ms.value


def wl_launch_count():
    return lib().wl_launch_count()


def wl_hash_bytes(data):
    """FNV-1a 64 of a bytes object, computed by the library (host only)"""
    buf = C.create_string_buffer(bytes(data), len(data)) if len(data) else None
    return int(lib().wl_hash_bytes(buf, len(data)))


# ------------------------------------------------------------------ serving
class wl_server:
    """Owns a wl_server*; keeps the hierarchies it serves alive."""

    def __init__(self, ptr):
        self._p = ptr
        self.amgs = []
        self.by_cfg = {}
        _live_srv.add(self)

    @property
    def handle(self):
        return self._p

    def close(self):
        if self._p:
            lib().srv_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def srv_create(hbm_budget_bytes, max_slots_per_config):
    out = C.c_void_p()
    _chk(lib().srv_create(int(hbm_budget_bytes), max_slots_per_config, C.byref(out)), "srv_create")
    return wl_server(out)


def srv_add(srv, amg):
    cid = C.c_int()
    _chk(lib().srv_add(srv.handle, amg.handle, C.byref(cid)), "srv_add")
    srv.amgs.append(amg)
    srv.by_cfg[cid.value] = amg
    return cid.value


def srv_info(srv, cfg):
    """(slots, device bytes) reserved for configuration cfg."""
    n, b = C.c_int(), C.c_ulonglong()
    _chk(lib().srv_info(srv.handle, cfg, C.byref(n), C.byref(b)), "srv_info")
    return n.value, b.value


def srv_start(srv):
    return _chk(lib().srv_start(srv.handle), "srv_start")


def srv_submit(srv, cfg, b, x, nrhs, tol):
    if cfg not in srv.by_cfg:
        raise ValueError("no configuration %r on this server" % (cfg,))
    op = srv.by_cfg[cfg].op
    need = _full(op, nrhs)
    rid = C.c_longlong()
    _chk(lib().srv_submit(srv.handle, cfg, _buf(b, need, op.device, "b"), _buf(x, need, op.device, "x"), nrhs,
                          tol, C.byref(rid)), "srv_submit")
    return rid.value


def srv_poll(srv, req_id, nrhs):
    done, lat = C.c_int(), C.c_double()
    info = (wl_info * nrhs)()
    rc = lib().srv_poll(srv.handle, req_id, C.byref(done), info, C.byref(lat))
    _chk(rc, "srv_poll", ok=(WL_OK, WL_NOT_CONVERGED, WL_NAN))
    return bool(done.value), [i.as_dict() for i in info], lat.value


def srv_drain(srv):
    return _chk(lib().srv_drain(srv.handle), "srv_drain")


def srv_destroy(srv):
    srv.close()


def wl_dhat_apply_noalloc(op, x, y, nrhs):
    """y = Dhat x through the allocation-free entry point (see the C header)."""
    need = _even(op, nrhs)
    return _chk(lib().wl_dhat_apply_noalloc(op.handle, _buf(x, need, op.device, "x"),
                                            _buf(y, need, op.device, "y"), nrhs), "wl_dhat_apply_noalloc")


# ------------------------------------------------- aggregation coarse space
class wl_agg:
    """Owns a wl_agg* (aggregation coarse space of one level of a hierarchy);
    keeps the hierarchy object alive."""

    def __init__(self, ptr, amg, level, B, k):
        self._p = ptr
        self.amg, self.level, self.B, self.k = amg, level, B, k
        nc, Nc, kk = C.c_int(), C.c_int(), C.c_int()
        _chk(lib().agg_info(ptr, C.byref(nc), C.byref(Nc), C.byref(kk)), "agg_info")
        self.nc, self.Nc = nc.value, Nc.value
        self.nf = amg.n(level) // 2
        _live_agg.add(self)

    @property
    def handle(self):
        return self._p

    def close(self):
        if self._p:
            lib().agg_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_live_agg = weakref.WeakSet()


def _close_all_agg():
    for g in list(_live_agg):
        g.close()


atexit.register(_close_all_agg)   # runs before _close_all (atexit is last-in, first-out)


def agg_create(amg, level, B, k, V):
    """Aggregation coarse space of `level` from the k test vectors V
    ([k][n_l][2] complex128 on the device)."""
    dev = amg.op.device
    need = k * amg.n(level)
    out = C.c_void_p()
    _chk(lib().agg_create(amg.handle, level, B, k, _buf(V, need, dev, "V"), C.byref(out)), "agg_create")
    return wl_agg(out, amg, level, B, k)


def agg_import(amg, level, B, k, Q, Ac):
    dev = amg.op.device
    nc = (amg.Nl[level] // B) ** 2 // 2
    out = C.c_void_p()
    _chk(lib().agg_import(amg.handle, level, B, k, _buf(Q, nc * 2 * B * B * k, dev, "Q"),
                          _buf(Ac, nc * 9 * 4 * k * k, dev, "Ac"), C.byref(out)), "agg_import")
    return wl_agg(out, amg, level, B, k)


def agg_export(g, Q, Ac):
    dev = g.amg.op.device
    return _chk(lib().agg_export(g.handle, _buf(Q, g.nc * 2 * g.B * g.B * g.k, dev, "Q"),
                                 _buf(Ac, g.nc * 9 * 4 * g.k * g.k, dev, "Ac")), "agg_export")


def agg_apply(g, x, y, nrhs, kernel=WL_AGG_FP64):
    need = _nrhs(nrhs) * g.nc * 2 * g.k
    dev = g.amg.op.device
    return _chk(lib().agg_apply(g.handle, _buf(x, need, dev, "x"), _buf(y, need, dev, "y"), nrhs, kernel),
                "agg_apply")


def agg_restrict(g, r, fc, nrhs):
    dev = g.amg.op.device
    return _chk(lib().agg_restrict(g.handle, _buf(r, _nrhs(nrhs) * 2 * g.nf, dev, "r"),
                                   _buf(fc, _nrhs(nrhs) * g.nc * 2 * g.k, dev, "fc"), nrhs), "agg_restrict")


def agg_prolong(g, e, x, nrhs):
    dev = g.amg.op.device
    return _chk(lib().agg_prolong(g.handle, _buf(e, _nrhs(nrhs) * g.nc * 2 * g.k, dev, "e"),
                                  _buf(x, _nrhs(nrhs) * 2 * g.nf, dev, "x"), nrhs), "agg_prolong")


def agg_time_apply(g, nrhs, kernel, reps):
    ms = C.c_double()
    _chk(lib().agg_time_apply(g.handle, nrhs, kernel, reps, C.byref(ms)), "agg_time_apply")
    return ms.value



def agg_info(g):
    """(coarse sites, coarse lattice side, k)"""
    return g.nc, g.Nc, g.k


def agg_destroy(g):
    g.close()
