"""Compute the shift m of every seeded workload and write wl_inputs/shifts.json.

TEST INFRASTRUCTURE (input preparation): calls only the oracle's operator and
SciPy's shift-invert Arnoldi.

Reading of the shift rule: the workloads ask that the smallest |eigenvalue| of
D = D_0 + m I equal a target t while every eigenvalue keeps a positive real
part (Sec. 2.2: m is chosen so that eta_min(D) is positive and close to 0).
With the eigenvalues of D_0 nearest the left edge of the spectrum, f(m) =
min |lambda + m| increases with m once m > -eta_0 (eta_0 = min Re lambda), and
f(-eta_0 + t) >= t, so m is found by bisection on (-eta_0, -eta_0 + t].  If
f(-eta_0) > t already (the leftmost eigenvalues are a complex pair far from
the axis), eta_min(D) = t is used instead.

    python oracle/make_shifts.py [NAME ...]
"""
import json
import os
import sys
import time

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as sla

_HERE = os.path.dirname(os.path.abspath(__file__))
sys.path[0] = os.path.dirname(_HERE)  # repo root, not this folder
from oracle import oracle as O  # noqa: E402
from wl_inputs import workloads as W  # noqa: E402


def near_eigs(A, sigma, k):
    """k eigenvalues of A nearest sigma: shift-invert Arnoldi with a sparse
    LU (minimum-degree ordering on the structurally symmetric A + A^T)."""
    n = A.shape[0]
    lu = sla.splu((A - sigma * sp.identity(n, format="csc", dtype=A.dtype)).tocsc(),
                  permc_spec="MMD_AT_PLUS_A", options=dict(SymmetricMode=True))
    op = sla.LinearOperator(A.shape, matvec=lu.solve, dtype=A.dtype)
    mu = sla.eigs(op, k=k, which="LM", return_eigenvectors=False, tol=1e-10, ncv=max(2 * k + 1, 24))
    return sigma + 1.0 / mu


def shift_for(N, U, t):
    D0 = O.wilson_csr(N, U, 0.0).tocsc()
    ev = near_eigs(D0, 0.0, 12)
    eta0 = ev.real.min()
    ev = np.concatenate([ev, near_eigs(D0, eta0, 12)])
    f = lambda m: np.abs(ev + m).min()  # noqa: E731
    lo, hi = -eta0, -eta0 + t
    if f(lo) > t:
        m = -eta0 + t
        rule = "eta_min"
    else:
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if f(mid) < t:
                lo = mid
            else:
                hi = mid
        m = 0.5 * (lo + hi)
        rule = "min_abs"
    if N <= 128:   # independent check with a fresh factorisation of D itself
        check = near_eigs((D0 + m * sp.identity(D0.shape[0], format="csc")).tocsc(), 0.0, 6)
        min_abs = float(np.abs(check).min())
    else:          # the second Arnoldi run already brackets -m
        min_abs = float(np.abs(ev + m).min())
    return dict(m=float(m), rule=rule, eta0=float(eta0), min_abs=min_abs,
                min_re=float((ev + m).real.min()))


def eta0_for(N, U):
    """eta0 = min Re lambda(D_0): the eigenvalues nearest 0 locate the left
    edge of the spectrum, a second shift-invert run centred there refines
    it.  A run with eta_min(D) = eta then uses m = eta - eta0."""
    D0 = O.wilson_csr(N, U, 0.0).tocsc()
    ev = near_eigs(D0, 0.0, 12)
    eta0 = ev.real.min()
    ev = np.concatenate([ev, near_eigs(D0, eta0, 12)])
    return dict(eta0=float(ev.real.min()), m=None, rule="eta_sweep")


def _update(path, entries):
    """Merge entries into the JSON file under an exclusive lock, so that
    several runs on different workloads can proceed in parallel."""
    import fcntl
    with open(path + ".lock", "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        out = {}
        if os.path.exists(path):
            with open(path) as f:
                out = json.load(f)
        out.update(entries)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(out, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def main(names):
    path = os.path.join(os.path.dirname(_HERE), "wl_inputs", "shifts.json")
    for name in names:
        t0 = time.time()
        w = W.workload(name)
        if w.get("eta_sweep"):
            r = eta0_for(w["N"], w["U"])
        else:
            r = shift_for(w["N"], w["U"], w["target"])
        r["seconds"] = round(time.time() - t0, 1)
        entries = {name: r}
        for other, ow in W.WORKLOADS.items():   # workloads sharing this gauge and target
            if other != name and all(ow[k] == w[k] for k in ("N", "beta", "sweeps", "seed", "target")):
                entries[other] = dict(r, same_as=name)
        print(name, r, flush=True)
        _update(path, entries)


if __name__ == "__main__":
    main(sys.argv[1:] or ["T16", "T32", "T64", "C1", "C2"])
