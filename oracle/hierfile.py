"""Writer and reader of the hierarchy file format (TEST INFRASTRUCTURE): the
writer stores hierarchies built by the oracle, the reader loads a file that
either side wrote so the oracle can solve on the same operators.  Format,
little endian:

  "WLAMGH01" | int32 version = 1 | int32 L | int32 N[L] | int32 B[L] |
  float64 m | uint64 FNV-1a-64 of the gauge bytes (complex128 [2][N][N]) |
  complex128 P weights [n_l][2][4] for l = 0 .. L-2 |
  complex128 coarse stencils [n_l][9][2][2] for l = 1 .. L-1 |
  uint64 FNV-1a-64 of all preceding bytes
"""
import struct

import numpy as np

_FNV_OFF = 14695981039346656037  # FNV-1a 64 offset basis
_FNV_PRIME = 1099511628211


def fnv1a64(data: bytes, h: int = _FNV_OFF) -> int:
    # vectorised in blocks: h = (h ^ byte) * prime mod 2^64 is sequential, so
    # process bytes in a plain loop over a memoryview (fast enough for MBs)
    mask = (1 << 64) - 1
    for b in memoryview(data):
        h = ((h ^ b) * _FNV_PRIME) & mask
    return h


def gauge_hash(U) -> int:
    return fnv1a64(np.ascontiguousarray(U, dtype=np.complex128).tobytes())


def write(path, U, m, Nl, Bl, Pw, As):
    L = len(Nl)
    Bfull = list(Bl[: L - 1]) + [0]
    parts = [b"WLAMGH01", struct.pack("<ii", 1, L), struct.pack("<%di" % L, *Nl),
             struct.pack("<%di" % L, *Bfull), struct.pack("<d", float(m)),
             struct.pack("<Q", gauge_hash(U))]
    for l in range(L - 1):
        parts.append(np.ascontiguousarray(Pw[l], dtype=np.complex128).tobytes())
    for l in range(1, L):
        parts.append(np.ascontiguousarray(As[l - 1], dtype=np.complex128).tobytes())
    body = b"".join(parts)
    with open(path, "wb") as f:
        f.write(body)
        f.write(struct.pack("<Q", fnv1a64(body)))


def write_hierarchy(path, h):
    """h: oracle.Hierarchy"""
    Pw, As = h.export()
    write(path, h.U, h.m, h.Nl, h.Bl, Pw, As)


def read(path):
    """Parse a hierarchy file; returns dict(Nl, Bl (one per coarsening step),
    m, gauge_hash, Pw, As).  Raises ValueError on a bad magic, version, size
    or checksum."""
    with open(path, "rb") as f:
        data = f.read()
    if len(data) < 8 + 8 + 8 or data[:8] != b"WLAMGH01":
        raise ValueError("not a hierarchy file")
    body, (chk,) = data[:-8], struct.unpack("<Q", data[-8:])
    if fnv1a64(body) != chk:
        raise ValueError("hierarchy file checksum mismatch")
    ver, L = struct.unpack_from("<ii", body, 8)
    if ver != 1 or not 2 <= L <= 8:
        raise ValueError("unsupported hierarchy file (version %d, %d levels)" % (ver, L))
    off = 16
    Nl = list(struct.unpack_from("<%di" % L, body, off))
    off += 4 * L
    Bl = list(struct.unpack_from("<%di" % L, body, off))
    off += 4 * L
    (m,) = struct.unpack_from("<d", body, off)
    off += 8
    (gh,) = struct.unpack_from("<Q", body, off)
    off += 8
    Pw, As = [], []
    for l in range(L - 1):
        n = Nl[l] ** 2 // 2 * 8
        Pw.append(np.frombuffer(body, np.complex128, n, off).reshape(Nl[l] ** 2 // 2, 2, 4).copy())
        off += 16 * n
    for l in range(1, L):
        n = Nl[l] ** 2 // 2 * 36
        As.append(np.frombuffer(body, np.complex128, n, off).reshape(Nl[l] ** 2 // 2, 9, 2, 2).copy())
        off += 16 * n
    if off != len(body):
        raise ValueError("hierarchy file size mismatch")
    return dict(Nl=Nl, Bl=Bl[:L - 1], m=m, gauge_hash=gh, Pw=Pw, As=As)

