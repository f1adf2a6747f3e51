"""The hierarchy file (oracle/hierfile.py, read by the oracle and by the
library's amg_import): its checksum is FNV-1a 64, pinned to the published
test vectors of that hash, the same on the library's side
(wl_hash_bytes, host code, no GPU needed); a written hierarchy reads back
unchanged; corruption, truncation and a wrong magic are refused."""
import os

import numpy as np
import pytest

from oracle import hierfile as HF

# FNV-1a 64 test vectors (the FNV reference's published values)
VECTORS = [(b"", 0xcbf29ce484222325), (b"a", 0xaf63dc4c8601ec8c), (b"foobar", 0x85944171f73967e8)]


def test_fnv1a64_published_vectors():
    for data, want in VECTORS:
        assert HF.fnv1a64(data) == want, data


def test_library_hash_equals_the_file_format_hash():
    W = pytest.importorskip("paper_1308_5992_gb300.wilson_amg")
    try:
        W.lib()
    except (OSError, RuntimeError) as e:  # pragma: no cover - the build step makes it
        pytest.skip("library not built: %s" % e)
    for data, want in VECTORS:
        assert W.wl_hash_bytes(data) == want, data
    rng = np.random.default_rng(5)
    for n in (1, 7, 4096):
        data = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
        assert W.wl_hash_bytes(data) == HF.fnv1a64(data)


@pytest.fixture(scope="module")
def small(O, tmp_path_factory):
    from wl_inputs import workload
    w = workload("T32")
    h = O.Hierarchy.setup(w["N"], w["U"], w["m"], O.setup_params(w["blocks"], k_r=4, k_e=4, seed=w["seed"]))
    path = str(tmp_path_factory.mktemp("hf") / "t32.wlh")
    HF.write_hierarchy(path, h)
    return h, w, path


def test_round_trip(small):
    h, w, path = small
    d = HF.read(path)
    Pw, As = h.export()
    assert d["Nl"] == list(h.Nl) and d["Bl"] == list(h.Bl[: len(h.Nl) - 1])
    assert d["m"] == w["m"] and d["gauge_hash"] == HF.gauge_hash(w["U"])
    assert all(np.array_equal(a, b) for a, b in zip(d["Pw"], Pw))
    assert all(np.array_equal(a, b) for a, b in zip(d["As"], As))


def test_corruption_is_refused(small, tmp_path):
    h, w, path = small
    data = bytearray(open(path, "rb").read())
    cases = {"flip": None, "magic": None, "short": None}
    flip = bytearray(data)
    flip[len(flip) // 2] ^= 0x40
    cases["flip"] = flip
    magic = bytearray(data)
    magic[:8] = b"XLAMGH01"
    cases["magic"] = magic
    cases["short"] = data[:-24]
    for name, blob in cases.items():
        p = os.path.join(str(tmp_path), name + ".wlh")
        with open(p, "wb") as f:
            f.write(bytes(blob))
        with pytest.raises(ValueError):
            HF.read(p)
