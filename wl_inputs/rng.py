"""Counter-based generator: the SplitMix64 output function (Steele, Lea &
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014).

    sm(z)             = mix13(z + 0x9E3779B97F4A7C15)
    u64(seed, s, i)   = sm(sm(sm(seed) + s) + i)        (all mod 2^64)
    uniform(seed,s,i) = ((u64 >> 11) + 1) * 2^-53        in (0, 1]
    cgauss(seed,s,i)  = Box-Muller on uniform(2i), uniform(2i+1):
                        sqrt(-2 ln u1) * (cos 2 pi u2 + i sin 2 pi u2)

Re and Im of cgauss are independent N(0, 1).  The definition is restated,
not shared, by every consumer that needs it.
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK = (1 << 64) - 1


def _sm_scalar(z: int) -> int:
    z = (z + 0x9E3779B97F4A7C15) & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def _sm_vec(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = z + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def rng_u64(seed: int, stream: int, idx) -> np.ndarray:
    key = _sm_scalar((_sm_scalar(int(seed) & _MASK) + int(stream)) & _MASK)
    i = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _sm_vec(i + np.uint64(key))


def uniform01(seed: int, stream: int, idx) -> np.ndarray:
    u = rng_u64(seed, stream, idx)
    return ((u >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def cgauss(seed: int, stream: int, n: int) -> np.ndarray:
    i = np.arange(n, dtype=np.uint64)
    u1 = uniform01(seed, stream, 2 * i)
    u2 = uniform01(seed, stream, 2 * i + np.uint64(1))
    r = np.sqrt(-2.0 * np.log(u1))
    t = 2.0 * np.pi * u2
    return r * np.cos(t) + 1j * (r * np.sin(t))
