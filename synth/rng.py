"""Counter-based random numbers (SplitMix64 finaliser + Box-Muller).

SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) maps a 64-bit counter to a
64-bit output with an add of the golden-ratio constant followed by two
xor-shift-multiply rounds.  Hashing (seed, stream, index) this way makes every
value addressable: element e of stream s under seed k is a pure function of
(k, s, e), so a block of a large tensor can be regenerated without drawing the
ones before it.

Normal deviates use the cosine branch of the Box-Muller transform on two
uniforms taken from counters 2e and 2e+1.
"""

from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM_MUL = np.uint64(0xD1B54A32D192ED03)


def _mix(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied elementwise to uint64 counters."""
    with np.errstate(over="ignore"):
        z = x + _GOLDEN
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def _key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        k = _mix(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
        k ^= _mix(np.array([(stream * 0x632BE59BD9B4E019) & 0xFFFFFFFFFFFFFFFF],
                           dtype=np.uint64))[0] * _STREAM_MUL
    return np.uint64(k)


def _raw(seed: int, stream: int, counters: np.ndarray) -> np.ndarray:
    key = _key(seed, stream)
    with np.errstate(over="ignore"):
        return _mix(counters ^ key)


def _to_unit_open(raw: np.ndarray) -> np.ndarray:
    """53 high bits -> (0, 1]."""
    return ((raw >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def _to_unit_half(raw: np.ndarray) -> np.ndarray:
    """53 high bits -> [0, 1)."""
    return (raw >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_stream(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Uniform [0,1) values for counters start .. start+count-1."""
    idx = np.arange(start, start + count, dtype=np.uint64)
    return _to_unit_half(_raw(seed, stream, idx))


def _normal_chunk(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    idx = np.arange(start, start + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        two = idx * np.uint64(2)
        u1 = _to_unit_open(_raw(seed, stream, two))
        u2 = _to_unit_half(_raw(seed, stream, two + np.uint64(1)))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos((2.0 * np.pi) * u2)


def normal_stream(seed: int, stream: int, start: int, count: int,
                  out: np.ndarray | None = None, threads: int | None = None) -> np.ndarray:
    """N(0,1) deviates for element counters start .. start+count-1.

    Large requests are split across threads (numpy releases the GIL inside
    its ufuncs); the values do not depend on the split.
    """
    if out is None:
        out = np.empty(count, dtype=np.float64)
    chunk = 1 << 22
    if count <= chunk:
        out[:count] = _normal_chunk(seed, stream, start, count)
        return out
    nthreads = threads or min(32, os.cpu_count() or 1)

    def work(i0: int) -> None:
        n = min(chunk, count - i0)
        out[i0:i0 + n] = _normal_chunk(seed, stream, start + i0, n)

    with ThreadPoolExecutor(max_workers=nthreads) as ex:
        list(ex.map(work, range(0, count, chunk)))
    return out
