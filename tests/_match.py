"""Helpers for comparing particle sets whose order differs.

In 1D3V the field has only an x component, so a push never changes vy and vz
(Appendix A with E along x).  Their FP32 bit patterns therefore identify a
particle across a step, on the GPU and in the oracle alike; compaction of
absorbed particles reorders the GPU store, so comparisons match by this key.
"""
import numpy as np


def key_of(v: np.ndarray) -> np.ndarray:
    v32 = np.ascontiguousarray(np.asarray(v, dtype=np.float32).reshape(-1, 3))
    b = v32.view(np.uint32)
    return (b[:, 1].astype(np.uint64) << np.uint64(32)) | b[:, 2].astype(np.uint64)


def match(key_a: np.ndarray, key_b: np.ndarray):
    """Indices (ia, ib) with key_a[ia] == key_b[ib], for keys unique in b."""
    order = np.argsort(key_b, kind="stable")
    sb = key_b[order]
    pos = np.searchsorted(sb, key_a)
    pos = np.minimum(pos, sb.size - 1) if sb.size else pos
    ok = (sb.size > 0) & (sb[pos] == key_a) if sb.size else np.zeros(key_a.size, bool)
    ia = np.nonzero(ok)[0]
    return ia, order[pos[ok]]


def unique_keys(v: np.ndarray) -> bool:
    k = key_of(v)
    return np.unique(k).size == k.size


def periodic_diff(a, b, L):
    return (np.asarray(a) - np.asarray(b) + 0.5 * L) % L - 0.5 * L
