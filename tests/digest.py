"""SHA-256 of a factor / X exported from the library, in the byte layout
tests/golden/make_golden.py uses for the oracle's (int32 sign, int32 exp,
n uint32 limbs per number, little endian; factor column by column)."""
import hashlib

import numpy as np


def _update(h, s, e, m):
    s = np.ascontiguousarray(s, "<i4")
    e = np.ascontiguousarray(e, "<i4")
    m = np.ascontiguousarray(m, "<u4")
    rec = np.zeros(len(s), dtype=[("s", "<i4"), ("e", "<i4"), ("m", "<u4", (m.shape[1],))])
    rec["s"], rec["e"], rec["m"] = s, e, m
    h.update(rec.tobytes())


def factor_digest(h_, hk, N, chunk=65536):
    h = hashlib.sha256()
    total = N * (N + 1) // 2
    for first in range(0, total, chunk):
        cnt = min(chunk, total - first)
        _update(h, *h_.export(hk.HK_FACTOR, first, cnt))
    return h.hexdigest()


def x_digest(h_, hk, N, k):
    h = hashlib.sha256()
    _update(h, *h_.export(hk.HK_X, 0, N * k))
    return h.hexdigest()
