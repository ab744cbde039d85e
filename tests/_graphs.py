"""Structured synthetic graphs in the input format, built directly with numpy
(test input only): long chains, closed chains, mixed strands, shuffled ids."""
from __future__ import annotations

from types import SimpleNamespace

import numpy as np


def structured(seed: int, sizes, closed=None, min_len=8, max_len=40, align=1, lone=0):
    """Chains of the given sizes (closed ones for the flags in `closed`), plus
    `lone` reads without overlaps; read ids are shuffled, strands random."""
    rng = np.random.default_rng(seed)
    closed = closed or [False] * len(sizes)
    n = int(sum(sizes)) + lone
    perm = rng.permutation(n).astype(np.int64)
    lens = rng.integers(min_len, max_len + 1, size=n).astype(np.int32)
    strand = rng.integers(0, 2, size=n).astype(np.int64)
    us, vs = [], []
    pos = 0
    for q, cl in zip(sizes, closed):
        ids = perm[pos:pos + q]
        if q >= 2:
            us.append(ids[:-1])
            vs.append(ids[1:])
        if cl and q >= 3:
            us.append(ids[-1:])
            vs.append(ids[:1])
        pos += q
    u = np.concatenate(us) if us else np.zeros(0, np.int64)
    v = np.concatenate(vs) if vs else np.zeros(0, np.int64)
    code_uv = (1 - strand[u]) | (strand[v] << 1)
    code_vu = ((code_uv & 1) << 1) | (code_uv >> 1)
    suf_uv = 1 + (rng.integers(0, 1 << 30, size=len(u)) % (lens[v] - 1))
    suf_vu = 1 + (rng.integers(0, 1 << 30, size=len(u)) % (lens[u] - 1))
    rows = np.concatenate([u, v])
    cols = np.concatenate([v, u])
    codes = np.concatenate([code_uv, code_vu]).astype(np.uint8)
    sufs = np.concatenate([suf_uv, suf_vu]).astype(np.int32)
    order = np.lexsort((cols, rows))
    rows, cols, codes, sufs = rows[order], cols[order], codes[order], sufs[order]
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, rows + 1, 1)
    rp = np.cumsum(rp)
    off = np.zeros(n, np.int64)
    stride = (lens.astype(np.int64) + align - 1) // align * align
    off[1:] = np.cumsum(stride)[:-1]
    total = int(off[-1] + stride[-1]) if n else 0
    packed = rng.integers(0, 256, size=max(1, (total + 3) // 4), dtype=np.uint8)
    return SimpleNamespace(row_ptr=rp, col=cols.astype(np.int32), code=codes, suf=sufs, len=lens, off=off,
                           packed=packed, n=n, m=len(cols))
