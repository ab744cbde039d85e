"""Test inputs for the read exchange: each rank's slice of the reads, repacked
into a 2-bit stream of that rank's own layout (test input construction only)."""
from __future__ import annotations

from types import SimpleNamespace

import numpy as np


def unpack2(packed: np.ndarray) -> np.ndarray:
    """Base codes (0..3) of a 2-bit stream: base i from byte i >> 2, bits 2 (i & 3)."""
    p = np.asarray(packed, dtype=np.uint8)
    out = np.empty(p.size * 4, dtype=np.uint8)
    for k in range(4):
        out[k::4] = (p >> (2 * k)) & 3
    return out


def pack_codes(codes: np.ndarray) -> np.ndarray:
    """The 2-bit stream of base codes, padded to whole 16-byte units."""
    n = codes.size
    padded = np.zeros((n + 63) // 64 * 64, dtype=np.uint8)
    padded[:n] = codes
    q = padded.reshape(-1, 4)
    return (q[:, 0] | (q[:, 1] << 2) | (q[:, 2] << 4) | (q[:, 3] << 6)).astype(np.uint8)


def read_slices(G, read_first, lead: int = 3):
    """Per rank r: (stream, off) holding reads [read_first[r], read_first[r+1]),
    each read's bases copied from G's stream, laid out from base `lead` on with a
    gap of v % 5 bases after read v, so that the ranks' phases differ from the
    graph's own layout."""
    codes = unpack2(G.packed)
    out = []
    for r in range(len(read_first) - 1):
        a, b = int(read_first[r]), int(read_first[r + 1])
        pos = lead
        offs = np.empty(b - a, dtype=np.int64)
        parts = [np.zeros(lead, np.uint8)]
        for i, v in enumerate(range(a, b)):
            offs[i] = pos
            L = int(G.len[v])
            parts.append(codes[int(G.off[v]):int(G.off[v]) + L])
            gap = v % 5
            parts.append(np.zeros(gap, np.uint8))
            pos += L + gap
        out.append((pack_codes(np.concatenate(parts)), offs))
    return out


def without_reads(G):
    """G's graph arrays with no packed reads and the size of G's stream, for a
    load with NO_READS."""
    return SimpleNamespace(row_ptr=G.row_ptr, col=G.col, code=G.code, suf=G.suf, len=G.len, off=G.off, packed=None,
                           packed_bytes=int(G.packed.nbytes), pre=getattr(G, "pre", None),
                           post=getattr(G, "post", None))
