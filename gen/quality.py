"""Assembly quality against the generator's ground truth (evaluation only).

The synthetic counterpart of the contig quality table the paper reports with
QUAST (Table 4: number of contigs, longest contig, completeness, misassembled
contigs). The generator knows where every read came from, so no alignment is
needed:

- genome fraction: the share of genome bases that lie under at least one read
  placed in a contig (a read occurs verbatim at its placement);
- misassembled contigs: contigs whose walk joins two consecutive reads through
  an overlap the generator did not derive from their placements (a repeat
  overlap, `is_true` = 0);
- number of contigs, longest contig, total length and N50 from the contig
  offsets.

Inputs are the per-read chain id and rank of any implementation (the CUDA
path's cg_chains, or the oracle) and its contig offsets.
"""
from __future__ import annotations

import numpy as np


def n50(lengths) -> int:
    """The largest L such that contigs of length >= L hold at least half of all bases."""
    x = np.sort(np.asarray(lengths, dtype=np.int64))[::-1]
    if x.size == 0:
        return 0
    c = np.cumsum(x)
    return int(x[np.searchsorted(c, (c[-1] + 1) // 2)])


def covered_bases(starts, ends) -> int:
    """Size of the union of the half-open intervals [starts[i], ends[i])."""
    s = np.asarray(starts, dtype=np.int64)
    e = np.asarray(ends, dtype=np.int64)
    if s.size == 0:
        return 0
    o = np.argsort(s, kind="stable")
    s, e = s[o], e[o]
    reach = np.maximum.accumulate(e)
    # an interval starts a new merged run when it begins after everything before it ends
    new = np.ones(s.size, bool)
    new[1:] = s[1:] > reach[:-1]
    run = np.cumsum(new) - 1
    run_start = s[new]
    run_end = np.zeros(run_start.size, np.int64)
    np.maximum.at(run_end, run, e)
    return int((run_end - run_start).sum())


def entry_is_true(G, u, v) -> np.ndarray:
    """is_true of the CSR entries (u[i] -> v[i]); every pair must be an entry."""
    rp = np.asarray(G.row_ptr, dtype=np.int64)
    col = np.asarray(G.col, dtype=np.int64)
    n = rp.shape[0] - 1
    key = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp)) * n + col
    order = np.argsort(key, kind="stable")
    q = np.asarray(u, dtype=np.int64) * n + np.asarray(v, dtype=np.int64)
    pos = np.searchsorted(key[order], q)
    ok = (pos < key.size) & (key[order][np.minimum(pos, key.size - 1)] == q)
    if not ok.all():
        i = int(np.nonzero(~ok)[0][0])
        raise ValueError(f"reads {u[i]} and {v[i]} are consecutive in a contig but share no overlap entry")
    return np.asarray(G.is_true)[order[pos]].astype(np.uint8)


def contig_quality(G, chain_id, rank, contig_off, genome_len: int | None = None) -> dict:
    """Quality of one assembly of generated graph G (see the module docstring)."""
    cid = np.asarray(chain_id, dtype=np.int64)
    rk = np.asarray(rank, dtype=np.int64)
    lengths = np.diff(np.asarray(contig_off, dtype=np.int64))
    placed = np.nonzero(cid >= 0)[0]
    order = placed[np.lexsort((rk[placed], cid[placed]))]          # walk order, contig by contig
    same = cid[order][1:] == cid[order][:-1]
    u, v = order[:-1][same], order[1:][same]
    true = entry_is_true(G, u, v) if u.size else np.zeros(0, np.uint8)
    bad_contigs = np.unique(cid[u][true == 0])
    gl = int(genome_len if genome_len is not None else G.cfg["genome_len"])
    ln = np.asarray(G.len, dtype=np.int64)
    gs = np.asarray(G.gstart, dtype=np.int64)
    cov = covered_bases(gs[placed], gs[placed] + ln[placed])
    return {
        "contigs": int(lengths.size),
        "longest_contig": int(lengths.max()) if lengths.size else 0,
        "total_length": int(lengths.sum()),
        "n50": n50(lengths),
        "genome_fraction_pct": 100.0 * cov / gl if gl else 0.0,
        "misassembled_contigs": int(bad_contigs.size),
        "false_joins": int((true == 0).sum()),
        "joins": int(true.size),
    }
