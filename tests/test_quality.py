"""The synthetic quality table (gen/quality.py) on CPU: its parts against
brute force, and its sense on generated graphs assembled by the oracle."""
import numpy as np

import gen
import oracle
from gen import quality


def test_n50_and_union_brute_force():
    rng = np.random.default_rng(1)
    for _ in range(200):
        k = int(rng.integers(0, 12))
        s = rng.integers(0, 60, size=k)
        e = s + rng.integers(1, 20, size=k)
        cover = np.zeros(100, bool)
        for a, b in zip(s, e):
            cover[a:b] = True
        assert quality.covered_bases(s, e) == int(cover.sum())
        L = rng.integers(1, 50, size=max(k, 1))
        # N50 by definition: the largest L with sum of lengths >= L at least half the total
        best = max(x for x in L if L[L >= x].sum() * 2 >= L.sum())
        assert quality.n50(L) == best


def test_tiny_genome_assembly():
    G = gen.generate("tiny-1Mb", threads=4)
    orc = oracle.run(G, min_chain_reads=2)
    q = quality.contig_quality(G, orc.chain_id, orc.rank, orc.contig_off)
    assert q["contigs"] == orc.n_contigs and q["total_length"] == orc.total_bases
    assert q["longest_contig"] == int(np.diff(orc.contig_off).max())
    assert 0 < q["genome_fraction_pct"] <= 100
    assert q["joins"] == int(orc.chain_id[orc.chain_id >= 0].size) - orc.n_contigs
    # a contig built only from true overlaps spells a stretch of the genome (or
    # its reverse complement), so at least the contigs free of false joins match
    ok = 0
    for c in range(orc.n_contigs):
        seq = orc.contig(c)
        ok += any(seq in gen_seq for gen_seq in (_genome(G), _genome_rc(G)))
    assert ok >= q["contigs"] - q["misassembled_contigs"]


_cache = {}


def _genome(G):
    if "g" not in _cache:
        _cache["g"] = G.genome(0, G.cfg["genome_len"])
    return _cache["g"]


def _genome_rc(G):
    if "rc" not in _cache:
        _cache["rc"] = oracle.revcomp(_genome(G).decode()).encode()
    return _cache["rc"]


def test_false_join_is_counted():
    G = gen.generate("tiny-1Mb", threads=4)
    orc = oracle.run(G, min_chain_reads=2)
    q = quality.contig_quality(G, orc.chain_id, orc.rank, orc.contig_off)
    # mark the first join of contig 0 as false: one more misassembled contig at most
    H = type("H", (), {})()
    for k in ("row_ptr", "col", "len", "gstart", "cfg"):
        setattr(H, k, getattr(G, k))
    H.is_true = np.ones_like(G.is_true)
    q1 = quality.contig_quality(H, orc.chain_id, orc.rank, orc.contig_off)
    assert q1["misassembled_contigs"] == 0 and q1["false_joins"] == 0
    c0 = np.nonzero(orc.chain_id == orc.chain_id[orc.chain_id >= 0].min())[0]
    a, b = c0[np.argsort(orc.rank[c0])][:2]
    rp = np.asarray(G.row_ptr)
    x = rp[a] + int(np.nonzero(np.asarray(G.col)[rp[a]:rp[a + 1]] == b)[0][0])
    H.is_true[x] = 0
    q2 = quality.contig_quality(H, orc.chain_id, orc.rank, orc.contig_off)
    assert q2["misassembled_contigs"] == 1 and q2["false_joins"] == 1
    assert q["genome_fraction_pct"] == q2["genome_fraction_pct"]
