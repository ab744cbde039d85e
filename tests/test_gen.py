"""The seeded input generator: determinism and ground truth. The generator is
input only; these tests check that its graphs are what its recipe says."""
import hashlib

import numpy as np
import pytest

import gen
import oracle
from tests._pins import rc


def _digest(g):
    h = hashlib.sha256()
    for a in (g.row_ptr, g.col, g.code, g.suf, g.len, g.off, g.packed, g.is_true, g.gstart, g.strand, g.contained):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def test_deterministic_across_threads():
    a = gen.generate("tiny-1Mb", threads=1)
    b = gen.generate("tiny-1Mb", threads=7)
    assert _digest(a) == _digest(b)
    c = gen.generate(dict(gen.WORKLOADS["tiny-1Mb"](), seed=12345), threads=3)
    assert _digest(a) != _digest(c)


@pytest.mark.parametrize("align", [1, 4, 32])
def test_reads_are_genome_substrings(align):
    g = gen.generate("tiny-1Mb", threads=4, off_align=align)
    assert g.n == g.info["n_sampled"] == 1000
    codes = np.array([ord(c) for c in "ACGT"], dtype=np.uint8)
    for r in range(0, g.n, 7):
        o, L = int(g.off[r]), int(g.len[r])
        idx = np.arange(o, o + L)
        stored = codes[(g.packed[idx >> 2] >> (2 * (idx & 3))) & 3].tobytes().decode()
        truth = g.genome(int(g.gstart[r]), L).decode()
        assert stored == (truth if g.strand[r] == 0 else rc(truth))
        if align > 1:
            assert o % align == 0


def test_containment_and_transitive_reduction():
    g = gen.generate("tiny-1Mb", threads=4)
    s = g.gstart.astype(np.int64)
    e = s + g.len
    n = g.n
    # contained: [s,e) inside another read (ties broken as in the sorted order: the longer, earlier read stays)
    order = np.lexsort((-e, s))
    cont = np.zeros(n, bool)
    best_e = -1
    for r in order:
        if e[r] <= best_e:
            cont[r] = True
        best_e = max(best_e, e[r])
    assert np.array_equal(cont, g.contained.astype(bool))
    assert all(g.row_ptr[r + 1] == g.row_ptr[r] for r in np.nonzero(cont)[0])
    # true edges = transitive reduction of the >= 2 kb overlap graph of the non-contained reads
    keep = [int(r) for r in order if not cont[r]]
    ov = {}
    for i, a in enumerate(keep):
        for b in keep[i + 1:]:
            if s[b] >= e[a]:
                break
            if e[a] - s[b] >= 2000:
                ov.setdefault(a, set()).add(b)
    reduced = set()
    for a, succ in ov.items():
        for b in succ:
            if not any(b in ov.get(c, ()) for c in succ if c != b):
                reduced.add((min(a, b), max(a, b)))
    true_pairs = set()
    for u in range(n):
        for x in range(g.row_ptr[u], g.row_ptr[u + 1]):
            if g.is_true[x]:
                true_pairs.add((min(u, int(g.col[x])), max(u, int(g.col[x]))))
    assert true_pairs == reduced
    assert g.info["n_rep_pairs"] > 0


def test_generated_graphs_are_valid_string_graphs():
    for name in ("tiny-1Mb", "genome-100Mb"):
        g = gen.generate(name, threads=4)
        ok, msg = oracle.validate(g)
        assert ok, msg
    for j in (0, 511):
        g = gen.generate(gen.batched_graph(j), threads=4)
        assert oracle.validate(g)[0]
