"""Pins for the CPU oracle: checks against what the paper and the mathematics
fix, independent of the oracle's own code. Each pin takes an OracleLib (the
default oracle, or a copy with a planted mistake) and raises AssertionError
when the oracle disagrees.

Sources of truth used here:
  * worked examples printed in the paper (tests/golden/*.txt, each cited);
  * brute force: every maximal valid walk of the unbranched graph, enumerated
    directly from the definition of a valid walk (Sec. 2) and of the contig
    set (Sec. 4.2) on tiny random graphs;
  * the generator's ground truth (true read positions and strands);
  * structural invariants stated in Sec. 4.4 (roots, intermediates, 2(q-1)
    edge entries) and Graham's LPT bound quoted in Sec. 4.3;
  * a library routine (networkx connected components) for the labels.
"""
from __future__ import annotations

import itertools
import os
import random
from types import SimpleNamespace

import numpy as np

import gen

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
_COMP = str.maketrans("ACGT", "TGCA")


def rc(s: str) -> str:
    """Reverse complement written from Sec. 2 (A<->T, C<->G, reversed)."""
    return s.translate(_COMP)[::-1]


def golden(name: str):
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(line.split())
    return out


def graph_from(reads, entries, align=1):
    """Graph in the input format from ASCII reads and (u, v, code, suf) entries."""
    ln, off, packed = gen.pack_reads(reads, align)
    rp, col, code, suf = gen.csr_from_entries(len(reads), entries)
    return SimpleNamespace(row_ptr=rp, col=col, code=code, suf=suf, len=ln, off=off, packed=packed,
                           n=len(reads), m=len(col), reads=list(reads))


def swap(code: int) -> int:
    return ((code & 1) << 1) | (code >> 1)


def contigs_of(res) -> list[str]:
    return [res.contig(i).decode() for i in range(res.n_contigs)]


# ------------------------------------------------------------------ paper
def pin_paper_mask_example(orc):
    """Sec. 4.2: v3 (degree 3) is masked; chains {v1,v2}, {v4,v5,v6}, {v7,v8}."""
    g = {k[0]: k[1:] for k in golden("paper_mask_example.txt")}
    pairs = [tuple(int(x[1:]) - 1 for x in e.split("-")) for e in g["edges"]]
    rnd = random.Random(7)
    reads = ["".join(rnd.choice("ACGT") for _ in range(12)) for _ in range(8)]
    # every read forward, each overlap joins the 3' end of u to the 5' end of v
    ent = []
    for u, v in pairs:
        ent.append((u, v, 1 | (0 << 1), 5))
        ent.append((v, u, swap(1), 4))
    G = graph_from(reads, ent)
    for mcr in (1, 2):
        res = orc.run(G, min_chain_reads=mcr)
        want_branch = {int(x[1:]) - 1 for x in g["branches"]}
        assert set(np.nonzero(res.is_branch)[0].tolist()) == want_branch, "masked set"
        chains = [[int(x.strip()[1:]) - 1 for x in c.strip().split(",")] for c in " ".join(g["chains"]).split("|")]
        assert res.n_contigs == len(chains)
        for c in chains:
            assert all(res.chain_id[v] == min(c) for v in c), "chain membership"
            assert sorted(res.rank[v] for v in c) == list(range(len(c)))
        assert res.chain_id[2] == -1 and res.orient[2] == 255


def _prepost_contig(reads, pp):
    """The paper's concatenation formula on (pre, post) pairs, forward reads."""
    names = list(reads)
    out = reads[names[0]][0:pp[0][2] + 1]
    for i in range(1, len(names) - 1):
        out += reads[names[i]][pp[i - 1][3]:pp[i][2] + 1]
    out += reads[names[-1]][pp[-1][3]:]
    return out


def _concat_graph(stored1_rc: bool):
    lines = golden("paper_concat_example.txt")
    reads = {l[1]: l[2] for l in lines if l[0] == "read"}
    pp = [(l[1], l[2], int(l[3]), int(l[4])) for l in lines if l[0] == "prepost"]
    want = [l[1] for l in lines if l[0] == "contig"][0]
    assert _prepost_contig(reads, pp) == want, "fixture self-check"
    l0, l1, l2 = reads["l0"], reads["l1"], reads["l2"]
    # suffix of v beyond the overlap = |l_v| - post - (|l_u| - 1 - pre)
    s01 = len(l1) - pp[0][3] - (len(l0) - 1 - pp[0][2])
    s12 = len(l2) - pp[1][3] - (len(l1) - 1 - pp[1][2])
    # walking back: the bases of u before its overlap with v
    s10 = pp[0][2] + 1
    s21 = pp[1][2] + 1
    if not stored1_rc:
        ent = [(0, 1, 1 | (0 << 1), s01), (1, 0, swap(1), s10), (1, 2, 1 | (0 << 1), s12), (2, 1, swap(1), s21)]
        return graph_from([l0, l1, l2], ent), want
    # l1 stored as its reverse complement: l0 meets its 3' end, l2 its 5' end
    ent = [(0, 1, 1 | (1 << 1), s01), (1, 0, swap(3), s10), (1, 2, 0 | (0 << 1), s12), (2, 1, swap(0), s21)]
    return graph_from([l0, rc(l1), l2], ent), want


def pin_paper_concat_example(orc):
    """Sec. 4.4 / Fig. 3: l0, l1, l2 with (pre, post) = (1,0), (4,2) spell AGAACTGAAGAA."""
    G, want = _concat_graph(False)
    for mcr in (1, 2, 3):
        res = orc.run(G, min_chain_reads=mcr)
        assert res.n_branch == 0
        assert contigs_of(res) == [want]
        assert res.rank.tolist() == [0, 1, 2] and res.orient.tolist() == [0, 0, 0]
    res = orc.run(G, min_chain_reads=4)
    assert res.n_contigs == 0 and res.chain_id.tolist() == [-1, -1, -1]


def pin_paper_rc_example(orc):
    """Sec. 4.4: l1 may be stored as its reverse complement CTTCAGTT; the contig is unchanged."""
    G, want = _concat_graph(True)
    assert G.reads[1] == [l[2] for l in golden("paper_revcomp_example.txt") if l[1] == "AACTGAAG"][0]
    res = orc.run(G)
    assert contigs_of(res) == [want]
    assert res.orient.tolist() == [0, 1, 0]


def pin_revcomp(orc):
    """Sec. 2: the reverse complement of ATTCG is CGAAT."""
    for _, s, want in golden("paper_revcomp_example.txt"):
        assert orc.revcomp(s) == want


def pin_same_end_rule(orc):
    """Sec. 2: a valid walk enters a read through one end and leaves through the
    other, so a read whose two overlaps both touch its 3' end is a branch; a
    read with one overlap per end is not."""
    reads = ["ACGTACGTAC", "CCGGTTAACC", "GATTACAGAT"]
    # read 1 (middle) has both overlaps on its 3' end
    ent = [(0, 1, 1 | (1 << 1), 6), (1, 0, swap(3), 5), (1, 2, 1 | (0 << 1), 7), (2, 1, swap(1), 5)]
    res = orc.run(graph_from(reads, ent), min_chain_reads=1)
    assert res.is_branch.tolist() == [0, 1, 0]
    assert res.n_contigs == 2 and contigs_of(res) == [reads[0], reads[2]]
    ent = [(0, 1, 1 | (0 << 1), 6), (1, 0, swap(1), 5), (1, 2, 1 | (0 << 1), 7), (2, 1, swap(1), 5)]
    res = orc.run(graph_from(reads, ent), min_chain_reads=1)
    assert res.is_branch.tolist() == [0, 0, 0] and res.n_contigs == 1
    # the rule looks only at overlaps left after removing degree >= 3 reads:
    # read 1 keeps one overlap (to read 0) once read 2 (degree 3) is gone
    reads5 = reads + ["TTGACCAGTA", "ACCATGGTCA"]
    ent = [(0, 1, 1 | (1 << 1), 6), (1, 0, swap(3), 5), (1, 2, 1 | (0 << 1), 7), (2, 1, swap(1), 5),
           (2, 3, 1, 4), (3, 2, swap(1), 4), (2, 4, 0, 3), (4, 2, swap(0), 3)]
    res = orc.run(graph_from(reads5, ent), min_chain_reads=1)
    assert res.is_branch.tolist() == [0, 0, 1, 0, 0]
    assert res.chain_id.tolist()[:2] == [0, 0]


# ------------------------------------------------------------ brute force
def random_tiny_graph(rnd: random.Random, n: int, p_edge: float, min_len=4, max_len=9):
    reads = ["".join(rnd.choice("ACGT") for _ in range(rnd.randint(min_len, max_len))) for _ in range(n)]
    ent = []
    for u, v in itertools.combinations(range(n), 2):
        if rnd.random() < p_edge:
            c = rnd.randrange(4)
            ent.append((u, v, c, rnd.randint(1, len(reads[v]) - 1)))
            ent.append((v, u, swap(c), rnd.randint(1, len(reads[u]) - 1)))
    return graph_from(reads, ent)


def random_chain_graph(rnd: random.Random, n: int, n_extra: int):
    """Reads on one or more paths/cycles with random strands, plus a few random extra edges."""
    reads = ["".join(rnd.choice("ACGT") for _ in range(rnd.randint(5, 10))) for _ in range(n)]
    order = list(range(n))
    rnd.shuffle(order)
    strand = [rnd.randrange(2) for _ in range(n)]
    have, ent = set(), []

    def add(u, v, c):
        if u == v or (min(u, v), max(u, v)) in have:
            return
        have.add((min(u, v), max(u, v)))
        ent.append((u, v, c, rnd.randint(1, len(reads[v]) - 1)))
        ent.append((v, u, swap(c), rnd.randint(1, len(reads[u]) - 1)))

    i = 0
    while i < n:
        k = rnd.randint(1, n - i)
        seg = order[i:i + k]
        for a, b in zip(seg, seg[1:]):
            add(a, b, (1 - strand[a]) | (strand[b] << 1))
        if k >= 3 and rnd.random() < 0.3:       # close it into a cycle
            add(seg[-1], seg[0], (1 - strand[seg[-1]]) | (strand[seg[0]] << 1))
        i += k
    for _ in range(n_extra):
        add(rnd.randrange(n), rnd.randrange(n), rnd.randrange(4))
    return graph_from(reads, ent)


def brute_force_contigs(G, is_branch, min_chain_reads):
    """Contig set by enumeration: all maximal valid walks of L (Sec. 2, 4.2)."""
    n = G.n
    adj = {v: [] for v in range(n)}                       # (w, E_v, E_w, suf(v->w))
    for v in range(n):
        if is_branch[v]:
            continue
        for x in range(G.row_ptr[v], G.row_ptr[v + 1]):
            w = int(G.col[x])
            if not is_branch[w]:
                adj[v].append((w, int(G.code[x]) & 1, int(G.code[x]) >> 1, int(G.suf[x])))
    alive = [v for v in range(n) if not is_branch[v]]

    def nexts(v, o):
        return [(w, ew, s) for (w, ev, ew, s) in adj[v] if ev == 1 - o]

    def prevs(v, o):
        return [(w, 1 - ew) for (w, ev, ew, s) in adj[v] if ev == o]

    walks = []
    for s in alive:
        for o in (0, 1):
            stack = [[(s, o)]]
            while stack:
                w = stack.pop()
                seen = {r for r, _ in w}
                ext = [(x, ox) for x, ox, _ in nexts(*w[-1]) if x not in seen]
                closes = any(x == w[0][0] and ox == w[0][1] for x, ox, _ in nexts(*w[-1]))
                if ext:
                    for x, ox in ext:
                        stack.append(w + [(x, ox)])
                    continue
                pre_ext = [p for p in prevs(*w[0]) if p[0] not in seen]
                if pre_ext:
                    continue
                walks.append((tuple(w), closes))

    def suf_of(u, v):
        for x in range(G.row_ptr[u], G.row_ptr[u + 1]):
            if G.col[x] == v:
                return int(G.suf[x])
        raise AssertionError("no edge")

    def spell(w):
        out = G.reads[w[0][0]] if w[0][1] == 0 else rc(G.reads[w[0][0]])
        for (u, _), (v, ov) in zip(w, w[1:]):
            s = G.reads[v] if ov == 0 else rc(G.reads[v])
            out += s[len(s) - suf_of(u, v):]
        return out

    contigs = {}
    for w, closes in walks:
        reads = frozenset(r for r, _ in w)
        if closes and len(w) >= 3:
            m = min(reads)
            k = [r for r, _ in w].index(m)
            rot = w[k:] + w[:k]
            if rot[0][1] != 0:
                continue                              # the other direction of the cycle
            contigs[reads] = (rot, True)
        else:
            if w[0][0] > w[-1][0] or (len(w) == 1 and w[0][1] != 0):
                continue                              # keep the copy from the smaller-id end
            contigs[reads] = (w, False)
    out = []
    for reads, (w, cyc) in sorted(contigs.items(), key=lambda kv: min(kv[0])):
        if len(w) >= min_chain_reads:
            out.append((min(reads), w, spell(w), cyc))
    return out


def brute_force_mask(G):
    """Branch reads from first principles: degree >= 3 in S (Sec. 4.2), or a
    read with exactly two neighbours left after that whose two overlaps admit
    no valid walk u -> v -> w through it (Sec. 2), found by trying every such
    walk."""
    n = G.n
    deg = [int(G.row_ptr[v + 1] - G.row_ptr[v]) for v in range(n)]
    b1 = [d >= 3 for d in deg]
    out = list(b1)
    for v in range(n):
        if b1[v]:
            continue
        nb = [(int(G.col[x]), int(G.code[x])) for x in range(G.row_ptr[v], G.row_ptr[v + 1]) if not b1[G.col[x]]]
        if len(nb) != 2:
            continue
        passable = False
        for (u, cu), (w, cw) in ((nb[0], nb[1]), (nb[1], nb[0])):
            for o_v in (0, 1):
                # enter v from u through end o_v, leave to w through end 1 - o_v
                if (cu & 1) == o_v and (cw & 1) == 1 - o_v:
                    passable = True
        out[v] = not passable
    return np.array(out, dtype=np.uint8)


def check_brute_force(orc, G, mcr):
    res = orc.run(G, min_chain_reads=mcr)
    assert np.array_equal(res.is_branch, brute_force_mask(G)), "branch mask"
    bf = brute_force_contigs(G, res.is_branch, mcr)
    assert res.n_contigs == len(bf), "contig count"
    assert contigs_of(res) == [b[2] for b in bf], "contig strings"
    for cid, w, _, _ in bf:
        for k, (r, o) in enumerate(w):
            assert res.chain_id[r] == cid and res.rank[r] == k and res.orient[r] == o, "per-read chain arrays"
    assert res.n_cycles == sum(1 for b in bf if b[3]) or mcr > 3
    # no surviving read breaks the valid-walk rule (Sec. 2)
    for v in range(G.n):
        if res.is_branch[v]:
            continue
        ends = [int(G.code[x]) & 1 for x in range(G.row_ptr[v], G.row_ptr[v + 1]) if not res.is_branch[G.col[x]]]
        assert len(ends) <= 2 and len(set(ends)) == len(ends), "surviving read with a bad end pair"


def pin_brute_force(orc, n_graphs=120, seed=11):
    rnd = random.Random(seed)
    for t in range(n_graphs):
        if t % 2 == 0:
            G = random_tiny_graph(rnd, rnd.randint(1, 7), rnd.choice([0.15, 0.3, 0.5]))
        else:
            G = random_chain_graph(rnd, rnd.randint(1, 9), rnd.randint(0, 2))
        check_brute_force(orc, G, rnd.choice([1, 2]))


def pin_cycles(orc):
    """Closed chains: a 4-cycle with mixed strands starts at its smallest read,
    forward, and leaves through its 3' end."""
    rnd = random.Random(3)
    reads = ["".join(rnd.choice("ACGT") for _ in range(8)) for _ in range(4)]
    strand = [0, 1, 1, 0]
    cyc = [2, 0, 3, 1]
    ent = []
    for a, b in zip(cyc, cyc[1:] + cyc[:1]):
        c = (1 - strand[a]) | (strand[b] << 1)
        ent.append((a, b, c, rnd.randint(1, 7)))
        ent.append((b, a, swap(c), rnd.randint(1, 7)))
    G = graph_from(reads, ent)
    res = orc.run(G)
    assert res.n_cycles == 1 and res.n_contigs == 1
    assert res.rank[0] == 0 and res.orient[0] == 0
    check_brute_force(orc, G, 2)


# -------------------------------------------------------- generated graphs
_cache = {}


def tiny_generated():
    if "tiny" not in _cache:
        _cache["tiny"] = gen.generate("tiny-1Mb", threads=4)
    return _cache["tiny"]


def small_generated(seed):
    key = ("small", seed)
    if key not in _cache:
        d = gen._cfg(seed, 300_000, [(0.08, 3000, 6000, 4, 10, 0.0)], 12, 1, 6000, 3000, 2500)
        _cache[key] = gen.generate(d, threads=4, off_align=1 if seed % 2 else 32)
    return _cache[key]


def chains_of(res):
    """{chain_id: [reads in rank order]} from the per-read arrays."""
    out = {}
    idx = np.nonzero(res.chain_id >= 0)[0]
    for v in idx[np.lexsort((res.rank[idx], res.chain_id[idx]))]:
        out.setdefault(int(res.chain_id[v]), []).append(int(v))
    return out


def entry(G, u, v):
    for x in range(int(G.row_ptr[u]), int(G.row_ptr[u + 1])):
        if G.col[x] == v:
            return x
    return None


def pin_generator_truth(orc):
    """Chains made only of true overlaps spell genome[a, b) (or its reverse
    complement), a = first true base and b = last, from the read positions."""
    checked = 0
    for G in [tiny_generated()] + [small_generated(s) for s in (101, 102)]:
        res = orc.run(G, min_chain_reads=2)
        for i, (cid, reads) in enumerate(sorted(chains_of(res).items())):
            xs = [entry(G, a, b) for a, b in zip(reads, reads[1:])]
            if any(x is None or not G.is_true[x] for x in xs):
                continue
            a = min(int(G.gstart[r]) for r in reads)
            b = max(int(G.gstart[r]) + int(G.len[r]) for r in reads)
            seq = res.contig(i).decode()
            truth = G.genome(a, b - a).decode()
            assert seq == truth or seq == rc(truth), "true chain does not spell the genome"
            checked += 1
    assert checked >= 10


def pin_invariants(orc):
    """Sec. 4.4 structure: every unmasked read in exactly one contig (with
    singletons allowed), contig length = first read + suffixes, two roots and
    q-2 intermediates per path, 2(q-1) edge entries per path walk."""
    import networkx as nx
    for G in [tiny_generated(), small_generated(101), small_generated(102)]:
        res1 = orc.run(G, min_chain_reads=1)
        unmasked = res1.is_branch == 0
        assert np.array_equal(res1.chain_id >= 0, unmasked)
        ch = chains_of(res1)
        assert res1.n_contigs == len(ch) == res1.n_components
        assert np.array_equal(res1.label_uf, res1.label_bfs)
        # labels against a library connected-components routine on L
        H = nx.Graph()
        H.add_nodes_from(int(v) for v in np.nonzero(unmasked)[0])
        for u in np.nonzero(unmasked)[0]:
            for x in range(int(G.row_ptr[u]), int(G.row_ptr[u + 1])):
                if unmasked[G.col[x]]:
                    H.add_edge(int(u), int(G.col[x]))
        for comp in nx.connected_components(H):
            lab = {int(res1.label_uf[v]) for v in comp}
            assert lab == {min(comp)}
        walked = 0
        for i, (cid, reads) in enumerate(sorted(ch.items())):
            q = len(reads)
            tot = int(G.len[reads[0]])
            for a, b in zip(reads, reads[1:]):
                x = entry(G, a, b)
                assert x is not None
                tot += int(G.suf[x])
                # the walk leaves a through end 1-o_a and enters b through o_b
                assert (int(G.code[x]) & 1) == 1 - res1.orient[a] and (int(G.code[x]) >> 1) == res1.orient[b]
            assert tot == res1.contig_off[i + 1] - res1.contig_off[i]
            degs = [sum(1 for x in range(int(G.row_ptr[v]), int(G.row_ptr[v + 1])) if unmasked[G.col[x]]) for v in reads]
            closed = q >= 3 and entry(G, reads[-1], reads[0]) is not None
            if q >= 2 and not closed:
                assert sorted(degs).count(1) == 2 and degs.count(2) == q - 2
                walked += 2 * (q - 1)
            elif closed:
                walked += 2 * q
            assert cid == min(reads)
            assert reads[0] == (min(reads) if closed else min(reads[0], reads[-1]))
        assert walked == res1.edges_walked
        res2 = orc.run(G, min_chain_reads=2)
        assert res2.n_contigs == sum(1 for r in ch.values() if len(r) >= 2)
        keep = np.concatenate([[0], np.cumsum([res1.contig_off[i + 1] - res1.contig_off[i]
                                               for i, r in enumerate(sorted(ch.items())) if len(r[1]) >= 2])])
        assert np.array_equal(res2.contig_off, keep)


# ------------------------------------------------------------------- LPT
def _opt_makespan(sizes, P):
    best = None
    for assign in itertools.product(range(P), repeat=len(sizes)):
        loads = [0] * P
        for s, b in zip(sizes, assign):
            loads[b] += s
        m = max(loads)
        best = m if best is None or m < best else best
    return best


def pin_lpt(orc):
    """Sec. 4.3: sorted greedy partitioning is within (4P-1)/(3P) of optimal;
    Graham's tight example reaches the bound."""
    g = {k[0]: k[1:] for k in golden("graham_lpt_tight.txt")}
    P = int(g["P"][0])
    sizes = [int(x) for x in g["sizes"]]
    assign, loads = orc.lpt(sizes, P)
    assert int(loads.max()) == int(g["lpt_makespan"][0])
    assert _opt_makespan(sizes, P) == int(g["optimum"][0])
    for b in range(P):
        assert loads[b] == sum(s for s, a in zip(sizes, assign) if a == b)
    # the tie rules, on a hand-worked example: equal sizes in input order, ties to the lowest part
    t = {k[0]: k[1:] for k in golden("lpt_ties.txt")}
    assign, loads = orc.lpt([int(x) for x in t["sizes"]], int(t["P"][0]))
    assert [int(a) for a in assign] == [int(x) for x in t["assign"]]
    assert [int(x) for x in loads] == [int(x) for x in t["loads"]]
    rnd = random.Random(5)
    for _ in range(60):
        P = rnd.randint(1, 4)
        k = rnd.randint(1, 8 if P > 2 else 10)
        sizes = [rnd.randint(1, 30) for _ in range(k)]
        assign, loads = orc.lpt(sizes, P)
        opt = _opt_makespan(sizes, P)
        assert int(loads.max()) * 3 * P <= (4 * P - 1) * opt
        assert all(0 <= a < P for a in assign)
        for b in range(P):
            assert loads[b] == sum(s for s, a in zip(sizes, assign) if a == b)


# ------------------------------------------------------------- validation
def pin_validation(orc):
    """Malformed graphs are rejected: each planted defect breaks one rule of a
    string graph (Sec. 2, 4.2)."""
    G, _ = _concat_graph(False)
    ok, msg = orc.validate(G)
    assert ok, msg

    def variant(**kw):
        H = SimpleNamespace(**{k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in vars(G).items()})
        for k, f in kw.items():
            f(getattr(H, k))
        return H

    bad = [
        variant(code=lambda c: c.__setitem__(1, 0)),               # mirror code not swapped
        variant(col=lambda c: c.__setitem__(0, 7)),                # column out of range
        variant(col=lambda c: c.__setitem__(0, 0)),                # self overlap
        variant(suf=lambda s: s.__setitem__(0, 0)),                # empty suffix
        variant(suf=lambda s: s.__setitem__(0, 8)),                # suffix = whole read
        variant(code=lambda c: c.__setitem__(0, 4)),               # code out of range
        variant(off=lambda o: o.__setitem__(2, 10**6)),            # read outside the stream
        variant(off=lambda o: o.__setitem__(0, -1)),               # read starting before the stream
        variant(len=lambda ln: ln.__setitem__(0, 0)),               # empty read
    ]
    for H in bad:
        ok, _ = orc.validate(H)
        assert not ok
    # duplicate pair and missing mirror: rebuild the CSR
    l0, l1, l2 = G.reads
    dup = graph_from(G.reads, [(0, 1, 1, 4), (0, 1, 1, 3), (1, 0, 2, 2), (1, 2, 1, 2), (2, 1, 2, 5)])
    assert not orc.validate(dup)[0]
    nomirror = graph_from(G.reads, [(0, 1, 1, 4), (1, 0, 2, 2), (1, 2, 1, 2)])
    assert not orc.validate(nomirror)[0]
    # a read overlapping itself and nothing else wrong: code 3 is its own mirror (its two
    # end bits swapped), the suffix is in range, no pair repeats
    selfloop = graph_from([l0], [(0, 0, 3, 2)])
    assert not orc.validate(selfloop)[0]
    H = variant(row_ptr=lambda r: r.__setitem__(1, 5))             # row_ptr not monotone
    assert not orc.validate(H)[0]
    # one entry more than row_ptr[n] counts (a well-formed entry after the last row)
    H = variant()
    H.col, H.code, H.suf = (np.append(a, a[0]).astype(a.dtype) for a in (G.col, G.code, G.suf))
    assert not orc.validate(H)[0]
    # the packed stream's end: a read whose last base is the stream's last base is
    # in bounds, one base further is not
    end = len(G.packed) * 4
    H = variant(off=lambda o: o.__setitem__(2, end - int(G.len[2])))
    assert orc.validate(H)[0]
    H = variant(off=lambda o: o.__setitem__(2, end - int(G.len[2]) + 1))
    assert not orc.validate(H)[0]


# ------------------------------------------------------------ x-drop form
def _xdrop_cases():
    """The cases of xdrop_examples.txt: name -> (reads, [(pre, post) of l0->l1, of l1->l2], contig)."""
    out, cur = {}, None
    for row in golden("xdrop_examples.txt"):
        if row[0] == "case":
            cur = out.setdefault(row[1], {"reads": {}, "pp": [], "contig": None})
        elif row[0] == "read":
            cur["reads"][row[1]] = row[2]
        elif row[0] == "prepost":
            cur["pp"].append((int(row[3]), int(row[4])))
        elif row[0] == "contig":
            cur["contig"] = row[1]
    return out


def xdrop_chain(reads, pp, stored1_rc: bool):
    """l0 - l1 - l2 in the x-drop form. pp holds the walk-direction (pre, post)
    of the entries l0->l1 and l1->l2 in l1's walk coordinates; with stored1_rc
    l1 is stored as its reverse complement, so its indices become 7 - i and
    the codes change ends. The mirror entries get in-range values (the
    canonical walk starts at l0 and never uses them)."""
    l0, l1, l2 = reads["l0"], reads["l1"], reads["l2"]
    L1 = len(l1)
    t = (lambda i: L1 - 1 - i) if stored1_rc else (lambda i: i)
    (pre01, post01), (pre12, post12) = pp
    if not stored1_rc:
        codes = {(0, 1): 1, (1, 0): 2, (1, 2): 1, (2, 1): 2}
    else:
        codes = {(0, 1): 3, (1, 0): 3, (1, 2): 0, (2, 1): 0}
    vals = {(0, 1): (pre01, t(post01)), (1, 2): (t(pre12), post12),
            (1, 0): (t(4), len(l0) - 1), (2, 1): (len(l2) - 2, t(L1 - 1))}
    keys = sorted(vals)
    ent = [(u, v, codes[(u, v)], 1) for u, v in keys]
    G = graph_from([l0, rc(l1) if stored1_rc else l1, l2], ent)
    G.suf = None
    G.pre = np.array([vals[k][0] for k in keys], np.int32)
    G.post = np.array([vals[k][1] for k in keys], np.int32)
    return G


def pin_xdrop_examples(orc):
    """Sec. 4.4, x-drop form: the paper's (pre, post) example spells
    AGAACTGAAGAA; an overlap reported one base later on one read skips that
    base; crossing overlaps leave the middle read empty; overlaps meeting at
    one base of the middle read let it add exactly that base (hand-derived)."""
    for name, c in _xdrop_cases().items():
        for stored1_rc in (False, True):
            G = xdrop_chain(c["reads"], c["pp"], stored1_rc)
            ok, msg = orc.validate(G)
            assert ok, (name, msg)
            for mcr in (1, 3):
                res = orc.run(G, min_chain_reads=mcr)
                assert contigs_of(res) == [c["contig"]], (name, stored1_rc)
                assert res.rank.tolist() == [0, 1, 2]
                assert res.orient.tolist() == [0, 1 if stored1_rc else 0, 0]


def circular_graph(seed: int, genome_len: int = 600, read_len: int = 90, step: int = 30):
    """Reads tiling a circular genome at a fixed step, random strands: one
    closed chain whose overlaps are exact (test input)."""
    rnd = random.Random(seed)
    genome = "".join(rnd.choice("ACGT") for _ in range(genome_len))
    q = genome_len // step
    reads, strand = [], []
    for i in range(q):
        s = (genome + genome)[i * step: i * step + read_len]
        st = rnd.randint(0, 1)
        reads.append(rc(s) if st else s)
        strand.append(st)
    ent = []
    for i in range(q):
        u, v = i, (i + 1) % q
        code = (1 - strand[u]) | (strand[v] << 1)
        ent.append((u, v, code, step))
        ent.append((v, u, swap(code), step))
    return graph_from(reads, ent)


def pin_xdrop_matches_suffix_form(orc):
    """Exact overlaps reported with equal early starts on both reads (any
    trim) spell the same contigs in the x-drop form as in the suffix form:
    the walk is the same and the pieces tile the same sequence. Generated
    graphs (open chains, both strands) and a closed chain."""
    graphs = [tiny_generated(), small_generated(3), circular_graph(4), circular_graph(9, 900, 120, 45)]
    for G in graphs:
        want = orc.run(G, min_chain_reads=1)
        for trim, seed in ((0, 0), (40, 1), (5000, 2)):
            X = gen.with_xdrop(G, max_trim=trim, seed=seed, consistent=True)
            got = orc.run(X, min_chain_reads=1)
            assert np.array_equal(got.contig_off, want.contig_off)
            assert np.array_equal(got.bases, want.bases)
            assert np.array_equal(got.chain_id, want.chain_id) and np.array_equal(got.rank, want.rank)
    # unequal starts change the contigs (the skewed and crossed cases pin how)
    X = gen.with_xdrop(graphs[2], max_trim=20, seed=3, consistent=False)
    assert not np.array_equal(orc.run(X, min_chain_reads=1).bases, orc.run(graphs[2], min_chain_reads=1).bases)


def pin_xdrop_validation(orc):
    """x-drop coordinates index the stored reads: pre into u, post into v."""
    c = _xdrop_cases()["paper"]
    G = xdrop_chain(c["reads"], c["pp"], False)      # len l0 = 6, l1 = 8, l2 = 7
    def with_(i, pre=None, post=None):
        H = SimpleNamespace(**{k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in vars(G).items()})
        if pre is not None:
            H.pre[i] = pre
        if post is not None:
            H.post[i] = post
        return H
    # entries in CSR order: (0,1), (1,0), (1,2), (2,1)
    assert orc.validate(with_(2, pre=7))[0]           # pre = len(l1) - 1 of u = l1 (> len(l2) - 1)
    assert not orc.validate(with_(0, pre=6))[0]       # pre = len(l0) of u = l0 (< len(l1) - 1)
    assert not orc.validate(with_(0, pre=-1))[0]
    assert orc.validate(with_(0, post=7))[0]          # post into v = l1
    assert not orc.validate(with_(2, post=7))[0]      # post = len(l2) of v = l2
    assert not orc.validate(with_(1, post=-1))[0]


# ------------------------------------------------- transitive reduction
def _tr_triangle(c01, c12, c02, s01, s12, s02, s10, s21, s20):
    """Reads 0, 1, 2 (100 bases each) with overlaps 0-1, 1-2, 0-2 given by the
    codes and suffixes of one direction and the mirror suffixes."""
    rnd = random.Random(11)
    reads = ["".join(rnd.choice("ACGT") for _ in range(100)) for _ in range(3)]
    ent = [(0, 1, c01, s01), (1, 0, swap(c01), s10), (1, 2, c12, s12), (2, 1, swap(c12), s21),
           (0, 2, c02, s02), (2, 0, swap(c02), s20)]
    return graph_from(reads, ent)


def _pairs(S):
    rp = np.asarray(S.row_ptr)
    return sorted((u, int(w)) for u in range(len(rp) - 1) for w in np.asarray(S.col)[rp[u]:rp[u + 1]])


def pin_transitive_reduction_cases(orc):
    """Alg. 1 / Sec. 2, by hand: the overlap 0-2 is redundant exactly when the
    walk 0 -> 1 -> 2 is valid (leaves 0 and enters 2 through the same ends as
    0 -> 2, passes through 1) and its suffixes add up to 0 -> 2's (within the
    tolerance); a pair goes when either direction is redundant."""
    line = [(0, 1), (1, 0), (1, 2), (2, 1)]
    every = sorted(line + [(0, 2), (2, 0)])
    cases = [  # (codes 01, 12, 02), suffixes 01, 12, 02, 10, 21, 20, fuzz, expected pairs
        ((1, 1, 1), (10, 15, 25, 30, 20, 50), 0, line),     # forward line: redundant both ways
        ((1, 1, 0), (10, 15, 25, 30, 20, 50), 0, every),    # 0 -> 2 leaves 0 through its 5' end
        ((1, 0, 1), (10, 15, 25, 30, 20, 50), 0, every),    # 1 entered and left through one end
        ((1, 1, 3), (10, 15, 25, 30, 20, 50), 0, every),    # 0 -> 2 enters 2 through its 3' end
        ((1, 1, 1), (10, 15, 26, 30, 20, 51), 0, every),    # sums off by one both ways
        ((1, 1, 1), (10, 15, 26, 30, 20, 51), 1, line),     # ... within a tolerance of 1
        ((1, 1, 1), (10, 15, 30, 30, 20, 55), 1, every),    # 5 short both ways, beyond the tolerance
        ((1, 1, 1), (10, 15, 26, 30, 20, 50), 0, line),     # only 2 -> 0 redundant: the pair goes
        ((3, 2, 3), (10, 15, 25, 30, 20, 50), 0, line),     # 1 and 2 stored reversed: the same walk
    ]
    for (c01, c12, c02), (s01, s12, s02, s10, s21, s20), fuzz, want in cases:
        G = _tr_triangle(c01, c12, c02, s01, s12, s02, s10, s21, s20)
        assert orc.validate(G)[0]
        S = orc.transitive_reduction(G, fuzz)
        assert _pairs(S) == sorted(want), ((c01, c12, c02), (s01, s12, s02, s10, s21, s20), fuzz)


def _csr_equal(S, R):
    for k in ("row_ptr", "col", "code", "suf"):
        a, b = np.asarray(getattr(S, k)), np.asarray(getattr(R, k))
        if a.shape != b.shape or not np.array_equal(a.astype(np.int64), b.astype(np.int64)):
            return False
    return True


def pin_transitive_reduction_interval_graphs(orc):
    """Exact overlaps among reads of one genome (no repeat overlaps): the
    reduction of the graph of all overlaps is the graph of consecutive
    overlaps, entry for entry; the reduction is idempotent with repeats too."""
    for d in (dict(gen.WORKLOADS["tiny-1Mb"](), k_rep=0),
              dict(gen._cfg(77, 400_000, [(0.05, 2000, 6000, 2, 6, 0.0)], 15, 1, 7000, 3000, 2500), k_rep=0)):
        full = gen.generate(dict(d, full_overlaps=1), threads=4, off_align=1)
        red = gen.generate(d, threads=4, off_align=1)
        assert full.m > 2 * red.m
        assert _csr_equal(orc.transitive_reduction(full), red)
    R = gen.generate(dict(gen.WORKLOADS["tiny-1Mb"](), full_overlaps=1), threads=4)
    S = orc.transitive_reduction(R)
    assert _csr_equal(orc.transitive_reduction(S), S)
    assert orc.validate(S)[0]


ALL_PINS = [pin_paper_mask_example, pin_paper_concat_example, pin_paper_rc_example, pin_revcomp,
            pin_same_end_rule, pin_brute_force, pin_cycles, pin_generator_truth, pin_invariants, pin_lpt,
            pin_validation, pin_xdrop_examples, pin_xdrop_matches_suffix_form, pin_xdrop_validation,
            pin_transitive_reduction_cases, pin_transitive_reduction_interval_graphs]
