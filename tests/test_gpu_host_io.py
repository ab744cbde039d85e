"""Host-resident inputs and outputs on GB300's host link, against the oracle,
bit-exact: CG_HOST_READS (the packed reads stay in pinned host memory and the
kernels read only the bases they spell) and pinned host outputs written in
place by the kernels, in the ASCII and the 2-bit forms; the copying paths give
the same bytes. Memory that is not pinned is refused for CG_HOST_READS and
staged for outputs."""
import numpy as np
import pytest

import gen
import oracle
from paper_2207_04350_gb300 import cg
from tests._graphs import structured

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2207_04350_gb300 import _build
    _build.build()
    assert torch.cuda.is_available()
    c = cg.cg_create(0)
    yield c
    c.close()


_keep = []


def pinned(a):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    _keep.append(t)
    return t.numpy()


def pinned_graph(G):
    P = type("P", (), {})()
    for k in ("row_ptr", "col", "code", "suf", "len", "off", "packed"):
        setattr(P, k, pinned(getattr(G, k)))
    return P


def outputs(ctx, g, pin_out: bool):
    n_contigs, total = cg.cg_emit_contigs(g)
    off = np.empty(n_contigs + 1, np.int64)
    bases = np.empty(max(total, 16), np.uint8)
    if pin_out:
        off, bases = pinned(off), pinned(bases)
    cg.cg_emit_contigs(g, off, bases)
    n2 = cg.packed_bytes_2bit(total)
    packed = np.empty(max(n2, 16), np.uint8)
    if pin_out:
        packed = pinned(packed)
    cg.cg_emit_contigs_2bit(g, None, packed)
    return off, bases[:total], packed[:n2]


def check(ctx, G, mcr=2):
    orc = oracle.run(G, min_chain_reads=mcr)
    want2 = np.zeros(cg.packed_bytes_2bit(orc.total_bases), np.uint8)
    p2 = oracle.pack2(orc.bases)
    want2[: p2.size] = p2
    P = pinned_graph(G)
    for flags in (cg.HOST_READS, 0):
        for pin_out in (True, False):
            for direct in (True, False):
                cg.cg_set_host_direct(ctx, direct)
                g = cg.cg_load_graph(ctx, P, flags=flags, min_chain_reads=mcr)
                try:
                    off, bases, packed = outputs(ctx, g, pin_out)
                finally:
                    g.close()
                assert np.array_equal(off, orc.contig_off), (flags, pin_out, direct)
                assert np.array_equal(bases, orc.bases), (flags, pin_out, direct)
                assert np.array_equal(packed, want2), (flags, pin_out, direct)
    cg.cg_set_host_direct(ctx, True)


def test_tiny_workload(ctx):
    for align in (1, 32):
        check(ctx, gen.generate("tiny-1Mb", threads=8, off_align=align), 2)


def test_reads_at_the_end_of_the_stream(ctx):
    # short reads, unaligned offsets: the last reads' bases end in the stream's last bytes
    sizes = [3000, 5, 7] + [2] * 100
    G = structured(12, sizes, [False, True, True] + [False] * 100, min_len=9, max_len=70, align=1)
    check(ctx, G, 1)


def test_generated_graphs(ctx):
    for j in (0, 5):
        check(ctx, gen.generate(gen.batched_graph(j), threads=8), 2)


def test_refusals(ctx):
    import torch
    G = gen.generate("tiny-1Mb", threads=8)
    with pytest.raises(cg.CgError) as e:            # packed not pinned
        cg.cg_load_graph(ctx, G, flags=cg.HOST_READS)
    assert e.value.status == cg.CG_EINVAL
    D = type("D", (), {})()
    for k in ("row_ptr", "col", "code", "suf", "len", "off", "packed"):
        setattr(D, k, torch.from_numpy(np.ascontiguousarray(getattr(G, k))).cuda())
    with pytest.raises(cg.CgError) as e:            # device inputs
        cg.cg_load_graph(ctx, D, flags=cg.HOST_READS)
    assert e.value.status == cg.CG_EINVAL
    g = cg.cg_load_graph(ctx, pinned_graph(G), flags=cg.HOST_READS)   # still usable
    g.close()


def test_batch_with_host_reads(ctx):
    """A batch whose reads stay in pinned host memory: the pieces are gathered
    from each graph's own stream; every graph's contigs exact, in both forms."""
    graphs = [gen.generate(gen.batched_graph(j), threads=8, off_align=(1, 4, 32)[j % 3]) for j in (0, 3, 7, 19, 40)]
    S = structured(12, [3000, 5, 7] + [2] * 100, [False, True, True] + [False] * 100, min_len=9, max_len=70, align=1)
    S.row_ptr = S.row_ptr.astype(graphs[0].row_ptr.dtype)    # a batch has one row_ptr width
    graphs.append(S)
    want = [oracle.run(G, min_chain_reads=2) for G in graphs]
    P = [pinned_graph(G) for G in graphs]
    for flags in (cg.HOST_READS, 0):
        g = cg.cg_load_batch(ctx, P, flags=flags, min_chain_reads=2)
        try:
            off, bases = cg.contigs_host(g)
            off2, packed, total = cg.contigs_2bit_host(g)
            fc, fb = cg.cg_batch_ranges(g)
            off_again, bases_again = cg.contigs_host(g)      # a second spelling gathers again
        finally:
            g.close()
        assert np.array_equal(off_again, off) and np.array_equal(bases_again, bases)
        for j, w in enumerate(want):
            assert np.array_equal(off[fc[j]:fc[j + 1] + 1] - fb[j], w.contig_off), (flags, j)
            assert np.array_equal(bases[fb[j]:fb[j + 1]], w.bases), (flags, j)
        assert np.array_equal(packed[: (total + 3) // 4], oracle.pack2(bases))
    with pytest.raises(cg.CgError) as e:                 # one graph's reads not pinned
        cg.cg_load_batch(ctx, P[:2] + [graphs[2]], flags=cg.HOST_READS)
    assert e.value.status == cg.CG_EINVAL


def test_server_with_pinned_requests(ctx):
    """Requests whose reads are pinned: the server gathers their pieces over the
    host link; every result exact, alone and batched, mixed with unpinned ones."""
    graphs = [gen.generate(gen.served_graph(j), threads=8) for j in (1, 2, 6)]
    want = [oracle.run(G, min_chain_reads=2) for G in graphs]
    P = [pinned_graph(G) for G in graphs]
    srv = cg.Server(0, hbm_budget_bytes=16 << 30, max_batch=8, workers=2)
    try:
        ids = [(srv.submit(P[i % 3] if i % 4 else graphs[i % 3]), i % 3) for i in range(12)]
        for rid, j in ids:
            r = srv.wait(rid)
            assert r["status"] == cg.CG_OK
            assert np.array_equal(r["contig_off"], want[j].contig_off) and np.array_equal(r["bases"], want[j].bases)
            srv.release(rid)
    finally:
        srv.stop()
