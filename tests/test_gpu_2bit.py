"""2-bit contig output (cg_emit_contigs_2bit) against the oracle's contigs in
the 2-bit layout (oracle.pack2 of the oracle's ASCII contigs), bit-exact,
including the zero bits past the last base up to the 16-byte chunk.

The cases stress what is particular to this form: pieces shorter than a
64-base chunk (several pieces in one chunk, chunks open across groups of 32
pieces), reverse-complement pieces at every bit shift, read offsets that are
not word-aligned, reads at both ends of the packed stream, every tile size,
and outputs that end inside a chunk.
"""
import random

import numpy as np
import pytest

import gen
import oracle
from paper_2207_04350_gb300 import cg
from tests import _pins
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


def expect(orc):
    want = oracle.pack2(orc.bases)
    full = np.zeros(cg.packed_bytes_2bit(orc.total_bases), np.uint8)
    full[: want.size] = want
    return full


def check(ctx, G, mcr=2, device=False):
    orc = oracle.run(G, min_chain_reads=mcr)
    g = cg.cg_load_graph(ctx, G, min_chain_reads=mcr)
    try:
        if device:
            import torch
            n_contigs, total = cg.cg_emit_contigs_2bit(g)
            off_t = torch.empty(n_contigs + 1, dtype=torch.int64, device="cuda")
            pk_t = torch.full((max(cg.packed_bytes_2bit(total), 16),), 0xAB, dtype=torch.uint8, device="cuda")
            cg.cg_emit_contigs_2bit(g, off_t, pk_t)
            cg.cg_sync(ctx)
            off, packed = off_t.cpu().numpy(), pk_t.cpu().numpy()[: cg.packed_bytes_2bit(total)]
        else:
            off, packed, total = cg.contigs_2bit_host(g)
    finally:
        g.close()
    assert total == orc.total_bases
    assert np.array_equal(off, orc.contig_off)
    want = expect(orc)
    if not np.array_equal(packed, want):
        bad = int(np.nonzero(packed != want)[0][0])
        raise AssertionError(f"byte {bad} of {want.size}: got {packed[bad]:#04x}, want {want[bad]:#04x}")
    return orc


def test_paper_examples(ctx):
    for stored_rc in (False, True):
        G, want = _pins._concat_graph(stored_rc)
        orc = check(ctx, G, 2)
        assert orc.contig(0).decode() == want


def test_brute_force_graphs(ctx):
    rnd = random.Random(77)
    for t in range(120):
        if t % 2 == 0:
            G = _pins.random_tiny_graph(rnd, rnd.randint(1, 8), rnd.choice([0.15, 0.3, 0.5]))
        else:
            G = _pins.random_chain_graph(rnd, rnd.randint(1, 12), rnd.randint(0, 3))
        check(ctx, G, rnd.choice([1, 2, 3]))


@pytest.mark.parametrize("align", [1, 4, 32])
def test_short_pieces(ctx, align):
    # reads of 8..40 bases: pieces far shorter than a chunk, many per chunk
    rng = np.random.default_rng(align)
    sizes = list(rng.integers(1, 60, size=3000)) + [5000]
    G = structured(40 + align, sizes, lone=100, align=align)
    check(ctx, G, 1)
    check(ctx, G, 2, device=True)


@pytest.mark.parametrize("bt,bps", [(128, 16), (128, 3), (512, 2), (512, 1)])
def test_block_sizes(bt, bps):
    """The spelling CTA size and blocks per SM change no byte of either form."""
    c = cg.cg_create(0)
    try:
        cg.cg_set_tuning(c, tile_bytes=4096, emit_blocks_per_sm=bps, emit_block_threads=bt)
        rng = np.random.default_rng(bt + bps)
        G = structured(60 + bps, list(rng.integers(1, 60, size=2000)) + [3000] * 3, lone=50, align=1)
        for mcr in (1, 2):
            check(c, G, mcr)
        check(c, gen.generate("tiny-1Mb", threads=8, off_align=4), 2, device=True)
    finally:
        c.close()


def test_long_reads_and_cycles(ctx):
    sizes = [30_000, 3, 4, 5, 7, 16, 33, 100] + [2] * 200
    closed = [False] + [True] * 7 + [False] * 200
    G = structured(8, sizes, closed, min_len=100, max_len=3000, lone=20, align=1)
    for mcr in (1, 2):
        check(ctx, G, mcr)


@pytest.mark.parametrize("align", [1, 4, 32])
def test_tiny_1mb(ctx, align):
    G = gen.generate("tiny-1Mb", threads=8, off_align=align)
    check(ctx, G, 2)
    check(ctx, G, 1, device=True)


def test_generated_sweep(ctx):
    for seed in range(4):
        d = gen._cfg(2000 + seed, 2_000_000, [(0.06, 2000, 9000, 2, 12, 0.0)], 25, 1, 8000, 4000, 2500)
        G = gen.generate(d, threads=8, off_align=(1, 4, 32, 1)[seed])
        check(ctx, G, 1 + seed % 2)


@pytest.mark.parametrize("tile", [4096, 8192, 16384, 32768, 65536, 131072])
def test_tile_sizes(tile):
    c = cg.cg_create(0)
    try:
        cg.cg_set_tuning(c, tile_bytes=tile, emit_blocks_per_sm=2)
        check(c, structured(21, [50_000, 3, 4, 17] + [2] * 40 + [6] * 30, [False, True, True, True] + [False] * 70,
                            lone=50, align=1), 1)
        check(c, gen.generate(gen.batched_graph(11), threads=8), 2)
    finally:
        c.close()


def test_empty_and_capacity(ctx):
    lone = structured(2, [1] * 50)
    orc = check(ctx, lone, 2)                # no contigs: total 0
    assert orc.total_bases == 0
    G = gen.generate("tiny-1Mb", threads=8)
    g = cg.cg_load_graph(ctx, G)
    try:
        n_contigs, total = cg.cg_emit_contigs_2bit(g)
        with pytest.raises(cg.CgError) as e:
            cg.cg_emit_contigs_2bit(g, None, np.empty(cg.packed_bytes_2bit(total) - 1, np.uint8))
        assert e.value.status == cg.CG_EINVAL
        import torch
        small = torch.empty(cg.packed_bytes_2bit(total) - 16, dtype=torch.uint8, device="cuda")
        cg.cg_emit_contigs_2bit(g, None, small, want_counts=False)
        with pytest.raises(cg.CgError) as e:
            cg.cg_sync(ctx)
        assert e.value.status == cg.CG_EINVAL
        # ASCII and 2-bit outputs of one graph, interleaved
        off, bases = cg.contigs_host(g)
        off2, packed, total2 = cg.contigs_2bit_host(g)
        assert np.array_equal(off, off2) and total2 == total
        assert np.array_equal(packed[: (total + 3) // 4], oracle.pack2(bases))
    finally:
        g.close()


def test_genome_100mb(ctx):
    G = gen.generate("genome-100Mb", threads=16)
    check(ctx, G, 2)
