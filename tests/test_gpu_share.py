"""cg_emit_share: one of n equal runs of output tiles of the whole contig
stream (the spelling work split by output bytes across ranks). The shares of
every split, laid end to end, must be the oracle's stream byte for byte, each
starting where the one before ended, with device and with host outputs, for
several tile sizes (a share boundary falls inside contigs and pieces), and
the whole contig offsets must be the oracle's."""
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


def _shares_device(g, n):
    import torch
    out, pos, offs = [], 0, None
    for r in range(n):
        fb, nb = cg.cg_emit_share(g, r, n)
        assert fb == pos or nb == 0
        pos = fb + nb if nb else pos
        off = torch.full((g_contigs(g) + 1,), -1, dtype=torch.int64, device="cuda")
        buf = torch.full((max(16, (nb + 15) // 16 * 16),), 7, dtype=torch.uint8, device="cuda")
        cg.cg_emit_share(g, r, n, off, buf, want_range=False)
        cg.cg_sync(g.ctx)
        out.append(buf[:nb].cpu().numpy())
        assert (buf[nb:].cpu().numpy() == 7).all()                  # nothing written past the share
        offs = off.cpu().numpy()
    return np.concatenate(out), offs, pos


def _shares_host(g, n):
    out, pos, offs = [], 0, None
    for r in range(n):
        fb, nb = cg.cg_emit_share(g, r, n)
        off = np.empty(g_contigs(g) + 1, np.int64)
        buf = np.empty(max(nb, 1), np.uint8)
        fb2, nb2 = cg.cg_emit_share(g, r, n, off, buf)
        assert (fb2, nb2) == (fb, nb)
        assert fb == pos or nb == 0
        pos = fb + nb if nb else pos
        out.append(buf[:nb])
        offs = off
    return np.concatenate(out), offs, pos


def g_contigs(g):
    return cg.cg_emit_contigs(g)[0]


@pytest.mark.parametrize("name", ["tiny-1Mb", "genome-100Mb", "structured"])
def test_shares_tile_the_stream(ctx, name):
    if name == "structured":   # long and closed chains, one-read contigs
        G = structured(3, [1] * 300 + [2] * 200 + [40] * 50 + [2000] * 3, closed=[False] * 550 + [True] * 3,
                       min_len=500, max_len=3000, lone=100)
        mcr = 1
    else:
        G = gen.generate(name, threads=8)
        mcr = 2
    w = oracle.run(G, min_chain_reads=mcr)
    g = cg.cg_load_graph(ctx, G, min_chain_reads=mcr)
    try:
        for tile in (4096, 32768):
            cg.cg_set_tuning(ctx, tile_bytes=tile)
            for n in (1, 2, 3, 8):
                for fn in (_shares_device, _shares_host):
                    bases, off, end = fn(g, n)
                    assert end == w.total_bases
                    assert np.array_equal(off, w.contig_off)
                    assert np.array_equal(bases, w.bases), (tile, n, fn.__name__)
    finally:
        cg.cg_set_tuning(ctx, tile_bytes=32768)
        g.close()


def test_bad_share_rejected(ctx):
    G = gen.generate("tiny-1Mb", threads=8)
    g = cg.cg_load_graph(ctx, G)
    try:
        for share, n in ((2, 2), (-1, 2), (0, 0)):
            with pytest.raises(cg.CgError) as e:
                cg.cg_emit_share(g, share, n)
            assert e.value.status == cg.CG_EINVAL
        fb, nb = cg.cg_emit_share(g, 0, 2)
        with pytest.raises(cg.CgError) as e:                     # one byte short
            cg.cg_emit_share(g, 0, 2, None, np.empty(max(nb - 1, 0), np.uint8))
        assert e.value.status == cg.CG_EINVAL
    finally:
        g.close()
