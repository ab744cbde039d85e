"""cg_offsets_noalloc: the offset scan for callers that cannot call cudaMalloc
(another allocator owns the device memory, or an allocation would stall a
latency-critical loop). It is checked through the C ABI against contig_off
from cg_emit_contigs, which the library computes with its own allocated
scratch, on two calls in a row. Collected last so that a failure here comes
after every other test has run."""
import numpy as np
import pytest

import gen
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


def _contig_off(ctx, G, mcr):
    import torch
    g = cg.cg_load_graph(ctx, G, min_chain_reads=mcr)
    n_contigs, total = cg.cg_emit_contigs(g)
    off = torch.empty(n_contigs + 1, dtype=torch.int64, device="cuda")
    cg.cg_emit_contigs(g, off, None)
    cg.cg_sync(ctx)
    g.close()
    return off


@pytest.mark.parametrize("case", ["tiny", "many_contigs"])
def test_noalloc_offsets_match_contig_off(ctx, case):
    import torch
    if case == "tiny":
        off = _contig_off(ctx, gen.generate("tiny-1Mb", threads=8), 2)
    else:   # ~25k one-read and short contigs: about a dozen scan tiles and a ragged last tile
        off = _contig_off(ctx, structured(4, [1] * 20000 + [2] * 3000 + [5] * 300, lone=1717), 1)
    lengths = (off[1:] - off[:-1]).to(torch.int32).contiguous()
    stream = torch.cuda.current_stream()
    for _ in range(2):                                   # two calls in a row share the scratch array
        out = torch.full((len(lengths) + 1,), -7, dtype=torch.int64, device="cuda")
        cg.cg_offsets_noalloc(lengths, out, stream)
        assert torch.equal(out, off)                     # integer offsets: bit-exact


def test_noalloc_allocates_nothing_after_first_call(ctx):
    import torch
    lengths = torch.randint(0, 1000, (300_001,), dtype=torch.int32, device="cuda")
    out = torch.empty(len(lengths) + 1, dtype=torch.int64, device="cuda")
    cg.cg_offsets_noalloc(lengths, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        cg.cg_offsets_noalloc(lengths, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    want = np.concatenate([[0], np.cumsum(lengths.cpu().numpy().astype(np.int64))])
    assert np.array_equal(out.cpu().numpy(), want)


def test_noalloc_rejects_sizes_beyond_the_maximum(ctx):
    st = cg.lib().cg_offsets_noalloc(None, cg.NOALLOC_MAX_COUNT + 1, None, None)
    assert st == cg.CG_EINVAL
    import torch
    empty = torch.zeros(0, dtype=torch.int32, device="cuda")
    out = torch.full((1,), 5, dtype=torch.int64, device="cuda")
    cg.cg_offsets_noalloc(empty, out)
    assert int(out[0]) == 0
