"""Runs the CUDA path through the C ABI and compares it with the oracle."""
from __future__ import annotations

from types import SimpleNamespace

import numpy as np

from paper_2207_04350_gb300 import cg


def run_gpu(ctx, G, min_chain_reads=2, inputs="host", outputs="host", flags=0):
    import torch
    src = G
    if inputs == "device":
        keys = ["row_ptr", "col", "code", "suf", "len", "off", "packed", "pre", "post"]
        src = SimpleNamespace(**{k: torch.from_numpy(np.ascontiguousarray(getattr(G, k))).cuda()
                                 if getattr(G, k, None) is not None else None for k in keys})
    g = cg.cg_load_graph(ctx, src, flags=flags, min_chain_reads=min_chain_reads)
    try:
        n = g.n
        if outputs == "host":
            isb = np.empty(n, np.uint8)
            nb = cg.cg_mask_branches(g, isb)
            cid, rank, orient, nc, ncy = cg.chains_host(g)
            off, bases = cg.contigs_host(g)
        else:
            isb_t = torch.empty(n, dtype=torch.uint8, device="cuda")
            nb = cg.cg_mask_branches(g, isb_t)
            cid_t = torch.empty(n, dtype=torch.int32, device="cuda")
            rank_t = torch.empty(n, dtype=torch.int32, device="cuda")
            or_t = torch.empty(n, dtype=torch.uint8, device="cuda")
            nc, ncy = cg.cg_chains(g, cid_t, rank_t, or_t)
            n_contigs, total = cg.cg_emit_contigs(g)
            off_t = torch.empty(n_contigs + 1, dtype=torch.int64, device="cuda")
            bases_t = torch.empty(max(total, 16), dtype=torch.uint8, device="cuda")
            cg.cg_emit_contigs(g, off_t, bases_t)
            cg.cg_sync(ctx)
            isb, cid, rank, orient = isb_t.cpu().numpy(), cid_t.cpu().numpy(), rank_t.cpu().numpy(), or_t.cpu().numpy()
            off, bases = off_t.cpu().numpy(), bases_t.cpu().numpy()[:total]
        return SimpleNamespace(n_branch=nb, is_branch=isb, chain_id=cid, rank=rank, orient=orient, n_contigs=nc,
                               n_cycles=ncy, contig_off=off, bases=bases)
    finally:
        g.close()


def assert_parity(gpu, orc):
    """Element-by-element: everything here is integer or byte work, so bit-exact."""
    assert gpu.n_branch == orc.n_branch
    assert np.array_equal(gpu.is_branch, orc.is_branch)
    assert gpu.n_contigs == orc.n_contigs
    assert gpu.n_cycles == orc.n_cycles
    assert np.array_equal(gpu.chain_id, orc.chain_id)
    assert np.array_equal(gpu.rank, orc.rank)
    assert np.array_equal(gpu.orient, orc.orient)
    assert np.array_equal(gpu.contig_off, orc.contig_off)
    assert len(gpu.bases) == len(orc.bases)
    if not np.array_equal(gpu.bases, orc.bases):
        bad = int(np.nonzero(gpu.bases != orc.bases)[0][0])
        raise AssertionError(f"bases differ first at {bad} (of {len(orc.bases)})")
