"""The read exchange (cg_exchange_sizes, cg_exchange_pack,
cg_emit_share_received): ranks that each hold only a slice of the reads,
every rank loading the whole graph without reads. Checked in one process
(every rank's context on the one GPU, the all-to-all done by slicing the send
buffers on the host) for 1 to 4 ranks, uneven slices and rank layouts whose
phases differ from the graph's own; and by two processes through
shard.ExchangeRun with a gloo all-to-all. The shares laid end to end must be
the oracle's stream byte for byte, and the contig offsets the oracle's."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import gen
import oracle
from paper_2207_04350_gb300 import cg
from tests._exchange import read_slices, without_reads
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


def _bounds(n, world, skew):
    cuts = [0] + [min(n, int(n * (r + skew * (r % 2)) / world)) for r in range(1, world)] + [n]
    return np.maximum.accumulate(np.array(cuts, dtype=np.int64))


def _run_all(ctx, G, world, rf, mcr):
    import torch
    graphs = [cg.cg_load_graph(ctx, without_reads(G), flags=cg.NO_READS, min_chain_reads=mcr) for _ in range(world)]
    try:
        slices = read_slices(G, rf)
        sizes = [cg.cg_exchange_sizes(graphs[r], world, rf, r) for r in range(world)]
        for r in range(world):
            for s in range(world):
                assert sizes[r][1][s] == sizes[s][0][r]          # what s sends r is what r expects from s
        sends = []
        for r in range(world):
            mp_, mo = slices[r]
            send = torch.zeros(max(16, int(sizes[r][0].sum())), dtype=torch.uint8, device="cuda")
            cg.cg_exchange_pack(graphs[r], world, rf, r, torch.from_numpy(mp_).cuda(), torch.from_numpy(mo).cuda(),
                                send)
            sends.append(send.cpu().numpy())
        shares, offs, firsts = [], [], []
        for r in range(world):
            segs = []
            for s in range(world):
                start = int(sizes[s][0][:r].sum())
                segs.append(sends[s][start:start + int(sizes[s][0][r])])
            recv = torch.from_numpy(np.concatenate(segs) if segs else np.zeros(0, np.uint8)).cuda()
            n_contigs, _ = cg.cg_emit_contigs(graphs[r])
            _, nb = cg.cg_emit_share(graphs[r], r, world)
            off = torch.empty(n_contigs + 1, dtype=torch.int64, device="cuda")
            bases = torch.full((max(16, (nb + 15) // 16 * 16),), 7, dtype=torch.uint8, device="cuda")
            fb, nb2 = cg.cg_emit_share_received(graphs[r], world, rf, r, recv, off, bases)
            assert nb2 == nb
            shares.append(bases[:nb].cpu().numpy())
            offs.append(off.cpu().numpy())
            firsts.append(fb)
        return shares, offs, firsts
    finally:
        for g in graphs:
            g.close()


@pytest.mark.parametrize("world", [1, 2, 3, 4])
@pytest.mark.parametrize("name", ["tiny-1Mb", "recipe-20Mb", "structured"])
def test_exchange_gives_the_oracle_stream(ctx, name, world):
    mcr = 2
    if name == "structured":   # long, closed and one-read chains, reads at any base offset
        G = structured(17, [1] * 200 + [2] * 150 + [30] * 40 + [900] * 3, closed=[False] * 390 + [True] * 3,
                       min_len=300, max_len=2500, lone=50, align=1)
        mcr = 1
    elif name == "recipe-20Mb":
        G = gen.generate(dict(gen.WORKLOADS["genome-3.1Gb"](), genome_len=20_000_000), threads=8)
    else:
        G = gen.generate(name, threads=8)
    want = oracle.run(G, min_chain_reads=mcr)
    rf = _bounds(G.n, world, 0.3)
    for tile in (4096, 32768):
        cg.cg_set_tuning(ctx, tile_bytes=tile)
        try:
            shares, offs, firsts = _run_all(ctx, G, world, rf, mcr)
        finally:
            cg.cg_set_tuning(ctx, tile_bytes=32768)
        pos = 0
        for r in range(world):
            assert firsts[r] == pos or len(shares[r]) == 0
            pos += len(shares[r])
            assert np.array_equal(offs[r], want.contig_off)
        assert np.array_equal(np.concatenate(shares), want.bases), (name, world, tile)


def test_exchange_refusals(ctx):
    import torch
    G = gen.generate("tiny-1Mb", threads=8)
    rf = np.array([0, G.n // 2, G.n], np.int64)
    g = cg.cg_load_graph(ctx, without_reads(G), flags=cg.NO_READS)
    full = cg.cg_load_graph(ctx, G)
    try:
        n_contigs, total = cg.cg_emit_contigs(g)                   # sizes need no reads
        assert total == oracle.run(G).total_bases
        with pytest.raises(cg.CgError) as e:                       # spelling does
            cg.cg_emit_contigs(g, np.empty(n_contigs + 1, np.int64), np.empty(total, np.uint8))
        assert e.value.status == cg.CG_EINVAL
        for bad in ([1, G.n // 2, G.n], [0, G.n // 2, G.n - 1], [0, G.n, G.n // 2]):   # bounds from 0 to n, rising
            with pytest.raises(cg.CgError) as e:
                cg.cg_exchange_sizes(g, 2, np.array(bad, np.int64), 0)
            assert e.value.status == cg.CG_EINVAL
        with pytest.raises(cg.CgError) as e:                       # a rank outside the split
            cg.cg_exchange_sizes(g, 2, rf, 2)
        assert e.value.status == cg.CG_EINVAL
        with pytest.raises(cg.CgError) as e:                       # a graph loaded with its reads
            cg.cg_exchange_sizes(full, 2, rf, 0)
        assert e.value.status == cg.CG_EINVAL
        send, recv = cg.cg_exchange_sizes(g, 2, rf, 1)
        short = torch.zeros(max(16, int(recv.sum()) - 4), dtype=torch.uint8, device="cuda")
        with pytest.raises(cg.CgError) as e:                       # not what the layout needs
            cg.cg_emit_share_received(g, 2, rf, 1, short[: int(recv.sum()) - 4], None, None)
        assert e.value.status == cg.CG_EINVAL
    finally:
        g.close()
        full.close()


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2207_04350_gb300 import shard
        torch.cuda.set_device(0)
        G = gen.generate(dict(gen.WORKLOADS["genome-3.1Gb"](), genome_len=20_000_000), threads=4)
        rf = _bounds(G.n, world, 0.2)
        my_packed, my_off = read_slices(G, rf)[rank]
        ctx = cg.cg_create(0)
        run = shard.ExchangeRun(ctx, without_reads(G), torch.from_numpy(my_packed).cuda(),
                                torch.from_numpy(my_off).cuda(), rf, rank, world)
        for _ in range(2):                                  # the second step lays out and exchanges again
            run.step()
        off, bases, first = run.result()
        run.close()
        ctx.close()
        whole = shard.gather_shares(bases, first, rank, world)
        out = {}
        if rank == 0:
            w = oracle.run(G, min_chain_reads=2)
            out = {"off": bool(np.array_equal(off, w.contig_off)), "bases": bool(np.array_equal(whole, w.bases))}
        q.put((rank, out))
    except Exception as e:
        q.put((rank, {"error": repr(e)}))
    finally:
        dist.destroy_process_group()


def test_two_ranks_exchange_their_reads():
    from paper_2207_04350_gb300 import _build
    _build.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=600) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert "error" not in res[0] and "error" not in res[1], res
    assert res[0]["off"] is True and res[0]["bases"] is True
