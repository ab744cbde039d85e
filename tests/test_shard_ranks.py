"""The host side of a run split over several ranks (paper_2207_04350_gb300.shard)
on CPU: two gloo ranks. Each rank's share is made here from the oracle's
contigs (test input), then the module's collectives bring the shares to
rank 0, which must get the oracle's whole stream back:

- "tiles": the stream cut into two runs of whole 4 KiB layout tiles;
- "lpt": whole contigs split by GreedyPartitioning (the oracle's LPT, weights
  = bases); two ranks that computed different partitions are refused.
"""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

TILE = 4096                                          # the library's layout tile


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _share(total, r, world, tile=TILE):
    T = (total + tile - 1) // tile
    t0, t1 = r * T // world, (r + 1) * T // world
    return t0 * tile, max(0, min(total, t1 * tile) - t0 * tile)


def _worker(rank, world, port, q, skew):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import gen
        import oracle
        from paper_2207_04350_gb300 import shard
        G = gen.generate(dict(gen.WORKLOADS["genome-100Mb"](), genome_len=20_000_000), threads=2)
        w = oracle.run(G, min_chain_reads=2)
        out = {}
        fb, nb = _share(w.total_bases, rank, world)
        whole = shard.gather_shares(w.bases[fb:fb + nb], fb, rank, world)
        out["tiles"] = None if whole is None else bool(np.array_equal(whole, w.bases))
        lens = np.diff(w.contig_off)
        part, _ = oracle.lpt(lens, world)
        if skew and rank == 1:
            part = part.copy()
            part[0] ^= 1                              # this rank disagrees on one contig
        mine = np.concatenate([w.bases[w.contig_off[c]:w.contig_off[c + 1]] for c in np.nonzero(part == rank)[0]])
        try:
            parts = shard.gather_parts(mine, part, rank, world)
            if parts is not None:                     # rank 0 puts every contig back in place
                pos = [0] * world
                got = []
                for c in range(len(lens)):
                    p = int(part[c])
                    got.append(parts[p][pos[p]:pos[p] + lens[c]])
                    pos[p] += int(lens[c])
                out["lpt"] = bool(np.array_equal(np.concatenate(got), w.bases))
        except RuntimeError as e:
            out["lpt_error"] = str(e)
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def _run(skew):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q, skew)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


def test_shares_and_parts_come_back_whole():
    res = _run(skew=False)
    assert res[0]["tiles"] is True and res[1]["tiles"] is None
    assert res[0]["lpt"] is True


def test_ranks_with_different_partitions_are_refused():
    res = _run(skew=True)
    assert "different partitions" in res[0]["lpt_error"] and "different partitions" in res[1]["lpt_error"]
