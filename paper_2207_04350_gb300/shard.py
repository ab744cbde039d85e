"""One string graph's contigs over several GPUs: each rank (one process, one
GPU) holds the whole graph and its reads, runs BranchRemoval and the chain
stage itself, and spells its own share of the contigs (Alg. 2: the ranks'
LocalAssembly of the contigs assigned to them, Sec. 4.3-4.4).

With the reads replicated (ShardedRun; the 3.1 Gb graph's 23 GB of packed
reads fit in every GPU's HBM) the data path has no collective: the paper's
induced-subgraph redistribution and read exchange only moved data between
address spaces that here all hold it already. With each rank holding a slice
of the reads (ExchangeRun), one all-to-all moves to every rank the bases of
the pieces it spells: the paper's read exchange. Every rank computes the same
chains, as the path is deterministic.

Two splits of the spelling work (ShardedRun; ExchangeRun spells tiles):
- "tiles" (cg_emit_share): the output stream is cut into `world` runs of
  whole output tiles, so every rank spells the same number of bytes whatever
  the contig sizes; a contig may span two ranks.
- "lpt" (cg_partition_contigs + cg_emit_part): the paper's GreedyPartitioning
  of whole contigs (longest processing time first) into `world` parts, which
  every rank computes identically on its GPU; rank r spells part r.

Collecting the shares in one place (gather_shares, gather_parts) is not part
of the path: the paper leaves each process with its own contigs. These two
helpers only move finished output to rank 0 over torch.distributed, with any
backend (gloo with host tensors, NCCL with device tensors).
"""
from __future__ import annotations

import hashlib

import numpy as np

from . import cg

MODES = ("tiles", "lpt")


class ShardedRun:
    """One rank's share of one graph: the graph loaded on this rank's context,
    device output buffers sized once, and step() queued on the context's
    stream with no host wait."""

    def __init__(self, ctx: cg.Context, graph, rank: int, world: int, mode: str = "tiles",
                 weight: int = cg.WEIGHT_BASES, min_chain_reads: int = 2, flags: int = 0):
        import torch
        if mode not in MODES:
            raise ValueError(f"mode must be one of {MODES}")
        if not 0 <= rank < world:
            raise ValueError("rank must be in [0, world)")
        self.ctx, self.rank, self.world, self.mode, self.weight = ctx, rank, world, mode, weight
        self.g = cg.cg_load_graph(ctx, graph, flags=flags, min_chain_reads=min_chain_reads)
        self.n_contigs, self.total = cg.cg_emit_contigs(self.g)
        self.contig_off = torch.empty(self.n_contigs + 1, dtype=torch.int64, device="cuda")
        if mode == "tiles":
            self.first_base, self.n_bases = cg.cg_emit_share(self.g, rank, world)
            cap = self.n_bases
            self.part = None
        else:
            self.part = torch.empty(max(self.n_contigs, 1), dtype=torch.int32, device="cuda")
            self.part_weight = torch.empty(world, dtype=torch.int64, device="cuda")
            cg.cg_partition_contigs(self.g, world, weight, self.part, self.part_weight)
            _, self.n_bases = cg.cg_emit_part(self.g, self.part, rank)
            self.first_base = None
            cap = self.n_bases
        self.bases = torch.empty(max(16, (cap + 15) // 16 * 16), dtype=torch.uint8, device="cuda")

    def step(self):
        """Queues one pass of the path for this rank: mask, chains, then this
        rank's spelling (with the LPT partition first in "lpt" mode)."""
        g = self.g
        cg.cg_mask_branches(g, want_count=False)
        cg.cg_chains(g, want_counts=False)
        if self.mode == "tiles":
            cg.cg_emit_share(g, self.rank, self.world, self.contig_off, self.bases, want_range=False)
        else:
            cg.cg_partition_contigs(g, self.world, self.weight, self.part, self.part_weight)
            cg.cg_emit_part(g, self.part, self.rank, self.contig_off, self.bases, want_counts=False)

    def result(self):
        """(contig_off, bases, first_base, part) as host arrays after the last
        step: in "tiles" mode contig_off is the whole stream's and bases holds
        stream bytes [first_base, first_base + len); in "lpt" mode contig_off
        gives every contig's range in this rank's output (empty for the other
        ranks' contigs) and part the assignment."""
        cg.cg_sync(self.ctx)
        off = self.contig_off.cpu().numpy()
        bases = self.bases[: self.n_bases].cpu().numpy()
        part = self.part[: self.n_contigs].cpu().numpy() if self.part is not None else None
        return off, bases, self.first_base, part

    def close(self):
        self.g.close()


class ExchangeRun:
    """One rank's share of one graph when every rank holds only a slice of the
    reads: reads [read_first[rank], read_first[rank + 1]) are this rank's, in
    my_packed (a device 2-bit stream of this rank's own layout; my_off[i] = the
    first base of read read_first[rank] + i in it). The rank loads the whole
    graph without its reads (`graph` with packed None and packed_bytes = the size
    of the virtual stream its `off` places the reads in), runs the mask, chain
    and layout steps, sends every share the bases of the pieces it needs from
    this rank's reads and receives those of its own share from every rank (one
    all-to-all: the paper's read exchange, Sec. 4.3), then spells its share of
    the output tiles, as ShardedRun's "tiles" mode does from the whole stream."""

    def __init__(self, ctx: cg.Context, graph, my_packed, my_off, read_first, rank: int, world: int,
                 min_chain_reads: int = 2, group=None):
        import torch
        self.ctx, self.rank, self.world, self.group = ctx, rank, world, group
        self.read_first = np.ascontiguousarray(read_first, dtype=np.int64)
        self.my_packed, self.my_off = my_packed, my_off
        self.g = cg.cg_load_graph(ctx, graph, flags=cg.NO_READS, min_chain_reads=min_chain_reads)
        self.n_contigs, self.total = cg.cg_emit_contigs(self.g)
        self.send_bytes, self.recv_bytes = cg.cg_exchange_sizes(self.g, world, self.read_first, rank)
        self.send = torch.empty(max(16, int(self.send_bytes.sum())), dtype=torch.uint8, device="cuda")
        self.recv = torch.empty(max(16, int(self.recv_bytes.sum())), dtype=torch.uint8, device="cuda")
        self.first_base, self.n_bases = cg.cg_emit_share(self.g, rank, world)
        self.bases = torch.empty(max(16, (self.n_bases + 15) // 16 * 16), dtype=torch.uint8, device="cuda")
        self.contig_off = torch.empty(self.n_contigs + 1, dtype=torch.int64, device="cuda")

    def _all_to_all(self):
        import torch
        import torch.distributed as dist
        ins, outs = [int(x) for x in self.send_bytes], [int(x) for x in self.recv_bytes]
        send = self.send[: sum(ins)]
        recv = self.recv[: sum(outs)]
        if self.world == 1:
            recv.copy_(send)
            return
        if dist.get_backend(self.group) == "nccl":
            dist.all_to_all_single(recv, send, outs, ins, group=self.group)
        else:                                   # gloo moves host tensors
            r = torch.empty(sum(outs), dtype=torch.uint8)
            dist.all_to_all_single(r, send.cpu(), outs, ins, group=self.group)
            recv.copy_(r)
        torch.cuda.synchronize()                # the library reads recv on its own stream

    def step(self):
        """One pass: mask, chains, layout, the exchange, then this rank's share."""
        g = self.g
        cg.cg_mask_branches(g, want_count=False)
        cg.cg_chains(g, want_counts=False)
        cg.cg_exchange_pack(g, self.world, self.read_first, self.rank, self.my_packed, self.my_off, self.send)
        self._all_to_all()
        cg.cg_emit_share_received(g, self.world, self.read_first, self.rank, self.recv[: int(self.recv_bytes.sum())],
                                  self.contig_off, self.bases)

    def result(self):
        """(contig_off of the whole stream, this share's bases, first_base) as host arrays."""
        cg.cg_sync(self.ctx)
        return self.contig_off.cpu().numpy(), self.bases[: self.n_bases].cpu().numpy(), self.first_base

    def close(self):
        self.g.close()


def partition_digest(part) -> bytes:
    """A digest of an assignment, to check that every rank computed the same one."""
    return hashlib.sha256(np.ascontiguousarray(part, dtype=np.int32).tobytes()).digest()


def _send_recv_bytes(arr, rank: int, world: int, group=None):
    """Every rank's uint8 array on rank 0 (a list by rank); None elsewhere."""
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    n = torch.tensor([len(arr)], dtype=torch.int64, device=dev)
    sizes = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(x.item()) for x in sizes]
    if rank == 0:
        out = [np.asarray(arr)]
        for r in range(1, world):
            buf = torch.empty(max(sizes[r], 1), dtype=torch.uint8, device=dev)
            dist.recv(buf, src=r, group=group)
            out.append(buf[: sizes[r]].cpu().numpy())
        return out
    t = torch.from_numpy(np.ascontiguousarray(arr, dtype=np.uint8))
    if t.numel() == 0:
        t = torch.zeros(1, dtype=torch.uint8)
    dist.send(t.to(dev), dst=0, group=group)
    return None


def gather_shares(bases, first_base: int, rank: int, world: int, group=None):
    """The whole output stream on rank 0 from every rank's "tiles" share (the
    shares are consecutive runs of the stream, in rank order); None elsewhere.
    Checks that the shares tile the stream without gaps."""
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    fb = torch.tensor([int(first_base)], dtype=torch.int64, device=dev)
    firsts = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(firsts, fb, group=group)
    parts = _send_recv_bytes(bases, rank, world, group)
    if rank != 0:
        return None
    pos = 0
    for r in range(world):
        if int(firsts[r].item()) != pos:
            raise RuntimeError(f"share {r} starts at {int(firsts[r].item())}, expected {pos}")
        pos += len(parts[r])
    return np.concatenate(parts) if parts else np.zeros(0, np.uint8)


def gather_parts(bases, part, rank: int, world: int, group=None):
    """Every rank's "lpt" output on rank 0, as a list by part; also checks that
    all ranks computed the same partition. None elsewhere."""
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    d = torch.tensor(np.frombuffer(partition_digest(part), dtype=np.uint8).copy(), device=dev)
    ds = [torch.zeros_like(d) for _ in range(world)]
    dist.all_gather(ds, d, group=group)
    if any(not torch.equal(x, ds[0]) for x in ds):
        raise RuntimeError("ranks computed different partitions")
    return _send_recv_bytes(bases, rank, world, group)
