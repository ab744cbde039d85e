"""Thin Python binding of include/cg.h (ctypes; argument marshalling only).

Every step of contig generation runs in the CUDA library libcg.so; this module
only turns numpy arrays / torch tensors into pointers and sizes. Buffers that
are torch CUDA tensors are passed as device memory, numpy arrays and CPU
tensors as host memory. If libcg.so has not been built the first call raises.
"""
from __future__ import annotations

import sys
import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcg.so")

CG_OK, CG_EINVAL, CG_ENOMEM, CG_ECUDA, CG_EGRAPH, CG_ETIMEOUT, CG_EBUSY, CG_EKERNEL = range(8)
MEM_HOST, MEM_DEVICE = 0, 1
BORROW_DEVICE, NO_VALIDATE, HOST_READS, NO_READS = 1, 2, 4, 8

_lock = threading.Lock()
_lib = None


class CgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status


def _status_name(s):
    return ["CG_OK", "CG_EINVAL", "CG_ENOMEM", "CG_ECUDA", "CG_EGRAPH", "CG_ETIMEOUT", "CG_EBUSY",
            "CG_EKERNEL"][s] if 0 <= s < 8 else f"status {s}"


class GraphDesc(ctypes.Structure):
    _fields_ = [("n_reads", ctypes.c_int64), ("n_entries", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("row_ptr_bytes", ctypes.c_int32), ("mem", ctypes.c_int32), ("col", ctypes.c_void_p),
                ("code", ctypes.c_void_p), ("suf", ctypes.c_void_p), ("len", ctypes.c_void_p),
                ("off", ctypes.c_void_p), ("packed", ctypes.c_void_p), ("packed_bytes", ctypes.c_int64),
                ("min_chain_reads", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("pre", ctypes.c_void_p), ("post", ctypes.c_void_p)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_int32), ("workers", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_uint64)]


class ServerResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("batch_size", ctypes.c_int32), ("n_contigs", ctypes.c_int64),
                ("total_bases", ctypes.c_int64), ("contig_off", ctypes.POINTER(ctypes.c_int64)),
                ("bases", ctypes.POINTER(ctypes.c_uint8)), ("t_submit_ns", ctypes.c_int64),
                ("t_start_ns", ctypes.c_int64), ("t_done_ns", ctypes.c_int64)]


API = {
    "cg_create": [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p],
    "cg_destroy": [ctypes.c_void_p],
    "cg_load_graph": [ctypes.c_void_p, ctypes.POINTER(GraphDesc), ctypes.c_uint32, ctypes.POINTER(ctypes.c_void_p)],
    "cg_free_graph": [ctypes.c_void_p],
    "cg_load_batch": [ctypes.c_void_p, ctypes.POINTER(GraphDesc), ctypes.c_int, ctypes.c_uint32,
                      ctypes.POINTER(ctypes.c_void_p)],
    "cg_batch_ranges": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int],
    "cg_mask_branches": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)],
    "cg_chains": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                  ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
    "cg_emit_contigs": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                        ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
    "cg_emit_part": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                     ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                     ctypes.POINTER(ctypes.c_int64)],
    "cg_emit_share": [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64,
                      ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                      ctypes.POINTER(ctypes.c_int64)],
    "cg_exchange_sizes": [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                          ctypes.c_void_p],
    "cg_exchange_pack": [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                         ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64],
    "cg_emit_share_received": [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                               ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                               ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
    "cg_emit_contigs_2bit": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                             ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
    "cg_transitive_reduction": [ctypes.c_void_p, ctypes.POINTER(GraphDesc), ctypes.c_int32, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                ctypes.POINTER(ctypes.c_int64)],
    "cg_partition_contigs": [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64,
                             ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)],
    "cg_sync": [ctypes.c_void_p],
    "cg_selftest_wait_timeout": [ctypes.c_void_p, ctypes.c_int32],
    "cg_set_timing": [ctypes.c_void_p, ctypes.c_int],
    "cg_set_graphs": [ctypes.c_void_p, ctypes.c_int],
    "cg_set_pdl": [ctypes.c_void_p, ctypes.c_int],
    "cg_set_host_direct": [ctypes.c_void_p, ctypes.c_int],
    "cg_set_fault": [ctypes.c_void_p, ctypes.c_char_p],
    "cg_set_tuning": [ctypes.c_void_p, ctypes.c_void_p],
    "cg_get_tuning": [ctypes.c_void_p, ctypes.c_void_p],
    "cg_kernel_time": [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_float)],
    "cg_get_stats": [ctypes.c_void_p, ctypes.c_void_p],
    "cg_server_start": [ctypes.c_int, ctypes.POINTER(ServerOpts), ctypes.POINTER(ctypes.c_void_p)],
    "cg_server_submit": [ctypes.c_void_p, ctypes.POINTER(GraphDesc), ctypes.POINTER(ctypes.c_uint64)],
    "cg_server_poll": [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)],
    "cg_server_wait": [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(ServerResult)],
    "cg_server_release": [ctypes.c_void_p, ctypes.c_uint64],
    "cg_server_stats": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                        ctypes.POINTER(ctypes.c_uint64)],
    "cg_server_kernels": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)],
    "cg_server_contexts_replaced": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)],
    "cg_server_stop": [ctypes.c_void_p],
    "cg_offsets_noalloc": [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p],
    "cg_status_str": [ctypes.c_int],
    "cg_last_error": [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t],
}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                                   "(python -c 'import __graft_entry__ as g; g.build()')")
            L = ctypes.CDLL(LIB_PATH)
            for name, args in API.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = ctypes.c_char_p if name == "cg_status_str" else ctypes.c_int
            _lib = L
    return _lib


# ---------------------------------------------------------------- marshal
def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _mem_of(a) -> int:
    if _is_torch(a):
        return MEM_DEVICE if a.is_cuda else MEM_HOST
    return MEM_HOST


def _ptr(a):
    if a is None:
        return None
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("buffers must be C-contiguous numpy arrays or torch tensors")
    return ctypes.c_void_p(a.ctypes.data)


def _nbytes(a) -> int:
    return a.numel() * a.element_size() if _is_torch(a) else a.nbytes


def _check(ctx_ptr, st: int):
    if st != CG_OK:
        buf = ctypes.create_string_buffer(512)
        if ctx_ptr:
            lib().cg_last_error(ctx_ptr, buf, 512)
        raise CgError(st, buf.value.decode(errors="replace"))


def _mem_of_all(arrays):
    mems = {_mem_of(a) for a in arrays if a is not None}
    if len(mems) > 1:
        raise ValueError("all buffers of one call must be in the same memory (host or device)")
    return mems.pop() if mems else MEM_HOST


class Context:
    """A cg_ctx: one device, one stream."""

    def __init__(self, ptr):
        self.ptr = ptr

    def close(self):
        if self.ptr:
            lib().cg_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        if sys.is_finalizing():       # the process is exiting: the CUDA driver releases everything
            return
        try:
            self.close()
        except Exception:
            pass


class Graph:
    """A loaded cg_graph (keeps borrowed inputs alive)."""

    def __init__(self, ctx: Context, ptr, keep, n: int):
        self.ctx, self.ptr, self._keep, self.n = ctx, ptr, keep, n

    def close(self):
        if self.ptr:
            lib().cg_free_graph(self.ptr)
            self.ptr = None
            self._keep = None

    def __del__(self):
        if sys.is_finalizing():       # the process is exiting: the CUDA driver releases everything
            return
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ the C ABI
def cg_create(device: int = 0, hbm_budget_bytes: int = 0, stream=None) -> Context:
    """cg_create: stream may be a torch.cuda.Stream, a raw cudaStream_t int, or None."""
    handle = None
    if stream is not None:
        handle = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    out = ctypes.c_void_p()
    st = lib().cg_create(ctypes.byref(out), int(device), int(hbm_budget_bytes), handle)
    if st != CG_OK:
        raise CgError(st, "cg_create failed")
    return Context(out)


def cg_destroy(ctx: Context):
    ctx.close()


def cg_load_graph(ctx: Context, graph, flags: int = 0, min_chain_reads: int = 2) -> Graph:
    """cg_load_graph from any object with row_ptr, col, code, suf, len, off, packed
    (and pre, post for the x-drop form)."""
    d = _desc(graph, min_chain_reads)
    out = ctypes.c_void_p()
    _check(ctx.ptr, lib().cg_load_graph(ctx.ptr, ctypes.byref(d), int(flags), ctypes.byref(out)))
    keep = [getattr(graph, k, None) for k in ("row_ptr", "col", "code", "suf", "len", "off", "packed", "pre", "post")]
    return Graph(ctx, out, keep if flags & (BORROW_DEVICE | HOST_READS) else None, d.n_reads)


def _np_addr(a) -> int:
    """The data address of a C-contiguous numpy array (the fast path of _desc:
    a ctypes view of a writable buffer is the cheapest way to it)."""
    if not a.flags.c_contiguous:
        raise ValueError("buffers must be C-contiguous numpy arrays or torch tensors")
    try:
        return ctypes.addressof(ctypes.c_char.from_buffer(a))
    except (TypeError, ValueError, BufferError):       # read-only or empty
        return a.__array_interface__["data"][0]


def _desc(graph, min_chain_reads):
    """The cg_graph_desc of `graph`: an object with row_ptr, col, code, suf, len,
    off and packed (numpy arrays or torch tensors); with `pre` and `post` as
    well it is in the x-drop form and suf may be None."""
    pre, post = getattr(graph, "pre", None), getattr(graph, "post", None)
    if pre is None or post is None:
        pre = post = None
    suf = getattr(graph, "suf", None)
    arrs = [graph.row_ptr, graph.col, graph.code, suf, graph.len, graph.off, graph.packed, pre, post]
    nd = np.ndarray
    if all(a is None or type(a) is nd for a in arrs):     # all host numpy arrays: fewer Python steps
        d = GraphDesc()
        d.n_reads = len(graph.len)
        d.n_entries = len(graph.col)
        d.row_ptr, d.row_ptr_bytes, d.mem = _np_addr(graph.row_ptr), graph.row_ptr.dtype.itemsize, MEM_HOST
        d.col, d.code = _np_addr(graph.col), _np_addr(graph.code)
        d.suf = _np_addr(suf) if suf is not None else None
        d.pre = _np_addr(pre) if pre is not None else None
        d.post = _np_addr(post) if post is not None else None
        d.len, d.off = _np_addr(graph.len), _np_addr(graph.off)
        if graph.packed is not None:
            d.packed, d.packed_bytes = _np_addr(graph.packed), graph.packed.nbytes
        else:
            d.packed, d.packed_bytes = None, int(getattr(graph, "packed_bytes", 0))
        d.min_chain_reads = int(min_chain_reads)
        return d
    mem = _mem_of_all(arrs)
    rp = graph.row_ptr
    d = GraphDesc()
    d.n_reads = len(graph.len)
    d.n_entries = len(graph.col)
    d.row_ptr, d.row_ptr_bytes, d.mem = _ptr(rp), (rp.element_size() if _is_torch(rp) else rp.dtype.itemsize), mem
    d.col, d.code, d.suf = _ptr(graph.col), _ptr(graph.code), _ptr(suf)
    d.pre, d.post = _ptr(pre), _ptr(post)
    d.len, d.off, d.packed = _ptr(graph.len), _ptr(graph.off), _ptr(graph.packed)
    # a graph without its reads (NO_READS) gives the size of its virtual stream instead
    d.packed_bytes = _nbytes(graph.packed) if graph.packed is not None else int(getattr(graph, "packed_bytes", 0))
    d.min_chain_reads = int(min_chain_reads)
    return d


def cg_load_batch(ctx: Context, graphs, flags: int = 0, min_chain_reads: int = 2) -> Graph:
    """cg_load_batch: the graphs as one union graph (see cg_batch_ranges)."""
    k = len(graphs)
    descs = (GraphDesc * k)(*[_desc(gr, min_chain_reads) for gr in graphs])
    out = ctypes.c_void_p()
    _check(ctx.ptr, lib().cg_load_batch(ctx.ptr, descs, k, int(flags), ctypes.byref(out)))
    g = Graph(ctx, out, list(graphs) if flags & HOST_READS else None, int(sum(len(gr.len) for gr in graphs)))
    g.batch_k = k
    return g


def cg_batch_ranges(g: Graph, first_contig=None, first_base=None):
    """Per graph of a batch: first contig and first base in the union outputs (k+1 entries)."""
    if first_contig is None and first_base is None:
        first_contig = np.empty(g.batch_k + 1, np.int64)
        first_base = np.empty(g.batch_k + 1, np.int64)
    mem = _mem_of_all([first_contig, first_base])
    _check(g.ctx.ptr, lib().cg_batch_ranges(g.ptr, _ptr(first_contig), _ptr(first_base), mem))
    return first_contig, first_base


def cg_free_graph(g: Graph):
    g.close()


def cg_mask_branches(g: Graph, is_branch=None, want_count: bool = True):
    nb = ctypes.c_int64(-1)
    _check(g.ctx.ptr, lib().cg_mask_branches(g.ptr, _ptr(is_branch), _mem_of_all([is_branch]),
                                             ctypes.byref(nb) if want_count else None))
    return nb.value if want_count else None


def cg_chains(g: Graph, chain_id=None, rank=None, orient=None, want_counts: bool = True):
    nc, ncy = ctypes.c_int64(-1), ctypes.c_int64(-1)
    mem = _mem_of_all([chain_id, rank, orient])
    _check(g.ctx.ptr, lib().cg_chains(g.ptr, _ptr(chain_id), _ptr(rank), _ptr(orient), mem,
                                      ctypes.byref(nc) if want_counts else None,
                                      ctypes.byref(ncy) if want_counts else None))
    return (nc.value, ncy.value) if want_counts else None


def cg_emit_contigs(g: Graph, contig_off=None, bases=None, want_counts: bool = True):
    nc, tot = ctypes.c_int64(-1), ctypes.c_int64(-1)
    mem = _mem_of_all([contig_off, bases])
    ocap = len(contig_off) if contig_off is not None else 0
    bcap = _nbytes(bases) if bases is not None else 0
    _check(g.ctx.ptr, lib().cg_emit_contigs(g.ptr, _ptr(contig_off), ocap, _ptr(bases), bcap, mem,
                                            ctypes.byref(nc) if want_counts else None,
                                            ctypes.byref(tot) if want_counts else None))
    return (nc.value, tot.value) if want_counts else None


def cg_emit_contigs_2bit(g: Graph, contig_off=None, packed=None, want_counts: bool = True):
    """Contigs in the 2-bit layout (base i at byte i >> 2, bits 2 (i & 3)); `packed`
    holds at least packed_bytes_2bit(total_bases) bytes. NULL outputs: sizes only."""
    nc, tot = ctypes.c_int64(-1), ctypes.c_int64(-1)
    mem = _mem_of_all([contig_off, packed])
    ocap = len(contig_off) if contig_off is not None else 0
    pcap = _nbytes(packed) if packed is not None else 0
    _check(g.ctx.ptr, lib().cg_emit_contigs_2bit(g.ptr, _ptr(contig_off), ocap, _ptr(packed), pcap, mem,
                                                 ctypes.byref(nc) if want_counts else None,
                                                 ctypes.byref(tot) if want_counts else None))
    return (nc.value, tot.value) if want_counts else None


def packed_bytes_2bit(total_bases: int) -> int:
    """Output bytes of the 2-bit form: whole 16-byte chunks of 64 bases."""
    return 16 * ((int(total_bases) + 63) // 64)


def cg_transitive_reduction(ctx: Context, graph, fuzz: int = 0, device: bool = False):
    """TransitiveReduction (Alg. 1, Sec. 2) of the overlap graph `graph` (suffix
    form, rows sorted). Returns the string graph: row_ptr (int64), col, code,
    suf (numpy, or torch CUDA tensors with device=True) plus graph's len, off and
    packed, ready for cg_load_graph. Two calls: the size, then the arrays."""
    from types import SimpleNamespace
    d = _desc(graph, 2)
    cnt = ctypes.c_int64(-1)
    _check(ctx.ptr, lib().cg_transitive_reduction(ctx.ptr, ctypes.byref(d), int(fuzz), None, None, None, None, 0,
                                                  MEM_HOST, ctypes.byref(cnt)))
    k, n = int(cnt.value), int(d.n_reads)
    if device:
        import torch
        rp = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        col = torch.empty(max(k, 1), dtype=torch.int32, device="cuda")
        code = torch.empty(max(k, 1), dtype=torch.uint8, device="cuda")
        suf = torch.empty(max(k, 1), dtype=torch.int32, device="cuda")
        mem = MEM_DEVICE
    else:
        rp = np.empty(n + 1, np.int64)
        col, code, suf = np.empty(max(k, 1), np.int32), np.empty(max(k, 1), np.uint8), np.empty(max(k, 1), np.int32)
        mem = MEM_HOST
    _check(ctx.ptr, lib().cg_transitive_reduction(ctx.ptr, ctypes.byref(d), int(fuzz), _ptr(rp), _ptr(col), _ptr(code),
                                                  _ptr(suf), k, mem, ctypes.byref(cnt)))
    return SimpleNamespace(row_ptr=rp, col=col[:k], code=code[:k], suf=suf[:k], len=graph.len, off=graph.off,
                           packed=graph.packed, n=n, m=k)


WEIGHT_READS, WEIGHT_BASES = 0, 1
MAX_PARTS = 1024


def cg_partition_contigs(g: Graph, n_parts: int, weight: int = WEIGHT_READS, part=None, part_weight=None):
    """GreedyPartitioning of the contigs into n_parts parts (Sec. 4.3).

    With no buffers given, returns host arrays (part per contig, weight sum per
    part); otherwise fills `part` (>= n_contigs entries) and `part_weight`
    (n_parts entries), both host or both device, and returns n_contigs.
    """
    if part is None and part_weight is None:
        nc, _ = cg_emit_contigs(g)
        part = np.empty(max(nc, 1), dtype=np.int32)
        part_weight = np.empty(max(int(n_parts), 1), dtype=np.int64)
        out = ctypes.c_int64(-1)
        _check(g.ctx.ptr, lib().cg_partition_contigs(g.ptr, int(n_parts), int(weight), _ptr(part), len(part),
                                                     _ptr(part_weight), MEM_HOST, ctypes.byref(out)))
        return part[:out.value], part_weight[:n_parts]
    mem = _mem_of_all([part, part_weight])
    out = ctypes.c_int64(-1)
    _check(g.ctx.ptr, lib().cg_partition_contigs(g.ptr, int(n_parts), int(weight), _ptr(part),
                                                 len(part) if part is not None else 0, _ptr(part_weight), mem,
                                                 ctypes.byref(out)))
    return out.value


def cg_emit_part(g: Graph, part, p: int, contig_off=None, bases=None, want_counts: bool = True):
    """The contigs c with part[c] == p back to back, each spelled as cg_emit_contigs
    spells it (Sec. 4.3-4.4); contig_off (n_contigs + 1) gets every contig's range
    in that output, empty for the contigs of other parts. part is int32 (at least
    n_contigs entries); part, contig_off and bases are all host or all device.
    NULL bases: sizes only. Returns (the graph's n_contigs, the part's bases)."""
    if part is not None:
        dt = str(part.dtype)
        if dt not in ("int32", "torch.int32"):
            raise ValueError("part must be int32")
    nc, tot = ctypes.c_int64(-1), ctypes.c_int64(-1)
    mem = _mem_of_all([part, contig_off, bases])
    pcap = len(part) if part is not None else 0
    ocap = len(contig_off) if contig_off is not None else 0
    bcap = _nbytes(bases) if bases is not None else 0
    _check(g.ctx.ptr, lib().cg_emit_part(g.ptr, _ptr(part), pcap, int(p), _ptr(contig_off), ocap, _ptr(bases), bcap,
                                         mem, ctypes.byref(nc) if want_counts else None,
                                         ctypes.byref(tot) if want_counts else None))
    return (nc.value, tot.value) if want_counts else None


def cg_emit_share(g: Graph, share: int, n_shares: int, contig_off=None, bases=None, want_range: bool = True):
    """Share `share` of n_shares equal runs of output tiles of the whole contig
    stream (Sec. 4.3-4.4 with the work split by output bytes): bases[:n] = stream
    bytes [first_base, first_base + n). contig_off (n_contigs + 1) gets the whole
    stream's offsets. Buffers all host or all device. Returns (first_base, n)."""
    fb, nb = ctypes.c_int64(-1), ctypes.c_int64(-1)
    mem = _mem_of_all([contig_off, bases])
    ocap = len(contig_off) if contig_off is not None else 0
    bcap = _nbytes(bases) if bases is not None else 0
    _check(g.ctx.ptr, lib().cg_emit_share(g.ptr, int(share), int(n_shares), _ptr(contig_off), ocap, _ptr(bases), bcap,
                                          mem, ctypes.byref(fb) if want_range else None,
                                          ctypes.byref(nb) if want_range else None))
    return (fb.value, nb.value) if want_range else None


def _read_first(read_first, n_shares):
    rf = np.ascontiguousarray(read_first, dtype=np.int64)
    if rf.shape != (n_shares + 1,):
        raise ValueError("read_first needs n_shares + 1 entries")
    return rf


def cg_exchange_sizes(g: Graph, n_shares: int, read_first, rank: int):
    """Bytes this rank sends to each share and receives from each rank (the read
    exchange of a split whose ranks hold slices of the reads; graph loaded with
    NO_READS). Returns (send_bytes, recv_bytes) as host int64 arrays."""
    rf = _read_first(read_first, n_shares)
    send = np.zeros(n_shares, np.int64)
    recv = np.zeros(n_shares, np.int64)
    _check(g.ctx.ptr, lib().cg_exchange_sizes(g.ptr, int(n_shares), _ptr(rf), int(rank), _ptr(send), _ptr(recv)))
    return send, recv


def cg_exchange_pack(g: Graph, n_shares: int, read_first, rank: int, my_packed, my_off, send_buf):
    """This rank's segments for every share into send_buf (device uint8): the
    pieces of each share whose reads this rank owns, from my_packed (device, this
    rank's reads; my_off[i] = first base of read read_first[rank] + i in it)."""
    rf = _read_first(read_first, n_shares)
    for name, t in (("my_packed", my_packed), ("my_off", my_off), ("send_buf", send_buf)):
        if t is not None and not (_is_torch(t) and t.is_cuda):
            raise ValueError(f"{name} must be a CUDA tensor")
    _check(g.ctx.ptr, lib().cg_exchange_pack(g.ptr, int(n_shares), _ptr(rf), int(rank), _ptr(my_packed),
                                             _nbytes(my_packed) if my_packed is not None else 0, _ptr(my_off),
                                             _ptr(send_buf), _nbytes(send_buf)))


def cg_emit_share_received(g: Graph, n_shares: int, read_first, rank: int, recv_buf, contig_off=None, bases=None):
    """Spells this rank's share from recv_buf (device uint8: every rank's segment for
    this rank, by source rank); outputs device tensors as for cg_emit_share.
    Returns (first_base, n_bases)."""
    rf = _read_first(read_first, n_shares)
    fb, nb = ctypes.c_int64(-1), ctypes.c_int64(-1)
    ocap = len(contig_off) if contig_off is not None else 0
    bcap = _nbytes(bases) if bases is not None else 0
    _check(g.ctx.ptr, lib().cg_emit_share_received(g.ptr, int(n_shares), _ptr(rf), int(rank), _ptr(recv_buf),
                                                   _nbytes(recv_buf) if recv_buf is not None else 0, _ptr(contig_off),
                                                   ocap, _ptr(bases), bcap, ctypes.byref(fb), ctypes.byref(nb)))
    return fb.value, nb.value


def contigs_part_host(g: Graph, part, p: int):
    """Host copies (contig_off, bases) of part p's spelling (see cg_emit_part);
    part may be None for a graph without contigs."""
    if part is not None:
        part = np.ascontiguousarray(part, dtype=np.int32)
    nc, tot = cg_emit_part(g, part, p)
    off = np.empty(nc + 1, dtype=np.int64)
    bases = np.empty(max(tot, 1), dtype=np.uint8)
    cg_emit_part(g, part, p, off, bases)
    return off, bases[:tot]


def cg_sync(ctx: Context):
    _check(ctx.ptr, lib().cg_sync(ctx.ptr))


def cg_selftest_wait_timeout(ctx: Context, tiles: int = 2) -> int:
    """Runs the look-back scan with its first tile withheld so that the bounded
    device wait runs out; returns the status (CG_ETIMEOUT expected; the context
    then refuses work until it is destroyed)."""
    return int(lib().cg_selftest_wait_timeout(ctx.ptr, int(tiles)))


class Tuning(ctypes.Structure):
    _fields_ = [("ruler_log2", ctypes.c_int32), ("tile_bytes", ctypes.c_int32), ("emit_blocks_per_sm", ctypes.c_int32),
                ("emit_block_threads", ctypes.c_int32)]


def cg_set_tuning(ctx: Context, ruler_log2: int = 0, tile_bytes: int = 0, emit_blocks_per_sm: int = 0,
                  emit_block_threads: int = 0):
    t = Tuning(int(ruler_log2), int(tile_bytes), int(emit_blocks_per_sm), int(emit_block_threads))
    _check(ctx.ptr, lib().cg_set_tuning(ctx.ptr, ctypes.byref(t)))


def cg_get_tuning(ctx: Context) -> dict:
    t = Tuning()
    _check(ctx.ptr, lib().cg_get_tuning(ctx.ptr, ctypes.byref(t)))
    return {"ruler_log2": t.ruler_log2, "tile_bytes": t.tile_bytes, "emit_blocks_per_sm": t.emit_blocks_per_sm,
            "emit_block_threads": t.emit_block_threads}


class Stats(ctypes.Structure):
    _fields_ = [("kernels_launched", ctypes.c_uint64), ("stage_ms", ctypes.c_float * 4)]


def cg_set_fault(ctx: Context, spec: str | None):
    """Host-side fault injection plan of a context ("site:n[:ms],..."; None clears)."""
    _check(ctx.ptr, lib().cg_set_fault(ctx.ptr, spec.encode() if spec else None))


def cg_set_host_direct(ctx: Context, enable: bool):
    """Kernels write pinned host outputs in place (True, the default) or via a device copy (False)."""
    _check(ctx.ptr, lib().cg_set_host_direct(ctx.ptr, 1 if enable else 0))


def cg_set_graphs(ctx: Context, enable: bool):
    _check(ctx.ptr, lib().cg_set_graphs(ctx.ptr, 1 if enable else 0))


def cg_set_pdl(ctx: Context, enable: bool):
    """Programmatic dependent launch between consecutive kernels of a stage (on by default)."""
    _check(ctx.ptr, lib().cg_set_pdl(ctx.ptr, 1 if enable else 0))


def cg_set_timing(ctx: Context, level):
    """0 off, 1 (or True) stage events, 2 stage and per-kernel events, 3 events around the spelling stage only."""
    _check(ctx.ptr, lib().cg_set_timing(ctx.ptr, int(level)))


def cg_get_stats(ctx: Context) -> dict:
    """kernels launched so far and the last mask / chain / offset / emission stage times (ms)."""
    s = Stats()
    _check(ctx.ptr, lib().cg_get_stats(ctx.ptr, ctypes.byref(s)))
    return {"kernels_launched": int(s.kernels_launched), "stage_ms": [float(x) for x in s.stage_ms]}


class Server:
    """cg_server: continuous batching over the batched form (host inputs and outputs).
    `workers` batches are in flight at once, each on its own context and stream."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 150 << 30, max_batch: int = 64, workers: int = 8):
        self.ptr = ctypes.c_void_p()
        opts = ServerOpts(int(max_batch), int(workers), int(hbm_budget_bytes))
        st = lib().cg_server_start(int(device), ctypes.byref(opts), ctypes.byref(self.ptr))
        if st != CG_OK:
            raise CgError(st, "cg_server_start failed")
        self._keep = {}

    def submit(self, graph, min_chain_reads: int = 2) -> int:
        d = _desc(graph, min_chain_reads)
        if d.mem != MEM_HOST:
            raise ValueError("server requests take host buffers")
        rid = ctypes.c_uint64()
        st = lib().cg_server_submit(self.ptr, ctypes.byref(d), ctypes.byref(rid))
        if st != CG_OK:
            raise CgError(st, "cg_server_submit refused the request")
        self._keep[rid.value] = graph            # its buffers must outlive the request
        return rid.value

    def poll(self, rid: int) -> bool:
        done = ctypes.c_int()
        _check(None, lib().cg_server_poll(self.ptr, rid, ctypes.byref(done)))
        return bool(done.value)

    def wait(self, rid: int, timeout_ms: int = -1, copy: bool = True) -> dict:
        """Result of a request: status, counts, contig_off / bases (copies), timestamps (ns)."""
        r = ServerResult()
        _check(None, lib().cg_server_wait(self.ptr, rid, int(timeout_ms), ctypes.byref(r)))
        out = {"status": r.status, "batch_size": r.batch_size, "n_contigs": r.n_contigs,
               "total_bases": r.total_bases, "t_submit_ns": r.t_submit_ns, "t_start_ns": r.t_start_ns,
               "t_done_ns": r.t_done_ns}
        if copy and r.status == CG_OK:
            out["contig_off"] = np.ctypeslib.as_array(r.contig_off, shape=(r.n_contigs + 1,)).copy()
            out["bases"] = (np.ctypeslib.as_array(r.bases, shape=(r.total_bases,)).copy() if r.total_bases
                            else np.zeros(0, np.uint8))
        return out

    def release(self, rid: int):
        _check(None, lib().cg_server_release(self.ptr, rid))
        self._keep.pop(rid, None)

    def stats(self) -> dict:
        b, q, f = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(None, lib().cg_server_stats(self.ptr, ctypes.byref(b), ctypes.byref(q), ctypes.byref(f)))
        n, rep = ctypes.c_uint64(), ctypes.c_uint64()
        _check(None, lib().cg_server_kernels(self.ptr, ctypes.byref(n)))
        _check(None, lib().cg_server_contexts_replaced(self.ptr, ctypes.byref(rep)))
        return {"batches": b.value, "requests": q.value, "in_flight_bytes": f.value, "kernels_launched": n.value,
                "contexts_replaced": rep.value}

    def stop(self):
        if self.ptr:
            lib().cg_server_stop(self.ptr)
            self.ptr = None
            self._keep = {}

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass


NOALLOC_MAX_COUNT = 16777216


def cg_offsets_noalloc(lengths, offsets, stream=None):
    """cg_offsets_noalloc on device tensors: offsets[i] = sum(lengths[:i]), offsets[-1] = total.
    lengths: a CUDA int32 tensor; offsets: a CUDA int64 tensor of len(lengths) + 1 entries."""
    for name, t, dt in (("lengths", lengths, "torch.int32"), ("offsets", offsets, "torch.int64")):
        if not _is_torch(t) or not t.is_cuda or str(t.dtype) != dt:
            raise ValueError(f"{name} must be a CUDA tensor of {dt}")
    handle = None
    if stream is not None:
        handle = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    count = len(lengths)
    if len(offsets) < count + 1:
        raise ValueError("offsets needs count + 1 entries")
    _check(None, lib().cg_offsets_noalloc(_ptr(lengths), count, _ptr(offsets), handle))


def cg_kernel_times(ctx: Context) -> list:
    """[(kernel name, ms)] of the last run, with timing level 2 (cg_set_timing)."""
    out = []
    k = 0
    while True:
        name, ms = ctypes.c_char_p(), ctypes.c_float()
        if lib().cg_kernel_time(ctx.ptr, k, ctypes.byref(name), ctypes.byref(ms)) != CG_OK:
            return out
        out.append((name.value.decode(), float(ms.value)))
        k += 1


def cg_status_str(s: int) -> str:
    return lib().cg_status_str(int(s)).decode()


# ------------------------------------------------------- convenience
def contigs_2bit_host(g: Graph):
    """Two-call size query, then contig offsets and the 2-bit stream into host arrays."""
    n_contigs, total = cg_emit_contigs_2bit(g)
    off = np.empty(n_contigs + 1, dtype=np.int64)
    packed = np.empty(max(packed_bytes_2bit(total), 16), dtype=np.uint8)
    cg_emit_contigs_2bit(g, off, packed)
    return off, packed[: packed_bytes_2bit(total)], total


def contigs_host(g: Graph):
    """Two-call size query, then every output into host numpy arrays."""
    n_contigs, total = cg_emit_contigs(g)
    off = np.empty(n_contigs + 1, dtype=np.int64)
    bases = np.empty(max(total, 1), dtype=np.uint8)
    cg_emit_contigs(g, off, bases)
    return off, bases[:total]


def chains_host(g: Graph):
    cid = np.empty(g.n, dtype=np.int32)
    rank = np.empty(g.n, dtype=np.int32)
    orient = np.empty(g.n, dtype=np.uint8)
    n_contigs, n_cycles = cg_chains(g, cid, rank, orient)
    return cid, rank, orient, n_contigs, n_cycles
