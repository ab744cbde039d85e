"""Seeded synthetic string-graph inputs (test and benchmark input only).

The generator lays out a genome with repeat families, samples long reads,
keeps contained reads as edgeless vertices and keeps the overlaps a perfect overlapper followed by
transitive reduction would keep, plus repeat-induced overlaps that create
branch reads (the string graph of Sec. 2; dataset shapes of Table 2). It holds
no step of contig generation itself. Both the CUDA path and the CPU oracle
consume what it produces.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_libcggen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile cg_gen.c into gen/_libcggen.so (gcc, pthreads)."""
    src = os.path.join(_HERE, "cg_gen.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= max(
        os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "cg_gen.h"))
    ):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.run(
        ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-pthread", "-o", tmp, src, "-lm"],
        check=True,
    )
    os.replace(tmp, _SO)
    return _SO


class RepClass(ctypes.Structure):
    _fields_ = [("share", ctypes.c_double), ("seg_min", ctypes.c_int32), ("seg_max", ctypes.c_int32),
                ("copies_min", ctypes.c_int32), ("copies_max", ctypes.c_int32), ("div_max", ctypes.c_double)]


class GenCfg(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("genome_len", ctypes.c_int64), ("n_classes", ctypes.c_int32),
                ("_pad0", ctypes.c_int32), ("cls", RepClass * 4), ("coverage", ctypes.c_double),
                ("len_kind", ctypes.c_int32), ("len_min", ctypes.c_int32), ("len_a", ctypes.c_double),
                ("len_b", ctypes.c_double), ("min_overlap", ctypes.c_int32), ("k_rep", ctypes.c_int32),
                ("rep_div_accept", ctypes.c_double), ("threads", ctypes.c_int32), ("shuffle_ids", ctypes.c_int32),
                ("off_align", ctypes.c_int32), ("full_overlaps", ctypes.c_int32)]


class GenInfo(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in (
        "genome_len", "n_sampled", "n_reads", "n_kept", "n_entries", "packed_bytes", "total_read_bases",
        "n_true_pairs", "n_rep_pairs", "n_copies", "n_families", "repeat_bases")]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            lib.cg_gen_plan.restype = ctypes.c_void_p
            lib.cg_gen_plan.argtypes = [ctypes.POINTER(GenCfg)]
            lib.cg_gen_error.restype = ctypes.c_char_p
            lib.cg_gen_error.argtypes = [ctypes.c_void_p]
            lib.cg_gen_get_info.argtypes = [ctypes.c_void_p, ctypes.POINTER(GenInfo)]
            lib.cg_gen_fill.restype = ctypes.c_int
            lib.cg_gen_fill.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 10
            lib.cg_gen_genome.restype = ctypes.c_int
            lib.cg_gen_genome.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]
            lib.cg_gen_free.argtypes = [ctypes.c_void_p]
            _lib = lib
    return _lib


# --------------------------------------------------------------------------
# Workloads. Seeds: the i-th named workload uses 220704350 + i; graph j of the
# batched / served pools uses (base seed) * 1000 + j.
SEED0 = 220704350


def _cfg(seed, G, classes, coverage, len_kind, a, b, len_min, rep_div_accept=0.0, k_rep=2, min_overlap=2000):
    return dict(seed=int(seed), genome_len=int(G), classes=list(classes), coverage=float(coverage),
                len_kind=int(len_kind), len_a=float(a), len_b=float(b), len_min=int(len_min),
                min_overlap=int(min_overlap), k_rep=int(k_rep), rep_div_accept=float(rep_div_accept))


def _loguniform(seed, j, lo, hi):
    # deterministic per-graph genome size: log-uniform in [lo, hi]
    x = np.random.default_rng([seed, j]).random()
    return int(round(math.exp(math.log(lo) + x * (math.log(hi) - math.log(lo)))))


WORKLOADS = {
    # 1 Mb uniform genome, 20 copies of one 5 kb repeat, 10x, read lengths U[5,15] kb
    "tiny-1Mb": lambda: _cfg(SEED0 + 0, 1_000_000, [(0.10, 5000, 5000, 20, 20, 0.0)], 10, 0, 5000, 15000, 1),
    # 100 Mb, 5% repeats (2-20 kb segments, 2-10 copies), 40x, lognormal(12 kb, 6 kb, min 2 kb)
    "genome-100Mb": lambda: _cfg(SEED0 + 1, 100_000_000, [(0.05, 2000, 20000, 2, 10, 0.0)], 40, 1, 12000, 6000, 2000),
    # 3.1 Gb, 45% repeats from 300 bp and 6 kb families at 0-15% divergence, 30x, lognormal(15 kb, 8 kb)
    "genome-3.1Gb": lambda: _cfg(SEED0 + 2, 3_100_000_000,
                                 [(0.20, 300, 300, 50000, 150000, 0.15), (0.25, 6000, 6000, 1000, 4000, 0.15)],
                                 30, 1, 15000, 8000, 2000, rep_div_accept=0.05),
}


def batched_graph(j: int):
    """Graph j of the 512-graph batch: genome log-U[0.5, 12] Mb, 2% repeats, 30x, LN(10 kb, 5 kb)."""
    seed = (SEED0 + 3) * 1000 + j
    G = _loguniform(SEED0 + 3, j, 0.5e6, 12e6)
    return _cfg(seed, G, [(0.02, 2000, 20000, 2, 10, 0.0)], 30, 1, 10000, 5000, 2000)


def served_graph(j: int):
    """Graph j of the served pool: genome log-U[1, 200] Mb, 5% repeats, 30x, LN(12 kb, 6 kb)."""
    seed = (SEED0 + 4) * 1000 + j
    G = _loguniform(SEED0 + 4, j, 1e6, 200e6)
    return _cfg(seed, G, [(0.05, 2000, 20000, 2, 10, 0.0)], 30, 1, 12000, 6000, 2000)


def make_cfg(d: dict, threads: int | None = None, off_align: int = 32, shuffle_ids: bool = True) -> GenCfg:
    c = GenCfg()
    c.seed = d["seed"]
    c.genome_len = d["genome_len"]
    cl = d["classes"]
    c.n_classes = len(cl)
    for i, (share, smin, smax, cmin, cmax, div) in enumerate(cl):
        c.cls[i] = RepClass(share, smin, smax, cmin, cmax, div)
    c.coverage = d["coverage"]
    c.len_kind = d["len_kind"]
    c.len_min = d["len_min"]
    c.len_a = d["len_a"]
    c.len_b = d["len_b"]
    c.min_overlap = d["min_overlap"]
    c.k_rep = d["k_rep"]
    c.rep_div_accept = d["rep_div_accept"]
    c.threads = int(threads or min(32, os.cpu_count() or 1))
    c.shuffle_ids = 1 if shuffle_ids else 0
    c.off_align = int(off_align)
    c.full_overlaps = int(d.get("full_overlaps", 0))
    return c


@dataclass
class Graph:
    """A generated string graph, CSR in read-id space, plus ground truth."""
    n: int
    m: int
    row_ptr: np.ndarray
    col: np.ndarray
    code: np.ndarray
    suf: np.ndarray
    len: np.ndarray
    off: np.ndarray
    packed: np.ndarray
    is_true: np.ndarray
    gstart: np.ndarray
    strand: np.ndarray
    contained: np.ndarray
    info: dict
    cfg: dict
    _handle: object = field(default=None, repr=False)

    @property
    def packed_bytes(self) -> int:
        return int(self.packed.shape[0])

    def genome(self, start: int, count: int) -> bytes:
        """ASCII genome[start, start+count) (ground truth for tests)."""
        if self._handle is None:
            raise RuntimeError("genome handle released")
        buf = np.empty(count, dtype=np.uint8)
        if _load().cg_gen_genome(self._handle.ptr, start, count, buf.ctypes.data) != 0:
            raise ValueError("genome range")
        return buf.tobytes()

    def release(self):
        if self._handle is not None:
            self._handle.close()
            self._handle = None


class _Handle:
    def __init__(self, ptr):
        self.ptr = ptr

    def close(self):
        if self.ptr:
            _load().cg_gen_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def generate(d: dict | str, threads: int | None = None, rp_bytes: int | None = None, off_align: int = 32,
             shuffle_ids: bool = True, keep_genome: bool = True, alloc=None, with_packed: bool = True) -> Graph:
    """Build one graph. `alloc(shape, dtype)` may supply (e.g. pinned) host buffers;
    with_packed=False leaves the read sequences out (graph statistics only)."""
    if isinstance(d, str):
        d = WORKLOADS[d]()
    lib = _load()
    cfg = make_cfg(d, threads, off_align, shuffle_ids)
    h = _Handle(lib.cg_gen_plan(ctypes.byref(cfg)))
    if not h.ptr:
        raise MemoryError("cg_gen_plan")
    err = lib.cg_gen_error(h.ptr).decode()
    if err:
        h.close()
        raise ValueError(err)
    inf = GenInfo()
    lib.cg_gen_get_info(h.ptr, ctypes.byref(inf))
    info = {k: int(getattr(inf, k)) for k, _ in GenInfo._fields_}
    n, m = info["n_reads"], info["n_entries"]
    if rp_bytes is None:
        rp_bytes = 8 if m > 2**31 - 1 or d["genome_len"] >= 1_000_000_000 else 4
    mk = alloc or (lambda shape, dt: np.empty(shape, dtype=dt))
    rp = mk((n + 1,), np.int64 if rp_bytes == 8 else np.int32)
    col, code, suf = mk((m,), np.int32), mk((m,), np.uint8), mk((m,), np.int32)
    ln, off = mk((n,), np.int32), mk((n,), np.int64)
    packed = mk((info["packed_bytes"],), np.uint8) if with_packed else np.zeros(1, np.uint8)
    is_true, gstart, strand = np.empty(m, np.uint8), np.empty(n, np.int64), np.empty(n, np.uint8)
    contained = np.empty(n, np.uint8)

    def p(a):
        return ctypes.c_void_p(a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr())

    rc = lib.cg_gen_fill(h.ptr, p(rp), rp_bytes, p(col), p(code), p(suf), p(ln), p(off),
                         p(packed) if with_packed else None,
                         p(is_true), p(gstart), p(strand), p(contained))
    if rc != 0:
        h.close()
        raise RuntimeError(f"cg_gen_fill failed ({rc})")
    g = Graph(n, m, rp, col, code, suf, ln, off, packed, is_true, gstart, strand, contained, info, d, h)
    if not keep_genome:
        g.release()
    return g


# --------------------------------------------------------------------------
# Small helpers for tests: hand-built graphs in the same input format.
_ENC = {ord("A"): 0, ord("C"): 1, ord("G"): 2, ord("T"): 3}


def pack_reads(seqs, align: int = 1):
    """Pack ASCII reads into one 2-bit stream; returns (len, off, packed)."""
    lens = np.array([len(s) for s in seqs], dtype=np.int32)
    offs = np.zeros(len(seqs), dtype=np.int64)
    acc = 0
    for i, s in enumerate(seqs):
        offs[i] = acc
        acc += (len(s) + align - 1) // align * align
    packed = np.zeros(max(1, (acc + 3) // 4), dtype=np.uint8)
    for i, s in enumerate(seqs):
        for t, ch in enumerate(s.encode() if isinstance(s, str) else s):
            q = int(offs[i]) + t
            packed[q >> 2] |= _ENC[ch] << (2 * (q & 3))
    return lens, offs, packed


def csr_from_entries(n: int, entries):
    """entries: iterable of (u, v, code, suf) directed CSR entries -> row_ptr/col/code/suf (rows sorted)."""
    ent = sorted(entries, key=lambda e: (e[0], e[1]))
    rp = np.zeros(n + 1, dtype=np.int64)
    for u, _, _, _ in ent:
        rp[u + 1] += 1
    rp = np.cumsum(rp).astype(np.int64)
    col = np.array([e[1] for e in ent], dtype=np.int32)
    code = np.array([e[2] for e in ent], dtype=np.uint8)
    suf = np.array([e[3] for e in ent], dtype=np.int32)
    return rp, col, code, suf


def xdrop_form(g, max_trim: int = 0, seed: int = 0, consistent: bool = True):
    """(pre, post) per CSR entry: the x-drop coordinates of each overlap.

    For entry (u -> v) the overlap covers the last ov = len[v] - suf bases of
    u and the first ov bases of v, both in walk orientation (u walked in
    orientation 1 - E_u, v in E_v); these are exact overlaps (the generator's
    and the suffix form's). An aligner that stops early reports the overlap
    starting t bases later: t_u on u, t_v on v, drawn per entry from `seed`
    (equal when `consistent`) in [0, cap] with cap = min(max_trim, ov - 1,
    slack of v), the slack of a read being the fewest bases it has before any
    of its overlaps minus one, so that the reported overlaps of a read never
    cross. pre = the stored index of u's last base before the reported overlap;
    post = the stored index of v's first base in it. Returns int32 (pre, post)."""
    rp = np.asarray(g.row_ptr, dtype=np.int64)
    col = np.asarray(g.col, dtype=np.int64)
    code = np.asarray(g.code, dtype=np.int64)
    suf = np.asarray(g.suf, dtype=np.int64)
    ln = np.asarray(g.len, dtype=np.int64)
    m = col.shape[0]
    u = np.repeat(np.arange(rp.shape[0] - 1, dtype=np.int64), np.diff(rp))
    lu, lv = ln[u], ln[col]
    ov = np.minimum(lv - suf, lu - 1)
    o_u, o_v = 1 - (code & 1), (code >> 1) & 1
    slack = np.full(ln.shape[0], np.iinfo(np.int64).max, dtype=np.int64)
    np.minimum.at(slack, u, lu - ov - 1)
    rng = np.random.default_rng(seed)
    cap = np.maximum(np.minimum(np.minimum(max_trim, ov - 1), slack[col]), 0)
    t_u = np.floor(rng.random(m) * (cap + 1)).astype(np.int64)
    t_v = t_u if consistent else np.floor(rng.random(m) * (cap + 1)).astype(np.int64)
    pre_w = lu - ov - 1 + t_u              # walk-orientation index in u
    post_w = t_v                           # walk-orientation index in v
    pre = np.where(o_u == 0, pre_w, lu - 1 - pre_w)
    post = np.where(o_v == 0, post_w, lv - 1 - post_w)
    return pre.astype(np.int32), post.astype(np.int32)


def with_xdrop(g, max_trim: int = 0, seed: int = 0, consistent: bool = True):
    """A view of graph `g` in the x-drop form: the same fields plus pre and post, suf left out."""
    from types import SimpleNamespace
    pre, post = xdrop_form(g, max_trim, seed, consistent)
    fields = {k: getattr(g, k) for k in ("row_ptr", "col", "code", "len", "off", "packed")}
    return SimpleNamespace(n=len(g.len), m=len(g.col), suf=None, pre=pre, post=post, **fields)
