"""CPU oracle for contig generation -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the `cpu_baseline` / reference
legs of `bench.py` may import this package. The product path (the CUDA
library and its Python binding) never does: the two share no code. The
oracle restates Alg. 2 of Guidi et al. (ICPP'22) as plain C (cg_oracle.c).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EGRAPH, ENOMEM, EINTERNAL = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile cg_oracle.c into oracle/_liboracle.so (gcc -O2, single thread)."""
    src = os.path.join(_HERE, "cg_oracle.c")
    hdr = os.path.join(_HERE, "cg_oracle.h")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr)):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, src], check=True)
    os.replace(tmp, _SO)
    return _SO


def _bind(lib):
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    lib.orc_validate.restype = ctypes.c_int
    lib.orc_validate.argtypes = [i64, i64] + [vp] * 6 + [i64, ctypes.c_char_p, ctypes.c_size_t]
    lib.orc_run.restype = vp
    lib.orc_run.argtypes = [i64, i64] + [vp] * 7 + [i64, i32, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    lib.orc_validate2.restype = ctypes.c_int
    lib.orc_validate2.argtypes = [i64, i64] + [vp] * 8 + [i64, ctypes.c_char_p, ctypes.c_size_t]
    lib.orc_run2.restype = vp
    lib.orc_run2.argtypes = [i64, i64] + [vp] * 9 + [i64, i32, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    for f in ("orc_n_branch", "orc_n_contigs", "orc_n_cycles", "orc_total_bases", "orc_n_components",
              "orc_edge_entries_walked"):
        getattr(lib, f).restype = i64
        getattr(lib, f).argtypes = [vp]
    lib.orc_get_branch.argtypes = [vp, vp]
    lib.orc_get_chains.argtypes = [vp, vp, vp, vp]
    lib.orc_get_contigs.argtypes = [vp, vp, vp]
    lib.orc_get_labels.argtypes = [vp, ctypes.c_int, vp]
    lib.orc_free.argtypes = [vp]
    lib.orc_revcomp.argtypes = [ctypes.c_char_p, i64, ctypes.c_char_p]
    lib.orc_transitive_reduction.restype = i64
    lib.orc_transitive_reduction.argtypes = [i64, i64] + [vp] * 4 + [i32] + [vp] * 4
    lib.orc_lpt.restype = ctypes.c_int
    lib.orc_lpt.argtypes = [vp, i64, i32, vp, vp]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_SO))
    return _lib


def compile_variant(src_text: str, so_path: str) -> "OracleLib":
    """Compile a modified copy of the oracle source (used by tests that plant a
    mistake in the oracle to check that the pins catch it)."""
    d = os.path.dirname(so_path)
    c_path = so_path[:-3] + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-I", _HERE, "-o", so_path, c_path], check=True,
                   cwd=d)
    return OracleLib(_bind(ctypes.CDLL(so_path)))


def source() -> str:
    with open(os.path.join(_HERE, "cg_oracle.c")) as f:
        return f.read()


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _inputs(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    code = np.ascontiguousarray(g.code, dtype=np.uint8)
    suf = getattr(g, "suf", None)
    suf = np.ascontiguousarray(suf, dtype=np.int32) if suf is not None else None
    ln = np.ascontiguousarray(g.len, dtype=np.int32)
    off = np.ascontiguousarray(g.off, dtype=np.int64)
    packed = np.ascontiguousarray(g.packed, dtype=np.uint8)
    return rp, col, code, suf, ln, off, packed


def _prepost(g):
    """The x-drop (pre, post) arrays of a graph, or (None, None) for the suffix form."""
    pre, post = getattr(g, "pre", None), getattr(g, "post", None)
    if pre is None or post is None:
        return None, None
    return np.ascontiguousarray(pre, dtype=np.int32), np.ascontiguousarray(post, dtype=np.int32)


@dataclass
class Result:
    n_branch: int
    n_contigs: int
    n_cycles: int
    n_components: int
    total_bases: int
    edges_walked: int
    is_branch: np.ndarray
    chain_id: np.ndarray
    rank: np.ndarray
    orient: np.ndarray
    contig_off: np.ndarray
    bases: np.ndarray
    label_uf: np.ndarray
    label_bfs: np.ndarray

    def contig(self, i: int) -> bytes:
        return self.bases[self.contig_off[i]:self.contig_off[i + 1]].tobytes()


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__({EGRAPH: "invalid graph", ENOMEM: "out of memory", EINTERNAL: "internal"}.get(code, code))
        self.code = code


class OracleLib:
    """The oracle's entry points bound to one compiled copy of cg_oracle.c."""

    def __init__(self, lib):
        self.lib = lib

    def validate(self, g) -> tuple[bool, str]:
        rp, col, code, suf, ln, off, packed = _inputs(g)
        pre, post = _prepost(g)
        msg = ctypes.create_string_buffer(200)
        rc = self.lib.orc_validate2(len(ln), len(col), _p(rp), _p(col), _p(code), _p(suf), _p(pre), _p(post),
                                   _p(ln), _p(off), packed.shape[0], msg, 200)
        return rc == OK, msg.value.decode()

    def run(self, g, min_chain_reads: int = 2, validate: bool = True) -> Result:
        """Contig generation on graph `g` (any object with row_ptr, col, code, suf, len, off, packed;
        with `pre` and `post` arrays as well, the x-drop form of Sec. 4.4 is used and suf is not read)."""
        lib = self.lib
        rp, col, code, suf, ln, off, packed = _inputs(g)
        pre, post = _prepost(g)
        n, m = len(ln), len(col)
        st = ctypes.c_int(0)
        h = lib.orc_run2(n, m, _p(rp), _p(col), _p(code), _p(suf), _p(pre), _p(post), _p(ln), _p(off), _p(packed),
                         packed.shape[0], int(min_chain_reads), 1 if validate else 0, ctypes.byref(st))
        if not h:
            raise OracleError(st.value)
        try:
            nb, nc = lib.orc_n_branch(h), lib.orc_n_contigs(h)
            tot = lib.orc_total_bases(h)
            isb = np.empty(n, np.uint8)
            cid, rk, orr = np.empty(n, np.int32), np.empty(n, np.int32), np.empty(n, np.uint8)
            coff, bases = np.empty(nc + 1, np.int64), np.empty(tot, np.uint8)
            luf, lbfs = np.empty(n, np.int32), np.empty(n, np.int32)
            lib.orc_get_branch(h, _p(isb))
            lib.orc_get_chains(h, _p(cid), _p(rk), _p(orr))
            lib.orc_get_contigs(h, _p(coff), _p(bases))
            lib.orc_get_labels(h, 0, _p(luf))
            lib.orc_get_labels(h, 1, _p(lbfs))
            return Result(nb, nc, lib.orc_n_cycles(h), lib.orc_n_components(h), tot, lib.orc_edge_entries_walked(h),
                          isb, cid, rk, orr, coff, bases, luf, lbfs)
        finally:
            lib.orc_free(h)

    def revcomp(self, s: str) -> str:
        b = s.encode()
        out = ctypes.create_string_buffer(len(b) + 1)
        self.lib.orc_revcomp(b, len(b), out)
        return out.raw[: len(b)].decode()

    def transitive_reduction(self, g, fuzz: int = 0):
        """The string graph S of overlap graph g (Alg. 1, Sec. 2): g's reads with the
        non-transitive entries of g (row_ptr int64, col, code, suf)."""
        from types import SimpleNamespace
        rp, col, code, suf, ln, off, packed = _inputs(g)
        n, m = len(ln), len(col)
        orp = np.zeros(n + 1, np.int64)
        ocol, ocode, osuf = np.empty(max(m, 1), np.int32), np.empty(max(m, 1), np.uint8), np.empty(max(m, 1), np.int32)
        k = self.lib.orc_transitive_reduction(n, m, _p(rp), _p(col), _p(code), _p(suf), int(fuzz), _p(orp), _p(ocol),
                                              _p(ocode), _p(osuf))
        return SimpleNamespace(row_ptr=orp, col=ocol[:k].copy(), code=ocode[:k].copy(), suf=osuf[:k].copy(), len=ln,
                               off=off, packed=packed, n=n, m=int(k))

    def lpt(self, sizes, P: int):
        sizes = np.ascontiguousarray(sizes, dtype=np.int64)
        assign = np.empty(len(sizes), np.int32)
        loads = np.empty(P, np.int64)
        rc = self.lib.orc_lpt(_p(sizes), len(sizes), int(P), _p(assign), _p(loads))
        if rc != OK:
            raise OracleError(rc)
        return assign, loads


_default = None


def default() -> OracleLib:
    global _default
    if _default is None:
        _default = OracleLib(_load())
    return _default


def run(g, min_chain_reads: int = 2, validate: bool = True) -> Result:
    """Contig generation on graph `g` (any object with row_ptr, col, code, suf, len, off, packed)."""
    return default().run(g, min_chain_reads, validate)


def validate(g):
    return default().validate(g)


def revcomp(s: str) -> str:
    return default().revcomp(s)


def lpt(sizes, P: int):
    return default().lpt(sizes, P)


def transitive_reduction(g, fuzz: int = 0):
    return default().transitive_reduction(g, fuzz)


_CODE2 = np.full(256, 255, dtype=np.uint8)
for _i, _ch in enumerate(b"ACGT"):
    _CODE2[_ch] = _i


def pack2(ascii_bases) -> np.ndarray:
    """The 2-bit form of an ASCII base stream, by definition: base i goes to
    byte i >> 2, bits 2 (i & 3), with A=0 C=1 G=2 T=3 -- the layout of the
    packed read buffers that Sec. 4.4 concatenates from. ceil(len / 4) bytes."""
    a = np.frombuffer(bytes(ascii_bases), dtype=np.uint8) if not isinstance(ascii_bases, np.ndarray) else ascii_bases
    code = _CODE2[a]
    if code.size and code.max() == 255:
        raise ValueError("not an A/C/G/T stream")
    out = np.zeros((code.size + 3) // 4, dtype=np.uint8)
    for k in range(4):
        part = code[k::4]
        out[: part.size] |= (part << (2 * k)).astype(np.uint8)
    return out
