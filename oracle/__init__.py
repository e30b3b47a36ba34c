"""CPU oracle for twofold summation (E. Latkin, "Twofold fast summation").

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use this package; the product library never
does.  It is plain C (``oracle/*.c``, strict IEEE, no contraction) behind this
ctypes wrapper over numpy arrays.

* primitives: FAST-TWO-SUM (Thm 1), TWO-SUM (Thm 2), TwoProduct (definition)
* the paper's sequential loops (Examples 1-3, the double-accumulator listing,
  and the dot forms)
* ``exact``: an exact superaccumulator (the plain definition of the sum)
* ``replay_flat`` / ``replay_csr``: the kernels' documented reduction order
  replayed one IEEE operation at a time; ``merge_pairs``: the rank-order
  merge of shard pairs (one vector split over several GPUs or calls)

Every function here is pinned by the ``-m "not gpu"`` tests to something
other than itself (theorems checked exhaustively on tiny formats, exact
rationals, closed forms, the paper's 100-hours table).  The values of the
paper's first Table 2 are not: its generator's seeds and mapping are not
published, so only their magnitudes are checked (parity of those values is
unpinned).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

F32, F64 = 0, 1
OPS = {"sum": 0, "dot": 1}
VARIANTS = {"plain": 0, "fast": 1, "rigorous": 2, "wide": 3, "kahan": 4, "fast_literal": 5,
            "rigorous_literal": 6}

_lib = None


class Exact(C.Structure):
    """Result of the exact superaccumulator (all fields rounded once)."""
    _fields_ = [("s", C.c_double), ("s_lo", C.c_double), ("sabs", C.c_double),
                ("rv", C.c_double), ("r", C.c_double), ("s32", C.c_float),
                ("cls", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        i64 = C.c_int64
        for dt in ("f32", "f64"):
            for nm in ("fast_two_sum", "two_sum", "two_product"):
                f = getattr(L, "orc_%s_%s" % (nm, dt))
                f.argtypes = [P, P, i64, P, P]
                f.restype = None
            for nm in ("sum", "sumk", "sumtf", "sumt"):
                f = getattr(L, "orc_%s_%s" % (nm, dt))
                f.argtypes = [i64, P, P]
                f.restype = None
            for nm in ("dot", "dotk", "dottf", "dott", "dottf2", "dott2"):
                f = getattr(L, "orc_%s_%s" % (nm, dt))
                f.argtypes = [i64, P, P, P]
                f.restype = None
        L.orc_sumd_f32.argtypes = [i64, P]
        L.orc_sumd_f32.restype = C.c_double
        L.orc_dotd_f32.argtypes = [i64, P, P]
        L.orc_dotd_f32.restype = C.c_double
        L.orc_sumq_f64.argtypes = [i64, P, P]
        L.orc_sumq_f64.restype = None
        L.orc_exact.argtypes = [C.c_int, P, P, i64, C.c_double, C.c_double, C.c_int,
                                C.POINTER(Exact)]
        L.orc_exact.restype = C.c_int
        L.orc_exact_batched.argtypes = [C.c_int, P, P, P, i64, P, P, C.c_int, P]
        L.orc_exact_batched.restype = C.c_int
        L.orc_exact_add_doubles.argtypes = [P, C.c_int]
        L.orc_exact_add_doubles.restype = C.c_double
        L.orc_replay_flat.argtypes = [C.c_int, C.c_int, C.c_int, P, P, i64, C.c_int,
                                      C.c_int, i64, C.c_int, P]
        L.orc_replay_flat.restype = C.c_int
        L.orc_replay_csr.argtypes = [C.c_int, C.c_int, C.c_int, P, P, P, i64, C.c_int,
                                     i64, C.c_int, C.c_int, P]
        L.orc_replay_csr.restype = C.c_int
        L.orc_merge_pairs.argtypes = [C.c_int, C.c_int, P, i64, C.c_int, P]
        L.orc_merge_pairs.restype = C.c_int
        L.orc_default_threads.argtypes = []
        L.orc_default_threads.restype = C.c_int
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _dt(a):
    if a.dtype == np.float32:
        return F32, "f32"
    if a.dtype == np.float64:
        return F64, "f64"
    raise TypeError("oracle: float32 or float64 arrays only, got %s" % a.dtype)


def _c(a):
    return np.ascontiguousarray(a)


# ------------------------------------------------------------- primitives
def _prim(name, a, b):
    a, b = _c(a), _c(b)
    assert a.dtype == b.dtype and a.shape == b.shape
    _, sfx = _dt(a)
    x = np.empty_like(a)
    y = np.empty_like(a)
    getattr(lib(), "orc_%s_%s" % (name, sfx))(_ptr(a), _ptr(b), a.size, _ptr(x), _ptr(y))
    return x, y


def fast_two_sum(a, b):
    """Dekker FAST-TWO-SUM (Theorem 1), elementwise: returns (x, y)."""
    return _prim("fast_two_sum", a, b)


def two_sum(a, b):
    """Knuth TWO-SUM (Theorem 2), elementwise: returns (x, y)."""
    return _prim("two_sum", a, b)


def two_product(a, b):
    """TwoProduct from its definition, elementwise: returns (p, e)."""
    return _prim("two_product", a, b)


# ------------------------------------------------------- sequential loops
def loop(method, x, y=None):
    """Run one of the paper's sequential loops.

    method: 'sum', 'sumk', 'sumtf', 'sumt', 'sumd' (binary32 data),
    'sumq' (binary64 data, binary128 accumulator), or for dots 'dot', 'dotk',
    'dottf', 'dott', 'dottf2', 'dott2', 'dotd'.  Returns (value, error) as
    numpy scalars of the data type ('sumd'/'dotd' return one binary64 value
    and 0.0; 'sumq' returns the binary128 accumulator as two doubles).
    """
    x = _c(x)
    _, sfx = _dt(x)
    L = lib()
    if method == "sumd":
        assert sfx == "f32"
        return np.float64(L.orc_sumd_f32(x.size, _ptr(x))), np.float64(0.0)
    if method == "dotd":
        y = _c(y)
        assert sfx == "f32" and y.dtype == x.dtype and y.size == x.size
        return np.float64(L.orc_dotd_f32(x.size, _ptr(x), _ptr(y))), np.float64(0.0)
    out = np.zeros(2, dtype=x.dtype)
    if method == "sumq":
        assert sfx == "f64"
        L.orc_sumq_f64(x.size, _ptr(x), _ptr(out))
    elif method.startswith("dot"):
        y = _c(y)
        assert y.dtype == x.dtype and y.size == x.size
        getattr(L, "orc_%s_%s" % (method, sfx))(x.size, _ptr(x), _ptr(y), _ptr(out))
    else:
        getattr(L, "orc_%s_%s" % (method, sfx))(x.size, _ptr(x), _ptr(out))
    return out[0], out[1]


# --------------------------------------------------------- exact results
def exact(x, y=None, v=0.0, e=0.0, nthreads=0):
    """Exact sum (y None) or dot of arrays, rounded once; residuals of (v, e)."""
    x = _c(x)
    code, _ = _dt(x)
    if y is not None:
        y = _c(y)
        assert y.dtype == x.dtype and y.size == x.size
    r = Exact()
    rc = lib().orc_exact(code, _ptr(x), _ptr(y), x.size, float(v), float(e), int(nthreads),
                         C.byref(r))
    if rc != 0:
        raise ValueError("orc_exact failed")
    return r


def exact_batched(x, offsets, y=None, v=None, e=None, nthreads=0):
    """Exact per-segment results; returns a structured numpy array."""
    x = _c(x)
    code, _ = _dt(x)
    off = _c(np.asarray(offsets, dtype=np.int64))
    nseg = off.size - 1
    if y is not None:
        y = _c(y)
    vv = None if v is None else _c(np.asarray(v, dtype=np.float64))
    ee = None if e is None else _c(np.asarray(e, dtype=np.float64))
    out = (Exact * max(nseg, 1))()
    rc = lib().orc_exact_batched(code, _ptr(x), _ptr(y), _ptr(off), nseg, _ptr(vv), _ptr(ee),
                                 int(nthreads), C.cast(out, C.c_void_p))
    if rc != 0:
        raise ValueError("orc_exact_batched: bad offsets")
    dt = np.dtype([(k, np.float64) for k in ("s", "s_lo", "sabs", "rv", "r")] +
                  [("s32", np.float32), ("cls", np.int32)])
    arr = np.frombuffer(bytearray(out), dtype=dt, count=max(nseg, 1))[:nseg]
    return arr.copy()


def exact_add(*vals):
    """RN64 of the exact sum of a few binary64 values (e.g. v + e)."""
    t = np.asarray(vals, dtype=np.float64)
    return lib().orc_exact_add_doubles(_ptr(t), t.size)


# ----------------------------------------------------------------- replay
def replay_flat(op, variant, x, y=None, *, block, unroll, grid, out_f64=False):
    """Replay the single-vector kernel order; returns the output pair."""
    x = _c(x)
    code, _ = _dt(x)
    if y is not None:
        y = _c(y)
    odt = np.float64 if (code == F64 or out_f64) else np.float32
    out = np.zeros(2, dtype=odt)
    rc = lib().orc_replay_flat(code, OPS[op], VARIANTS[variant], _ptr(x), _ptr(y), x.size,
                               int(block), int(unroll), int(grid), int(bool(out_f64)), _ptr(out))
    if rc != 0:
        raise ValueError("orc_replay_flat: bad arguments")
    return out


def replay_csr(op, variant, x, offsets, y=None, *, unroll, tile, out_f64=False, nthreads=0):
    """Replay the segmented kernel order; returns an (nseg, 2) array."""
    x = _c(x)
    code, _ = _dt(x)
    if y is not None:
        y = _c(y)
    off = _c(np.asarray(offsets, dtype=np.int64))
    nseg = off.size - 1
    odt = np.float64 if (code == F64 or out_f64) else np.float32
    out = np.zeros((max(nseg, 1), 2), dtype=odt)
    rc = lib().orc_replay_csr(code, OPS[op], VARIANTS[variant], _ptr(x), _ptr(y), _ptr(off),
                              nseg, int(unroll), int(tile), int(bool(out_f64)), int(nthreads),
                              _ptr(out))
    if rc != 0:
        raise ValueError("orc_replay_csr: bad arguments")
    return out[:nseg]


def merge_pairs(pairs, dtype, variant, out_f64=False):
    """Merge G shard pairs (a (G, 2) binary64 array: each shard's pair as a
    binary32 call with the binary64 output, or a binary64 call, writes it) in
    rank order; returns the output pair in the reductions' output format."""
    pr = _c(np.asarray(pairs, dtype=np.float64).reshape(-1, 2))
    code = F32 if np.dtype(dtype) == np.float32 else F64
    odt = np.float64 if (code == F64 or out_f64) else np.float32
    out = np.zeros(2, dtype=odt)
    rc = lib().orc_merge_pairs(code, VARIANTS[variant], _ptr(pr), pr.shape[0], int(bool(out_f64)),
                               _ptr(out))
    if rc != 0:
        raise ValueError("orc_merge_pairs: bad arguments")
    return out


def default_threads():
    return lib().orc_default_threads()


def library_path():
    return os.path.abspath(_build.LIB)
