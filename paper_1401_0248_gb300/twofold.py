"""Thin Python binding of libtwofold.so (include/twofold.h), same names as the C ABI.

Argument marshalling only: tensors supply device pointers, the current torch
stream supplies the cudaStream_t, and every step of the reduction runs in the
library's CUDA kernels.  There is no CPU fallback: if the library is missing
or no sm_103a GPU is present, the calls raise.

    out = sum(x, "fast")                 # tensor([value, error]) on x's device
    out = dot(x, y, "rigorous")
    out = sum_batched(x, offsets, "fast")    # (nseg, 2)
    v, e = sum_host(x_pinned, "fast")        # host data, synchronous (end to end)
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtwofold.so")
DEFAULT_PLANS = os.path.join(_HERE, "plans_gb300.txt")

DTYPES = {torch.float32: 0, torch.float64: 1}
VARIANTS = {"plain": 0, "fast": 1, "rigorous": 2, "wide": 3, "kahan": 4}
OPS = {"sum": 0, "dot": 1}
OUT_F64 = 0x1
DOT_LITERAL = 0x2
# plan classes (the `batched` argument of the plan calls): single vectors of
# more than SMALL_N elements, batched calls, single vectors of at most SMALL_N
PLAN_FLAT, PLAN_BATCHED, PLAN_FLAT_SMALL = 0, 1, 2
SMALL_N = 1 << 22


def plan_class(n, batched=False):
    """The plan class a call of n elements uses."""
    if batched:
        return PLAN_BATCHED
    return PLAN_FLAT_SMALL if n <= SMALL_N else PLAN_FLAT


STATUS = {0: "TF_OK", 1: "TF_ERR_ARG", 2: "TF_ERR_DTYPE", 3: "TF_ERR_WORKSPACE",
          4: "TF_ERR_ALIGN", 5: "TF_ERR_CUDA", 6: "TF_ERR_OFFSETS", 7: "TF_ERR_TIMEOUT",
          8: "TF_ERR_UNSUPPORTED", 9: "TF_ERR_UNDRAINED"}

# every symbol declared in include/twofold.h, with its ctypes signature
_P, _I64, _I32, _SZ, _U32 = C.c_void_p, C.c_int64, C.c_int32, C.c_size_t, C.c_uint32
SIGNATURES = {
    "tf_sum": ([_P, _I64, C.c_int, C.c_int, _P, _P, _SZ, _U32, _P], C.c_int),
    "tf_dot": ([_P, _P, _I64, C.c_int, C.c_int, _P, _P, _SZ, _U32, _P], C.c_int),
    "tf_sum_batched": ([_P, _I64, _P, _I64, C.c_int, C.c_int, _P, _P, _SZ, _U32, _P], C.c_int),
    "tf_dot_batched": ([_P, _P, _I64, _P, _I64, C.c_int, C.c_int, _P, _P, _SZ, _U32, _P], C.c_int),
    "tf_sum_host_async": ([_P, _I64, C.c_int, C.c_int, _P, _P, _P, _SZ, _U32, _P, _P], C.c_int),
    "tf_dot_host_async": ([_P, _P, _I64, C.c_int, C.c_int, _P, _P, _P, _P, _SZ, _U32, _P, _P],
                          C.c_int),
    "tf_sum_host": ([_P, _I64, C.c_int, C.c_int, _P, _P, _P, _SZ, _U32, _P], C.c_int),
    "tf_sum_noalloc": ([_P, _I64, C.c_int, C.c_int, _P, _U32, _P], C.c_int),
    "tf_dot_host": ([_P, _P, _I64, C.c_int, C.c_int, _P, _P, _P, _P, _SZ, _U32, _P], C.c_int),
    "tf_workspace_size": ([C.c_int, C.c_int, C.c_int, C.c_int, _I64, _I64, C.POINTER(_SZ)], C.c_int),
    "tf_workspace_reset": ([_P, _SZ, _P], C.c_int),
    "tf_get_device_error": ([_P, _SZ, C.POINTER(_I32), _P], C.c_int),
    "tf_plan_get": ([C.c_int, C.c_int, C.c_int, C.c_int, _P], C.c_int),
    "tf_plan_set": ([C.c_int, C.c_int, C.c_int, C.c_int, _P], C.c_int),
    "tf_launch_shape": ([C.c_int, C.c_int, C.c_int, C.c_int, _I64, C.POINTER(_I32),
                         C.POINTER(_I32), C.POINTER(_I64), C.POINTER(_I64)], C.c_int),
    "tf_tune": ([C.c_int, C.c_int, C.c_int, C.c_int, _P, _P, _I64, _P, _I64, _P, _P, _SZ,
                 C.c_int, _P, _P], C.c_int),
    "tf_plan_save": ([C.c_char_p], C.c_int),
    "tf_plan_load": ([C.c_char_p], C.c_int),
    "tf_prim": ([C.c_int, C.c_int, _P, _P, _P, _P, _I64, _P], C.c_int),
    "tf_merge_pairs": ([_P, _I64, C.c_int, C.c_int, _P, _U32, _P], C.c_int),
    "tf_count_large_errors": ([_P, _I64, C.c_int, C.c_double, _P, _P], C.c_int),
    "tf_probe_read": ([_P, _P, _I64, _P, _I32, _I32, _I32, _P], C.c_int),
    "tf_probe_alu": ([C.c_int, _I64, _P, _I32, _I32, _P], C.c_int),
    "tf_probe_wait": ([_I32, _I64, _P, _P], C.c_int),
    "tf_status_string": ([C.c_int], C.c_char_p),
    "tf_device_sm_count": ([], _I32),
}


class Plan(C.Structure):
    _fields_ = [("block", _I32), ("unroll", _I32), ("blocks_per_sm", _I32), ("tile", _I32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TwofoldError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__("%s failed: %s (%d)" % (fn, STATUS.get(code, "?"), code))
        self.code = code


_lib = None
_lock = threading.Lock()


def lib():
    """Load libtwofold.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                if not os.path.exists(LIB_PATH):
                    raise RuntimeError("libtwofold.so is not built (run __graft_entry__.build() or "
                                       "python -m paper_1401_0248_gb300.build)")
                L = C.CDLL(LIB_PATH)
                for name, (args, res) in SIGNATURES.items():
                    f = getattr(L, name)
                    f.argtypes = args
                    f.restype = res
                # the launch plans tuned on GB300 (TF_PLANS=<file> picks another
                # file, TF_PLANS=none keeps the library's built-in defaults)
                plans = os.environ.get("TF_PLANS", DEFAULT_PLANS)
                if plans != "none" and os.path.exists(plans):
                    rc = L.tf_plan_load(os.fsencode(plans))
                    if rc != 0:
                        raise TwofoldError("tf_plan_load(%s)" % plans, rc)
                _lib = L
    return _lib


def _check(fn, rc):
    if rc != 0:
        raise TwofoldError(fn, rc)


def _stream(t=None):
    return C.c_void_p(torch.cuda.current_stream(t.device if t is not None else None).cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _dt(x):
    if x.dtype not in DTYPES:
        raise TypeError("twofold: float32 or float64 tensors only, got %s" % x.dtype)
    return DTYPES[x.dtype]


def _flat(x):
    if x.dim() != 1 or not x.is_contiguous():
        raise ValueError("twofold: 1-D contiguous tensor expected")
    if not x.is_cuda:
        raise ValueError("twofold: CUDA tensor expected (use sum_host for host data)")
    return x


# -------------------------------------------------------------- workspace
_ws_cache = {}


def workspace_size(op="sum", batched=False, dtype=torch.float32, variant="fast", n=0, nseg=0):
    b = C.c_size_t(0)
    _check("tf_workspace_size", lib().tf_workspace_size(OPS[op], int(batched), DTYPES[dtype],
                                                        VARIANTS[variant], int(n), int(nseg),
                                                        C.byref(b)))
    return b.value


def workspace(nbytes, device=None):
    """A zero-filled uint8 workspace of at least nbytes on `device`, cached per
    (device, current stream) and grown on demand (allocated by torch, never by
    the library).  Calls in flight on different streams thus never share one:
    a workspace holds the per-call tickets and block pairs."""
    dev = torch.device(device if device is not None else "cuda")
    if dev.index is None:
        dev = torch.device("cuda", torch.cuda.current_device())
    key = (dev, torch.cuda.current_stream(dev).cuda_stream)
    ws = _ws_cache.get(key)
    if ws is None or ws.numel() < nbytes:
        ws = torch.zeros(max(nbytes, 1 << 16), dtype=torch.uint8, device=dev)
        _ws_cache[key] = ws
    return ws


def workspace_reset(ws):
    """Zero-fill a workspace on the current stream (tf_workspace_reset): the
    state a workspace needs before its first use."""
    _check("tf_workspace_reset", lib().tf_workspace_reset(_ptr(ws), ws.numel(), _stream(ws)))
    return ws


# ------------------------------------------------------------ reductions
def _out(x, n_pairs, out_f64, out):
    odt = torch.float64 if (x.dtype == torch.float64 or out_f64) else x.dtype
    shape = (2,) if n_pairs is None else (n_pairs, 2)
    if out is None:
        return torch.empty(shape, dtype=odt, device=x.device)
    if out.dtype != odt or out.numel() < 2 * (1 if n_pairs is None else n_pairs) or not out.is_contiguous():
        raise ValueError("twofold: out must be a contiguous %s tensor of %s" % (odt, shape))
    return out


def sum(x, variant="fast", *, out_f64=False, out=None, ws=None):  # noqa: A001 - the paper's name
    """Twofold sum of a 1-D CUDA tensor: tensor([value, error])."""
    x = _flat(x)
    out = _out(x, None, out_f64, out)
    if ws is None:
        ws = workspace(workspace_size("sum", False, x.dtype, variant, x.numel()), x.device)
    rc = lib().tf_sum(_ptr(x), x.numel(), _dt(x), VARIANTS[variant], _ptr(out), _ptr(ws),
                      ws.numel(), OUT_F64 if out_f64 else 0, _stream(x))
    _check("tf_sum", rc)
    return out


def dot(x, y, variant="fast", *, out_f64=False, out=None, ws=None, literal=False):
    """Twofold dot product of two 1-D CUDA tensors: tensor([value, error]).
    literal=True: the paper's dot form (products rounded, their errors not
    tracked) for the fast and rigorous variants."""
    x, y = _flat(x), _flat(y)
    if x.dtype != y.dtype or x.numel() != y.numel() or x.device != y.device:
        raise ValueError("twofold.dot: x and y must match in dtype, length and device")
    out = _out(x, None, out_f64, out)
    if ws is None:
        ws = workspace(workspace_size("dot", False, x.dtype, variant, x.numel()), x.device)
    flags = (OUT_F64 if out_f64 else 0) | (DOT_LITERAL if literal else 0)
    rc = lib().tf_dot(_ptr(x), _ptr(y), x.numel(), _dt(x), VARIANTS[variant], _ptr(out), _ptr(ws),
                      ws.numel(), flags, _stream(x))
    _check("tf_dot", rc)
    return out


def _offsets(offsets, x):
    if offsets.dtype != torch.int64 or offsets.dim() != 1 or not offsets.is_contiguous():
        raise ValueError("twofold: offsets must be a contiguous 1-D int64 tensor")
    if offsets.device != x.device:
        raise ValueError("twofold: offsets must live on x's device")
    return offsets


def sum_batched(x, offsets, variant="fast", *, out_f64=False, out=None, ws=None):
    """One twofold sum per CSR segment [offsets[s], offsets[s+1]): (nseg, 2)."""
    x = _flat(x)
    offsets = _offsets(offsets, x)
    nseg = offsets.numel() - 1
    out = _out(x, nseg, out_f64, out)
    if ws is None:
        ws = workspace(workspace_size("sum", True, x.dtype, variant, x.numel(), nseg), x.device)
    rc = lib().tf_sum_batched(_ptr(x), x.numel(), _ptr(offsets), nseg, _dt(x), VARIANTS[variant],
                              _ptr(out), _ptr(ws), ws.numel(), OUT_F64 if out_f64 else 0,
                              _stream(x))
    _check("tf_sum_batched", rc)
    return out


def dot_batched(x, y, offsets, variant="fast", *, out_f64=False, out=None, ws=None, literal=False):
    """One twofold dot product per CSR segment: (nseg, 2)."""
    x, y = _flat(x), _flat(y)
    if x.dtype != y.dtype or x.numel() != y.numel() or x.device != y.device:
        raise ValueError("twofold.dot_batched: x and y must match in dtype, length and device")
    offsets = _offsets(offsets, x)
    nseg = offsets.numel() - 1
    out = _out(x, nseg, out_f64, out)
    if ws is None:
        ws = workspace(workspace_size("dot", True, x.dtype, variant, x.numel(), nseg), x.device)
    flags = (OUT_F64 if out_f64 else 0) | (DOT_LITERAL if literal else 0)
    rc = lib().tf_dot_batched(_ptr(x), _ptr(y), x.numel(), _ptr(offsets), nseg, _dt(x),
                              VARIANTS[variant], _ptr(out), _ptr(ws), ws.numel(), flags,
                              _stream(x))
    _check("tf_dot_batched", rc)
    return out


def shard_bounds(n, G, dtype=torch.float32):
    """Contiguous shards of one vector of n elements for G GPUs (or calls):
    shard g is [g*m, min((g+1)*m, n)) with m = ceil(n / (G*V)) * V elements,
    V = 16 / element size, so that every shard starts on a 16-byte boundary
    of a 16-byte-aligned vector (the last shards may be short or empty)."""
    if G < 1 or n < 0:
        raise ValueError("G >= 1 and n >= 0")
    V = 4 if dtype == torch.float32 else 2
    m = -(-n // (G * V)) * V
    return [(min(g * m, n), min((g + 1) * m, n)) for g in range(G)]


def merge_pairs(pairs, dtype, variant="fast", *, out_f64=False, out=None):
    """Merge the (G, 2) binary64 device tensor of shard pairs (rank order) of
    one vector reduced in G contiguous shards into one pair (tf_merge_pairs);
    dtype is the data's dtype (binary32 shards give their pairs with
    out_f64=True)."""
    if pairs.dtype != torch.float64 or pairs.dim() != 2 or pairs.shape[1] != 2:
        raise ValueError("pairs must be a (G, 2) float64 tensor")
    if not pairs.is_cuda:
        raise ValueError("pairs must be a CUDA tensor")
    pairs = pairs.contiguous()
    odt = torch.float64 if (dtype == torch.float64 or out_f64) else torch.float32
    if out is None:
        out = torch.empty(2, dtype=odt, device=pairs.device)
    _check("tf_merge_pairs", lib().tf_merge_pairs(_ptr(pairs), pairs.shape[0], DTYPES[dtype],
                                                  VARIANTS[variant], _ptr(out),
                                                  OUT_F64 if out_f64 else 0, _stream(pairs)))
    return out


def count_large_errors(pairs, tau, count=None):
    """Number of pairs (value, error) with |error| > tau * |value| (or not
    finite), as a device int32 tensor; pairs is an (n, 2) or (2,) tensor."""
    if not pairs.is_cuda or not pairs.is_contiguous() or pairs.dtype not in DTYPES:
        raise ValueError("count_large_errors: a contiguous CUDA float32/float64 tensor of pairs")
    if count is None:
        count = torch.empty(1, dtype=torch.int32, device=pairs.device)
    _check("tf_count_large_errors", lib().tf_count_large_errors(_ptr(pairs), pairs.numel() // 2,
                                                                _dt(pairs), float(tau), _ptr(count),
                                                                _stream(pairs)))
    return count


def device_error(ws=None, device=None):
    """Read and clear the device error word of a workspace (0 = none)."""
    if ws is None:
        ws = workspace(0, device)
    code = C.c_int32(0)
    _check("tf_get_device_error", lib().tf_get_device_error(_ptr(ws), ws.numel(), C.byref(code),
                                                            _stream(ws)))
    return code.value


# ------------------------------------------------------- host buffers (e2e)
def sum_host(x, variant="fast", *, out_f64=False, x_dev=None, ws=None, device=None):
    """Twofold sum of host data through the C ABI's host-buffer call: copies x
    (pinned for full speed) to the device, reduces, returns (value, error)."""
    if x.is_cuda or x.dim() != 1 or not x.is_contiguous():
        raise ValueError("sum_host: a 1-D contiguous CPU tensor expected")
    dev = torch.device(device if device is not None else "cuda")
    if x_dev is None:
        x_dev = torch.empty_like(x, device=dev)
    if ws is None:
        ws = workspace(workspace_size("sum", False, x.dtype, variant, x.numel()), dev)
    res = (C.c_double * 2)() if (x.dtype == torch.float64 or out_f64) else (C.c_float * 2)()
    rc = lib().tf_sum_host(_ptr(x), x.numel(), _dt(x), VARIANTS[variant], C.cast(res, C.c_void_p),
                           _ptr(x_dev), _ptr(ws), ws.numel(), OUT_F64 if out_f64 else 0,
                           _stream(x_dev))
    _check("tf_sum_host", rc)
    return res[0], res[1]


def dot_host(x, y, variant="fast", *, out_f64=False, x_dev=None, y_dev=None, ws=None, device=None):
    """Twofold dot product of host data (see sum_host)."""
    if (x.is_cuda or y.is_cuda or x.dtype != y.dtype or x.numel() != y.numel() or x.dim() != 1
            or y.dim() != 1 or not x.is_contiguous() or not y.is_contiguous()):
        raise ValueError("dot_host: two matching 1-D contiguous CPU tensors expected")
    dev = torch.device(device if device is not None else "cuda")
    if x_dev is None:
        x_dev = torch.empty_like(x, device=dev)
    if y_dev is None:
        y_dev = torch.empty_like(y, device=dev)
    if ws is None:
        ws = workspace(workspace_size("dot", False, x.dtype, variant, x.numel()), dev)
    res = (C.c_double * 2)() if (x.dtype == torch.float64 or out_f64) else (C.c_float * 2)()
    rc = lib().tf_dot_host(_ptr(x), _ptr(y), x.numel(), _dt(x), VARIANTS[variant],
                           C.cast(res, C.c_void_p), _ptr(x_dev), _ptr(y_dev), _ptr(ws), ws.numel(),
                           OUT_F64 if out_f64 else 0, _stream(x_dev))
    _check("tf_dot_host", rc)
    return res[0], res[1]


def _host_out(x, out_f64, out):
    odt = torch.float64 if (x.dtype == torch.float64 or out_f64) else torch.float32
    if out is None:
        out = torch.empty(2, dtype=odt, pin_memory=True)
    if out.is_cuda or out.dtype != odt or out.numel() != 2 or not out.is_contiguous():
        raise ValueError("out: a contiguous CPU tensor of two %s expected" % odt)
    return out


def sum_host_async(x, variant="fast", *, x_dev, ws, out=None, out_f64=False, copy_stream=None):
    """Enqueue a twofold sum of host data without waiting (tf_sum_host_async):
    x (pinned, 1-D) is copied to x_dev on copy_stream (default: the current
    stream of x_dev's device), the reduction runs on the current stream
    behind the copy, and the pair lands in `out` (a pinned CPU tensor,
    returned) once that stream reaches it."""
    if x.is_cuda or x.dim() != 1 or not x.is_contiguous():
        raise ValueError("sum_host_async: a 1-D contiguous CPU tensor expected")
    if x_dev.dtype != x.dtype or x_dev.numel() != x.numel() or not x_dev.is_cuda:
        raise ValueError("x_dev: a CUDA tensor of x's dtype and size expected")
    out = _host_out(x, out_f64, out)
    cs = None if copy_stream is None else C.c_void_p(copy_stream.cuda_stream)
    _check("tf_sum_host_async",
           lib().tf_sum_host_async(_ptr(x), x.numel(), _dt(x), VARIANTS[variant], _ptr(out),
                                   _ptr(x_dev), _ptr(ws), ws.numel(), OUT_F64 if out_f64 else 0,
                                   _stream(x_dev), cs))
    return out


def dot_host_async(x, y, variant="fast", *, x_dev, y_dev, ws, out=None, out_f64=False,
                   copy_stream=None):
    """The dot-product form of sum_host_async."""
    if (x.is_cuda or y.is_cuda or x.dtype != y.dtype or x.numel() != y.numel() or x.dim() != 1
            or y.dim() != 1 or not x.is_contiguous() or not y.is_contiguous()):
        raise ValueError("dot_host_async: two matching 1-D contiguous CPU tensors expected")
    for d in (x_dev, y_dev):
        if d.dtype != x.dtype or d.numel() != x.numel() or not d.is_cuda:
            raise ValueError("x_dev, y_dev: CUDA tensors of x's dtype and size expected")
    out = _host_out(x, out_f64, out)
    cs = None if copy_stream is None else C.c_void_p(copy_stream.cuda_stream)
    _check("tf_dot_host_async",
           lib().tf_dot_host_async(_ptr(x), _ptr(y), x.numel(), _dt(x), VARIANTS[variant],
                                   _ptr(out), _ptr(x_dev), _ptr(y_dev), _ptr(ws), ws.numel(),
                                   OUT_F64 if out_f64 else 0, _stream(x_dev), cs))
    return out


# ------------------------------------------------------------------- plans
def plan_get(op="sum", batched=False, dtype=torch.float32, variant="fast"):
    """The plan of a key; `batched` is the plan class (False/0 single vectors of
    more than SMALL_N elements, True/1 batched, 2 single vectors of at most
    SMALL_N elements; plan_class(n) gives the one a call uses)."""
    p = Plan()
    _check("tf_plan_get", lib().tf_plan_get(OPS[op], int(batched), DTYPES[dtype], VARIANTS[variant],
                                            C.byref(p)))
    return p.as_dict()


def plan_set(op, batched, dtype, variant, block, unroll, blocks_per_sm, tile=0):
    p = Plan(block, unroll, blocks_per_sm, tile)
    _check("tf_plan_set", lib().tf_plan_set(OPS[op], int(batched), DTYPES[dtype], VARIANTS[variant],
                                            C.byref(p)))


def launch_shape(op="sum", batched=False, dtype=torch.float32, variant="fast", n=0):
    """(block, unroll, grid, tile) of a call of n elements on the current device."""
    b, u, g, t = C.c_int32(), C.c_int32(), C.c_int64(), C.c_int64()
    _check("tf_launch_shape", lib().tf_launch_shape(OPS[op], int(batched), DTYPES[dtype],
                                                    VARIANTS[variant], int(n), C.byref(b),
                                                    C.byref(u), C.byref(g), C.byref(t)))
    return b.value, u.value, g.value, t.value


def tune(op, variant, x, y=None, offsets=None, reps=5, ws=None):
    """Time every candidate plan on this problem and keep the fastest."""
    x = _flat(x)
    batched = offsets is not None
    nseg = offsets.numel() - 1 if batched else 0
    out = _out(x, nseg if batched else None, False, None)
    if ws is None:
        ws = workspace(workspace_size(op, batched, x.dtype, variant, x.numel(), nseg), x.device)
    p = Plan()
    rc = lib().tf_tune(OPS[op], int(batched), _dt(x), VARIANTS[variant], _ptr(x), _ptr(y),
                       x.numel(), _ptr(offsets), nseg, _ptr(out), _ptr(ws), ws.numel(), int(reps),
                       _stream(x), C.byref(p))
    _check("tf_tune", rc)
    return p.as_dict()


def plan_save(path):
    _check("tf_plan_save", lib().tf_plan_save(os.fsencode(path)))


def plan_load(path):
    _check("tf_plan_load", lib().tf_plan_load(os.fsencode(path)))


# --------------------------------------------------------- building blocks
PRIMS = {"fast_two_sum": 0, "two_sum": 1, "two_product": 2, "two_sum_int": 3,
         "two_product_int": 4, "fast_two_sum_int": 5}


def prim(name, a, b):
    """Elementwise FAST-TWO-SUM / TWO-SUM / TwoProduct on the GPU: (x, y)."""
    a, b = _flat(a), _flat(b)
    x = torch.empty_like(a)
    y = torch.empty_like(a)
    _check("tf_prim", lib().tf_prim(PRIMS[name], _dt(a), _ptr(a), _ptr(b), _ptr(x), _ptr(y),
                                    a.numel(), _stream(a)))
    return x, y


def probe_read(x, y=None, blocks=None, threads=512, unroll=4, sink=None):
    """Launch the read-bandwidth probe over x (and y) once, `unroll` 16-byte
    loads of each array in flight per thread."""
    blocks = blocks or 4 * sm_count()
    if sink is None:
        sink = torch.empty(blocks, dtype=torch.int32, device=x.device)
    nbytes = x.numel() * x.element_size()
    _check("tf_probe_read", lib().tf_probe_read(_ptr(x), _ptr(y), nbytes, _ptr(sink), blocks, threads,
                                                unroll, _stream(x)))
    return sink


ALU_KINDS = {"fadd": 0, "dadd": 1, "ffma": 2, "dfma": 3, "iadd": 4, "fast_f32": 5,
             "rigorous_f32": 6, "fast_f64": 7, "rigorous_f64": 8, "dmul": 9, "dadd_as_fma": 10}
# operations per thread per iteration (8 chains; the step mixes count the
# paper's 4 and 7 operations per item)
ALU_OPS_PER_ITER = {0: 8, 1: 8, 2: 8, 3: 8, 4: 8, 5: 32, 6: 56, 7: 32, 8: 56, 9: 8, 10: 8}


def probe_alu(kind, iters, blocks, threads, sink=None, device=None):
    k = ALU_KINDS[kind]
    if sink is None:
        sink = torch.empty(blocks * threads, dtype=torch.int32, device=device or "cuda")
    _check("tf_probe_alu", lib().tf_probe_alu(k, int(iters), _ptr(sink), blocks, threads,
                                              _stream(sink)))
    return sink


def probe_wait(arrive, polls, device=None):
    """Run the batched kernel's bounded barrier wait on a barrier that is
    never completed (arrive=False) or completed first (arrive=True); returns
    True if the wait gave up."""
    flag = torch.full((1,), -1, dtype=torch.int32, device=device or "cuda")
    _check("tf_probe_wait", lib().tf_probe_wait(1 if arrive else 0, int(polls), _ptr(flag),
                                                _stream(flag)))
    return bool(int(flag.item()) == 1)


def sm_count():
    return int(lib().tf_device_sm_count())


def status_string(code):
    return lib().tf_status_string(int(code)).decode()
