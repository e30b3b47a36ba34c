"""Seeded synthetic inputs for twofold summation (no summation arithmetic here).

Every array is a pure function of (seed, stream, index) through SplitMix64
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014): the i-th 64-bit word of stream k under seed s is the SplitMix64
output function applied to the state (c + 1) * 0x9E3779B97F4A7C15 with
counter c = ((s * 4096 + k) << 40) + i.  It is written with wrapping int64
torch arithmetic, so the same code fills host or device memory; the float
conversions from those words are exact.  Distributions that need
transcendental functions (normal, log-normal, log-uniform lengths) may differ
in the last bits between devices, so tests hand the generated array itself to
the oracle.

The workloads follow the paper's and the benchmark's shapes: uniform data on
[-1, 1) (the paper's accuracy table), N(0,1) and signed log-normal(0, 2)
vectors, ragged CSR batches with log-uniform lengths, and ill-conditioned
vectors whose exact sum is known by construction (``ill_conditioned``).
``exact_dot_f32`` gives the known exact dot of a binary32 pair (each product
is an integer significand product times a power of two; the integers are
added exactly in 31-bit limbs), for reporting accuracy at sizes where no
construction fixes it.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import torch

_GAMMA = -7046029254386353131      # 0x9E3779B97F4A7C15 as int64
_M1 = -4658895280553007687         # 0xBF58476D1CE4E5B9
_M2 = -7723592293110705685         # 0x94D049BB133111EB
_CHUNK = 1 << 25


def _srl(z: torch.Tensor, k: int) -> torch.Tensor:
    """logical right shift of int64 words"""
    return (z >> k) & ((1 << (64 - k)) - 1)


def _mix(z: torch.Tensor) -> torch.Tensor:
    z = (z ^ _srl(z, 30)) * _M1
    z = (z ^ _srl(z, 27)) * _M2
    return z ^ _srl(z, 31)


def words(n: int, seed: int, stream: int, device="cpu", start: int = 0) -> torch.Tensor:
    """n SplitMix64 words (int64 bit patterns) of (seed, stream), from index start."""
    assert 0 <= seed < 4096 and 0 <= stream < 4096 and n + start < (1 << 40)
    base = ((seed * 4096 + stream) << 40) + start + 1
    if base >= 1 << 63:                      # the same 64-bit word, as a signed int64
        base -= 1 << 64
    out = torch.empty(n, dtype=torch.int64, device=device)
    for lo in range(0, n, _CHUNK):
        hi = min(n, lo + _CHUNK)
        c = torch.arange(lo, hi, dtype=torch.int64, device=device) + base   # counter + 1
        out[lo:hi] = _mix(c * _GAMMA)
    return out


def _torch_dtype(dtype):
    if dtype in ("f32", np.float32, torch.float32):
        return torch.float32
    if dtype in ("f64", np.float64, torch.float64):
        return torch.float64
    raise ValueError("dtype must be f32 or f64")


def uniform(n, dtype="f64", seed=0, stream=0, device="cpu", lo=-1.0) -> torch.Tensor:
    """Uniform on [lo, 1) for lo in {-1, 0}: binary64 k*2^-52 - 1 from the top
    53 bits (binary32: top 24 bits, k*2^-23 - 1); lo = 0 gives k*2^-53
    (k*2^-24).  All conversions are exact."""
    td = _torch_dtype(dtype)
    out = torch.empty(n, dtype=td, device=device)
    for a in range(0, n, _CHUNK):
        b = min(n, a + _CHUNK)
        w = words(b - a, seed, stream, device, start=a)
        if td == torch.float64:
            k = _srl(w, 11).to(torch.float64)
            out[a:b] = k * 2.0 ** -52 - 1.0 if lo == -1.0 else k * 2.0 ** -53
        else:
            k = _srl(w, 40).to(torch.float32)
            out[a:b] = k * 2.0 ** -23 - 1.0 if lo == -1.0 else k * 2.0 ** -24
    return out


def normal(n, dtype="f32", seed=0, stream=0, device="cpu") -> torch.Tensor:
    """N(0,1) by Box-Muller in binary64, rounded once to the data type."""
    td = _torch_dtype(dtype)
    out = torch.empty(n, dtype=td, device=device)
    for a in range(0, n, _CHUNK):
        b = min(n, a + _CHUNK)
        w1 = words(b - a, seed, stream, device, start=a)
        w2 = words(b - a, seed, stream + 1, device, start=a)
        u1 = (_srl(w1, 11).to(torch.float64) + 1.0) * 2.0 ** -53       # (0, 1]
        u2 = _srl(w2, 11).to(torch.float64) * 2.0 ** -53                 # [0, 1)
        z = torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)
        out[a:b] = z.to(td)
    return out


def signed_lognormal(n, dtype="f32", sigma=2.0, seed=0, stream=0, device="cpu") -> torch.Tensor:
    """|x| = exp(sigma * Z), Z ~ N(0,1), with a random sign."""
    td = _torch_dtype(dtype)
    z = normal(n, "f64", seed, stream, device)
    w = words(n, seed, stream + 2, device)
    sign = 1.0 - 2.0 * (w & 1).to(torch.float64)
    return (sign * torch.exp(sigma * z)).to(td)


def ternary_i8(n, seed=0, stream=0, device="cpu") -> torch.Tensor:
    """Values in {-1, 0, +1} (int8), from the word's bits 40..63 mod 3; built a
    chunk at a time so that n may exceed 2^31."""
    out = torch.empty(n, dtype=torch.int8, device=device)
    for lo in range(0, n, _CHUNK):
        hi = min(n, lo + _CHUNK)
        w = words(hi - lo, seed, stream, device, start=lo)
        out[lo:hi] = (_srl(w, 40) % 3 - 1).to(torch.int8)
    return out


def csr_lengths(nseg, lmin=16, lmax=1 << 18, seed=0, stream=0) -> np.ndarray:
    """Segment lengths floor(exp(U(ln lmin, ln lmax))) (log-uniform), host int64."""
    w = words(nseg, seed, stream, "cpu")
    u = _srl(w, 11).to(torch.float64).numpy() * 2.0 ** -53
    L = np.floor(np.exp(math.log(lmin) + u * (math.log(lmax) - math.log(lmin))))
    return np.clip(L, lmin, lmax).astype(np.int64)


def csr_offsets(lengths) -> np.ndarray:
    """Exclusive scan of the lengths: offsets[0] = 0, offsets[s+1] - offsets[s] = L_s."""
    off = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(np.asarray(lengths, dtype=np.int64), out=off[1:])
    return off


def permutation(n, seed=0, stream=0, device="cpu") -> torch.Tensor:
    """A seeded permutation of range(n): stable sort of SplitMix64 keys."""
    k = words(n, seed, stream, device)
    return torch.sort(k, stable=True).indices


# --------------------------------------------------------- ill-conditioned
def pow2(k: torch.Tensor) -> torch.Tensor:
    """2^k as binary64 for integer k in [-1022, 1023], built from its bits."""
    return ((k.to(torch.int64) + 1023) << 52).view(torch.float64)


class IllConditioned:
    """An ill-conditioned vector (or dot pair) whose exact sum is known by construction.

    Recipe (n elements, precision p = 24 or 53, top exponent E = ceil(log2 cond)):
      * h = (n - r) / 2 entries a_i = +-m_i * 2^(k_i - p + 1): significand m_i
        uniform in [2^(p-1), 2^p), exponent k_i uniform in 0..E, random sign;
      * h entries -a_i that cancel them exactly;
      * r positive residuals z_j = m_j * 2^(e_z - p + 1) with one exponent e_z,
        chosen so that the condition number sum|x| / |sum x| is near the
        target (r = min(1024, n/64), at least 1, with the parity of n);
      * a seeded permutation shuffles the whole vector.
    The exact sum is S = sum z_j, held as a Fraction; sum|x| is reported in
    binary64.  For a dot pair, y_i = +-2^(j_i) with j_i uniform in -2..2 and
    x_i = w_i * y_i^-1 (exact), so that x_i * y_i = w_i and the exact dot is S.
    """

    def __init__(self, n, dtype="f64", cond=1e8, seed=0, device="cpu", dot=False):
        assert n >= 3
        td = _torch_dtype(dtype)
        p = 24 if td == torch.float32 else 53
        E = max(1, int(math.ceil(math.log2(cond))))
        r = max(1, min(1024, n // 64))
        if (n - r) % 2:
            r += 1
        h = (n - r) // 2
        self.n, self.dtype, self.cond_target, self.E, self.p, self.r = n, dtype, cond, E, p, r
        wm = words(h, seed, 100, device)
        we = words(h, seed, 101, device)
        sig = _srl(wm, 64 - (p - 1)) + (1 << (p - 1))                     # [2^(p-1), 2^p)
        k = _srl(we, 11) % (E + 1)
        neg = (_srl(we, 1) & 1).bool()
        a = sig.to(torch.float64) * pow2(k - (p - 1))
        a = torch.where(neg, -a, a)
        abs_a = float(torch.sum(torch.abs(a)).item()) if h else 0.0
        target_S = max(2.0 * abs_a / cond, 1.0)
        ez = int(math.floor(math.log2(target_S / (1.5 * r))))
        ez = max(min(ez, 100), -100)
        wz = words(r, seed, 102, device)
        zsig = _srl(wz, 64 - (p - 1)) + (1 << (p - 1))
        z = zsig.to(torch.float64) * (2.0 ** (ez - (p - 1)))
        w = torch.cat([a, -a, z]).to(td)                     # every value exact in td
        self.S = Fraction(int(zsig.sum().item())) * (Fraction(2) ** (ez - (p - 1)))
        perm = permutation(n, seed, 103, device)
        w = w[perm]
        self.sum_abs = float(torch.sum(torch.abs(w.to(torch.float64))).item())
        self.cond = self.sum_abs / float(self.S)
        if not dot:
            self.x, self.y = w, None
        else:
            wj = words(n, seed, 104, device)
            j = (_srl(wj, 11) % 5) - 2
            sgn = 1.0 - 2.0 * (_srl(wj, 3) & 1).to(torch.float64)
            y = sgn * pow2(j)
            x = w.to(torch.float64) * sgn * pow2(-j)
            self.x, self.y = x.to(td), y.to(td)


def ill_conditioned(n, dtype="f64", cond=1e8, seed=0, device="cpu", dot=False):
    return IllConditioned(n, dtype, cond, seed, device, dot)


# ------------------------------------------------- exact binary32 dot value
_LIMB = 31
_EMIN32 = -149 - 149          # exponent of the least product's unit


def exact_dot_f32(x: torch.Tensor, y: torch.Tensor) -> Fraction:
    """The exact real sum of x_i * y_i for finite binary32 vectors, as a Fraction.

    Each x_i = mx * 2^ex with an integer significand mx < 2^24 (subnormals
    included), so x_i * y_i = (mx * my) * 2^(ex + ey), an integer below 2^48
    times a power of two.  Split into 24-bit halves and placed at bit offset
    ex + ey + 298 >= 0, every half lands in two 31-bit limbs; the limbs are
    added as int64 (each partial sum stays below 2^62 for up to 2^30 items)
    and combined as an exact integer.  No floating-point arithmetic touches
    the values; runs on the tensors' device, a chunk at a time."""
    assert x.dtype == torch.float32 and y.dtype == torch.float32 and x.shape == y.shape
    n = x.numel()
    assert n < (1 << 30) + 1, "limb sums are exact for at most 2^30 items"
    nlimb = (2 * 149 + 2 * 128 + 48) // _LIMB + 3
    acc = torch.zeros(nlimb, dtype=torch.int64, device=x.device)
    mask = (1 << _LIMB) - 1
    xf, yf = x.reshape(-1), y.reshape(-1)
    for a in range(0, n, _CHUNK):
        b = min(n, a + _CHUNK)
        parts = []
        for t in (xf[a:b], yf[a:b]):
            u = t.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
            e = (u >> 23) & 0xFF
            assert not bool((e == 0xFF).any()), "finite data only"
            m = (u & 0x7FFFFF) | torch.where(e > 0, 1 << 23, 0)
            parts.append((m, torch.clamp(e, min=1) - 150, u >> 31))
        (mx, ex, sx), (my, ey, sy) = parts
        M = mx * my                                        # < 2^48, exact
        off = ex + ey - _EMIN32                            # >= 0
        sign = 1 - 2 * (sx ^ sy)
        for half, shift in ((M & 0xFFFFFF, 0), (M >> 24, 24)):
            pos = off + shift
            limb = pos // _LIMB
            v = half << (pos % _LIMB)                       # < 2^54
            acc.index_add_(0, limb, sign * (v & mask))
            acc.index_add_(0, limb + 1, sign * (v >> _LIMB))
    total = 0
    for k, c in enumerate(acc.tolist()):
        total += c << (_LIMB * k)
    return Fraction(total) * (Fraction(2) ** _EMIN32)
