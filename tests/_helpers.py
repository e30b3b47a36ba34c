"""Shared test helpers: error bounds and bit comparisons (no method arithmetic)."""
import math

import numpy as np

U32 = 2.0 ** -24
U64 = 2.0 ** -53


def gamma(k, u):
    return k * u / (1 - k * u)


def flat_depth(n, V, block, unroll, grid):
    """Longest chain of dependent rounded additions in the single-vector order:
    a thread's chain, its tree, the warp and block butterflies, the grid fold
    (sequential part and butterflies), and the output conversion."""
    nv = -(-n // V)
    chain = -(-nv // (grid * block)) + 1
    W = max(block // 32, 1)
    tree = int(math.log2(unroll * V))
    fold = 5 + int(math.log2(W))
    return chain + tree + fold + (-(-grid // block)) + fold + 2


def csr_depth(length, V, unroll, tile):
    """Dependency depth of one segment in the batched order."""
    per_lane = -(-min(length, tile) // (32 * V)) + 1
    pieces = -(-length // tile) + 1
    return per_lane + int(math.log2(unroll * V)) + 5 + (-(-pieces // 32)) + 5 + 2


def twofold_bound(S, sabs, u, D):
    """|S - (v + e)| <= u|S| + gamma_D^2 sum|x| (Sum2/Dot2-type bound, depth D)."""
    g = gamma(D, u)
    return u * abs(S) + g * g * sabs


def same_bits(a, b):
    a = np.ascontiguousarray(a)
    b = np.ascontiguousarray(b)
    if a.dtype != b.dtype or a.shape != b.shape:
        return False
    na, nb = np.isnan(a), np.isnan(b)
    if not np.array_equal(na, nb):
        return False
    return np.array_equal(a[~na].view(np.uint8), b[~nb].view(np.uint8))
