"""The seeded input generators (CPU): SplitMix64 against its published
outputs, exact conversions, and the CSR helpers' shapes."""
import numpy as np
import torch

from paper_1401_0248_gb300 import inputs as I

M64 = (1 << 64) - 1
# the first outputs of SplitMix64 started from state 0 (the reference
# implementation of Steele, Lea and Flood's generator, as distributed with
# the xoshiro/xoroshiro generators for seeding)
SPLITMIX64_SEED0 = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F,
                    0xF88BB8A8724C81EC]


def test_words_are_splitmix64():
    w = [int(v) & M64 for v in I.words(4, 0, 0)]
    assert w == SPLITMIX64_SEED0
    # a later start continues the same sequence; streams and seeds differ
    assert [int(v) & M64 for v in I.words(2, 0, 0, start=2)] == SPLITMIX64_SEED0[2:]
    assert int(I.words(1, 0, 1)[0]) & M64 not in SPLITMIX64_SEED0
    assert int(I.words(1, 1, 0)[0]) & M64 not in SPLITMIX64_SEED0


def test_uniform_is_an_exact_function_of_the_words():
    n = 4096
    w = np.array([int(v) & M64 for v in I.words(n, 3, 2)], dtype=object)
    x64 = I.uniform(n, "f64", seed=3, stream=2).numpy()
    x32 = I.uniform(n, "f32", seed=3, stream=2).numpy()
    for i in range(0, n, 97):
        assert x64[i] == (w[i] >> 11) * 2.0 ** -52 - 1.0
        assert x32[i] == np.float32((w[i] >> 40) * 2.0 ** -23 - 1.0)
    assert x64.min() >= -1.0 and x64.max() < 1.0
    assert x32.min() >= -1.0 and x32.max() < 1.0
    # words generated in pieces (start offsets) equal one call
    a = I.words(1000, 5, 1)
    b = torch.cat([I.words(400, 5, 1), I.words(600, 5, 1, start=400)])
    assert torch.equal(a, b)


def test_csr_lengths_and_offsets():
    L = I.csr_lengths(16384, 16, 1 << 18, seed=0)
    assert len(L) == 16384 and int(np.min(L)) >= 16 and int(np.max(L)) <= 1 << 18
    off = I.csr_offsets(L)
    assert off.dtype == np.int64 and off[0] == 0 and len(off) == len(L) + 1
    assert np.array_equal(np.diff(off), np.asarray(L, dtype=np.int64))
    # log-uniform lengths: the mean of [16, 2^18] is (2^18 - 16) / ln(2^14)
    mean = (2 ** 18 - 16) / np.log(2 ** 14)
    assert 0.9 * mean < float(np.mean(L)) < 1.1 * mean


def test_exact_dot_f32_against_fractions_and_oracle():
    """The known exact dot of a binary32 pair (limb sums of the integer
    significand products) equals brute-force rational arithmetic on small
    vectors with subnormals, zeros and huge values, and the oracle's exact
    superaccumulator on larger N(0,1) and signed log-normal pairs."""
    from fractions import Fraction
    import oracle as O
    x = torch.tensor([1e-45, -3e-39, 3e38, 1.0, 0.0, -0.0, 2.5e-20, 7.0], dtype=torch.float32)
    y = torch.tensor([1e-45, 2e-39, -3e38, -0.0, 5.0, 3.0, 3.3e-21, -1.0 / 3], dtype=torch.float32)
    want = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x.tolist(), y.tolist()))
    assert I.exact_dot_f32(x, y) == want
    for gen in (I.normal, I.signed_lognormal):
        a = gen(200003, "f32", seed=3)
        b = gen(200003, "f32", seed=3, stream=6)
        S = I.exact_dot_f32(a, b)
        ex = O.exact(a.numpy(), b.numpy(), v=float(S))
        assert ex.s == float(S) and ex.s32 == np.float32(float(S))
        # the residual of RN64(S) is below half an ulp: S is exact, not rounded
        assert abs(ex.rv) <= abs(float(S)) * 2.0 ** -53
