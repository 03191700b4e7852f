"""The arithmetic behind the tolerances of the tensor-core paths, checked on
the CPU by emulating bf16 rounding: an fp32 value x splits into a bf16 high
part h = bf16(x) and a bf16 remainder l = bf16(x - h) with
|x - h - l| <= 2^-16 |x|, and the three-pass product hi*hi + hi*lo + lo*hi
of two such splits is within about 2^-15 of the exact product (the dropped
lo*lo term and the two remainders), so a K-term dot product accumulated in
fp32 is within (2^-15 + K 2^-24) sum |a_k b_k| of the exact one."""

import numpy as np


def bf16_round(x):
    """Round float32 values to bf16 (round to nearest, ties to even) and
    return them as float32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = (u + 0x7FFF + lsb) >> 16 << 16
    return r.astype(np.uint32).view(np.float32)


def split(x):
    x = np.asarray(x, dtype=np.float32)
    h = bf16_round(x)
    lo = bf16_round((x - h).astype(np.float32))
    return h, lo


def test_bf16_rounding_is_to_nearest():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(100000).astype(np.float32)
    h = bf16_round(x)
    # 8 significant bits: half an ulp is at most 2^-8 of |x|; h has no low bits
    assert np.all(np.abs(h.astype(np.float64) - x) <= 2.0 ** -8 * np.abs(x))
    assert np.all((h.view(np.uint32) & 0xFFFF) == 0)


def test_split_reconstructs_to_16_bits():
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(100000) * np.exp(rng.uniform(-20, 20, 100000))).astype(np.float32)
    h, lo = split(x)
    err = np.abs(x.astype(np.float64) - h.astype(np.float64) - lo.astype(np.float64))
    assert np.all(err <= 2.0 ** -16 * np.abs(x.astype(np.float64)))


def test_three_pass_dot_product_bound():
    rng = np.random.default_rng(2)
    for K in (16, 128, 1024):
        a = rng.standard_normal((200, K)).astype(np.float32)
        b = rng.standard_normal((200, K)).astype(np.float32)
        ha, la = split(a)
        hb, lb = split(b)
        # products of bf16 values are exact in fp32; accumulate in fp32
        terms = (ha * hb + ha * lb + la * hb).astype(np.float32)
        acc = np.zeros(200, dtype=np.float32)
        for k in range(K):
            acc = (acc + terms[:, k]).astype(np.float32)
        exact = np.sum(a.astype(np.float64) * b.astype(np.float64), axis=1)
        scale = np.sum(np.abs(a.astype(np.float64) * b.astype(np.float64)), axis=1)
        assert np.all(np.abs(acc - exact) <= (2.0 ** -15 + K * 2.0 ** -24) * scale), K
