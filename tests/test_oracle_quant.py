"""Pins for the low-precision oracle (BF16, FP8-E4M3, split BF16, per-tile FP8).

The conversions are checked against PyTorch's CPU casts (library routines that
implement the same IEEE-style round-to-nearest-even), against the decoded code
tables, and against closed-form properties of the formats.
"""
import numpy as np
import torch

from oracle import quant
from paper_1801_04348_gb300 import inputs


def _torch_bf16_bits(x):
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16)
    return t.view(torch.int16).numpy().view(np.uint16)


def _random_wide(n, seed):
    rng = np.random.default_rng(seed)
    mant = rng.uniform(1, 2, n)
    exps = rng.integers(-140, 128, n)
    sign = rng.choice([-1.0, 1.0], n)
    with np.errstate(over="ignore"):
        return (sign * np.ldexp(mant, exps)).astype(np.float32)


def test_bf16_matches_torch_random():
    x = np.concatenate([_random_wide(200000, 1), inputs.normal((50000,), 2)])
    assert np.array_equal(quant.bf16_bits(x), _torch_bf16_bits(x))


def test_bf16_ties_to_even():
    # exact midpoints between consecutive bf16 values: low 16 bits = 0x8000
    rng = np.random.default_rng(3)
    hi = rng.integers(0x0080, 0x7F00, 5000).astype(np.uint32)
    mid = ((hi << 16) | 0x8000).view(np.float32)
    got = quant.bf16_bits(mid).astype(np.uint32)
    want = np.where(hi % 2 == 0, hi, hi + 1)
    assert np.array_equal(got, want)
    assert np.array_equal(got, _torch_bf16_bits(mid).astype(np.uint32))


def test_bf16_specials():
    x = np.array([0.0, -0.0, np.inf, -np.inf, 3.4028235e38, 1e-45, -1e-45, 1.1754944e-38],
                 dtype=np.float32)
    got = quant.bf16_bits(x)
    assert np.array_equal(got, _torch_bf16_bits(x))
    assert got[4] == 0x7F80                       # rounds past the largest bf16 to inf
    assert np.isnan(quant.bf16_rn(np.array([np.nan], np.float32)))[0]


def test_e4m3_code_table_roundtrip():
    codes = np.arange(256, dtype=np.uint8)
    vals = quant.e4m3_value(codes)
    finite = ~np.isnan(vals)
    assert np.nanmax(vals) == 448.0 and np.nanmin(vals) == -448.0
    assert quant.e4m3_value(np.array([0x01], np.uint8))[0] == 2.0 ** -9
    assert quant.e4m3_value(np.array([0x08], np.uint8))[0] == 2.0 ** -6
    back = quant.e4m3_rn_sat(vals[finite].astype(np.float32))
    assert np.array_equal(back, codes[finite])


def test_e4m3_matches_torch_in_range():
    x = np.concatenate([inputs.normal((100000,), 5) * 50, inputs.uniform((50000,), 6, -448, 448),
                        inputs.normal((20000,), 7) * 1e-3]).astype(np.float32)
    t = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(quant.e4m3_rn_sat(x), t)


def test_e4m3_ties_and_saturation():
    pos = np.arange(0, 0x7E, dtype=np.uint8)                 # 0 .. 416
    lo, hi = quant.e4m3_value(pos), quant.e4m3_value(pos + 1)
    mid = ((lo + hi) / 2).astype(np.float32)                 # exact midpoints in binary32
    got = quant.e4m3_rn_sat(mid)
    want = np.where(pos % 2 == 0, pos, pos + 1).astype(np.uint8)
    assert np.array_equal(got, want)
    sat = quant.e4m3_rn_sat(np.array([448.0, 463.9, 464.0, 1e6, -1e30, -500.0], np.float32))
    assert list(sat) == [0x7E, 0x7E, 0x7E, 0x7E, 0xFE, 0xFE]


def test_split_bf16_properties():
    x = np.concatenate([inputs.normal((100000,), 8), _random_wide(100000, 9) * 0 + inputs.uniform((100000,), 10)])
    hi, lo = quant.split_bf16(x)
    xd = x.astype(np.float64)
    # x - hi is exact in binary32, and the two-term representation is 2^-16 accurate
    assert np.array_equal((x - hi).astype(np.float64), xd - hi.astype(np.float64))
    err = np.abs(xd - hi.astype(np.float64) - lo.astype(np.float64))
    assert np.all(err <= 2.0 ** -16 * np.abs(xd) + 1e-45)
    assert np.array_equal(quant.bf16_rn(hi), hi) and np.array_equal(quant.bf16_rn(lo), lo)


def test_fp8_tile_scaling_properties():
    X = inputs.normal((300, 200), 11) * 7.0        # ragged 128 tiles: 3 x 2
    codes, S = quant.fp8_tile_quant(X)
    assert S.shape == (3, 2)
    for i in range(3):
        for j in range(2):
            blk = codes[i * 128:(i + 1) * 128, j * 128:(j + 1) * 128]
            assert np.max(blk & 0x7F) == 0x7E               # amax maps to 448
    D = quant.fp8_dequant(codes, S)
    Sfull = np.repeat(np.repeat(S, 128, 0), 128, 1)[:300, :200].astype(np.float64)
    # per-element error at most half a spacing: 2^-4 relative, or 2^-10 * scale below 2^-6
    err = np.abs(D - X.astype(np.float64))
    assert np.all(err <= np.maximum(2.0 ** -4 * np.abs(X), 2.0 ** -10 * Sfull) * 1.0001)


def test_fp8_exact_on_small_integers_pow2_scale():
    # integers in [-7, 7] with a 7 in every tile: scale = 7/448 = 2^-6 exactly and
    # every x * 2^6 has at most 3 significant bits, so dequantisation is exact
    X = inputs.integers((256, 256), 12, -7, 7)
    X[::128, ::128] = 7.0
    codes, S = quant.fp8_tile_quant(X)
    assert np.all(S == np.float32(2.0 ** -6))
    assert np.array_equal(quant.fp8_dequant(codes, S), X.astype(np.float64))


def test_fp8_zero_tile_scale_one():
    X = np.zeros((130, 10), np.float32)
    codes, S = quant.fp8_tile_quant(X)
    assert np.all(S == 1.0) and np.all(codes == 0)
