"""Low-precision operand preparation, written from the number formats' definitions
-- TEST INFRASTRUCTURE ONLY (nothing in the product imports this module).

The paper computes in int32 (Fig. "cudamul"); the low-precision forms of the GEMM
are this library's extension, so the definitions come from the formats:

* BF16: 1 sign, 8 exponent (bias 127), 7 fraction bits; same exponent range as
  binary32, subnormal spacing 2^-133.  Conversion is round-to-nearest, ties to
  even; overflow goes to infinity.
* FP8 E4M3 ("fn" variant): 1 sign, 4 exponent (bias 7), 3 fraction bits, no
  infinities, S.1111.111 is NaN, largest finite 448, subnormal spacing 2^-9.
  Conversion is round-to-nearest-even with saturation to +-448 ("satfinite").
* Split BF16: hi = bf16(x), lo = bf16(x - hi); x - hi is exact in binary32.
* FP8 per-tile scaling: for every 128 x 128 tile, scale = amax / 448 (binary32
  division; 1 when amax == 0) and q = e4m3(x / scale) (binary32 division).  The
  binary32 decisions are taken in binary32 here too, so the quantised codes are
  reproducible bit for bit.

Every rounding below is carried out on exact binary64 values with numpy's
round-half-even `rint`, after scaling by a power of two (which is exact).
"""
from __future__ import annotations

import numpy as np

E4M3_MAX = 448.0


def _round_to_spacing(a: np.ndarray, min_exp: int, sig_bits: int) -> np.ndarray:
    """Round |values| a >= 0 (binary64, exact copies of the inputs) to the nearest
    number with `sig_bits` significant bits, or to a multiple of 2^min_exp below
    the normal range; ties to even."""
    _, e = np.frexp(a)                     # a = m * 2^e with 0.5 <= m < 1
    ulp_exp = np.maximum(e - sig_bits, min_exp)
    q = np.ldexp(a, -ulp_exp)              # exact: scaling by a power of two
    return np.ldexp(np.rint(q), ulp_exp)


def bf16_rn(x: np.ndarray) -> np.ndarray:
    """bfloat16 round-to-nearest-even of binary32 values, returned as binary32
    values (exactly representable in bf16)."""
    x = np.asarray(x, dtype=np.float32)
    xd = x.astype(np.float64)
    a = np.abs(xd)
    with np.errstate(invalid="ignore", over="ignore"):
        y = _round_to_spacing(np.where(np.isfinite(a), a, 0.0), -133, 8)
        y = np.where(y >= 2.0 ** 128, np.inf, y)           # overflow -> inf
        y = np.where(np.isfinite(a), y, a)                 # inf / nan pass through
        y = np.copysign(y, xd)
    return y.astype(np.float32)


def bf16_bits(x: np.ndarray) -> np.ndarray:
    """uint16 bit patterns of bf16_rn(x)."""
    y = bf16_rn(x)
    return (y.view(np.uint32) >> 16).astype(np.uint16)


def bf16_from_bits(bits: np.ndarray) -> np.ndarray:
    """Decode bf16 bit patterns to binary32 values."""
    b = np.asarray(bits, dtype=np.uint16).astype(np.uint32) << 16
    return b.view(np.float32)


def e4m3_value(code: np.ndarray) -> np.ndarray:
    """Decode E4M3 ("fn") codes to binary64 from the format definition."""
    c = np.asarray(code, dtype=np.uint8).astype(np.int64)
    sign = np.where(c & 0x80, -1.0, 1.0)
    exp = (c >> 3) & 0xF
    frac = c & 0x7
    normal = np.ldexp(1.0 + frac / 8.0, exp - 7)
    sub = np.ldexp(frac / 8.0, -6)
    v = np.where(exp == 0, sub, normal)
    v = np.where((exp == 0xF) & (frac == 0x7), np.nan, v)
    return sign * v


def e4m3_rn_sat(x: np.ndarray) -> np.ndarray:
    """E4M3 codes (uint8) of binary32 values: round to nearest even, saturate to
    +-448; NaN maps to 0x7F (0xFF when negative)."""
    x = np.asarray(x, dtype=np.float32)
    xd = x.astype(np.float64)
    a = np.abs(xd)
    nan = np.isnan(a)
    a0 = np.where(nan | np.isinf(a), E4M3_MAX, a)
    y = _round_to_spacing(a0, -9, 4)
    y = np.minimum(y, E4M3_MAX)
    # magnitude -> code
    code = np.zeros(y.shape, dtype=np.int64)
    sub = y < 2.0 ** -6
    code = np.where(sub, np.rint(y / 2.0 ** -9).astype(np.int64), code)
    _, e = np.frexp(np.where(sub, 1.0, y))
    E = e - 1                                   # y = (1 + f/8) * 2^E
    f = np.rint((np.ldexp(np.where(sub, 1.0, y), -E) - 1.0) * 8.0).astype(np.int64)
    code = np.where(sub, code, ((E + 7) << 3) | f)
    code = np.where(nan, 0x7F, code)
    sign = np.signbit(xd).astype(np.int64) << 7
    return (code | sign).astype(np.uint8)


def split_bf16(x: np.ndarray):
    """(hi, lo) bf16 values (as binary32) with hi = bf16(x), lo = bf16(x - hi)."""
    x = np.asarray(x, dtype=np.float32)
    hi = bf16_rn(x)
    r = (x - hi).astype(np.float32)             # exact in binary32 (Sterbenz)
    lo = bf16_rn(r)
    return hi, lo


def fp8_tile_scales(X: np.ndarray, tile: int = 128) -> np.ndarray:
    """binary32 scale per tile x tile block of X (ragged edge tiles included):
    amax / 448 evaluated as a binary32 division, 1 when the tile is all zero."""
    X = np.asarray(X, dtype=np.float32)
    R, C = X.shape
    tr, tc = -(-R // tile), -(-C // tile)
    S = np.empty((tr, tc), dtype=np.float32)
    for i in range(tr):
        for j in range(tc):
            blk = X[i * tile:(i + 1) * tile, j * tile:(j + 1) * tile]
            amax = np.float32(np.max(np.abs(blk))) if blk.size else np.float32(0)
            S[i, j] = np.float32(1.0) if amax == 0 else np.float32(amax) / np.float32(E4M3_MAX)
    return S


def fp8_tile_quant(X: np.ndarray, tile: int = 128):
    """Per-tile scaled E4M3 quantisation: returns (codes uint8 R x C, scales)."""
    X = np.asarray(X, dtype=np.float32)
    S = fp8_tile_scales(X, tile)
    Sfull = np.repeat(np.repeat(S, tile, axis=0), tile, axis=1)[: X.shape[0], : X.shape[1]]
    with np.errstate(over="ignore", invalid="ignore"):
        ratio = (X / Sfull).astype(np.float32)   # binary32 division
    return e4m3_rn_sat(ratio), S


def fp8_dequant(codes: np.ndarray, S: np.ndarray, tile: int = 128) -> np.ndarray:
    """binary64 values q * scale of a per-tile scaled E4M3 matrix."""
    v = e4m3_value(codes)
    Sfull = np.repeat(np.repeat(S.astype(np.float64), tile, axis=0), tile, axis=1)
    return v * Sfull[: v.shape[0], : v.shape[1]]
