"""CPU model of the FP8 sweep's shared-memory conversion (no GPU).

The FP8 form's converter warps turn a 128 x 128 tile of E4M3 codes, as a TMA
copy with 128-byte swizzle lays it out, into the BF16 tile a TMA copy of the
dequantised values would have produced.  That arithmetic is restated here and
checked against the oracle's E4M3 decoding and the swizzle's definition:

* bit formula: for a normal code c of a tile with exponent k, the BF16 bits of
  c 2^k are (c << 4) + ((120 + k) << 7), computed two codes per 32-bit word
  as 16-bit lanes, with the exponent term masked to lanes whose code is >= 8;
* layout: thread y reads row y's eight 16-byte chunks at positions c ^ (y % 8)
  and writes chunk c's 16 values as BF16 chunks 2 (c % 4) and 2 (c % 4) + 1 of
  box c / 4, each at its swizzled position.
"""
import numpy as np

from oracle import enmf_oracle as O


def _swizzled(y, b):
    """Byte offset of byte b of row y in a 128-byte-swizzled box of 128-byte
    rows (1024-byte aligned)."""
    return y * 128 + (((b >> 4) ^ (y & 7)) << 4) + (b & 15)


def _byte_perm(x, s):
    """CUDA __byte_perm(x, 0, s) on uint32 arrays: result byte n is byte
    (s >> 4n) & 7 of the 8-byte value (0, x)."""
    out = np.zeros_like(x)
    for n in range(4):
        sel = (s >> (4 * n)) & 7
        byte = (x >> (8 * sel)) & 0xFF if sel < 4 else np.zeros_like(x)
        out |= byte << (8 * n)
    return out


def _convert_words(w, e0):
    """Two uint32 outputs (BF16 pairs) per uint32 word of four codes."""
    w = w.astype(np.uint64)
    t = ((w + 0x78787878) & 0xFFFFFFFF) & 0x80808080
    lo = (_byte_perm(w, 0x4140) * 16 + _byte_perm(t, 0x4140) * e0) & 0xFFFFFFFF
    hi = (_byte_perm(w, 0x4342) * 16 + _byte_perm(t, 0x4342) * e0) & 0xFFFFFFFF
    return lo.astype(np.uint32), hi.astype(np.uint32)


def _bf16_bits_exact(v):
    f = np.asarray(v, dtype=np.float32)
    b = f.view(np.uint32)
    assert np.all((b & 0xFFFF) == 0), "value not exact in BF16"
    return (b >> 16).astype(np.uint16)


def _grid_values(codes):
    e, m = codes >> 3, codes & 7
    return np.where(codes == 0, 0.0, 2.0 ** (e.astype(np.int64) - 7) * (1 + m / 8.0))


def test_bit_formula_every_normal_code_and_exponent():
    codes = np.arange(8, 127, dtype=np.uint32)
    # one word per code pair: (c, c, c, c)
    w = codes | (codes << 8) | (codes << 16) | (codes << 24)
    for k in range(O.TILE_K_MIN, O.TILE_K_MAX + 1):
        lo, hi = _convert_words(w, 120 + k)
        want = _bf16_bits_exact(_grid_values(codes) * 2.0 ** k).astype(np.uint32)
        for half in (lo, hi):
            assert np.array_equal(half & 0xFFFF, want), k
            assert np.array_equal(half >> 16, want), k
    # the grid values are exactly the oracle's E4M3 values
    np.testing.assert_array_equal(O.e4m3_round(_grid_values(codes)), _grid_values(codes))


def test_zero_codes_stay_zero_beside_nonzero_ones():
    w = np.array([0x00380000, 0x7E000008, 0x0], dtype=np.uint32)
    lo, hi = _convert_words(w, 120)
    # word 0: codes (0, 0, 0x38, 0): 1.0 in the third lane only
    assert lo[0] == 0 and hi[0] == 0x3F80
    # word 1: codes (8, 0, 0, 0x7E): 2^-6 and 448
    assert lo[1] == _bf16_bits_exact(2.0 ** -6)[()] and hi[1] == (int(_bf16_bits_exact(448.0)) << 16)
    assert lo[2] == 0 and hi[2] == 0


def test_swizzled_tile_conversion_matches_dequantised_tile():
    rng = np.random.default_rng(4)
    for k in (-100, -7, 0, 33, 100):
        code = rng.integers(8, 127, (128, 128)).astype(np.uint32)
        code[rng.random((128, 128)) < 0.3] = 0
        Q = np.zeros(128 * 128, np.uint8)
        ys, bs = np.meshgrid(np.arange(128), np.arange(128), indexing="ij")
        Q[_swizzled(ys, bs)] = code
        A = np.zeros(2 * 128 * 128 * 2, np.uint8)         # two BF16 boxes of 16 KB
        for y in range(128):
            sw = y & 7
            for c in range(8):
                chunk = Q[y * 128 + ((c ^ sw) << 4): y * 128 + ((c ^ sw) << 4) + 16]
                words = chunk.view(np.uint32)
                lo, hi = _convert_words(words, 120 + k)
                out = np.empty(8, np.uint32)
                out[0::2], out[1::2] = lo, hi
                d = (c >> 2) * 16384 + y * 128
                cc = (c & 3) * 2
                for half, idx in ((0, cc), (1, cc + 1)):
                    off = d + ((idx ^ sw) << 4)
                    assert 0 <= off and off + 16 <= A.size
                    A[off:off + 16] = out[4 * half:4 * half + 4].view(np.uint8)
        bits = _bf16_bits_exact(_grid_values(code) * 2.0 ** k)
        E = np.zeros_like(A)
        col = np.arange(128)
        for y in range(128):
            box, j = col // 64, col % 64
            off = box * 16384 + _swizzled(y, 2 * j)
            E[off] = bits[y] & 0xFF
            E[off + 1] = bits[y] >> 8
        np.testing.assert_array_equal(A, E)
