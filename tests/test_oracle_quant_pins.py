"""Pins of the oracle's storage quantisers (BF16 and FP8 E4M3 with column scales).

BF16 is checked against torch's float32 -> bfloat16 conversion (round to
nearest even). E4M3 is checked against torch's float8_e4m3fn conversion for
in-range values and against hand-derived codes from the OCP E4M3 format
definition stored in tests/golden/e4m3_cases.txt.
"""
import os

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "e4m3_cases.txt")


def _edge_floats():
    vals = [0.0, -0.0, 1.0, -1.0, 3.0e38, -3.0e38, 1e-40, -1e-40, 1.17549435e-38,
            np.float32(1.0) + np.float32(2.0 ** -8), np.float32(1.0) + np.float32(3 * 2.0 ** -9),
            np.float32(1.0) + np.float32(2.0 ** -9), 65504.0, 0.1, -0.3333333, 7.0e-3]
    return np.array(vals, dtype=np.float32)


def test_bf16_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(100000).astype(np.float32),
                        (rng.standard_normal(10000) * 1e30).astype(np.float32),
                        (rng.standard_normal(10000) * 1e-38).astype(np.float32),
                        _edge_floats()])
    # ties: low 16 bits exactly 0x8000
    bits = rng.integers(0, 2**32, 5000, dtype=np.uint64).astype(np.uint32)
    bits = (bits & 0xFFFF0000) | 0x8000
    bits = bits[(bits & 0x7F800000) != 0x7F800000]
    x = np.concatenate([x, bits.view(np.float32)])
    ours = oracle.bf16_from_f32(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(ours, ref)
    back = oracle.bf16_to_f64(ours)
    np.testing.assert_array_equal(back, torch.from_numpy(x).to(torch.bfloat16).double().numpy())


def test_e4m3_golden_cases():
    """Codes derived by hand from the E4M3 definition (bias 7, 3 mantissa bits, max 448)."""
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                v, code = line.split()
                rows.append((float(v), int(code, 16)))
    assert len(rows) >= 20
    for v, code in rows:
        assert oracle.e4m3_from_f64(v) == code, (v, hex(code))
        if not (v > 448 or v < -448):
            # decoding the code gives the rounded value back
            dec = oracle.e4m3_value(code)
            assert abs(dec - v) <= abs(v) * 2.0 ** -4 + 2.0 ** -10


def test_e4m3_matches_torch_in_range():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-448, 448, 50000), rng.standard_normal(50000),
                        rng.uniform(-2.0 ** -6, 2.0 ** -6, 20000),
                        np.array([0.0, 448.0, -448.0, 2.0 ** -9, 2.0 ** -10, 3 * 2.0 ** -11])])
    x = x.astype(np.float32)
    ours = np.array([oracle.e4m3_from_f64(float(v)) for v in x], dtype=np.uint8)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    # signed zero: the format has -0 (0x80); torch keeps the sign as well
    np.testing.assert_array_equal(ours, ref)
    # every code decodes to the value torch decodes
    codes = np.arange(256, dtype=np.uint8)
    vals = oracle.e4m3_decode(codes)
    tv = torch.from_numpy(codes).view(torch.float8_e4m3fn).double().numpy()
    finite = ~np.isnan(tv)
    np.testing.assert_array_equal(vals[finite], tv[finite])
    assert np.isnan(vals[~finite]).all() and (~finite).sum() == 2


@pytest.mark.parametrize("amax", [0.0, 1.0, 448.0, 448.0000001, 5.3, 1e-6, 3.2e4, 2.0 ** -20])
def test_e4m3_column_scale_definition(amax):
    s = oracle.e4m3_column_scale(amax)
    m, e = np.frexp(s)
    assert m == 0.5  # power of two
    if amax == 0:
        assert s == 1.0
    else:
        assert 448.0 * s >= amax
        assert 448.0 * (s / 2) < amax


def test_quantize_e4m3_matrix():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((300, 7)).astype(np.float32)
    X[:, 0] = 1.0
    X[:, 3] = 0.0
    X[:, 4] *= 1000
    Q, s = oracle.quantize_e4m3(X, ld_q=16)
    assert Q.shape == (300, 16) and (Q[:, 7:] == 0).all()
    assert s[0] == 2.0 ** -8 and s[3] == 1.0
    deq = oracle.dequantize_e4m3(Q, s, p=7)
    # intercept column survives exactly; all values within half an E4M3 ulp
    assert (deq[:, 0] == 1.0).all()
    assert (deq[:, 3] == 0.0).all()
    err = np.abs(deq - X)
    assert (err <= np.abs(X) * 2.0 ** -4 + 2.0 ** -9 * s[None, :]).all()
    # column scaling then torch's conversion gives the same codes
    ref = torch.from_numpy((X / s[None, :]).astype(np.float32)).to(torch.float8_e4m3fn)
    np.testing.assert_array_equal(Q[:, :7], ref.view(torch.uint8).numpy())
