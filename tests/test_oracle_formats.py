"""Pins for fl(.) (Definition 1) and the formats of Table I."""
import json
import os
from decimal import Decimal

import numpy as np
import pytest
import torch

from oracle.formats import FORMATS, fl, quant_e4m3_rows, e4m3_block_scale


def _table1(golden_dir):
    with open(os.path.join(golden_dir, "table1_formats.json")) as f:
        return json.load(f)


def test_table1_parameters(golden_dir):
    t = _table1(golden_dir)
    for name, row in t["formats"].items():
        f = FORMATS[name]
        assert f.p == row["sig"]
        assert f.emax == 2 ** (row["exp"] - 1) - 1
        assert abs(Decimal(f.xmin) / Decimal(row["xmin"]) - 1) < Decimal("5e-3")
        assert abs(Decimal(f.xmax) / Decimal(row["xmax"]) - 1) < Decimal("5e-3")
        if name == "fp64":
            # Table I misprint: 4.88e-16 printed, 2^-53 for a 53-bit significand
            assert f.u == 2.0 ** -53
            assert abs(f.u / row["u"] - 1) > 0.5
        else:
            assert abs(f.u / row["u"] - 1) < 5e-3


def _samples(rng, n=20000):
    mags = 10.0 ** rng.uniform(-12, 12, n)
    x = mags * rng.choice([-1.0, 1.0], n)
    return np.concatenate([x, rng.standard_normal(n), [0.0, 1.0, -1.0]])


def test_fl_fp32_matches_ieee_single():
    x = _samples(np.random.default_rng(1))
    assert np.array_equal(fl(x, "fp32"), x.astype(np.float32).astype(np.float64))


def test_fl_fp16_matches_ieee_half_including_subnormals():
    rng = np.random.default_rng(2)
    x = np.concatenate([_samples(rng) * 1e-3, rng.uniform(-7e-5, 7e-5, 5000)])
    with np.errstate(over="ignore"):
        ref = x.astype(np.float16).astype(np.float64)
    assert np.array_equal(fl(x, "fp16"), ref)


def test_fl_bf16_matches_torch():
    x = _samples(np.random.default_rng(3))
    ref = torch.from_numpy(x).to(torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    # the float64 -> float32 step of the reference double-rounds; compare on
    # values exactly representable in float32 so only one rounding happens
    x32 = x.astype(np.float32).astype(np.float64)
    ref = torch.from_numpy(x32).to(torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(fl(x32, "bf16"), ref)


def test_fl_e4m3_matches_torch_in_range():
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.uniform(-448, 448, 20000), rng.uniform(-2e-2, 2e-2, 5000),
                        [448.0, -448.0, 0.0, 2.0 ** -9, 3 * 2.0 ** -10]])
    x = x.astype(np.float32).astype(np.float64)
    ref = torch.from_numpy(x).to(torch.float32).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(fl(x, "e4m3"), ref)


def test_fl_e4m3_saturates():
    assert fl(np.array([1e4, -500.0, 460.0]), "e4m3").tolist() == [448.0, -448.0, 448.0]


def test_ties_to_even_and_overflow():
    # midway between 1+2^-7 (odd last bit) and 1+2^-6 (even): goes to 1+2^-6
    assert fl(1 + 3 * 2.0 ** -8, "bf16") == 1 + 2.0 ** -6
    assert fl(1 + 2.0 ** -8, "bf16") == 1.0
    assert fl(1 + 2.0 ** -11, "fp16") == 1.0
    assert fl(65520.0, "fp16") == np.inf         # (xmax + half ulp) rounds to even -> overflow
    assert fl(65519.0, "fp16") == 65504.0


@pytest.mark.parametrize("fmt", ["bf16", "fp16", "fp32"])
def test_standard_model_definition2(fmt):
    """|fl(x) - x| <= u |x| for x in the normal range (Definition 2)."""
    f = FORMATS[fmt]
    rng = np.random.default_rng(5)
    x = rng.standard_normal(50000) * 10.0 ** rng.uniform(-3, 3, 50000)
    x = x[(np.abs(x) >= f.xmin) & (np.abs(x) <= f.xmax)]
    assert np.all(np.abs(fl(x, fmt) - x) <= f.u * np.abs(x))


def test_e4m3_block_scale_definition():
    rng = np.random.default_rng(6)
    amax = 10.0 ** rng.uniform(-6, 6, 10000)
    s = e4m3_block_scale(amax)
    k = np.log2(s)
    assert np.array_equal(k, np.round(k))          # powers of two
    assert np.all(amax <= 448 * s) and np.all(amax > 224 * s)   # smallest such power
    assert e4m3_block_scale(np.array([0.0]))[0] == 1.0
    assert e4m3_block_scale(np.array([448.0]))[0] == 1.0
    assert e4m3_block_scale(np.array([448.0 * (1 + 2 ** -20)]))[0] == 2.0


def test_e4m3_block_roundtrip_error():
    rng = np.random.default_rng(7)
    v = rng.standard_normal((64, 100)) * 10.0 ** rng.uniform(-3, 3, (64, 1))
    q, s = quant_e4m3_rows(v, 32)
    assert s.shape == (64, 4)
    big = np.abs(v) >= np.repeat(s, 32, axis=1)[:, :100] * 2.0 ** -6   # normal e4m3 range
    assert np.all(np.abs(q - v)[big] <= 2.0 ** -4 * np.abs(v)[big])
    assert np.all(np.abs(q - v) <= 2.0 ** -10 * np.repeat(s, 32, axis=1)[:, :100] + 2.0 ** -4 * np.abs(v))
