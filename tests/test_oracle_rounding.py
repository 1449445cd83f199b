"""Pins for the oracle's FP32/BF16 value rounding (IEEE nearest-even from FP64)."""
import numpy as np
import torch

import oracle


def test_bf16_matches_library_on_f32_exact_inputs():
    # for inputs already exact in FP32 the FP32 -> BF16 cast is a single rounding
    g = np.random.default_rng(1)
    v = (g.standard_normal(50000) * 10.0 ** g.integers(-30, 30, 50000)).astype(np.float32)
    ref = torch.from_numpy(v).to(torch.bfloat16).double().numpy()
    assert np.array_equal(oracle.round_to_bf16(v.astype(np.float64)), ref)


def test_bf16_ties_and_bound():
    one = 1.0
    ulp = 2.0 ** -7                       # BF16 spacing on [1, 2)
    # exact halfway cases go to the even neighbour
    assert oracle.round_to_bf16(np.array([one + ulp / 2]))[0] == one
    assert oracle.round_to_bf16(np.array([one + 3 * ulp / 2]))[0] == one + 2 * ulp
    # just above halfway rounds up (a bit FP32 cannot hold: double rounding would tie)
    assert oracle.round_to_bf16(np.array([one + ulp / 2 + 2.0 ** -40]))[0] == one + ulp
    g = np.random.default_rng(2)
    v = g.uniform(-1e3, 1e3, 100000)
    r = oracle.round_to_bf16(v)
    assert np.all(np.abs(r - v) <= 2.0 ** -8 * np.abs(v))
    # results are representable: rounding again changes nothing
    assert np.array_equal(oracle.round_to_bf16(r), r)


def test_f32_rounding():
    v = np.array([1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, 0.1])
    r = oracle.round_to_f32(v)
    assert r[0] == 1.0 and r[1] == 1.0 + 2.0 ** -22 and r[2] == np.float32(0.1)
