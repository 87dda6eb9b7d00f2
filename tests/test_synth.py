"""Pins of the shared seeded input generators (no GPU)."""
import numpy as np

import synth


def test_splitmix64_published_values():
    # SplitMix64 from state 0: first outputs as published with the generator
    z = synth.splitmix64(0, 3)
    assert int(z[0]) == 0xE220A8397B1DCDAF
    assert int(z[1]) == 0x6E789E6AA1B965F4
    assert int(z[2]) == 0x06C45D188009454F


def test_normal_moments_and_determinism():
    a = synth.normal(12345, 200001)
    assert abs(a.mean()) < 0.01 and abs(a.var() - 1.0) < 0.01
    assert np.array_equal(a[:10], synth.normal(12345, 10))
    B = synth.normal_rhs(100, 3, config=2)
    assert B.flags["F_CONTIGUOUS"]
    assert np.array_equal(B[:, 1], synth.normal(synth.rhs_seed(2, 0, 1), 100))


def test_workload_draws():
    probs = synth.batched_problems()
    assert len(probs) == 64
    assert all(6 <= n <= 16 and 1.0 <= k <= 10.0 for n, k in probs)
    reqs = synth.serving_requests()
    assert len(reqs) == 200 and all(1 <= r["nrhs"] <= 16 for r in reqs)
    ts = [r["t"] for r in reqs]
    assert all(b > a for a, b in zip(ts, ts[1:]))
