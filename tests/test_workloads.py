"""The seeded synthetic inputs: SplitMix64 against its reference outputs, and
the batch / serving generators (deterministic, in their stated ranges)."""
import math

import numpy as np

from paper_2202_06111_gb300 import workloads as W


def test_splitmix64_reference_outputs():
    """The first outputs of the reference SplitMix64 for seed 1234567."""
    r = W.SplitMix64(1234567)
    assert [r.next_u64() for _ in range(5)] == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                                                4593380528125082431, 16408922859458223821]


def test_uniform_draws_in_range():
    r = W.SplitMix64(7)
    u = np.array([r.uniform() for _ in range(20000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01
    k = np.array([r.randint(5, 11) for _ in range(7000)])
    assert k.min() == 5 and k.max() == 11
    e = np.array([r.exponential(0.005) for _ in range(20000)])
    assert abs(e.mean() - 0.005) < 0.0003 and e.min() > 0


def test_batch_512_deterministic_and_ranged():
    a, b = W.batch_512(), W.batch_512()
    assert len(a) == 512 and a == b
    for p in a:
        assert p["dyn"] in ("vdp", "cstr_dl") and p["n"] == 2 and p["k"] == 3
        assert 5 <= len(p["controls"]) <= 11 and 0 <= p["levels"] <= 3
        cells = p["n0"][0] * p["n0"][1]
        assert 30 ** 2 <= cells <= 513 ** 2
    kinds = [p["dyn"] for p in a]
    assert 200 < kinds.count("vdp") < 312


def test_serving_2000_arrivals():
    reqs = W.serving_2000()
    assert len(reqs) == 2000 and reqs == W.serving_2000()
    t = np.array([p["arrival_s"] for p in reqs])
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean(np.diff(t)) - 0.005) < 0.0005          # Poisson arrivals, mean 200 / s
    kinds = {p["dyn"] for p in reqs}
    assert kinds == {"vdp", "cstr_dl", "cartpole"}
    for p in reqs:
        assert 0 <= p["levels"] <= 3
        if p["dyn"] == "cartpole":
            assert 16 <= p["n0"][0] <= 48 and len(set(p["n0"])) == 1
        else:
            assert 30 ** 2 <= p["n0"][0] * p["n0"][1] <= 1030 ** 2
    assert not math.isnan(t[-1])
