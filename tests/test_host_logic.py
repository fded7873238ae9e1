"""Host-side logic that needs no GPU: the benchmark's roofline bookkeeping and oracle-error
helper, and the value keys of the autograd plan cache."""
import numpy as np
import pytest

import bench
from oracle import cauchy
from synthetic import normal_signals, random_unit_v

torch = pytest.importorskip("torch")


def test_roofline_of_picks_the_dominant_kernel():
    recs = [{"kernel": "k_dct_r8", "ms": 0.010, "bytes": 8.0e7, "flops": 1e9},
            {"kernel": "k_gemm_tc", "ms": 0.020, "bytes": 1e7, "flops": 1.0e13},
            {"kernel": "k_dct_r8", "ms": 0.010, "bytes": 8.0e7, "flops": 1e9},
            {"kernel": "k_gemm_tc", "ms": 0.030, "bytes": 1e7, "flops": 1.0e13}]
    r = bench.roofline_of(recs, 6000.0, 2000.0, "measured")
    assert r["kernel"] == "k_gemm_tc" and r["bound"] == "tensor" and r["launches_of_kernel"] == 2
    assert r["kernel_ms"] == pytest.approx(0.025)
    # achieved = flops per launch / mean launch time
    assert r["achieved"] == pytest.approx(1.0e13 / 25e-6 / 1e12)
    assert r["peak"] == pytest.approx(2000.0 * 1.1 / 2.25)
    assert r["share_of_step"] == pytest.approx(0.05 / 0.07)
    r3 = bench.roofline_of([{"kernel": "k_nfst_fast", "ms": 2.0, "bytes": 1e8, "flops": 1.0e9}],
                           6000.0, 2000.0, "measured")
    assert r3["bound"] == "alu" and r3["peak"] == bench.FP64_NOMINAL_TFLOPS
    assert r3["achieved"] == pytest.approx(1.0e9 / 2e-3 / 1e12)
    r2 = bench.roofline_of(recs[:1], 6000.0, 2000.0, "measured")
    assert r2["bound"] == "hbm" and r2["unit"] == "GB/s"
    assert r2["achieved"] == pytest.approx(8.0e7 / 10e-6 / 1e9)
    assert r2["frac"] == pytest.approx(r2["achieved"] / 6000.0)


def test_oracle_error_is_zero_on_the_oracle_and_sees_a_planted_error():
    n = 64
    v = random_unit_v(n)
    x = normal_signals(20, n, seed=3)
    y = cauchy.transform(cauchy.make_plan(n, v, 2.0), x)
    e = bench.oracle_error(n, v, 2.0, x, y)
    assert e["max_abs"] < 1e-12 and e["normwise_rel_max"] < 1e-12
    y_bad = y.copy()
    y_bad[:, 5] += 1e-3
    e = bench.oracle_error(n, v, 2.0, x, y_bad)
    assert e["max_abs"] == pytest.approx(1e-3, rel=1e-6)
    # the sampled-roots form finds the same rows
    e = bench.oracle_error(n, v, 2.0, x, y, root_sample=10)
    assert e["max_abs"] < 1e-12 and "sampled" in e["sample"]


def test_autograd_value_keys_are_memoised_per_tensor_version():
    import paper_2409_08970_gb300 as pkg
    calls = []

    def to_host(t):
        calls.append(1)
        return t.detach().numpy().tobytes()

    v = torch.arange(4, dtype=torch.float64)
    k1 = pkg._value_key(v, to_host)
    k2 = pkg._value_key(v, to_host)
    assert k1 == k2 and len(calls) == 1          # same unmodified tensor: no second copy
    v.add_(1.0)
    k3 = pkg._value_key(v, to_host)
    assert k3 != k1 and len(calls) == 2          # in-place change: new version, new key
    w = v.clone()
    assert pkg._value_key(w, to_host) == k3 and len(calls) == 3  # equal values, other tensor
    assert pkg._value_key(1.5, float) == 1.5     # plain numbers are their own key


def test_autotune_cache_record_and_lookup(tmp_path):
    """The autotune cache (host-only entry points): record, lookup by (device, n, batch
    bucket), replacement of an entry with the same key, other keys untouched, a missing file
    or key reported as no entry, and lines that do not parse skipped."""
    import json

    import paper_2409_08970_gb300 as pkg
    path = str(tmp_path / "tune.json")
    dev = "NVIDIA GB300"
    assert pkg.dctplus_tune_lookup(path, dev, 1024, 4096) is None          # no file yet
    pkg.dctplus_tune_record(path, dev, 1024, 4096, pkg.CAUCHY_HIER, 1, 0.061, [0.07, 0.061, 0.09, 0.5])
    pkg.dctplus_tune_record(path, dev, 4096, 4000, pkg.CAUCHY_HIER, 2, 0.2)
    pkg.dctplus_tune_record(path, "other device", 1024, 4096, pkg.CAUCHY_DENSE, 0, 0.05)
    assert pkg.dctplus_tune_lookup(path, dev, 1024, 4096) == (pkg.CAUCHY_HIER, 1)
    assert pkg.dctplus_tune_lookup(path, dev, 1024, 3000) == (pkg.CAUCHY_HIER, 1)   # same bucket 4096
    assert pkg.dctplus_tune_lookup(path, dev, 1024, 5000) is None                    # bucket 8192
    assert pkg.dctplus_tune_lookup(path, dev, 4096, 4096) == (pkg.CAUCHY_HIER, 2)
    assert pkg.dctplus_tune_lookup(path, "other device", 1024, 4096) == (pkg.CAUCHY_DENSE, 0)
    pkg.dctplus_tune_record(path, dev, 1024, 4096, pkg.CAUCHY_DENSE, 0, 0.05)     # replace
    assert pkg.dctplus_tune_lookup(path, dev, 1024, 4096) == (pkg.CAUCHY_DENSE, 0)
    d = json.load(open(path))                                                   # valid JSON
    assert len(d["entries"]) == 3
    e = [x for x in d["entries"] if x["n"] == 4096][0]
    assert e["batch_bucket"] == 4096 and e["far_field"] == 2 and e["ms_dense"] == -1
    # a damaged line is skipped, the others still read
    text = open(path).read().replace('"other device"', '"other device', 1)
    open(path, "w").write(text)
    assert pkg.dctplus_tune_lookup(path, dev, 4096, 4096) == (pkg.CAUCHY_HIER, 2)
    assert pkg.dctplus_tune_lookup(path, "other device", 1024, 4096) is None
    with pytest.raises(pkg.DctPlusError):
        pkg.dctplus_tune_record(path, dev, 1024, 4096, 9, 0, 0.1)                 # bad mode


def test_oracle_plans_are_cached_and_timed_without_planning():
    """The bench builds each oracle plan once per (n, v, rho, roots) and times the oracle's
    transform alone; the rate counts input samples per second."""
    n = 64
    v = random_unit_v(n)
    a = bench.oracle_plan(n, v, 2.0)
    assert bench.oracle_plan(n, v, 2.0) is a
    assert bench.oracle_plan(n, v, -0.3) is not a
    assert bench.oracle_plan(n, v, 2.0, roots=[0, 1]) is not a
    calls = []
    r = bench.oracle_rate(lambda: calls.append(1), 1000, "stub", budget_s=0.05)
    assert r["kind"] == "oracle" and r["unit"] == "GSamples/s" and r["cores"] >= 1
    assert r["value"] > 0 and len(calls) >= 1
