"""The autotuner on the GPU: it times every applicable Cauchy evaluation, records the fastest
correct one, and a plan with DCTPLUS_CAUCHY_AUTO and that cache takes it."""
import numpy as np
import pytest

from oracle import cauchy
from synthetic import normal_signals, random_unit_v

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_08970_gb300 as p
    from paper_2409_08970_gb300 import build
    build.build()
    return p


@pytest.mark.parametrize("n", [256, 1024, 4096])
def test_autotune_picks_the_fastest_correct_mode(pkg, n, tmp_path):
    cache = str(tmp_path / "tune.json")
    batch = 2048
    v = random_unit_v(n)
    res = pkg.dctplus_autotune(n, v, 2.0, batch, cache)
    ms = res["ms"]
    # every evaluation that applies at this n ran and agreed with the CUDA-core product
    assert all(ms[k] > 0 for k in ("dense", "hier_leaf", "hier_tree", "simt")), ms
    best = min(ms, key=lambda k: ms[k])
    want = {"dense": (pkg.CAUCHY_DENSE, 0), "hier_leaf": (pkg.CAUCHY_HIER, 1),
            "hier_tree": (pkg.CAUCHY_HIER, 2), "simt": (pkg.CAUCHY_SIMT, 0)}[best]
    assert (res["cauchy_mode"], res["far_field"]) == want
    name = torch.cuda.get_device_name(0)
    assert pkg.dctplus_tune_lookup(cache, name, n, batch) == want
    # AUTO with the cache takes the recorded choice and transforms correctly
    plan = pkg.Plan(n, v, 2.0, tune_cache=cache, batch_hint=batch)
    assert plan.cauchy_mode == want[0]
    if want[0] == pkg.CAUCHY_HIER:
        assert plan.far_field == want[1]
    x = normal_signals(64, n, seed=2)
    y = plan.forward(torch.tensor(x, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    ref = cauchy.transform(cauchy.make_plan(n, v, 2.0), x)
    assert (np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)).max() < 1e-6
    plan.close()
    # a batch in another bucket has no entry: the fixed rule
    plan = pkg.Plan(n, v, 2.0, tune_cache=cache, batch_hint=64)
    assert plan.cauchy_mode == (pkg.CAUCHY_HIER if n >= 1024 else pkg.CAUCHY_DENSE)
    plan.close()
    assert pkg.dctplus_sync_check(0) == 0
