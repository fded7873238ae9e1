"""Progressive multi-transform with pruning (Theorem 3.4) against the FP64 oracle."""
import numpy as np
import pytest

from oracle import cauchy
from synthetic import normal_signals, random_unit_v, self_loop_v

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32_TOL = 1e-6
RHOS = [0.25 * (k + 1) for k in range(8)]


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_08970_gb300 as p
    from paper_2409_08970_gb300 import build
    build.build()
    return p


def run_pruned(pkg, plans, x, m_out, c_p, ldy=None):
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    width = len(plans) * m_out
    ldy = ldy or width
    y = torch.full((x.shape[0], ldy), float("nan"), device="cuda")
    pkg.dctplus_execute_pruned([p.handle for p in plans], xd.data_ptr(), n_of(plans), y.data_ptr(), ldy,
                               x.shape[0], m_out, c_p, torch.cuda.current_stream().cuda_stream)
    return y[:, :width].double().cpu().numpy()


def n_of(plans):
    return plans[0].n


def check_blocks(pkg, plans, vs, x, m_out, c_p, got, rows=None):
    n = plans[0].n
    sig = np.arange(x.shape[0]) if rows is None else rows
    for k, (v, rho) in enumerate(vs):
        ref = cauchy.pruned_transform(cauchy.make_plan(n, v, rho), x[sig], m_out, c_p)
        blk = got[sig, k * m_out:(k + 1) * m_out]
        err = np.linalg.norm(blk - ref, axis=1) / np.linalg.norm(x[sig], axis=1)
        assert err.max() < F32_TOL, (k, err.max())


@pytest.mark.parametrize("c_p", [512, 128])
def test_pruned_n512_eight_self_loops(pkg, c_p):
    n, batch, m_out = 512, 300, 128
    vs = [(self_loop_v(n, 0), r) for r in RHOS]
    plans = [pkg.Plan(n, v, r) for v, r in vs]
    x = normal_signals(batch, n, seed=0)
    got = run_pruned(pkg, plans, x, m_out, c_p)
    check_blocks(pkg, plans, vs, x, m_out, c_p, got)
    if c_p == n:  # exact: equals the first m_out coefficients of the full transforms
        for k, p in enumerate(plans):
            full = p.forward(torch.tensor(x, dtype=torch.float32, device="cuda")).double().cpu().numpy()
            assert np.abs(got[:, k * m_out:(k + 1) * m_out] - full[:, :m_out]).max() < 1e-4
    else:  # Theorem 3.4's bound holds for the GPU result
        for k, (v, rho) in enumerate(vs):
            op = cauchy.make_plan(n, v, rho)
            full = cauchy.transform(op, x[:40])
            padded = np.zeros_like(full)
            padded[:, :c_p] = got[:40, k * m_out:(k + 1) * m_out]
            err = np.linalg.norm(full - padded, axis=1)
            assert np.all(err <= cauchy.pruning_bound(op, x[:40], c_p) * (1 + 1e-5))
    for p in plans:
        p.close()
    assert pkg.dctplus_sync_check(0) == 0


def test_pruned_cuda_core_path_and_mixed_updates(pkg):
    n = 256
    vs = [(random_unit_v(n, seed=11), -0.3), (self_loop_v(n, 0), 1.0), (random_unit_v(n, seed=12), 2.0)]
    plans = [pkg.Plan(n, v, r) for v, r in vs]
    x = normal_signals(129, n, seed=3)
    for m_out, c_p, ldy in [(100, 200, None), (33, 33, 101), (64, 256, None), (1, 1, None)]:
        got = run_pruned(pkg, plans, x, m_out, c_p, ldy)
        check_blocks(pkg, plans, vs, x, m_out, c_p, got)
    for p in plans:
        p.close()
    assert pkg.dctplus_sync_check(0) == 0


@pytest.mark.parametrize("n", [8, 32, 64, 96])
def test_pruned_small_n(pkg, n):
    vs = [(self_loop_v(n, 0), 0.5), (random_unit_v(n, seed=2), -0.5)]
    plans = [pkg.Plan(n, v, r) for v, r in vs]
    x = normal_signals(77, n, seed=5)
    for m_out, c_p in [(n // 2, n), (n // 4, n // 2), (n, n)]:
        got = run_pruned(pkg, plans, x, m_out, c_p)
        check_blocks(pkg, plans, vs, x, m_out, c_p, got)
    for p in plans:
        p.close()


def test_pruned_full_config_sampled(pkg):
    """n = 512, 16384 signals, K = 8, m = 128: the launch configuration the benchmark times."""
    n, batch, m_out = 512, 16384, 128
    vs = [(self_loop_v(n, 0), r) for r in RHOS]
    plans = [pkg.Plan(n, v, r) for v, r in vs]
    x = normal_signals(batch, n, seed=0)
    rng = np.random.default_rng(4)
    rows = np.sort(rng.choice(batch, 48, replace=False))
    for c_p in (512, 128):
        got = run_pruned(pkg, plans, x, m_out, c_p)
        assert np.isfinite(got).all()
        check_blocks(pkg, plans, vs, x, m_out, c_p, got, rows=rows)
    for p in plans:
        p.close()
    assert pkg.dctplus_sync_check(0) == 0


def test_pruned_cache_survives_destroy_and_rebuild(pkg):
    n = 256
    v = self_loop_v(n, 0)
    x = normal_signals(64, n, seed=1)
    a = [pkg.Plan(n, v, 1.0)]
    ya = run_pruned(pkg, a, x, 128, 256)
    a[0].close()
    b = [pkg.Plan(n, v, 2.0)]  # may reuse the freed plan's address
    yb = run_pruned(pkg, b, x, 128, 256)
    check_blocks(pkg, b, [(v, 2.0)], x, 128, 256, yb)
    assert np.abs(ya - yb).max() > 1e-3
    b[0].close()


def test_pruned_argument_errors(pkg):
    n = 256
    p1 = pkg.Plan(n, self_loop_v(n, 0), 1.0)
    p2 = pkg.Plan(128, self_loop_v(128, 0), 1.0)
    x = torch.zeros(4, n, device="cuda")
    y = torch.zeros(4, 512, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    lib = pkg._lib.load()
    import ctypes

    def call(plans, m_out, c_p, ldy=512, yp=None):
        arr = (ctypes.c_void_p * len(plans))(*[q.handle.value for q in plans])
        return lib.dctplus_execute_pruned(arr, len(plans), ctypes.c_void_p(x.data_ptr()), n,
                                          ctypes.c_void_p(yp or y.data_ptr()), ldy, 4, m_out, c_p,
                                          ctypes.c_void_p(s))
    assert call([p1], 64, 128) == 0
    assert call([p1], 129, 128) == 1      # m_out > c_p
    assert call([p1], 64, 257) == 1       # c_p > n
    assert call([p1], 0, 128) == 1
    assert call([p1, p2], 64, 128) == 1   # different n
    assert call([p1, p1], 300, 300, ldy=599) == 1  # ldy < K m_out
    assert call([p1], 64, 128, yp=x.data_ptr()) == 1  # overlaps x
    p1.close()
    p2.close()
