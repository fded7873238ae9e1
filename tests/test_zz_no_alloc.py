"""dctplus_execute_noalloc (fixed device scratch, no allocation at execute
time) against dctplus_execute and the FP64 oracle. This file is collected
last so it also runs after every other GPU test in one process."""
import ctypes

import numpy as np
import pytest

from oracle import cauchy
from synthetic import edge_update_v, normal_signals, random_unit_v

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32_TOL = 1e-6
MAX_SAMPLES = 1 << 22


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_08970_gb300 as p
    from paper_2409_08970_gb300 import build
    build.build()
    return p


def noalloc(lib, plan, x, y):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.dctplus_execute_noalloc(plan.handle, ctypes.c_void_p(x.data_ptr()), x.stride(0),
                                       ctypes.c_void_p(y.data_ptr()), y.stride(0), x.shape[0], stream)


def relerr(y, ref):
    return np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)


def oracle_rows(n, v, rho, x, rng):
    """Sampled oracle rows: all of them up to n = 4096, else about 40 secular-root rows
    (the sampled set of root numbers mapped to their output rows) and a few deflated rows."""
    if n <= 4096:
        return np.arange(n), cauchy.transform(cauchy.make_plan(n, v, rho), x)
    probe = cauchy.make_plan(n, v, rho, roots=[])
    K = int(probe.row_kind.sum())
    roots = np.unique(np.concatenate([rng.choice(K, min(K, 36), replace=False), [0, 1, K - 2, K - 1]]))
    plan = cauchy.make_plan(n, v, rho, roots=roots)
    root_rows = np.nonzero((plan.row_kind == 1) & np.isin(plan.row_index, roots))[0]
    defl = np.nonzero(plan.row_kind == 0)[0][:4]
    rows = np.sort(np.concatenate([root_rows, defl]))
    return rows, cauchy.transform(plan, x, rows=rows)


# n = 8192 and 16384 have no stored W table: the Cauchy product then generates W tile by
# tile on the CUDA cores, and n = 16384 runs the DCT with 512 threads and 70 KB of shared memory per signal
@pytest.mark.parametrize("n,batch", [(128, 300), (1024, 4096), (4096, 64), (8192, 512), (16384, 256)])
def test_noalloc_matches_execute_twice(pkg, n, batch):
    assert batch * n <= MAX_SAMPLES
    lib = pkg._lib.load()
    rng = np.random.default_rng(n)
    for v, rho in [(random_unit_v(n), 2.0), (edge_update_v(n, n // 2 - 1, n // 2), -0.5)]:
        plan = pkg.Plan(n, v, rho)
        xh = normal_signals(batch, n, seed=n + 5)
        x = torch.tensor(xh, dtype=torch.float32, device="cuda")
        ref = plan.forward(x).double().cpu().numpy()
        sig = np.arange(0, batch, max(1, batch // (32 if n <= 4096 else 6)))
        cols, want = oracle_rows(n, v, rho, xh[sig], rng)
        scale = np.linalg.norm(xh[sig], axis=1)[:, None]
        for call in range(2):
            y = torch.full_like(x, float("nan"))
            free0 = torch.cuda.mem_get_info()[0]
            assert noalloc(lib, plan, x, y) == 0
            torch.cuda.synchronize()
            if call == 1:  # the first call on the device may have done its one-time set-up
                assert torch.cuda.mem_get_info()[0] == free0
            got = y.double().cpu().numpy()
            assert np.isfinite(got).all()
            assert relerr(got, ref).max() < 2 * F32_TOL, (n, rho, call)
            if n <= 4096:
                assert relerr(got[sig], want).max() < F32_TOL, (n, rho, call)
            else:  # sampled rows: max error relative to the signal's norm
                assert (np.abs(got[sig][:, cols] - want) / scale).max() < F32_TOL, (n, rho, call)
        plan.close()
    assert pkg.dctplus_sync_check(0) == 0


def test_noalloc_limits(pkg):
    lib = pkg._lib.load()
    n = 1024
    plan = pkg.Plan(n, random_unit_v(n), 2.0)
    over = MAX_SAMPLES // n + 1
    x = torch.zeros(over, n, device="cuda")
    y = torch.zeros_like(x)
    assert noalloc(lib, plan, x, y) == pkg.ERR_SCRATCH_LIMIT
    assert b"scratch" in lib.dctplus_status_string(pkg.ERR_SCRATCH_LIMIT)
    assert noalloc(lib, plan, x[: over - 1], y[: over - 1]) == 0
    assert noalloc(lib, plan, x[:0], y[:0]) == 0
    plan.close()
    small = pkg.Plan(64, random_unit_v(64), 2.0)
    x = torch.zeros(8, 64, device="cuda")
    assert noalloc(lib, small, x, torch.zeros_like(x)) == 2  # UNSUPPORTED: n <= 64 needs no scratch
    small.close()
    torch.cuda.synchronize()
    assert pkg.dctplus_sync_check(0) == 0
