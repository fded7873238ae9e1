"""Parity of the CUDA path with the FP64 oracle, through the C ABI.

Tolerances: FP64 data within 1e-12 of the oracle (max abs, unit-norm rows);
FP32 data within a normwise relative error of 1e-6 per signal, the accuracy
the split-precision contractions are designed for (the CUDA-core FP32 path
reaches about 1e-7).
"""
import numpy as np
import pytest

from oracle import cauchy, common, definition
from synthetic import (edge_update_v, laplace_residuals, mixed_size_workload, normal_signals,
                       random_unit_v, self_loop_v)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32_TOL = 1e-6
F64_TOL = 1e-12


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_08970_gb300 as p
    from paper_2409_08970_gb300 import build
    build.build()
    return p


def relerr(y, ref):
    return np.linalg.norm(y - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-300)


def run32(plan, x):
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    return plan.forward(xt).double().cpu().numpy()


def run64(plan, x):
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    return plan.forward(xt).cpu().numpy()


SETUP_CASES = [
    (2, random_unit_v(2, seed=5), 0.7),
    (3, self_loop_v(3, 0), 1.0),
    (5, edge_update_v(5, 1, 2), -0.4),
    (8, edge_update_v(8, 3, 4), -0.5),
    (16, random_unit_v(16), 2.0),
    (33, random_unit_v(33), -0.3),
    (64, self_loop_v(64, 0), 1.0),
    (64, edge_update_v(64, 31, 32), -0.5),
    (100, random_unit_v(100), 0.0),
    (256, random_unit_v(256), 2.0),
    (1024, random_unit_v(1024), -0.3),
    (1024, edge_update_v(1024, 511, 512), -0.5),
]


@pytest.mark.parametrize("case", range(len(SETUP_CASES)))
def test_setup_stage_matches_oracle(pkg, case):
    n, v, rho = SETUP_CASES[case]
    plan = pkg.Plan(n, v, rho)
    info = plan.inspect()
    ref = cauchy.make_plan(n, v, rho)
    assert np.abs(info["z"] - ref.z).max() < 1e-14
    assert np.array_equal(info["row_kind"], ref.row_kind)
    assert np.abs(info["eigenvalues"] - ref.eigenvalues).max() < 1e-13 * max(1.0, abs(rho))
    roots = np.nonzero(ref.row_kind == 1)[0]
    if roots.size:
        i = ref.row_index[roots]
        mu_ref = ref.lam[ref.origin[i]] + ref.tau[i]
        mu = ref.lam[info["row_pole"][roots]] + info["row_tau"][roots]
        # the root offset from its pole carries full relative accuracy
        same = info["row_pole"][roots] == ref.origin[i]
        assert np.all(np.abs(info["row_tau"][roots][same] - ref.tau[i][same])
                      <= 1e-11 * np.abs(ref.tau[i][same]) + 1e-300)
        assert np.abs(mu - mu_ref).max() < 1e-13
        assert np.abs(info["row_a"][roots] - ref.a[i]).max() < 1e-11
    plan.close()


def test_secular_iteration_cap_reports_not_converged(pkg):
    with pytest.raises(pkg.DctPlusError) as e:
        pkg.Plan(64, random_unit_v(64), 2.0, max_secular_iter=1)
    assert e.value.status == 3


def test_fp64_unit_self_loop_n64_matches_jacobi_and_dst7(pkg):
    """FP64 n=64, v=e_0, rho=1, 1024 N(0,1) signals (seed 0): the DST-VII."""
    n = 64
    x = normal_signals(1024, n, seed=0)
    plan = pkg.Plan(n, self_loop_v(n, 0), 1.0)
    y = run64(plan, x)
    k = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    dst7 = 2.0 / np.sqrt(2 * n + 1) * np.sin(np.pi * (2 * k + 1) * (j + 1) / (2 * n + 1))
    assert np.abs(y - x @ dst7.T).max() < F64_TOL * np.abs(x).max() * 8
    y1 = definition.transform(n, self_loop_v(n, 0), 1.0, x)
    assert np.abs(y - y1).max() < 1e-11
    plan.close()


@pytest.mark.parametrize("n", [2, 3, 4, 5, 7, 8, 12, 16, 31, 32, 33, 48, 63, 64])
def test_small_n_fp32_and_fp64_match_oracle(pkg, n):
    for v, rho in [(self_loop_v(n, 0), 0.5), (random_unit_v(n, seed=n), -0.3),
                   (edge_update_v(n, n // 2 - 1, n // 2), -0.5)]:
        x = normal_signals(777, n, seed=n)  # ragged: 777 is not a multiple of any tile
        ref = cauchy.transform(cauchy.make_plan(n, v, rho), x)
        plan = pkg.Plan(n, v, rho)
        assert relerr(run32(plan, x), ref).max() < F32_TOL
        assert np.abs(run64(plan, x) - ref).max() < F64_TOL * 10
        plan.close()


@pytest.mark.parametrize("n", [128, 256, 512, 1024, 2048, 4096])
def test_large_n_fp32_matches_oracle(pkg, n):
    batch = 37
    for v, rho in [(random_unit_v(n), -0.3), (random_unit_v(n), 2.0), (self_loop_v(n, 0), 1.0)]:
        x = normal_signals(batch, n, seed=0)
        ref = cauchy.transform(cauchy.make_plan(n, v, rho), x)
        plan = pkg.Plan(n, v, rho)
        err = relerr(run32(plan, x), ref)
        assert err.max() < F32_TOL, (n, rho, err.max())
        plan.close()


def test_n16384_sampled_rows_match_oracle(pkg):
    n, batch = 16384, 512
    v = random_unit_v(n)
    for rho in (-0.3, 2.0):
        x = normal_signals(batch, n, seed=0)
        plan = pkg.Plan(n, v, rho)
        y = run32(plan, x)
        rng = np.random.default_rng(5)
        rows = np.sort(rng.choice(n, 48, replace=False))
        rows = np.unique(np.concatenate([rows, [0, 1, n - 2, n - 1]]))
        sig = np.sort(rng.choice(batch, 16, replace=False))
        ref_plan = cauchy.make_plan(n, v, rho, roots=rows)
        ref = cauchy.transform(ref_plan, x[sig], rows=rows)
        got = y[sig][:, rows]
        # sampled rows: error relative to the signal norm (rows are unit vectors)
        err = np.abs(got - ref).max(axis=1) / np.linalg.norm(x[sig], axis=1)
        assert err.max() < F32_TOL, err.max()
        # Parseval on every signal
        pr = np.abs(np.linalg.norm(y, axis=1) / np.linalg.norm(x, axis=1) - 1)
        assert pr.max() < 5e-6
        plan.close()


def test_rho_zero_gives_dct2(pkg):
    for n in (8, 64, 1024):
        x = normal_signals(50, n, seed=3)
        plan = pkg.Plan(n, random_unit_v(n), 0.0)
        assert relerr(run32(plan, x), common.dct2(x)).max() < F32_TOL
        plan.close()


def test_edge_cases(pkg):
    n = 64
    plan = pkg.Plan(n, self_loop_v(n, 0), 1.0)
    # empty batch
    x = torch.zeros((0, n), device="cuda")
    assert plan.forward(x).shape == (0, n)
    # one signal, strided input rows (ldx > n)
    xb = normal_signals(5, 2 * n, seed=1)
    xt = torch.tensor(xb, dtype=torch.float32, device="cuda")[:, :n]
    y = plan.forward(xt).double().cpu().numpy()
    ref = cauchy.transform(cauchy.make_plan(n, self_loop_v(n, 0), 1.0), xb[:, :n])
    assert relerr(y, ref).max() < F32_TOL
    # a view offset by one element (not 16-byte aligned, ld = n + 1) still transforms correctly
    xo = normal_signals(9, n + 1, seed=2)
    big = torch.tensor(xo, dtype=torch.float32, device="cuda")
    y = plan.forward(big[:, 1:]).double().cpu().numpy()
    assert relerr(y, cauchy.transform(cauchy.make_plan(n, self_loop_v(n, 0), 1.0), xo[:, 1:])).max() < F32_TOL
    # a pointer not aligned to the element size is rejected on the host
    with pytest.raises(pkg.DctPlusError) as e:
        pkg.dctplus_execute(plan.handle, pkg.F32, big.data_ptr() + 2, n + 1, big.data_ptr() + 4096,
                            n + 1, 1, 0)
    assert e.value.status == 1
    assert pkg.dctplus_sync_check(0) == 0
    plan.close()


def test_host_buffer_variant_matches_device_variant(pkg):
    for n in (16, 1024):
        x = normal_signals(300, n, seed=9).astype(np.float32)
        plan = pkg.Plan(n, random_unit_v(n), 2.0)
        yd = plan.forward(torch.tensor(x, device="cuda")).cpu().numpy()
        yh = plan.forward_host(x)
        assert np.array_equal(yd, yh)
        plan.close()


def _mixed_plans(pkg, wl):
    plans, index = [], {}
    for n, ups in wl.updates.items():
        for u, (v, rho) in enumerate(ups):
            index[(n, u)] = len(plans)
            plans.append(pkg.Plan(n, v, rho))
    return plans, index


def test_mixed_size_group_matches_oracle(pkg):
    wl = mixed_size_workload(total_rows=1 << 13)
    plans, index = _mixed_plans(pkg, wl)
    group = pkg.Group(plans)
    seg = np.array([[index[(s.n, s.update)], s.offset, s.rows] for s in wl.segments], dtype=np.int64)
    x = torch.tensor(wl.x, device="cuda")
    y = group.forward(x, seg).double().cpu().numpy()
    for s in wl.segments:
        v, rho = wl.updates[s.n][s.update]
        xs = wl.x[s.offset:s.offset + s.rows * s.n].astype(np.float64).reshape(s.rows, s.n)
        ref = cauchy.transform(cauchy.make_plan(s.n, v, rho), xs)
        got = y[s.offset:s.offset + s.rows * s.n].reshape(s.rows, s.n)
        nz = np.linalg.norm(ref, axis=1) > 0
        assert relerr(got[nz], ref[nz]).max() < F32_TOL, (s.n, s.update)
    # host-buffer variant gives the same bytes
    yh = group.forward_host(wl.x, seg)
    assert np.array_equal(yh, y.astype(np.float32))
    assert pkg.dctplus_sync_check(0) == 0
    group.close()
    for p in plans:
        p.close()


def test_mixed_size_full_workload_sampled(pkg):
    """2^20 rows, the launch configuration the benchmark times; sampled rows checked."""
    wl = mixed_size_workload()
    plans, index = _mixed_plans(pkg, wl)
    group = pkg.Group(plans)
    seg = np.array([[index[(s.n, s.update)], s.offset, s.rows] for s in wl.segments], dtype=np.int64)
    x = torch.tensor(wl.x, device="cuda")
    y = group.forward(x, seg).cpu().numpy()
    # the host-buffer path runs in overlapped chunks at this size; same bytes as the device path
    yh = group.forward_host(wl.x, seg)
    assert np.array_equal(yh, y)
    # segments given out of address order, with a gap left untouched in the output
    order = np.arange(len(seg))[::-1]
    gap = seg[3].copy()
    seg2 = np.delete(seg[order], len(seg) - 1 - 3, axis=0)
    yh2 = np.full_like(wl.x, 7.0)
    yh2 = group.forward_host(wl.x, seg2, out=yh2)
    lo, hi = gap[1], gap[1] + gap[2] * plans[gap[0]].n
    assert np.all(yh2[lo:hi] == 7.0)
    mask = np.ones(len(y), dtype=bool)
    mask[lo:hi] = False
    assert np.array_equal(yh2[mask], y[mask])
    rng = np.random.default_rng(11)
    for s in wl.segments:
        v, rho = wl.updates[s.n][s.update]
        rows = np.unique(np.concatenate([rng.choice(s.rows, 64, replace=False), [0, s.rows - 1]]))
        xs = wl.x[s.offset:s.offset + s.rows * s.n].astype(np.float64).reshape(s.rows, s.n)[rows]
        ref = cauchy.transform(cauchy.make_plan(s.n, v, rho), xs)
        got = y[s.offset:s.offset + s.rows * s.n].reshape(s.rows, s.n)[rows].astype(np.float64)
        nz = np.linalg.norm(ref, axis=1) > 0
        assert relerr(got[nz], ref[nz]).max() < F32_TOL, (s.n, s.update)
    assert pkg.dctplus_sync_check(0) == 0
    group.close()
    for p in plans:
        p.close()


@pytest.mark.parametrize("n", [4, 8, 16, 32, 64])
def test_tensor_core_path_tiles_and_tails(pkg, n):
    """Full packed rows go to the tcgen05 kernel, leftovers to the CUDA-core kernel."""
    per = 64 // n  # signals per packed row
    batches = [max(1, per - 1), 128 * per, 128 * per + max(1, per - 1), 129 * per,
               (3 * 152 + 7) * 128 * per + max(1, per // 2)]
    v, rho = random_unit_v(n, seed=7), 1.3
    ref_plan = cauchy.make_plan(n, v, rho)
    plan = pkg.Plan(n, v, rho)
    simt = pkg.Plan(n, v, rho, cauchy_mode=pkg.CAUCHY_SIMT)
    for batch in batches:
        x = normal_signals(batch, n, seed=batch % 1000)
        ref = cauchy.transform(ref_plan, x)
        y = run32(plan, x)
        assert relerr(y, ref).max() < F32_TOL, (n, batch, relerr(y, ref).max())
        ys = run32(simt, x)
        assert relerr(y, ys).max() < 2 * F32_TOL
    assert pkg.dctplus_sync_check(0) == 0
    plan.close()
    simt.close()


def test_tensor_core_path_integer_residuals(pkg):
    """Laplace integer residuals (exact in TF32) through the tensor-core path, all sizes."""
    for n in (4, 8, 16, 32, 64):
        x = laplace_residuals(5000 * n, seed=n).astype(np.float64).reshape(5000, n)
        for v, rho in [(self_loop_v(n, 0), 2.0), (edge_update_v(n, n // 2 - 1, n // 2), -0.5)]:
            ref = cauchy.transform(cauchy.make_plan(n, v, rho), x)
            plan = pkg.Plan(n, v, rho)
            y = run32(plan, x)
            nz = np.linalg.norm(ref, axis=1) > 0
            assert relerr(y[nz], ref[nz]).max() < F32_TOL
            plan.close()


def test_tensor_core_path_mixed_exact_and_inexact_tiles(pkg):
    """Tiles whose samples are all exact in TF32 (x_lo = 0) next to tiles, row blocks and
    single rows with inexact samples, in one launch. The kernel always issues the x_lo
    product; this guards that a tile's x_lo buffer never leaks into the next tile."""
    n = 16
    rows = 128 * 64 // n * 6 + 37  # six full 128-row tiles of packed rows plus a ragged tail
    x = laplace_residuals(rows * n, seed=3).astype(np.float64).reshape(rows, n)
    per_tile = 128 * 64 // n
    x[per_tile:2 * per_tile] += 0.1                       # tile 1: every sample inexact
    x[3 * per_tile + 40] += 1e-3                          # tile 3: one inexact sample
    x[4 * per_tile:5 * per_tile:7, 5] = 1.0 / 3.0         # tile 4: a sparse set of inexact samples
    for v, rho in [(self_loop_v(n, 0), 1.0), (edge_update_v(n, n // 2 - 1, n // 2), -0.5)]:
        ref = cauchy.transform(cauchy.make_plan(n, v, rho), x)
        plan = pkg.Plan(n, v, rho)
        y = run32(plan, x)
        nz = np.linalg.norm(ref, axis=1) > 0
        assert relerr(y[nz], ref[nz]).max() < F32_TOL
        plan.close()
    assert pkg.dctplus_sync_check(0) == 0
