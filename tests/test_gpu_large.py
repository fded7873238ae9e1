"""Large-n paths against the FP64 oracle: dense split-TF32 tensor-core Cauchy
product, the CUDA-core product, and the dense-GFT comparison baseline."""
import numpy as np
import pytest

from oracle import cauchy
from synthetic import edge_update_v, normal_signals, random_unit_v, self_loop_v

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32_TOL = 1e-6


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_08970_gb300 as p
    from paper_2409_08970_gb300 import build
    build.build()
    return p


def relerr(y, ref):
    return np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)


def run32(plan, x):
    return plan.forward(torch.tensor(x, dtype=torch.float32, device="cuda")).double().cpu().numpy()


@pytest.mark.parametrize("n", [128, 256, 1024, 4096])
def test_dense_tensor_core_mode_matches_oracle(pkg, n):
    batch = 300 if n <= 1024 else 130  # ragged: not a multiple of the 128-row tile
    for v, rho in [(random_unit_v(n), -0.3), (random_unit_v(n), 2.0), (edge_update_v(n, n // 2 - 1, n // 2), -0.5)]:
        x = normal_signals(batch, n, seed=n)
        ref = cauchy.transform(cauchy.make_plan(n, v, rho), x)
        plan = pkg.Plan(n, v, rho, cauchy_mode=pkg.CAUCHY_DENSE)
        assert plan.cauchy_mode == pkg.CAUCHY_DENSE
        err = relerr(run32(plan, x), ref)
        assert err.max() < F32_TOL, (n, rho, err.max())
        plan.close()
    assert pkg.dctplus_sync_check(0) == 0


def test_dense_and_cuda_core_modes_agree(pkg):
    n, batch = 512, 257
    v = random_unit_v(n)
    x = normal_signals(batch, n, seed=1)
    a = pkg.Plan(n, v, 2.0, cauchy_mode=pkg.CAUCHY_DENSE)
    b = pkg.Plan(n, v, 2.0, cauchy_mode=pkg.CAUCHY_SIMT)
    ya, yb = run32(a, x), run32(b, x)
    assert relerr(ya, yb).max() < 2 * F32_TOL
    a.close()
    b.close()


def test_auto_mode_choice(pkg):
    for n, want in [(128, pkg.CAUCHY_DENSE), (512, pkg.CAUCHY_DENSE), (1024, pkg.CAUCHY_HIER), (4096, pkg.CAUCHY_HIER),
                    (16384, pkg.CAUCHY_HIER)]:
        p = pkg.Plan(n, self_loop_v(n, 0), 1.0)
        assert p.cauchy_mode == want, n
        p.close()


def test_unsupported_modes_are_rejected(pkg):
    with pytest.raises(pkg.DctPlusError) as e:
        pkg.Plan(16384, self_loop_v(16384, 0), 1.0, cauchy_mode=pkg.CAUCHY_DENSE)
    assert e.value.status == 2
    with pytest.raises(pkg.DctPlusError) as e:
        pkg.Plan(8192, self_loop_v(8192, 0), 1.0, cauchy_mode=pkg.CAUCHY_DENSE_GFT)
    assert e.value.status == 2


@pytest.mark.parametrize("n", [256, 1024, 2048, 4096])
def test_dense_gft_baseline_matches_oracle(pkg, n):
    batch = 200 if n <= 1024 else 40
    v = random_unit_v(n)
    x = normal_signals(batch, n, seed=3)
    ref = cauchy.transform(cauchy.make_plan(n, v, 2.0), x)
    plan = pkg.Plan(n, v, 2.0, cauchy_mode=pkg.CAUCHY_DENSE_GFT)
    err = relerr(run32(plan, x), ref)
    assert err.max() < F32_TOL, err.max()
    plan.close()


@pytest.mark.parametrize("far_field", [1, 2])
@pytest.mark.parametrize("n", [256, 512, 1024, 4096])
def test_hierarchical_mode_matches_oracle(pkg, n, far_field):
    """Both far-field forms (leaf level, multipole tree) against the Cauchy formula; the
    batch is ragged for the 128-signal GEMM tiles and the 256-signal tree CTAs."""
    batch = 150 if n < 4096 else 300
    cases = [(random_unit_v(n), -0.3), (random_unit_v(n), 2.0), (self_loop_v(n, 0), 1.0),
             (edge_update_v(n, n // 2 - 1, n // 2), -0.5), (edge_update_v(n, 5, 6), 3.0)]
    for v, rho in cases:
        x = normal_signals(batch, n, seed=n + 1)
        ref = cauchy.transform(cauchy.make_plan(n, v, rho), x)
        plan = pkg.Plan(n, v, rho, cauchy_mode=pkg.CAUCHY_HIER, far_field=far_field)
        assert plan.cauchy_mode == pkg.CAUCHY_HIER and plan.far_field == far_field
        err = relerr(run32(plan, x), ref)
        assert err.max() < F32_TOL, (n, rho, far_field, err.max())
        plan.close()
    assert pkg.dctplus_sync_check(0) == 0


def test_far_field_forms_agree_and_default(pkg):
    """The two far-field forms give the same transform; the default is the tree from n = 8192."""
    n, batch = 2048, 200
    v = random_unit_v(n)
    x = normal_signals(batch, n, seed=5)
    a = pkg.Plan(n, v, 2.0, cauchy_mode=pkg.CAUCHY_HIER, far_field=1)
    b = pkg.Plan(n, v, 2.0, cauchy_mode=pkg.CAUCHY_HIER, far_field=2)
    assert relerr(run32(a, x), run32(b, x)).max() < 2 * F32_TOL
    a.close()
    b.close()
    for m, want in [(4096, 1), (8192, 2), (16384, 2)]:
        p = pkg.Plan(m, self_loop_v(m, 0), 1.0, cauchy_mode=pkg.CAUCHY_HIER)
        assert p.far_field == want, m
        p.close()
    d = pkg.Plan(1024, v[:1024] / np.linalg.norm(v[:1024]), 1.0, cauchy_mode=pkg.CAUCHY_DENSE)
    assert d.far_field == 0
    d.close()
    with pytest.raises(pkg.DctPlusError):
        pkg.Plan(1024, self_loop_v(1024, 0), 1.0, cauchy_mode=pkg.CAUCHY_HIER, far_field=3)


@pytest.mark.parametrize("far_field", [1, 2])
def test_hierarchical_unaligned_input_view(pkg, far_field):
    """x as a view offset by one element (ld = n + 1, not 16-byte aligned): the DCT kernel
    reads it with scalar loads instead of float4; the result must not change."""
    n, batch = 1024, 130
    v = random_unit_v(n)
    xo = normal_signals(batch, n + 1, seed=11)
    big = torch.tensor(xo, dtype=torch.float32, device="cuda")
    ref = cauchy.transform(cauchy.make_plan(n, v, 2.0), xo[:, 1:])
    plan = pkg.Plan(n, v, 2.0, cauchy_mode=pkg.CAUCHY_HIER, far_field=far_field)
    y = plan.forward(big[:, 1:]).double().cpu().numpy()
    assert relerr(y, ref).max() < F32_TOL
    y2 = run32(plan, xo[:, 1:])  # the same rows, contiguous and aligned
    assert np.abs(y - y2).max() <= 1e-6 * np.abs(y2).max()
    plan.close()
    assert pkg.dctplus_sync_check(0) == 0


def test_leaf_to_leaf_product_widths_agree(pkg):
    """The leaf-level far field's product runs 64 columns wide when its 128-wide tiles would not
    cover the SMs (small batches) and 128 wide otherwise: n = 2048 with 8192 signals takes the
    wide tiles, the first 1000 of them alone the narrow ones. Both agree with each other and
    with the Cauchy formula on sampled signals."""
    n = 2048
    v = random_unit_v(n)
    x = normal_signals(8192, n, seed=13)
    plan = pkg.Plan(n, v, 2.0, cauchy_mode=pkg.CAUCHY_HIER, far_field=1)
    y_wide = run32(plan, x)
    y_narrow = run32(plan, x[:1000])
    assert np.abs(y_wide[:1000] - y_narrow).max() <= 1e-6 * np.abs(y_narrow).max()
    rng = np.random.default_rng(4)
    sig = np.sort(rng.choice(1000, 24, replace=False))
    ref = cauchy.transform(cauchy.make_plan(n, v, 2.0), x[sig])
    assert relerr(y_wide[sig], ref).max() < F32_TOL
    assert relerr(y_narrow[sig], ref).max() < F32_TOL
    plan.close()
    assert pkg.dctplus_sync_check(0) == 0


def test_hierarchical_n16384_sampled(pkg):
    n, batch = 16384, 512
    v = random_unit_v(n)
    x = normal_signals(batch, n, seed=0)
    for rho in (-0.3, 2.0):
        plan = pkg.Plan(n, v, rho, cauchy_mode=pkg.CAUCHY_HIER)
        y = run32(plan, x)
        rng = np.random.default_rng(7)
        rows = np.unique(np.concatenate([rng.choice(n, 40, replace=False), [0, 1, n - 2, n - 1]]))
        sig = np.sort(rng.choice(batch, 8, replace=False))
        ref = cauchy.transform(cauchy.make_plan(n, v, rho, roots=rows), x[sig], rows=rows)
        err = np.abs(y[sig][:, rows] - ref).max(axis=1) / np.linalg.norm(x[sig], axis=1)
        assert err.max() < F32_TOL, err.max()
        pr = np.abs(np.linalg.norm(y, axis=1) / np.linalg.norm(x, axis=1) - 1)
        assert pr.max() < 2e-6
        plan.close()
    assert pkg.dctplus_sync_check(0) == 0


@pytest.mark.parametrize("n", [1024, 4096])
@pytest.mark.parametrize("far_field", [1, 2])
def test_hierarchical_full_batch_sampled(pkg, far_field, n):
    """n = 1024 and 4096, batch 4096 in the hierarchical mode: the launch configurations the
    benchmark times (at n = 4096 the leaf-to-leaf product takes its 128-wide tiles), checked on
    128 sampled signals against the Cauchy formula."""
    batch = 4096
    v = random_unit_v(n)
    x = normal_signals(batch, n, seed=0)
    for rho in (-0.3, 2.0):
        plan = pkg.Plan(n, v, rho, cauchy_mode=pkg.CAUCHY_HIER, far_field=far_field)
        y = run32(plan, x)
        rng = np.random.default_rng(3)
        sig = np.sort(rng.choice(batch, 128, replace=False))
        ref = cauchy.transform(cauchy.make_plan(n, v, rho), x[sig])
        assert relerr(y[sig], ref).max() < F32_TOL
        plan.close()
    assert pkg.dctplus_sync_check(0) == 0


@pytest.mark.parametrize("n", [1024, 4096])
def test_dense_mode_full_batch_sampled(pkg, n):
    """n = 1024 and 4096, batch 4096: the launch configurations the benchmark times."""
    batch = 4096
    v = random_unit_v(n)
    x = normal_signals(batch, n, seed=0)
    for rho in (-0.3, 2.0):
        plan = pkg.Plan(n, v, rho, cauchy_mode=pkg.CAUCHY_DENSE)
        y = run32(plan, x)
        rng = np.random.default_rng(2)
        sig = np.sort(rng.choice(batch, 128, replace=False))
        ref = cauchy.transform(cauchy.make_plan(n, v, rho), x[sig])
        assert relerr(y[sig], ref).max() < F32_TOL
        pr = np.abs(np.linalg.norm(y, axis=1) / np.linalg.norm(x, axis=1) - 1)
        assert pr.max() < 2e-6
        plan.close()
    assert pkg.dctplus_sync_check(0) == 0


@pytest.mark.parametrize("n", [96, 100, 160, 384, 1000, 3000])
def test_lengths_without_an_fft_match_oracle(pkg, n):
    batch = 70
    for v, rho in [(random_unit_v(n), -0.3), (edge_update_v(n, n // 2 - 1, n // 2), 1.5)]:
        x = normal_signals(batch, n, seed=n)
        ref = cauchy.transform(cauchy.make_plan(n, v, rho), x)
        plan = pkg.Plan(n, v, rho)
        err = relerr(run32(plan, x), ref)
        assert err.max() < F32_TOL, (n, rho, err.max())
        plan.close()
    assert pkg.dctplus_sync_check(0) == 0


def run_multi(pkg, plans, x):
    """dctplus_execute_multi over FP32 signals x: a [batch, len(plans) n] array."""
    n = plans[0].n
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    y = torch.empty((x.shape[0], len(plans) * n), dtype=torch.float32, device="cuda")
    pkg.dctplus_execute_multi([p.handle for p in plans], xd.data_ptr(), n, y.data_ptr(), len(plans) * n,
                              x.shape[0], torch.cuda.current_stream().cuda_stream)
    return y.double().cpu().numpy()


@pytest.mark.parametrize("count", [2, 3])
@pytest.mark.parametrize("mode", ["hier_leaf", "hier_tree", "dense"])
@pytest.mark.parametrize("n", [256, 1024, 4096])
def test_execute_multi_matches_plan_by_plan(pkg, n, mode, count):
    """Several updates over the same signals in one call: the hierarchical plans share one DCT-II
    (their moments and dense rows formed from the same s), the dense plans share it before their
    products. The first two plans have the same v, so their far field is formed once; with two
    or three plans the sets hold one or two far fields. Each plan's block equals its own
    dctplus_execute, and the first agrees with the Cauchy formula; the batch is ragged for every
    tile shape."""
    cm = pkg.CAUCHY_DENSE if mode == "dense" else pkg.CAUCHY_HIER
    far = {"hier_leaf": 1, "hier_tree": 2, "dense": 0}[mode]
    cases = [(random_unit_v(n, seed=3), -0.3), (random_unit_v(n, seed=3), 2.0), (self_loop_v(n, 0), 0.7)]
    plans = [pkg.Plan(n, v, rho, cauchy_mode=cm, far_field=far) for v, rho in cases[:count]]
    x = normal_signals(150, n, seed=17)
    y = run_multi(pkg, plans, x)
    for k, p in enumerate(plans):
        yk = run32(p, x)
        assert np.abs(y[:, k * n:(k + 1) * n] - yk).max() <= 1e-6 * np.abs(yk).max(), (n, mode, k)
    v, rho = cases[0]
    ref = cauchy.transform(cauchy.make_plan(n, v, rho), x[:20])
    assert relerr(y[:20, :n], ref).max() < F32_TOL
    for p in plans:
        p.close()
    assert pkg.dctplus_sync_check(0) == 0


def test_execute_multi_groups_mixed_sets_and_errors(pkg):
    """Five hierarchical plans take two groups (one DCT per group of four); a set mixing the
    dense and the hierarchical mode runs plan by plan; bad arguments are refused on the host."""
    n = 1024
    rhos = (-0.3, 0.4, 0.9, 2.0, 3.5)
    plans = [pkg.Plan(n, random_unit_v(n, seed=5), r, cauchy_mode=pkg.CAUCHY_HIER) for r in rhos]
    x = normal_signals(130, n, seed=19)
    y = run_multi(pkg, plans, x)
    for k, p in enumerate(plans):
        yk = run32(p, x)
        assert np.abs(y[:, k * n:(k + 1) * n] - yk).max() <= 1e-6 * np.abs(yk).max(), k
    twice = [plans[1], plans[2], plans[1]]  # a handle given twice runs plan by plan
    y = run_multi(pkg, twice, x)
    for k, p in enumerate(twice):
        yk = run32(p, x)
        assert np.abs(y[:, k * n:(k + 1) * n] - yk).max() <= 1e-6 * np.abs(yk).max(), k
    mixed = [plans[0], pkg.Plan(n, random_unit_v(n, seed=6), 1.0, cauchy_mode=pkg.CAUCHY_DENSE)]
    y = run_multi(pkg, mixed, x)
    for k, p in enumerate(mixed):
        yk = run32(p, x)
        assert np.abs(y[:, k * n:(k + 1) * n] - yk).max() <= 1e-6 * np.abs(yk).max(), k
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    yd = torch.empty((x.shape[0], 2 * n), dtype=torch.float32, device="cuda")
    sh = torch.cuda.current_stream().cuda_stream
    with pytest.raises(pkg.DctPlusError) as e:  # row stride below count * n
        pkg.dctplus_execute_multi([p.handle for p in mixed], xd.data_ptr(), n, yd.data_ptr(), n, x.shape[0], sh)
    assert e.value.status == 1
    other = pkg.Plan(512, random_unit_v(512), 1.0)
    with pytest.raises(pkg.DctPlusError) as e:  # lengths differ
        pkg.dctplus_execute_multi([plans[0].handle, other.handle], xd.data_ptr(), n, yd.data_ptr(), 2 * n,
                                  x.shape[0], sh)
    assert e.value.status == 1
    for p in plans + mixed[1:] + [other]:
        p.close()
    assert pkg.dctplus_sync_check(0) == 0


@pytest.mark.parametrize("far_field", [1, 2])
def test_execute_multi_in_a_cuda_graph(pkg, far_field):
    """The plans after the first run their products on side streams forked from the caller's
    stream; captured into a CUDA graph (after a first call on that stream, which sizes the
    workspaces and creates the side streams), the replays give the plan-by-plan results on
    fresh inputs."""
    n, batch = 1024, 300
    plans = [pkg.Plan(n, random_unit_v(n, seed=8), r, cauchy_mode=pkg.CAUCHY_HIER, far_field=far_field)
             for r in (-0.3, 2.0, 0.6)]
    x = torch.tensor(normal_signals(batch, n, seed=21), dtype=torch.float32, device="cuda")
    y = torch.zeros((batch, 3 * n), dtype=torch.float32, device="cuda")
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream
    handles = [p.handle for p in plans]
    with torch.cuda.stream(stream):
        pkg.dctplus_execute_multi(handles, x.data_ptr(), n, y.data_ptr(), 3 * n, batch, sh)
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        pkg.dctplus_execute_multi(handles, x.data_ptr(), n, y.data_ptr(), 3 * n, batch, sh)
    for seed in (22, 23):
        xh = normal_signals(batch, n, seed=seed)
        x.copy_(torch.tensor(xh, dtype=torch.float32))
        y.zero_()
        g.replay()
        torch.cuda.synchronize()
        got = y.double().cpu().numpy()
        for k, p in enumerate(plans):
            yk = run32(p, xh)
            assert np.abs(got[:, k * n:(k + 1) * n] - yk).max() <= 1e-6 * np.abs(yk).max(), (seed, k)
    del g
    for p in plans:
        p.close()
    assert pkg.dctplus_sync_check(0) == 0


@pytest.mark.parametrize("far_field", [1, 2])
def test_execute_multi_shared_far_field_and_slot_collisions(pkg, far_field):
    """Updates that differ in rho only share z, so one far field serves them all; each plan keeps
    its dense rows in its own pair of slots, taken in turn from sixteen. Seventeen plans made one
    after another: the first and the last have the same slots and so form their far fields apart,
    the first two share one. Every block equals the plan's own dctplus_execute."""
    n = 256
    v = random_unit_v(n, seed=12)
    plans = [pkg.Plan(n, v, 0.1 + 0.2 * i, cauchy_mode=pkg.CAUCHY_HIER, far_field=far_field) for i in range(17)]
    x = normal_signals(140, n, seed=23)
    for sel in ([0, 1], [0, 16], [0, 16, 1, 2]):
        chosen = [plans[i] for i in sel]
        y = run_multi(pkg, chosen, x)
        for k, p in enumerate(chosen):
            yk = run32(p, x)
            assert np.abs(y[:, k * n:(k + 1) * n] - yk).max() <= 1e-6 * np.abs(yk).max(), (sel, k)
    ref = cauchy.transform(cauchy.make_plan(n, v, 0.1 + 0.2 * 16), x[:16])
    assert relerr(run_multi(pkg, [plans[0], plans[16]], x)[:16, n:], ref).max() < F32_TOL
    for p in plans:
        p.close()
    assert pkg.dctplus_sync_check(0) == 0
