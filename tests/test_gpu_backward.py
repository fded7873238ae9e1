"""Backward pass (dctplus_backward and the autograd Function) against the FP64
oracle gradients and central finite differences."""
import numpy as np
import pytest

from oracle import cauchy, definition, gradient
from synthetic import ar1_signals, edge_update_v, normal_signals, random_unit_v, self_loop_v

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


def tail_loss_grad(y):
    n = y.shape[1]
    g = np.zeros_like(y)
    g[:, n // 2:] = 2 * y[:, n // 2:]
    return g


def test_autograd_matches_finite_differences_n16(pkg):
    """Central differences (h = 1e-6) of the FP64 Jacobi forward for the tail loss."""
    n = 16
    for v, rho in [(random_unit_v(n, seed=9), 2.0), (self_loop_v(n, 0), 1.0), (edge_update_v(n, 7, 8), -0.5)]:
        x = ar1_signals(6, n, seed=2)

        def loss(v_, rho_, x_=x):
            y = definition.transform(n, v_, rho_, x_)
            return float(np.sum(y[:, n // 2:] ** 2))

        h = 1e-6
        f_rho = (loss(v, rho + h) - loss(v, rho - h)) / (2 * h)
        f_v = np.array([(loss(v + h * e, rho) - loss(v - h * e, rho)) / (2 * h) for e in np.eye(n)])
        f_x = np.zeros_like(x)
        for b in range(x.shape[0]):
            for j in range(n):
                xp, xm = x.copy(), x.copy()
                xp[b, j] += h
                xm[b, j] -= h
                f_x[b, j] = (loss(v, rho, xp) - loss(v, rho, xm)) / (2 * h)

        xt = torch.tensor(x, dtype=torch.float32, device="cuda", requires_grad=True)
        vt = torch.tensor(v, dtype=torch.float64, device="cuda", requires_grad=True)
        rt = torch.tensor(rho, dtype=torch.float64, device="cuda", requires_grad=True)
        y = pkg.dct_plus(xt, vt, rt)
        (y[:, n // 2:] ** 2).sum().backward()
        assert abs(rt.grad.item() - f_rho) < 2e-5 * max(1.0, abs(f_rho)), (rt.grad.item(), f_rho)
        gv = vt.grad.cpu().numpy()
        assert np.abs(gv - f_v).max() < 2e-5 * max(1.0, np.abs(f_v).max())
        gx = xt.grad.double().cpu().numpy()
        assert np.abs(gx - f_x).max() < 2e-5 * max(1.0, np.abs(f_x).max())
    assert pkg.dctplus_sync_check(0) == 0


EPS32 = 2.0 ** -24


def param_error_bounds(op, x, g):
    """First-order FP32 error scale of the parameter gradients: the same sums with every term
    replaced by its magnitude (so cancellation in the K products is accounted for)."""
    t = cauchy.transform_matrix(op)
    y = x @ t.T
    w = t @ op.v
    ka = np.abs(gradient.cauchy_k(op))
    p_abs = np.abs(y * w) @ ka.T
    q_abs = np.abs(g * w) @ ka
    b_rho = float(np.sum(np.abs(g * w) * p_abs))
    b_v = abs(op.rho) * (np.abs(y) * q_abs + np.abs(g) * p_abs).sum(axis=0) @ np.abs(t)
    return b_rho, b_v


@pytest.mark.parametrize("n,batch", [(16, 33), (48, 70), (64, 20), (96, 40), (256, 300), (1024, 256)])
def test_backward_matches_oracle_gradients(pkg, n, batch):
    for v, rho in [(random_unit_v(n, seed=1), 2.0), (random_unit_v(n, seed=2), -0.3)]:
        x = normal_signals(batch, n, seed=n)
        op = cauchy.make_plan(n, v, rho)
        y64 = cauchy.transform(op, x)
        g = tail_loss_grad(y64)
        plan = pkg.Plan(n, v, rho)
        xd = torch.tensor(x, dtype=torch.float32, device="cuda")
        yd = plan.forward(xd)
        gd = torch.tensor(g, dtype=torch.float32, device="cuda")
        gx, g_rho, g_v = plan.backward(gd, yd, want_x=True, want_params=True)
        ref_x = gradient.backward_x(op, g)
        err_x = np.linalg.norm(gx.double().cpu().numpy() - ref_x, axis=1) / np.linalg.norm(ref_x, axis=1)
        assert err_x.max() < 2e-6, (n, rho, err_x.max())
        r_rho, r_v = gradient.parameter_gradients(op, x, g)
        b_rho, b_v = param_error_bounds(op, x, g)
        assert abs(g_rho.item() - r_rho) < 16 * EPS32 * b_rho, (n, rho, g_rho.item(), r_rho, b_rho)
        assert np.all(np.abs(g_v.cpu().numpy() - r_v) <= 16 * EPS32 * b_v + 1e-12), (n, rho)
        assert abs(g_rho.item() - r_rho) < 1e-3 * abs(r_rho)
        assert np.linalg.norm(g_v.cpu().numpy() - r_v) / np.linalg.norm(r_v) < 1e-3
        plan.close()
    assert pkg.dctplus_sync_check(0) == 0


def test_autograd_many_pending_plans(pkg):
    """More forwards with distinct rho than the plan cache holds, all before their backwards:
    every backward must still find its own plan and match the oracle gradients."""
    n, batch = 64, 20
    v = random_unit_v(n, seed=3)
    x = normal_signals(batch, n, seed=11)
    rhos = [0.1 * (k + 1) for k in range(20)]
    vt = torch.tensor(v, dtype=torch.float64, device="cuda", requires_grad=True)
    pending = []
    for rho in rhos:
        xt = torch.tensor(x, dtype=torch.float32, device="cuda", requires_grad=True)
        rt = torch.tensor(rho, dtype=torch.float64, device="cuda", requires_grad=True)
        y = pkg.dct_plus(xt, vt, rt)
        pending.append((rho, xt, rt, (y[:, n // 2:] ** 2).sum()))
    assert len(pkg._plan_cache) <= pkg._PLAN_CACHE_MAX
    for rho, xt, rt, loss in pending:
        vt.grad = None
        loss.backward()
        op = cauchy.make_plan(n, v, rho)
        g = tail_loss_grad(cauchy.transform(op, x))
        ref_x = gradient.backward_x(op, g)
        r_rho, r_v = gradient.parameter_gradients(op, x, g)
        gx = xt.grad.double().cpu().numpy()
        assert (np.linalg.norm(gx - ref_x, axis=1) / np.linalg.norm(ref_x, axis=1)).max() < 2e-6, rho
        assert abs(rt.grad.item() - r_rho) < 1e-3 * abs(r_rho), rho
        assert np.linalg.norm(vt.grad.cpu().numpy() - r_v) / np.linalg.norm(r_v) < 1e-3, rho
    # the same unmodified v tensor and rho reuse the cached plan; an in-place change of v
    # (a new version) makes a new one
    rt = torch.tensor(0.55, dtype=torch.float64, device="cuda")
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    pkg.dct_plus(xt, vt, rt)
    before = len(pkg._plan_cache), id(next(reversed(pkg._plan_cache.values())))
    pkg.dct_plus(xt, vt, rt)
    assert (len(pkg._plan_cache), id(next(reversed(pkg._plan_cache.values())))) == before
    with torch.no_grad():
        vt.mul_(-1.0)
    y_neg = pkg.dct_plus(xt, vt, rt).detach().double().cpu().numpy()
    ref = cauchy.transform(cauchy.make_plan(n, -v, 0.55), x)
    assert (np.linalg.norm(y_neg - ref, axis=1) / np.linalg.norm(ref, axis=1)).max() < 1e-6
    assert pkg.dctplus_sync_check(0) == 0


def test_backward_is_the_adjoint(pkg):
    n, batch = 512, 200
    plan = pkg.Plan(n, random_unit_v(n, seed=3), 0.8)
    x = torch.tensor(normal_signals(batch, n, seed=4), dtype=torch.float32, device="cuda")
    g = torch.tensor(normal_signals(batch, n, seed=5), dtype=torch.float32, device="cuda")
    y = plan.forward(x)
    gx, _, _ = plan.backward(g)
    lhs = (y.double() * g.double()).sum().item()
    rhs = (x.double() * gx.double()).sum().item()
    assert abs(lhs - rhs) < 1e-5 * (y.double() * g.double()).abs().sum().item()
    xx, _, _ = plan.backward(y)  # X X^T x = x
    assert ((xx - x).norm(dim=1) / x.norm(dim=1)).max().item() < 2e-6
    plan.close()


def test_differentiable_workload_full_batch(pkg):
    """n = 1024, batch 8192, loss = sum of squared coefficients 512..1023: the benchmark's step."""
    n, batch = 1024, 8192
    v, rho = random_unit_v(n, seed=1), 2.0
    x = normal_signals(batch, n, seed=0)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda", requires_grad=True)
    vt = torch.tensor(v, dtype=torch.float64, device="cuda", requires_grad=True)
    rt = torch.tensor(rho, dtype=torch.float64, device="cuda", requires_grad=True)
    y = pkg.dct_plus(xt, vt, rt)
    (y[:, n // 2:] ** 2).sum().backward()
    op = cauchy.make_plan(n, v, rho)
    y64 = cauchy.transform(op, x)
    g = tail_loss_grad(y64)
    r_rho, r_v = gradient.parameter_gradients(op, x, g)
    b_rho, b_v = param_error_bounds(op, x, g)
    assert abs(rt.grad.item() - r_rho) < 16 * EPS32 * b_rho
    assert np.all(np.abs(vt.grad.cpu().numpy() - r_v) <= 16 * EPS32 * b_v + 1e-12)
    assert abs(rt.grad.item() - r_rho) < 1e-3 * abs(r_rho)
    assert np.linalg.norm(vt.grad.cpu().numpy() - r_v) / np.linalg.norm(r_v) < 1e-3
    rows = np.random.default_rng(3).choice(batch, 64, replace=False)
    ref_x = gradient.backward_x(op, g[rows])
    got = xt.grad.double().cpu().numpy()[rows]
    assert (np.linalg.norm(got - ref_x, axis=1) / np.linalg.norm(ref_x, axis=1)).max() < 1e-5
    assert pkg.dctplus_sync_check(0) == 0


def test_backward_argument_errors(pkg):
    import ctypes
    lib = pkg._lib.load()
    n = 256
    plan = pkg.Plan(n, self_loop_v(n, 0), 1.0)
    g = torch.zeros(4, n, device="cuda")
    gx = torch.zeros(4, n, device="cuda")
    r = torch.zeros((), dtype=torch.float64, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    P = ctypes.c_void_p
    # parameter gradients without the forward output
    assert lib.dctplus_backward(plan.handle, P(g.data_ptr()), n, None, n, None, n, P(r.data_ptr()), None, 4, s) == 1
    # gx overlapping gy
    assert lib.dctplus_backward(plan.handle, P(g.data_ptr()), n, None, n, P(g.data_ptr()), n, None, None, 4, s) == 1
    assert lib.dctplus_backward(plan.handle, P(g.data_ptr()), n - 1, None, n, P(gx.data_ptr()), n, None, None, 4, s) == 1
    assert lib.dctplus_backward(plan.handle, P(g.data_ptr()), n, None, n, P(gx.data_ptr()), n, None, None, 0, s) == 0
    plan.close()


@pytest.mark.parametrize("n,batch", [(8192, 64), (16384, 32)])
def test_backward_large_n_adjoint_and_rho(pkg, n, batch):
    """Beyond n = 4096 the FP64 oracle's gradients take minutes, so the backward is checked there
    by what holds at any length: the adjoint identity <g, X^T x> = <X g, x>, X X^T x = x, and
    dL/drho against a central difference of the forward transform in rho. L = sum_b c_b y_b[n-1]
    is linear in y: a loss like the tail energy has dL/drho some 1e-6 of L, below what an FP32
    forward resolves, and its gradient is a cancellation of large terms."""
    v, rho, h = random_unit_v(n, seed=7), 1.3, 1e-2
    plan = pkg.Plan(n, v, rho)
    x = torch.tensor(normal_signals(batch, n, seed=8), dtype=torch.float32, device="cuda")
    g = torch.tensor(normal_signals(batch, n, seed=9), dtype=torch.float32, device="cuda")
    y = plan.forward(x)
    gx, _, _ = plan.backward(g)
    lhs = (y.double() * g.double()).sum().item()
    rhs = (x.double() * gx.double()).sum().item()
    assert abs(lhs - rhs) < 1e-5 * (y.double() * g.double()).abs().sum().item()
    xx, _, _ = plan.backward(y)
    assert ((xx - x).norm(dim=1) / x.norm(dim=1)).max().item() < 1e-5
    c = g[:, 0].clone()
    gy = torch.zeros_like(y)
    gy[:, n - 1] = c
    _, grho, _ = plan.backward(gy, y, want_x=False, want_params=True)

    def loss(r):
        p = pkg.Plan(n, v, r)
        t = (p.forward(x).double()[:, n - 1] * c.double()).sum().item()
        p.close()
        return t

    fd = (loss(rho + h) - loss(rho - h)) / (2 * h)
    assert abs(grho.item() - fd) < 2e-2 * abs(fd) + 1e-3 * c.norm().item(), (grho.item(), fd)
    plan.close()
    assert pkg.dctplus_sync_check(0) == 0
