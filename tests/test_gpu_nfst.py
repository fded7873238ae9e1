"""The paper's trigonometric route on the GPU (cauchy mode DCTPLUS_CAUCHY_NFST) against the
oracle's version of the same route and the Cauchy-formula oracle. Powers of two from 16 to 8192
run the O(n log n) kernel (FFT-based DCT-II and DST-I, nonuniform sine transform); other
lengths up to 1024 and n = 8 run the direct-sum kernel."""
import numpy as np
import pytest
import scipy.fft

from oracle import cauchy, nfst_route
from synthetic import edge_update_v, normal_signals, random_unit_v, self_loop_v

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


def conditioning(op):
    mu = op.mu
    inside = (mu > 0) & (mu < 4)
    th = 2 * np.arctan2(np.sqrt(mu[inside]), np.sqrt(4 - mu[inside]))
    return np.abs(np.sin(op.n * th)).min() if inside.any() else 1.0


def check_route(pkg, n, v, rho, signals):
    op = cauchy.make_plan(n, v, rho)
    x = normal_signals(signals, n, seed=n)
    plan = pkg.Plan(n, v, rho, cauchy_mode=pkg.CAUCHY_NFST)
    assert plan.cauchy_mode == pkg.CAUCHY_NFST
    y = plan.forward(torch.tensor(x, dtype=torch.float64, device="cuda")).cpu().numpy()
    same = nfst_route.transform(op, x)
    ref = cauchy.transform(op, x)
    tol = max(1e-12, 1e-13 * n / conditioning(op))
    e_same = np.linalg.norm(y - same, axis=1) / np.linalg.norm(same, axis=1)
    e_ref = np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert e_same.max() < tol, (n, rho, e_same.max(), tol)
    assert e_ref.max() < 2 * tol, (n, rho, e_ref.max(), tol)
    y32 = plan.forward(torch.tensor(x, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    e32 = np.linalg.norm(y32 - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert e32.max() < max(1e-6, 2 * tol), (n, rho, e32.max())
    plan.close()
    return op


@pytest.mark.parametrize("n", [8, 16, 64, 100, 256, 1024, 2048])
def test_route_matches_oracles(pkg, n):
    cases = [(random_unit_v(n, seed=7), 0.7), (random_unit_v(n, seed=8), -0.3), (self_loop_v(n, 0), 2.0)]
    if n >= 16:
        cases.append((edge_update_v(n, n // 2 - 1, n // 2), -0.5))
    for v, rho in cases:
        check_route(pkg, n, v, rho, 50)
    assert pkg.dctplus_sync_check(0) == 0


def test_fast_route_at_the_largest_length(pkg):
    """n = 8192: one CTA of 512 threads per signal, the 147 KB shared buffer, a root beyond 4."""
    op = check_route(pkg, 8192, random_unit_v(8192, seed=7), 0.7, 6)
    assert (op.mu >= 4.0).any()
    assert pkg.dctplus_sync_check(0) == 0


def test_route_conditioning_next_to_a_pole(pkg):
    """A tiny weight z_10 puts a root next to pole 10: the route loses digits there, the
    pole + offset form of the other modes does not."""
    n = 64
    z = np.random.default_rng(2).standard_normal(n)
    z[10] = 1e-5
    v = scipy.fft.idct(z, norm="ortho")
    v /= np.linalg.norm(v)
    op = cauchy.make_plan(n, v, 1.0)
    x = normal_signals(20, n, seed=1)
    ref = cauchy.transform(op, x)
    route = pkg.Plan(n, v, 1.0, cauchy_mode=pkg.CAUCHY_NFST)
    simt = pkg.Plan(n, v, 1.0, cauchy_mode=pkg.CAUCHY_SIMT)
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    e_route = np.abs(route.forward(xd).cpu().numpy() - ref).max()
    e_cauchy = np.abs(simt.forward(xd).cpu().numpy() - ref).max()
    assert e_route > 1e3 * e_cauchy and e_cauchy < 1e-12
    route.close()
    simt.close()


def test_route_size_limit(pkg):
    """Beyond 1024 only powers of two up to 8192 (the fast kernel's shared buffer) are taken."""
    for n in (1536, 16384):
        with pytest.raises(pkg.DctPlusError) as e:
            pkg.Plan(n, self_loop_v(n, 0), 1.0, cauchy_mode=pkg.CAUCHY_NFST)
        assert e.value.status == 2


def test_fast_route_edge_cases(pkg):
    """The O(n log n) kernel on an empty batch, on input views that are strided and not
    16-byte aligned (ld = n + 3, offset by three elements), with rho = 0 (every row deflated,
    so the result is the DCT-II itself), and on a batch much larger than its grid (each CTA
    loops over many signals)."""
    for n in (64, 1024):
        v = random_unit_v(n, seed=5)
        op = cauchy.make_plan(n, v, 0.9)
        plan = pkg.Plan(n, v, 0.9, cauchy_mode=pkg.CAUCHY_NFST)
        assert plan.forward(torch.zeros((0, n), dtype=torch.float64, device="cuda")).shape == (0, n)
        xo = normal_signals(7, n + 3, seed=4)
        big = torch.tensor(xo, dtype=torch.float64, device="cuda")
        y = plan.forward(big[:, 3:]).cpu().numpy()
        ref = cauchy.transform(op, xo[:, 3:])
        tol = max(1e-12, 1e-13 * n / conditioning(op))
        e = np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert e.max() < 2 * tol, (n, e.max())
        plan.close()
        zero = pkg.Plan(n, v, 0.0, cauchy_mode=pkg.CAUCHY_NFST)
        x = normal_signals(9, n, seed=6)
        y = zero.forward(torch.tensor(x, dtype=torch.float64, device="cuda")).cpu().numpy()
        assert np.abs(y - scipy.fft.dct(x, norm="ortho", axis=1)).max() < 1e-13 * np.abs(x).sum(axis=1).max()
        zero.close()
    n, batch = 16, 20000
    v = random_unit_v(n, seed=9)
    op = cauchy.make_plan(n, v, 1.3)
    plan = pkg.Plan(n, v, 1.3, cauchy_mode=pkg.CAUCHY_NFST)
    x = normal_signals(batch, n, seed=10)
    y = plan.forward(torch.tensor(x, dtype=torch.float64, device="cuda")).cpu().numpy()
    ref = cauchy.transform(op, x)
    tol = max(1e-12, 1e-13 * n / conditioning(op))
    assert (np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)).max() < 2 * tol
    plan.close()
    assert pkg.dctplus_sync_check(0) == 0


@pytest.mark.parametrize("n", [1024, 4096])
def test_fast_route_full_batch_sampled(pkg, n):
    """The route in the benchmark's launch configuration (batch 4096, FP32 data, two updates),
    checked on sampled signals against the oracle's route and the Cauchy formula."""
    batch = 4096
    x = normal_signals(batch, n, seed=0)
    rng = np.random.default_rng(5)
    sig = np.sort(rng.choice(batch, 12, replace=False))
    for rho in (-0.3, 2.0):
        v = random_unit_v(n)
        op = cauchy.make_plan(n, v, rho)
        plan = pkg.Plan(n, v, rho, cauchy_mode=pkg.CAUCHY_NFST)
        y = plan.forward(torch.tensor(x, dtype=torch.float32, device="cuda")).double().cpu().numpy()[sig]
        tol = max(1e-12, 1e-13 * n / conditioning(op))
        same = nfst_route.transform(op, x[sig])
        ref = cauchy.transform(op, x[sig])
        e_same = np.linalg.norm(y - same, axis=1) / np.linalg.norm(same, axis=1)
        e_ref = np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert e_same.max() < max(1e-6, 2 * tol), (n, rho, e_same.max())  # FP32 output rounding
        assert e_ref.max() < max(1e-6, 2 * tol), (n, rho, e_ref.max())
        plan.close()
    assert pkg.dctplus_sync_check(0) == 0
