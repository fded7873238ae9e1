"""The accuracy sweep behind Table 1: 10000 AR(0.99) signals per size, the three graphs of the
runtime experiment (edge (2,3) update, self-loop at vertex 1, edge (3,5) addition; 1-based as
printed, weight 1.5), GPU output against the FP64 oracle, SNR in dB averaged over signals."""
import os

import numpy as np
import pytest

from oracle import cauchy
from synthetic import ar1_signals, edge_update_v, self_loop_v

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = (8, 16, 32, 64, 96, 128, 160, 192, 224, 256)


def table1():
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_snr.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    return {int(r[0]): (float(r[1]), float(r[2]), float(r[3])) for r in rows}


def snr_db(y, ref):
    return float(np.mean(10 * np.log10(np.sum(ref ** 2, 1) / np.sum((y - ref) ** 2, 1))))


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_08970_gb300 as p
    from paper_2409_08970_gb300 import build
    build.build()
    return p


def test_snr_sweep_matches_or_beats_table1(pkg):
    printed = table1()
    lines = ["n    graph  FP64 GPU dB  FP32 GPU dB  Table 1 dB"]
    for n in SIZES:
        x = ar1_signals(10000, n, 0.99, seed=0)
        graphs = [("EU", edge_update_v(n, 1, 2)), ("SLA", self_loop_v(n, 0)), ("EA", edge_update_v(n, 2, 4))]
        for gi, (name, v) in enumerate(graphs):
            ref = cauchy.transform(cauchy.make_plan(n, v, 1.5), x)
            plan = pkg.Plan(n, v, 1.5)
            y64 = plan.forward(torch.tensor(x, dtype=torch.float64, device="cuda")).cpu().numpy()
            s64 = snr_db(y64, ref)
            y32 = plan.forward(torch.tensor(x, dtype=torch.float32, device="cuda")).double().cpu().numpy()
            s32 = snr_db(y32, ref)
            assert s32 >= 100.0, (n, name, s32)
            plan.close()
            if n in printed:
                assert s64 >= printed[n][gi], (n, name, s64, printed[n][gi])
            assert s64 >= 200.0, (n, name, s64)
            lines.append(f"{n:<4d} {name:<5s}  {s64:11.1f}  {s32:11.1f}  "
                         f"{printed[n][gi] if n in printed else float('nan'):10.1f}")
    print("\n" + "\n".join(lines))
    assert pkg.dctplus_sync_check(0) == 0
