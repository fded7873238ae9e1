"""Seeded input generators for the Fast DCT+ workloads.

Every generator uses NumPy's PCG64 (``numpy.random.default_rng(seed)``), so the
same seed gives the same bytes on x86 and Arm hosts.

Rank-one update vectors follow the two scenarios of Sec. 2.1 (Prop. 2.4):
a self-loop of weight w at vertex i is ``rho = w, v = e_i``; changing the
weight of edge (i, j) by w is ``rho = w, v = e_i - e_j``. Vertex indices are
0-based here, the paper's are 1-based.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SIZES_SMALL = (4, 8, 16, 32, 64)


def normal_signals(batch: int, n: int, seed: int = 0) -> np.ndarray:
    """``batch`` signals of length ``n`` with i.i.d. N(0,1) FP64 samples, row-major."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((batch, n))


def ar1_signals(batch: int, n: int, r: float = 0.99, seed: int = 0) -> np.ndarray:
    """Stationary AR(1) signals x_t = r x_{t-1} + sqrt(1-r^2) e_t with unit variance.

    This is the signal model of the paper's runtime experiment (Fig. 3 caption,
    AR(0.99) signals).
    """
    rng = np.random.default_rng(seed)
    e = rng.standard_normal((batch, n))
    x = np.empty((batch, n))
    x[:, 0] = e[:, 0]
    k = np.sqrt(1.0 - r * r)
    for t in range(1, n):
        x[:, t] = r * x[:, t - 1] + k * e[:, t]
    return x


def laplace_residuals(count: int, scale: float = 12.0, seed: int = 0) -> np.ndarray:
    """Integer prediction residuals: rint(Laplace(0, scale)) clipped to [-255, 255], as FP32."""
    rng = np.random.default_rng(seed)
    v = np.rint(rng.laplace(0.0, scale, size=count))
    return np.clip(v, -255.0, 255.0).astype(np.float32)


def random_unit_v(n: int, seed: int = 1) -> np.ndarray:
    """A dense random unit-norm update vector: g / ||g|| with g ~ N(0, I) in FP64."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(n)
    return g / np.linalg.norm(g)


def self_loop_v(n: int, vertex: int = 0) -> np.ndarray:
    """Update vector of a self-loop at ``vertex`` (scenario (i) of Sec. 2.1)."""
    v = np.zeros(n)
    v[vertex] = 1.0
    return v


def edge_update_v(n: int, i: int, j: int) -> np.ndarray:
    """Update vector of a weight change on edge (i, j) (scenario (ii) of Sec. 2.1)."""
    v = np.zeros(n)
    v[i] = 1.0
    v[j] = -1.0
    return v


@dataclass
class MixedSegment:
    """One contiguous run of rows that share a block size and a rank-one update."""

    n: int
    update: int  # index into MixedWorkload.updates[n]
    rows: int
    offset: int  # element offset of the first sample in the packed buffer


@dataclass
class MixedWorkload:
    """Mixed block sizes 4..64 with several updates per size, packed segment by segment."""

    x: np.ndarray  # FP32, all samples of all segments back to back
    segments: list = field(default_factory=list)
    updates: dict = field(default_factory=dict)  # n -> list of (v, rho)

    @property
    def total_rows(self) -> int:
        return sum(s.rows for s in self.segments)

    @property
    def total_samples(self) -> int:
        return int(self.x.size)


def small_size_updates(n: int) -> list:
    """The four rank-one updates used for every block size of the mixed workload.

    Three self-loops at vertex 0 with rho in {0.5, 1, 2} and one weight change
    of rho = -0.5 on the central edge (n/2 - 1, n/2).
    """
    ups = [(self_loop_v(n, 0), r) for r in (0.5, 1.0, 2.0)]
    ups.append((edge_update_v(n, n // 2 - 1, n // 2), -0.5))
    return ups


def mixed_size_workload(total_rows: int = 1 << 20, sizes=SIZES_SMALL,
                        seed_x: int = 0, seed_sizes: int = 2,
                        seed_updates: int = 3) -> MixedWorkload:
    """Video-residual-shaped rows of mixed length.

    Each of ``total_rows`` rows draws its length uniformly from ``sizes`` (seed 2)
    and one of four updates uniformly (seed 3); rows are grouped by
    (size, update) into contiguous segments, and the samples are Laplace
    residuals (seed 0) laid out segment after segment.
    """
    rs = np.random.default_rng(seed_sizes)
    ru = np.random.default_rng(seed_updates)
    size_idx = rs.integers(0, len(sizes), size=total_rows)
    upd = ru.integers(0, 4, size=total_rows)
    counts = np.zeros((len(sizes), 4), dtype=np.int64)
    np.add.at(counts, (size_idx, upd), 1)
    segs = []
    off = 0
    for si, n in enumerate(sizes):
        for u in range(4):
            rows = int(counts[si, u])
            if rows == 0:
                continue
            segs.append(MixedSegment(n=n, update=u, rows=rows, offset=off))
            off += rows * n
    x = laplace_residuals(off, seed=seed_x)
    updates = {n: small_size_updates(n) for n in sizes}
    return MixedWorkload(x=x, segments=segs, updates=updates)
