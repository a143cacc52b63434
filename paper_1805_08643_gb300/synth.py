"""Seeded synthetic workloads (random draws only; no arithmetic of the method).

The paper's inputs are synthetic by construction (tanh droplets and slabs in
periodic boxes, Sec. IV).  This module draws the random parameters of the
larger workloads so that the CUDA path, the tests and the benchmark see the
same inputs for a given seed.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SEED = 1805


def random_droplets(box: int = 512, n_per_axis: int = 3, r_lo: float = 12.0, r_hi: float = 40.0,
                    jitter: float = 40.0, seed: int = SEED):
    """Droplets on a jittered n^3 lattice of a periodic box: (centres (n^3, 3), radii (n^3,))."""
    rng = np.random.default_rng(seed)
    cell = box / n_per_axis
    idx = np.stack(np.meshgrid(*[np.arange(n_per_axis)] * 3, indexing="ij"), -1).reshape(-1, 3)
    centres = (idx + 0.5) * cell + rng.uniform(-jitter, jitter, idx.shape)
    radii = rng.uniform(r_lo, r_hi, len(idx))
    return np.mod(centres, box), radii


@dataclass
class BoxSpec:
    edge: int
    radius: float
    T_over_Tc: float


def batched_boxes(n: int = 512, edges=(32, 48, 64, 96), t_lo=0.6, t_hi=0.9, seed: int = SEED):
    """Independent periodic boxes, each a centred droplet with R ~ U[6, edge/3]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        e = int(rng.choice(edges))
        out.append(BoxSpec(e, float(rng.uniform(6.0, e / 3.0)), float(rng.uniform(t_lo, t_hi))))
    return out


@dataclass
class JobSpec:
    arrival: float  # seconds after the stream starts
    edge: int
    kind: str       # "droplet" | "flat"
    T_over_Tc: float
    operator: str   # "orth" | "nonorth"


def job_stream(n: int, rate_per_s: float, edge_lo=48, edge_hi=192, t_lo=0.6, t_hi=0.9,
               seed: int = SEED):
    """Poisson arrivals of droplet / flat-interface jobs with random box sizes."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, n))
    jobs = []
    for k in range(n):
        jobs.append(JobSpec(float(t[k]), int(rng.integers(edge_lo, edge_hi + 1)),
                            "droplet" if rng.random() < 0.5 else "flat",
                            float(rng.uniform(t_lo, t_hi)),
                            "orth" if rng.random() < 0.5 else "nonorth"))
    return jobs
