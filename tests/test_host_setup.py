"""Host-side set-up on CPU: the product's coexistence solver against the oracle's
equal-area quadrature, and the seeded workload generators against the recipes
they implement (counts, ranges, determinism, Poisson statistics)."""

import numpy as np
import pytest

from oracle import maxwell
from paper_1805_08643_gb300 import synth, thermo


@pytest.mark.parametrize("t", [0.6, 0.7, 0.8, 0.9])
@pytest.mark.parametrize("a", [1.0, 0.25])
def test_carnahan_starling_coexistence_matches_the_oracle(t, a):
    # equal chemical potential (product) and equal areas by quadrature (oracle) are the same rule
    rl, rv = thermo.coexistence_cs(t, a, 4.0, 1.0)
    ol, ov = maxwell.coexistence_cs(t, a=a, b=4.0, R=1.0)
    assert abs(rl / ol - 1) < 1e-10 and abs(rv / ov - 1) < 1e-10


def test_exponential_coexistence_matches_the_oracle():
    rl, rv = thermo.coexistence_exp()
    ol, ov = maxwell.coexistence_exp()
    assert abs(rl / ol - 1) < 1e-10 and abs(rv / ov - 1) < 1e-10


def test_critical_temperature_and_domain():
    assert thermo.critical_temperature(1.0, 4.0, 1.0) == pytest.approx(0.37733 / 4.0, rel=1e-15)
    for bad in (0.2, 1.0):
        with pytest.raises(ValueError):
            thermo.coexistence_cs(bad)


def test_random_droplets_recipe():
    c, r = synth.random_droplets()
    c2, r2 = synth.random_droplets()
    assert c.shape == (27, 3) and r.shape == (27,)
    assert np.array_equal(c, c2) and np.array_equal(r, r2)  # seeded
    assert np.all((r >= 12.0) & (r <= 40.0))
    assert np.all((c >= 0) & (c < 512))
    cell = 512 / 3
    idx = np.stack(np.meshgrid(*[np.arange(3)] * 3, indexing="ij"), -1).reshape(-1, 3)
    d = np.abs(c - (idx + 0.5) * cell)
    assert np.all(np.minimum(d, 512 - d) <= 40.0 + 1e-12)  # within the jitter of its cell centre
    c3, _ = synth.random_droplets(seed=7)
    assert not np.array_equal(c, c3)


def test_batched_boxes_recipe():
    boxes = synth.batched_boxes()
    assert len(boxes) == 512 and boxes == synth.batched_boxes()
    edges = np.array([b.edge for b in boxes])
    assert set(edges) == {32, 48, 64, 96}
    assert all(6.0 <= b.radius <= b.edge / 3 for b in boxes)
    assert all(0.6 <= b.T_over_Tc <= 0.9 for b in boxes)
    # edges uniform over the four values: each within 5 standard deviations of 128
    counts = np.array([np.sum(edges == e) for e in (32, 48, 64, 96)])
    assert np.all(np.abs(counts - 128) < 5 * np.sqrt(512 * 0.25 * 0.75))


def test_job_stream_is_a_poisson_stream_of_the_stated_jobs():
    rate, n = 4.0, 4000
    jobs = synth.job_stream(n, rate)
    t = np.array([j.arrival for j in jobs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    # exponential gaps: mean 1/rate, coefficient of variation 1 (5-sigma bounds for n = 4000)
    assert abs(gaps.mean() * rate - 1) < 5 / np.sqrt(n)
    assert abs(gaps.std() / gaps.mean() - 1) < 0.1
    assert all(48 <= j.edge <= 192 and 0.6 <= j.T_over_Tc <= 0.9 for j in jobs)
    assert {j.kind for j in jobs} == {"droplet", "flat"} and {j.operator for j in jobs} == {"orth", "nonorth"}
    frac_drop = np.mean([j.kind == "droplet" for j in jobs])
    assert abs(frac_drop - 0.5) < 5 * np.sqrt(0.25 / n)
    assert [j.arrival for j in synth.job_stream(10, rate)] == list(t[:10])  # seeded, prefix-stable
