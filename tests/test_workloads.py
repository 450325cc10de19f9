"""The seeded input recipe (no GPU): the splitmix64 generator against its published definition,
the readings of the configurations (nodes include the Dirichlet ring, k h = 0.6 exactly at the
corners, the random source confined to |x|_inf < 0.5, the ECS start on a node), and
reproducibility of every generator."""
import math

import numpy as np
import pytest

from paper_1012_4307_gb300 import workloads as W


def splitmix64_scalar(state, count):
    """splitmix64 written out one output at a time with Python integers (mod 2^64)."""
    mask = (1 << 64) - 1
    out = []
    for _ in range(count):
        state = (state + 0x9E3779B97F4A7C15) & mask
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        out.append(z ^ (z >> 31))
    return out


@pytest.mark.parametrize("seed", [0, 1, 12345, 2 ** 63 + 7])
def test_splitmix64_matches_the_scalar_definition(seed):
    assert [int(v) for v in W.splitmix64(seed, 50)] == splitmix64_scalar(seed, 50)


def test_uniform_and_normal_moments():
    u = W.uniform(7, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5e-3 and abs(u.var() - 1.0 / 12.0) < 5e-3
    g = W.normal(8, 200001)
    assert g.shape == (200001,)
    assert abs(g.mean()) < 1e-2 and abs(g.std() - 1.0) < 1e-2


@pytest.mark.parametrize("dim,n", [(2, 65), (2, 1025), (3, 33), (3, 257)])
def test_well_growth_reaches_kh_max_exactly_at_the_corners(dim, n):
    k2 = W.k2_well_growth(dim, n, kh_max=0.6)
    h = 2.0 / (n - 1)
    kh = np.sqrt(np.maximum(k2, 0.0)) * h
    corner = (0,) * dim
    assert kh[corner] == pytest.approx(0.6, rel=1e-12)
    assert kh.max() == pytest.approx(0.6, rel=1e-12)
    # the well: k^2 = 2 (E + V0) at the centre
    centre = ((n - 1) // 2,) * dim
    assert k2[centre] == pytest.approx(2.0 * (2.0 + 5.0), rel=1e-12)


def test_random_box_source_is_confined_and_reproducible():
    n = 129
    f = W.random_box_source(2, n, 1)
    x = np.linspace(-1.0, 1.0, n)
    inside = (np.abs(x)[None, :] < 0.5) & (np.abs(x)[:, None] < 0.5)
    assert np.all(f[~inside] == 0)
    assert np.count_nonzero(f[inside]) == inside.sum()
    assert np.array_equal(f, W.random_box_source(2, n, 1))
    assert not np.array_equal(f, W.random_box_source(2, n, 2))


def test_gaussian_source_centre_and_ring():
    n = 65
    f = W.gaussian_source(2, n, 0.05, 0)
    assert np.all(f[0, :] == 0) and np.all(f[-1, :] == 0) and np.all(f[:, 0] == 0) and np.all(f[:, -1] == 0)
    c = W.uniform(0, 2) - 0.5
    iy, ix = np.unravel_index(np.argmax(np.abs(f)), f.shape)
    x = np.linspace(-1.0, 1.0, n)
    assert abs(x[ix] - c[0]) <= 1.0 / (n - 1) and abs(x[iy] - c[1]) <= 1.0 / (n - 1)


@pytest.mark.parametrize("n", [65, 129, 257, 513, 1025])
def test_nodes_include_the_ring_and_the_layer_starts_on_a_node(n):
    P = W.config_2d_well(n) if n == 1025 else W.Problem("p", 2, n, W.k2_well_growth(2, n), W.random_box_source(2, n, 1))
    assert P.unknowns == (n - 2) ** 2
    h = 2.0 / (n - 1)
    j = (0.75 - (-1.0)) / h
    assert j == pytest.approx(round(j), abs=1e-9)


def test_batch_configuration_draws_sizes_and_energies_in_range():
    probs = W.config_batch()
    assert len(probs) == 64
    assert {P.n for P in probs} <= {129, 257, 513, 1025}
    assert len({P.n for P in probs}) == 4
    assert all(0.5 <= P.extra["E"] <= 4.0 for P in probs)
    again = W.config_batch()
    assert all(np.array_equal(a.f, b.f) and np.array_equal(a.k2, b.k2) for a, b in zip(probs, again))
    assert all(P.theta_a == W.WELL_THETA_A and P.tol == 1e-8 for P in probs)


def test_headline_configuration():
    P = W.config_2d_well()
    assert (P.dim, P.n, P.unknowns) == (2, 1025, 1023 ** 2)
    assert P.theta == pytest.approx(math.pi / 6) and P.theta_a == pytest.approx(math.pi / 10)
    assert (P.restart, P.tol, P.coarsest_n) == (30, 1e-8, 17)
