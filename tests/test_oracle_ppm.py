"""Pins for the oracle's PPM pieces (Colella & Woodward 1984, restated in the
oracle): each check is fixed by mathematics, not by the oracle's own formula."""
import numpy as np
import pytest

import oracle


def cubic_averages(edges, c):
    """Exact zone averages of the cubic sum c_k x^k (antiderivative)."""
    F = lambda x: c[0] * x + c[1] * x ** 2 / 2 + c[2] * x ** 3 / 3 + c[3] * x ** 4 / 4
    return (F(edges[1:]) - F(edges[:-1])) / np.diff(edges)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_interface_exact_for_cubics(seed):
    # The unlimited interface formula interpolates the cumulative integral by a
    # quartic, so it is exact for cubic profiles on any grid.
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.3, 1.7, size=24)
    e = np.concatenate([[0.0], np.cumsum(w)])
    c = rng.normal(size=4)
    a = cubic_averages(e, c)
    edge = oracle.ppm_edges(w, a, limited=False)
    x = e[1:]                                  # edge i sits at e[i+1]
    exact = c[0] + c[1] * x + c[2] * x ** 2 + c[3] * x ** 3
    ok = slice(1, len(a) - 2)
    scale = np.max(np.abs(exact))
    assert np.max(np.abs(edge[ok] - exact[ok])) < 1e-12 * scale


def test_interface_uniform_grid_closed_form():
    # On a uniform grid the interface value is 7/12 (a_i + a_{i+1}) - 1/12 (a_{i-1} + a_{i+2}).
    rng = np.random.default_rng(7)
    a = rng.normal(size=20)
    edge = oracle.ppm_edges(np.ones(20), a, limited=False)
    i = np.arange(1, 17)
    ref = 7.0 / 12.0 * (a[i] + a[i + 1]) - 1.0 / 12.0 * (a[i - 1] + a[i + 2])
    assert np.max(np.abs(edge[i] - ref)) < 1e-14


@pytest.mark.parametrize("seed", range(6))
def test_limited_interface_stays_between_neighbours(seed):
    # With the limited slopes the interface value of monotone data lies between
    # the two adjacent zone averages (CW84's purpose of the slope limiter).
    rng = np.random.default_rng(100 + seed)
    a = np.cumsum(rng.exponential(size=30) * (rng.uniform(size=30) < 0.7))
    w = rng.uniform(0.2, 3.0, size=30)
    edge = oracle.ppm_edges(w, a, limited=True)
    for i in range(1, 27):
        lo, hi = min(a[i], a[i + 1]), max(a[i], a[i + 1])
        assert lo - 1e-12 <= edge[i] <= hi + 1e-12


def parabola(aL, aR, a6, xi):
    return aL + xi * ((aR - aL) + a6 * (1.0 - xi))


@pytest.mark.parametrize("seed", range(8))
def test_parabola_average_and_monotone(seed):
    rng = np.random.default_rng(200 + seed)
    for _ in range(200):
        ai, aL, aR = rng.normal(size=3)
        f = rng.choice([0.0, 0.0, rng.uniform()])
        l, r, a6 = oracle.ppm_parabola(ai, aL, aR, f)
        # zone average of the parabola is a_i (Simpson is exact for quadratics)
        avg = (parabola(l, r, a6, 0.0) + 4 * parabola(l, r, a6, 0.5) + parabola(l, r, a6, 1.0)) / 6.0
        assert abs(avg - ai) < 1e-12 * (1 + abs(ai))
        # the constrained parabola is monotone on the zone and takes no value
        # outside [min(aL, aR), max(aL, aR)]
        xi = np.linspace(0, 1, 101)
        vals = parabola(l, r, a6, xi)
        d = np.diff(vals)
        assert np.all(d >= -1e-12) or np.all(d <= 1e-12)
        assert vals.min() >= min(l, r) - 1e-12 and vals.max() <= max(l, r) + 1e-12


def test_parabola_flattening_and_extremum():
    # full flattening gives the constant a_i; a zone that is a local extremum
    # (a_i outside the edge values) is made constant.
    assert np.allclose(oracle.ppm_parabola(0.3, -2.0, 5.0, 1.0), [0.3, 0.3, 0.0])
    assert np.allclose(oracle.ppm_parabola(2.0, 1.0, 1.5, 0.0), [2.0, 2.0, 0.0])


@pytest.mark.parametrize("seed", range(5))
def test_domain_of_dependence_averages(seed):
    # avg_right(y) is the mean of the parabola over the last fraction y of the
    # zone, avg_left(y) over the first fraction y (checked by quadrature).
    rng = np.random.default_rng(300 + seed)
    for _ in range(50):
        aL, aR, a6 = rng.normal(size=3)
        y = rng.uniform(0.01, 1.0)
        xs = np.linspace(1 - y, 1, 2001)
        ref_r = np.trapezoid(parabola(aL, aR, a6, xs), xs) / y
        xs = np.linspace(0, y, 2001)
        ref_l = np.trapezoid(parabola(aL, aR, a6, xs), xs) / y
        assert abs(oracle.avg_right(aL, aR, a6, y) - ref_r) < 1e-7
        assert abs(oracle.avg_left(aL, aR, a6, y) - ref_l) < 1e-7
    # y -> 0 gives the edge values, y = 1 the zone average
    aL, aR, a6 = 0.2, 1.1, -0.4
    assert oracle.avg_right(aL, aR, a6, 0.0) == aR
    assert oracle.avg_left(aL, aR, a6, 0.0) == aL
    mean = aL + 0.5 * (aR - aL) + a6 / 6.0
    assert abs(oracle.avg_right(aL, aR, a6, 1.0) - mean) < 1e-15
    assert abs(oracle.avg_left(aL, aR, a6, 1.0) - mean) < 1e-15
