"""The seeded input recipe (paper_2507_23613_gb300/inputs.py): determinism, frequency bands
and gaps, Gaussian centres and widths, the two-layer medium and the printed three-frequency
problem.  CPU only."""

import numpy as np
import pytest

from paper_2507_23613_gb300 import inputs


def _peak_centre(wl, m):
    """Grid coordinates of the forcing maximum of frequency m (x first)."""
    idx = np.unravel_index(np.argmax(wl.forcing[m]), wl.forcing[m].shape)
    coords = inputs.coordinates(wl.n, wl.length)
    return np.array([c[idx] for c in coords])


def test_same_seed_same_inputs():
    a, b = inputs.square_large(7, n=64), inputs.square_large(7, n=64)
    assert np.array_equal(a.omega, b.omega) and np.array_equal(a.forcing, b.forcing)
    c = inputs.square_large(8, n=64)
    assert not np.array_equal(a.omega, c.omega)
    assert np.array_equal(inputs.batch_workload(3).forcing, inputs.batch_workload(3).forcing)


def test_square_workloads():
    wl = inputs.square_small()
    assert wl.n == (64, 64) and wl.shape == (65, 65) and list(wl.omega) == [5.5, 9.3]
    assert wl.cfl == 0.5 and wl.n_p == 1 and wl.c2 == 1.0
    big = inputs.square_large()
    assert big.n == (1024, 1024) and big.nf == 8 and big.n_p == 2
    assert np.all((big.omega >= 10.0) & (big.omega <= 60.0)) and np.all(np.diff(big.omega) >= 1.0)
    assert big.forcing.shape == (8, 1025, 1025) and big.interior_points == 1023 ** 2
    for m in range(big.nf):
        x0 = _peak_centre(big, m)
        assert np.all((x0 >= 0.2 - 1e-3) & (x0 <= 0.8 + 1e-3))
        assert abs(big.forcing[m].max() - 1.0) < 0.05          # A = 1, peak near a grid point


def test_gaussian_width_is_b():
    """f = A exp(-b ||x - x0||^2) with b = 400: one grid step from the centre the value
    falls by exp(-b h^2)."""
    g = inputs.coordinates((100, 100), (1.0, 1.0))
    f = inputs.gaussian(g, (0.5, 0.5), 2.0, 400.0)
    assert f[50, 50] == 2.0
    assert abs(f[50, 51] / f[50, 50] - np.exp(-400.0 * 0.01 ** 2)) < 1e-14


def test_cube_two_layer_medium():
    wl = inputs.cube_layered(n=16)
    assert wl.nf == 4 and np.all((wl.omega >= 8.0) & (wl.omega <= 30.0))
    c2 = wl.c2
    z = inputs.coordinates(wl.n, wl.length)[2]
    assert np.all(c2[z < 0.5] == 1.0) and np.all(c2[z >= 0.5] == 2.25)
    assert wl.layer == {"c_lo": 1.0, "c_hi": 1.5, "interface": 0.5, "axis": 2}


@pytest.mark.parametrize("seed", range(6))
def test_batch_and_warm_start_draws(seed):
    wl = inputs.batch_workload(seed)
    assert wl.n[0] == wl.n[1] and wl.n[0] in inputs.BATCH_SIZES
    assert 1 <= wl.nf <= 16 and np.all((wl.omega >= 5.0) & (wl.omega <= 80.0))
    assert wl.nf == 1 or np.min(np.diff(wl.omega)) >= 1.5
    ws = inputs.warm_start_workload(seed, n=32)
    assert ws.nf == 6 and ws.n_p == 2 and np.min(np.diff(ws.omega)) >= 1.5
    assert np.all((ws.omega >= 15.0) & (ws.omega <= 45.0))


def test_printed_three_frequency_problem():
    """eq. Nf3parameters: omega = {5.1, 10.1, 15.1}, amplitudes {25, 100, 225}, width 15,
    centres (0.6, 0.45), (0.4, 0.5), (0.55, 0.5); N_p = 2."""
    wl = inputs.paper_three_frequency(100)
    assert list(wl.omega) == [5.1, 10.1, 15.1] and wl.n_p == 2
    for m, (amp, c) in enumerate([(25.0, (0.6, 0.45)), (100.0, (0.4, 0.5)), (225.0, (0.55, 0.5))]):
        assert np.allclose(_peak_centre(wl, m), c, atol=1e-12)
        assert abs(wl.forcing[m].max() - amp) < 1e-12
    cube = inputs.paper_three_frequency_cube(20)
    assert np.allclose(_peak_centre(cube, 0), (0.6, 0.45, 0.5), atol=1e-12)


def test_random_c2_field_is_seeded_and_in_range():
    a = inputs.random_c2((6, 5, 4), 3, 1.0, 1.5)
    b = inputs.random_c2((6, 5, 4), 3, 1.0, 1.5)
    assert a.shape == (5, 6, 7) and np.array_equal(a, b)
    assert a.min() >= 1.0 and a.max() <= 2.25
    assert not np.array_equal(a, inputs.random_c2((6, 5, 4), 4, 1.0, 1.5))
