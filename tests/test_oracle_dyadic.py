"""Pins of the dyadic patterns and the fast Hough transform (Sec. 4.4-4.5, Eq. 22)."""
import os

import numpy as np
import pytest

from oracle import combine_quarters, dyadic_pattern, fht_stages, pattern_backproject

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "dyadic_patterns_n3.txt")
RNG = np.random.default_rng(5)


def test_patterns_match_hand_derived_golden():
    want = np.loadtxt(GOLDEN, dtype=np.int64)
    got = np.stack([dyadic_pattern(3, t) for t in range(8)])
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("n", range(1, 10))
def test_pattern_is_a_digital_line(n):
    N = 1 << n
    i = np.arange(N)
    worst = 0.0
    for tau in range(N):
        d = dyadic_pattern(n, tau)
        assert d[0] == 0 and d[-1] == tau
        assert set(np.unique(np.diff(d))) <= {0, 1}
        worst = max(worst, np.abs(d - tau * i / (N - 1)).max())
    # dyadic approximations deviate from the straight line by at most log2(N)/6
    assert worst <= n / 6 + 1e-12
    if n % 2 == 0:
        assert worst == pytest.approx(n / 6)


@pytest.mark.parametrize("N", [2, 4, 8, 16])
@pytest.mark.parametrize("extra", [0, 5])
def test_stage_recursion_equals_pattern_sums(N, extra):
    W = 2 * N + extra
    L = RNG.integers(-1000, 1001, size=(N, W)).astype(np.float64)
    want = pattern_backproject(L)
    np.testing.assert_array_equal(fht_stages(L, np.float64), want)
    np.testing.assert_array_equal(fht_stages(L, np.float32).astype(np.float64), want)
    Lr = RNG.normal(size=(N, W))
    np.testing.assert_allclose(fht_stages(Lr, np.float64), pattern_backproject(Lr), atol=1e-12)


def test_integer_inputs_are_exact_in_float32_at_n64():
    N = 64
    L = RNG.integers(-1024, 1025, size=(N, 2 * N)).astype(np.float64)
    np.testing.assert_array_equal(fht_stages(L, np.float32).astype(np.float64), pattern_backproject(L))


def test_delta_back_projects_onto_one_digital_line():
    N, n = 32, 5
    i0, c0 = 19, 40
    L = np.zeros((N, 2 * N))
    L[i0, c0] = 1.0
    F = fht_stages(L, np.float64)
    for tau in range(N):
        u = c0 - dyadic_pattern(n, tau)[i0]
        expect = np.zeros(N)
        if 0 <= u < N:
            expect[u] = 1.0
        np.testing.assert_array_equal(F[tau], expect)


def test_combine_maps_quarters_to_pixels():
    N = 8
    F = np.zeros((4, N, N))
    F[0, 2, 5] = 1      # v-: [y][x]       -> pixel (y=2, x=5)
    F[1, 3, 1] = 10     # v+: [y][N-1-x]   -> pixel (y=3, x=6)
    F[2, 4, 7] = 100    # h-: [x][y]       -> pixel (y=7, x=4)
    F[3, 6, 2] = 1000   # h+: [x][N-1-y]   -> pixel (y=5, x=6)
    img = combine_quarters(F)
    assert img[2, 5] == 1 and img[3, 6] == 10 and img[7, 4] == 100 and img[5, 6] == 1000
    assert img.sum() == 1111
