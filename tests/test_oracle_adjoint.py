"""Pins of the oracle's adjoints: each transpose against its forward map through the
identity <A x, y> = <x, A^T y> on random float64 data, exact special cases, and the
transposed float32 stage recursion against brute force on integer data."""
import numpy as np
import pytest

import oracle


def dot(a, b):
    return float(np.sum(np.asarray(a, np.float64) * np.asarray(b, np.float64)))


def close(a, b, rtol=1e-12):
    assert abs(a - b) <= rtol * max(1.0, abs(a), abs(b)), (a, b)


@pytest.mark.parametrize("N", [2, 4, 8, 16])
def test_pattern_backprojection_adjoint_identity(N):
    rng = np.random.default_rng(N)
    L = rng.normal(size=(N, 2 * N))
    G = rng.normal(size=(N, N))
    close(dot(oracle.pattern_backproject(L), G), dot(L, oracle.pattern_backproject_adjoint(G, 2 * N)))


@pytest.mark.parametrize("N", [2, 4, 8, 16, 32])
def test_transposed_stages_equal_brute_force(N):
    rng = np.random.default_rng(100 + N)
    G = rng.integers(-512, 512, size=(N, N)).astype(np.float64)
    brute = oracle.pattern_backproject_adjoint(G, 2 * N)
    np.testing.assert_array_equal(oracle.fht_stages_adjoint(G, 2 * N, np.float64), brute)
    np.testing.assert_array_equal(oracle.fht_stages_adjoint(G, 2 * N, np.float32), brute)


def test_one_pixel_spreads_along_its_dyadic_lines():
    # G = delta at (tau, u): L-bar is 1 exactly at (i, u + d_tau(i)) for every row i.
    N, n = 16, 4
    for tau, u in [(0, 0), (5, 3), (15, 15), (9, 0)]:
        G = np.zeros((N, N))
        G[tau, u] = 1.0
        lb = oracle.fht_stages_adjoint(G, 2 * N, np.float64)
        want = np.zeros((N, 2 * N))
        want[np.arange(N), u + oracle.dyadic_pattern(n, tau)] = 1.0
        np.testing.assert_array_equal(lb, want)


def test_quarter_sum_adjoint_identity():
    rng = np.random.default_rng(3)
    N = 8
    F = rng.normal(size=(4, N, N))
    g = rng.normal(size=(N, N))
    close(dot(oracle.combine_quarters(F), g), dot(F, oracle.quarter_gradients(g)))


def test_back_projection_adjoint_float32_matches_float64():
    rng = np.random.default_rng(4)
    N = 32
    g = rng.normal(size=(N, N))
    f32 = oracle.fht_backproject_adjoint(g.astype(np.float32))
    f64 = oracle.fht_backproject_adjoint(g, brute=True)
    assert np.abs(f32 - f64).max() <= 1e-5 * np.abs(f64).max()


@pytest.mark.parametrize("N,K,M", [(8, 12, 12), (16, 24, 23), (16, 7, 30)])
def test_linogram_adjoint_identity(N, K, M):
    rng = np.random.default_rng(N * K + M)
    pt = rng.normal(size=(K, M))
    lb = rng.normal(size=(4, N, 2 * N))
    close(dot(oracle.linogram(pt, N), lb), dot(pt, oracle.linogram_adjoint(lb, N, K, M)))


def test_linogram_adjoint_of_one_sample_is_its_bilinear_weights():
    # one linogram sample's transpose is w_i times the four bilinear weights (summing to w_i)
    N, K, M = 16, 24, 23
    for q, i, c in [(0, 3, 5), (1, 0, 7), (2, 15, 20), (3, 9, 12)]:
        lb = np.zeros((4, N, 2 * N))
        lb[q, i, c] = 1.0
        pb = oracle.linogram_adjoint(lb, N, K, M)
        assert np.count_nonzero(pb) <= 4
        assert abs(pb.sum() - oracle.row_weights(N)[i]) <= 1e-12 or np.count_nonzero(pb) < 4
        basis = np.zeros((K, M))
        for k, m in zip(*np.nonzero(pb)):
            basis[:] = 0.0
            basis[k, m] = 1.0
            close(oracle.linogram_at(basis, q, np.array([i]), np.array([c]), N)[0], pb[k, m])


def test_filter_is_symmetric():
    rng = np.random.default_rng(5)
    b, a = [0.2, -0.35, 0.15], list(np.poly([0.9, 0.4 + 0.3j, 0.4 - 0.3j]).real[1:])
    x = rng.normal(size=(3, 50))
    y = rng.normal(size=(3, 50))
    close(dot(oracle.iir_filter(x, b, a), y), dot(x, oracle.iir_filter(y, b, a)))


def test_fast_fbp_adjoint_identity():
    rng = np.random.default_rng(6)
    N, K, M = 16, 24, 23
    b, a = [0.2, -0.35, 0.15], list(np.poly([0.8, 0.5, -0.2])[1:])
    x = rng.normal(size=(K, M))
    g = rng.normal(size=(N, N))
    close(dot(oracle.fast_fbp(x, N, b, a), g), dot(x, oracle.fast_fbp_adjoint(g, N, K, M, b, a)),
          rtol=1e-10)
