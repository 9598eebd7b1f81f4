"""Pins of the quarter geometry (Sec. 4.1-4.2, Eq. 14-15) and the row weights."""
import numpy as np
import pytest

from oracle import linogram_at, quarter_angle, quarter_r, row_weights, slopes

RANGES = {0: (0.0, np.pi / 4), 1: (3 * np.pi / 4, np.pi), 2: (np.pi / 4, np.pi / 2),
          3: (np.pi / 2, 3 * np.pi / 4)}     # v-, v+, h-, h+ (Sec. 4.1)


@pytest.mark.parametrize("q", range(4))
def test_angles_lie_in_the_papers_quarter_ranges(q):
    th = quarter_angle(q, slopes(64))
    lo, hi = RANGES[q]
    assert th.min() >= lo - 1e-15 and th.max() <= hi + 1e-15


def _paper_line(q, sigma):
    """Eq. 14: tan(theta) = -(N/t)^p with p = -1 for v lines, +1 for h lines; t/N = +-sigma."""
    t_over_n = sigma if q in (1, 3) else -sigma
    return t_over_n


@pytest.mark.parametrize("q", range(4))
def test_angle_and_offset_agree_with_eq14(q):
    N = 32
    c0 = (N - 1) / 2
    sig = slopes(N)[1:-1]                 # avoid tan singularities at the ends
    th = quarter_angle(q, sig)
    tn = _paper_line(q, sig)
    tan_paper = -tn if q in (0, 1) else -1.0 / tn
    np.testing.assert_allclose(np.tan(th), tan_paper, rtol=1e-12)
    # Offset: Eq. 14 gives r = s N / sqrt(t^2 + N^2) from the corner origin for the line
    # through the boundary point at coordinate s (x = s + (t/N) y for v, y = s + (t/N) x for h).
    # Its normal angle theta_p solves Eq. 14 with cos(theta_p) > 0 (v) or sin(theta_p) > 0 (h).
    for c in (0, 5, N - 1, N + 3, 2 * N - 2):
        u = c if q in (0, 2) else N - 1 - c
        r_corner = u / np.sqrt(1 + tn ** 2)
        theta_p = np.arctan(tan_paper)
        if q in (2, 3):
            theta_p = np.where(theta_p < 0, theta_p + np.pi, theta_p)
        r_centre = r_corner - c0 * np.cos(theta_p) - c0 * np.sin(theta_p)
        same = np.isclose(np.cos(th), np.cos(theta_p)) & np.isclose(np.sin(th), np.sin(theta_p))
        flip = np.isclose(np.cos(th), -np.cos(theta_p)) & np.isclose(np.sin(th), -np.sin(theta_p))
        assert np.all(same | flip)
        want = np.where(same, r_centre, -r_centre)
        np.testing.assert_allclose(quarter_r(q, sig, c, N), want, rtol=0, atol=1e-11)


@pytest.mark.parametrize("q", range(4))
def test_normal_is_perpendicular_to_the_quarter_line(q):
    # Two points of the stated line (x = u -+ sigma y or y = u -+ sigma x) both satisfy
    # (x - c0) cos(theta) + (y - c0) sin(theta) = r.
    N = 16
    c0 = (N - 1) / 2
    for i in range(N):
        s = i / (N - 1)
        th = quarter_angle(q, s)
        for c in range(2 * N):
            u = c if q in (0, 2) else N - 1 - c
            sign = -1.0 if q in (0, 2) else 1.0
            if q in (0, 1):
                pts = [(u, 0.0), (u + sign * s * (N - 1), N - 1.0)]
            else:
                pts = [(0.0, u), (N - 1.0, u + sign * s * (N - 1))]
            r = quarter_r(q, s, c, N)
            for x, y in pts:
                assert (x - c0) * np.cos(th) + (y - c0) * np.sin(th) == pytest.approx(r, abs=1e-10)


@pytest.mark.parametrize("N", [4, 16, 256, 2048])
def test_weights_follow_euler_maclaurin(N):
    # Trapezoid rule for int_0^1 d sigma / (1 + sigma^2) = pi/4 has error -h^2/24 + O(h^6)
    # (f'''(0) = f'''(1) = 0), so the four quarters sum to pi - h^2/6 + O(h^6).
    h = 1.0 / (N - 1)
    total = 4.0 * row_weights(N).sum()
    assert total == pytest.approx(np.pi - h * h / 6.0, abs=2 * h ** 6 + 1e-14)


def test_single_linogram_sample_reads_the_right_sinogram_point():
    # A sinogram that is 1 at exactly one (k, m) and 0 elsewhere; the linogram sample whose
    # (theta, r) lands exactly on that grid point must equal the row weight.
    N, K, M = 16, 24, 23
    pt = np.zeros((K, M))
    k, m = 3, 14
    pt[k, m] = 1.0
    theta = k * np.pi / K                       # v- covers [0, pi/4]
    sigma = np.tan(theta)
    # column whose r equals m - (M-1)/2, from r = (u - c0 - sigma c0)/sqrt(1 + sigma^2)
    c0 = (N - 1) / 2
    u = (m - (M - 1) / 2) * np.sqrt(1 + sigma ** 2) + c0 + sigma * c0
    i = sigma * (N - 1)
    # pick the nearest stored row/column and evaluate the bilinear weight independently
    ii, cc = int(round(i)), int(round(u))
    s = ii / (N - 1)
    th = np.arctan(s)
    tk = th * K / np.pi
    mm = (cc - c0 - s * c0) / np.sqrt(1 + s * s) + (M - 1) / 2
    wt = max(0.0, 1 - abs(tk - k)) * max(0.0, 1 - abs(mm - m))
    got = linogram_at(pt, 0, np.array([ii]), np.array([cc]), N)[0]
    assert got == pytest.approx(row_weights(N)[ii] * wt, abs=1e-14)
