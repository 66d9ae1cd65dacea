"""R-D selection over a ladder (host logic): upper convex hull of (bytes, PSNR),
budgeted choice per frame, PSNR from squared-error sums and of rendered views."""
import numpy as np

from paper_2606_05650_gb300 import rd


def test_upper_hull_drops_dominated_and_concave_points():
    rate = [1, 2, 3, 4, 5]
    q = [10, 15, 16, 22, 21]
    # (3, 16) lies below the segment (2, 15)-(4, 22); (5, 21) costs more for less
    assert rd.upper_hull(rate, q) == [0, 1, 3]


def test_upper_hull_is_concave_and_increasing():
    rng = np.random.default_rng(0)
    for _ in range(50):
        r = rng.uniform(0, 100, 12)
        q = rng.uniform(0, 50, 12)
        h = rd.upper_hull(r, q)
        rr, qq = r[h], q[h]
        assert (np.diff(rr) > 0).all() and (np.diff(qq) > 0).all()
        slopes = np.diff(qq) / np.diff(rr)
        assert (np.diff(slopes) < 1e-12).all()  # concave
        # every point lies on or below the hull's piecewise-linear interpolation (within its rate range)
        inside = (r >= rr[0]) & (r <= rr[-1])
        assert (q[inside] <= np.interp(r[inside], rr, qq) + 1e-9).all()


def test_select_under_budget():
    rate = np.array([[100, 60, 40, 30, 25], [50, 40, 30, 20, 10]], float)
    q = np.array([[40, 36, 33, 30, 28], [30, 29, 27, 24, 20]], float)
    sel = rd.select(rate, q, [55, 5])
    assert sel[0] == 2  # 40 bytes fit (33 dB); 60 does not
    assert sel[1] == 4  # nothing fits: the smallest stream


def test_psnr_from_error_sums():
    e = np.full((1, 2, 4), 0.01 * 100)  # MSE 0.01 over 100 voxels and 4 channels
    e[0, 1] *= 10
    p = rd.psnr(e, [100])
    assert np.allclose(p, [[20.0, 10.0]])
    assert np.allclose(rd.psnr(e, [100], channels=[0, 1]), [[20.0, 10.0]])


def test_image_psnr_closed_form_and_clamping():
    ref = np.full((4, 5, 3), 0.5)
    for d in (0.1, 0.01, 0.001):
        assert np.isclose(rd.image_psnr(ref + d, ref), -20 * np.log10(d))
    # values beyond [0, 1] are clamped before the difference
    assert np.isclose(rd.image_psnr(np.full((2, 2, 3), 1.7), np.full((2, 2, 3), 0.9)), -20 * np.log10(0.1))


def test_rendered_psnr_averages_views_of_both_frames():
    calls = []

    def render(pos, attr, view):
        calls.append((pos, view))
        return np.full((2, 2, 3), 0.25 + (0.1 * view if pos == "dec" else 0.0))
    v = rd.rendered_psnr(render, ("orig", None), ("dec", None), [0.1, 0.01])
    assert np.isclose(v, np.mean([-20 * np.log10(0.01), -20 * np.log10(0.001)]))
    assert sorted(calls) == sorted([("dec", 0.1), ("orig", 0.1), ("dec", 0.01), ("orig", 0.01)])
