"""GPU splat rasteriser (gsnfs_render) against the oracle's FP64 renderer,
pixel by pixel: synthetic scenes seen from orbit cameras on ragged image
sizes (partial edge tiles), the closed-form single Gaussian, an opaque front
splat hiding one behind it, empty and fully culled scenes, and argument
errors.  The oracle marks the pixels whose value hangs on a decision taken
within rounding of its threshold (alpha at the 1/255 cut, transmittance at
the 1e-4 stop, a tile rectangle edge, depths equal in FP32); every other
pixel must lie within the oracle's first-order bound on the error of an FP32
evaluation of that pixel (Sec. 5.1 renders decoded frames to score them)."""
import numpy as np
import pytest

from paper_2606_05650_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

VIEW = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]], dtype=np.float64)


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_05650_gb300 import gsnfs
    return gsnfs


def _both(G, orc, pos, attr, view, f, W, H, bg=(0.0, 0.0, 0.0)):
    """GPU image and the oracle's (image, threshold flags, FP32 error bounds)."""
    cx, cy = W / 2, H / 2
    ref = orc.render(pos, attr, view, f, f, cx, cy, W, H, bg=bg, check=True)
    img = G.render(torch.from_numpy(pos).cuda(), torch.from_numpy(attr).cuda(), view, f, f, cx, cy, W, H,
                   background=bg).cpu().numpy()
    return img, ref


def _close(img, ref):
    """Every pixel not flagged by the oracle within its error bound, in all three channels; flagged pixels are
    counted and rare."""
    want, flag, tol = ref
    d = np.abs(img.astype(np.float64) - want).max(axis=2)
    ok = flag == 0
    bad = ok & (d > tol)
    assert not bad.any(), (int(bad.sum()), float(d[bad].max()), float(tol[bad].min()))
    assert flag.mean() < 5e-3, flag.mean()
    return d, flag


@pytest.mark.parametrize("seed,W,H", [(1, 200, 150), (2, 97, 131), (3, 256, 256)])
def test_scene_matches_oracle(G, orc, seed, W, H):
    pos, attr = syn.static_gs_frame(seed, n=8_000)
    for view in syn.orbit_views(2, radius=1.5 + 0.2 * seed):
        img, ref = _both(G, orc, pos, attr, view, 0.9 * W, W, H, bg=(0.1, 0.2, 0.3))
        _close(img, ref)
        assert ref[0].std() > 0.02  # the scene is visible


def test_single_gaussian_closed_form(G):
    f, W, H, s, zc = 100.0, 64, 64, 0.02, 2.0
    a = np.zeros((1, 56), dtype=np.float32)
    a[0, 0:3] = np.log(s)
    a[0, 3] = 1.0
    a[0, 8:11] = [1.0, -1.0, 0.5]
    p = np.array([[0, 0, zc]], dtype=np.float32)
    bg = np.array([0.1, 0.2, 0.3])
    img = G.render(torch.from_numpy(p).cuda(), torch.from_numpy(a).cuda(), VIEW, f, f, W / 2 + 0.5, H / 2 + 0.5,
                   W, H, background=bg).cpu().numpy()
    var = (f * s / zc) ** 2 + 0.3
    col = np.maximum(0.5 / np.sqrt(np.pi) * np.array([1.0, -1.0, 0.5]) + 0.5, 0)
    for dx, dy in ((0, 0), (1, 0), (0, 2), (2, 1), (-1, -1)):
        alpha = min(0.99, 0.5 * np.exp(-(dx * dx + dy * dy) / (2 * var)))
        want = col * alpha + (1 - alpha) * bg if alpha >= 1 / 255 else bg
        assert np.allclose(img[32 + dy, 32 + dx], want, atol=2e-6), (dx, dy)
    assert np.allclose(img[0, 0], bg)


def test_occlusion_and_order(G, orc):
    a = np.zeros((3, 56), dtype=np.float32)
    a[:, 0:3] = np.log(0.2)
    a[:, 3] = 1.0
    a[:, 7] = 4.0  # alpha up to 0.982: transmittance 3.2e-4 after two, clear of the 1e-4 stop
    a[0, 8:11] = [1.0, 0, 0]
    a[1, 8:11] = [0, 1.0, 0]
    a[2, 8:11] = [0, 0, 1.0]
    p = np.array([[0, 0, 3.0], [0, 0, 2.0], [0, 0, 2.0]], dtype=np.float32)  # 1 and 2 tie in depth: index order
    img, ref = _both(G, orc, p, a, VIEW, 100.0, 48, 40)
    _close(img, ref)
    c0 = 0.5 / np.sqrt(np.pi)
    # splat 1 (green) is in front and first of the tie; 1% of the rest goes to splat 2, then splat 0
    assert img[20, 24, 1] > 0.95 * (c0 + 0.5)


def test_empty_and_culled(G, orc):
    bg = (0.25, 0.5, 0.75)
    e = torch.zeros((0, 3), device="cuda"), torch.zeros((0, 56), device="cuda")
    img = G.render(e[0], e[1], VIEW, 50, 50, 20, 20, 40, 33, background=bg).cpu().numpy()
    assert np.array_equal(img, np.broadcast_to(np.float32(bg), img.shape))
    pos, attr = syn.static_gs_frame(5, n=2000)
    pos = pos - np.float32(5.0)  # every point behind the camera (z < 0)
    img, ref = _both(G, orc, pos, attr, VIEW, 50.0, 40, 33, bg=bg)
    assert np.array_equal(img, ref[0].astype(np.float32)) and not ref[1].any()


def test_bad_arguments(G):
    p = torch.zeros((4, 3), device="cuda")
    a = torch.zeros((4, 56), device="cuda")
    with pytest.raises(G.GsnfsError):
        G.render(p, a, VIEW, 50, 50, 20, 20, 40, 33, znear=0.0)
    with pytest.raises(G.GsnfsError):
        G.render(p, a, VIEW, 50, 50, 20, 20, 0, 33)
    with pytest.raises(ValueError):
        G.render(p, a[:3], VIEW, 50, 50, 20, 20, 40, 33)
