"""Oracle splat rasteriser (the renderer behind rendered-view PSNR): pinned
by the orthonormality of its real SH basis on the sphere, closed-form pixels
of one projected Gaussian (EWA footprint with the 0.3 px dilation), the SH
colour of a known direction, front-to-back occlusion, the background of an
empty or culled scene."""
import numpy as np

VIEW = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]], dtype=np.float64)  # camera at the origin, +z


def _gauss(pos, logscale, logit, dc, ac=None):
    a = np.zeros(56, dtype=np.float32)
    a[0:3] = logscale
    a[3] = 1.0  # identity rotation
    a[7] = logit
    a[8:11] = dc
    if ac is not None:
        a[11:56] = ac
    return np.array(pos, dtype=np.float32), a


def test_sh_basis_is_orthonormal(orc):
    n = 200_000  # Fibonacci sphere quadrature
    k = np.arange(n) + 0.5
    z = 1 - 2 * k / n
    phi = np.pi * (1 + 5 ** 0.5) * k
    r = np.sqrt(1 - z * z)
    d = np.stack([r * np.cos(phi), r * np.sin(phi), z], 1)
    Y = np.array([orc.sh_basis(x) for x in d[:: 20]])  # 10,000 points
    G = Y.T @ Y * (4 * np.pi / Y.shape[0])
    assert np.abs(G - np.eye(16)).max() < 5e-3


def test_single_gaussian_closed_form(orc):
    f, W, H = 100.0, 64, 64
    s, zc = 0.02, 2.0
    p, a = _gauss([0, 0, zc], np.log(s), 0.0, [1.0, -1.0, 0.5])  # opacity 0.5
    bg = np.array([0.1, 0.2, 0.3])
    img = orc.render(p[None], a[None], VIEW, f, f, W / 2 + 0.5, H / 2 + 0.5, W, H, bg=bg)
    # the mean projects to the centre of pixel (32, 32); footprint variance (f s / z)^2 + 0.3
    var = (f * s / zc) ** 2 + 0.3
    c0 = 0.5 / np.sqrt(np.pi)
    col = np.maximum(c0 * np.array([1.0, -1.0, 0.5]) + 0.5, 0)
    for dx, dy in ((0, 0), (1, 0), (0, 2), (2, 1), (-1, -1)):
        alpha = min(0.99, 0.5 * np.exp(-(dx * dx + dy * dy) / (2 * var)))
        want = col * alpha + (1 - alpha) * bg if alpha >= 1 / 255 else bg
        assert np.allclose(img[32 + dy, 32 + dx], want, atol=1e-12), (dx, dy)
    assert np.allclose(img[0, 0], bg)  # outside the footprint square's tiles


def test_view_dependent_colour(orc):
    ac = np.zeros(45, dtype=np.float32)
    ac[1] = 0.3  # R, degree 1, the z-term (AC function 2)
    p, a = _gauss([0, 0, 2.0], np.log(0.05), 20.0, [0, 0, 0], ac)  # opaque (alpha capped at 0.99)
    img = orc.render(p[None], a[None], VIEW, 100, 100, 32.5, 32.5, 64, 64)
    y = orc.sh_basis([0, 0, 1.0])
    assert np.isclose(img[32, 32, 0], 0.99 * (0.5 + 0.3 * y[2]))
    assert np.isclose(img[32, 32, 1], 0.99 * 0.5)


def test_front_to_back_occlusion_and_empty(orc):
    p1, a1 = _gauss([0, 0, 2.0], np.log(0.05), 20.0, [1.5, -1.5, -1.5])
    p2, a2 = _gauss([0, 0, 3.0], np.log(0.05), 20.0, [-1.5, -1.5, 1.5])
    for order in ((0, 1), (1, 0)):  # input order does not matter, depth does
        P = np.stack([p1, p2])[list(order)]
        A = np.stack([a1, a2])[list(order)]
        img = orc.render(P, A, VIEW, 100, 100, 32.5, 32.5, 64, 64)
        c1 = np.maximum(0.5 / np.sqrt(np.pi) * np.array([1.5, -1.5, -1.5]) + 0.5, 0)
        c2 = np.maximum(0.5 / np.sqrt(np.pi) * np.array([-1.5, -1.5, 1.5]) + 0.5, 0)
        assert np.allclose(img[32, 32], 0.99 * c1 + 0.01 * 0.99 * c2)
    bg = np.array([0.3, 0.4, 0.5])
    assert np.allclose(orc.render(np.zeros((0, 3)), np.zeros((0, 56)), VIEW, 100, 100, 32, 32, 32, 32, bg=bg), bg)
    behind, ab = _gauss([0, 0, -1.0], np.log(0.05), 20.0, [1, 1, 1])
    assert np.allclose(orc.render(behind[None], ab[None], VIEW, 100, 100, 16, 16, 32, 32, bg=bg), bg)


def test_sh_basis_equals_library_real_harmonics(orc):
    """Every sign and constant of the 16 functions: the real harmonics built
    from scipy's complex ones (Condon-Shortley phase kept): sqrt(2) Im Y_l^|m|
    for m < 0, Y_l^0, sqrt(2) Re Y_l^m for m > 0, in the order l, m = -l..l."""
    sp = __import__("pytest").importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        __import__("pytest").skip("scipy without sph_harm_y")
    rng = np.random.default_rng(4)
    d = rng.normal(size=(64, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    for v in d:
        theta, phi = np.arccos(v[2]), np.arctan2(v[1], v[0])
        ref = []
        for l in range(4):
            for m in range(-l, l + 1):
                Y = sp.sph_harm_y(l, abs(m), theta, phi)
                ref.append(Y.real if m == 0 else np.sqrt(2) * (Y.real if m > 0 else Y.imag))
        assert np.allclose(orc.sh_basis(v), ref, atol=1e-12)


def test_rotated_anisotropic_gaussian_closed_form(orc):
    """A Gaussian turned by 0.6 rad about the viewing axis with unequal scales:
    its footprint is (f/z)^2 R2 diag(s1^2, s2^2) R2^T + 0.3 I, which pins the
    quaternion-to-rotation convention, the covariance and the conic."""
    f, W, H, zc, th = 100.0, 64, 64, 2.0, 0.6
    s = np.array([0.05, 0.01, 0.02])
    p, a = _gauss([0, 0, zc], np.log(s), 0.0, [0.3, 0.2, 0.1])
    a[3:7] = [np.cos(th / 2), 0, 0, np.sin(th / 2)]  # (w, x, y, z): rotation by th about z
    img = orc.render(p[None], a[None], VIEW, f, f, W / 2 + 0.5, H / 2 + 0.5, W, H)
    R2 = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    S2 = (f / zc) ** 2 * R2 @ np.diag(s[:2] ** 2) @ R2.T + 0.3 * np.eye(2)
    Q = np.linalg.inv(S2)
    col = np.maximum(0.5 / np.sqrt(np.pi) * np.array([0.3, 0.2, 0.1]) + 0.5, 0)
    for dx, dy in ((0, 0), (2, 1), (-2, -1), (1, -2), (3, 2), (0, 3)):
        d = np.array([dx, dy], dtype=np.float64)
        alpha = min(0.99, 0.5 * np.exp(-0.5 * d @ Q @ d))
        want = col * alpha if alpha >= 1 / 255 else np.zeros(3)
        assert np.allclose(img[32 + dy, 32 + dx], want, atol=1e-12), (dx, dy)
    # the long axis follows the rotation: (2, 1) lies near it, (1, -2) across it
    assert img[33, 34, 0] > img[30, 33, 0]


# ---- threshold flags and FP32 error bounds of the check mode (pins of what the GPU parity test excuses) ----
def _check(orc, ps, As, view, f, cx, cy, W, H, bg=(0.1, 0.2, 0.3)):
    return orc.render(np.array(ps, np.float32), np.array(As, np.float32), view, f, f, cx, cy, W, H, bg=bg,
                      check=True)


def test_check_mode_image_equals_render_and_generic_pixels_are_not_flagged(orc):
    from paper_2606_05650_gb300 import synthetic as syn
    pos, attr = syn.static_gs_frame(4, n=3000)
    view = syn.orbit_views(1, radius=1.8)[0]
    img = orc.render(pos, attr, view, 90.0, 90.0, 50, 40, 100, 80)
    img2, flag, tol = orc.render(pos, attr, view, 90.0, 90.0, 50, 40, 100, 80, check=True)
    assert np.array_equal(img, img2)
    assert flag.mean() < 0.01 and (tol >= 0).all()
    p, a = _gauss([0, 0, 2.0], np.log(0.02), 0.0, [1.0, -1.0, 0.5])
    _, flag, tol = _check(orc, [p], [a], VIEW, 100.0, 32.5, 32.5, 64, 64)
    assert not flag.any()
    # background only: the bound is the accumulation term alone, 6 ulp of the largest value
    _, flag, tol = _check(orc, np.zeros((0, 3)), np.zeros((0, 56)), VIEW, 100.0, 32, 32, 20, 10, bg=(0.25, 0.5, 1.0))
    assert not flag.any() and np.allclose(tol, 6 * 2.0 ** -24)


def test_flag_alpha_at_the_cut(orc):
    logit = np.log((1 / 255) / (1 - 1 / 255))  # opacity 1/255 to float rounding: alpha at the centre is the cut
    p, a = _gauss([0, 0, 2.0], np.log(0.02), logit, [1.0, 1.0, 1.0])
    _, flag, _ = _check(orc, [p], [a], VIEW, 100.0, 32.5, 32.5, 64, 64)
    assert flag[32, 32] == 1 and flag.sum() <= 9  # the centre (and at most its neighbours)
    p, a = _gauss([0, 0, 2.0], np.log(0.02), logit + 0.5, [1.0, 1.0, 1.0])  # clear of the cut: nothing flagged
    _, flag, _ = _check(orc, [p], [a], VIEW, 100.0, 32.5, 32.5, 64, 64)
    assert not flag.any()


def test_flag_transmittance_at_the_stop(orc):
    # two splats clamped at alpha 0.99 at the centre: transmittance 0.01 x 0.01 = the 1e-4 stop
    g = [_gauss([0, 0, z], np.log(0.05), 8.0, [1.0, 0.0, 0.0]) for z in (2.0, 3.0)]
    _, flag, _ = _check(orc, [x[0] for x in g], [x[1] for x in g], VIEW, 100.0, 32.5, 32.5, 64, 64)
    assert flag[32, 32] == 1
    g = [_gauss([0, 0, z], np.log(0.05), 3.0, [1.0, 0.0, 0.0]) for z in (2.0, 3.0)]  # alpha 0.95: well above
    _, flag, _ = _check(orc, [x[0] for x in g], [x[1] for x in g], VIEW, 100.0, 32.5, 32.5, 64, 64)
    assert not flag.any()


def test_flag_depths_equal_in_fp32(orc):
    # camera z = z_world + 1e-7 x_world: depths 2 and 2 + 1e-10 are distinct in FP64 and equal in FP32; the
    # farther splat has the lower index, so FP64 depth order and (FP32 depth, index) order disagree
    view = VIEW.copy()
    view[2, 0] = 1e-7
    g = [_gauss([1e-3, 0, 2.0], np.log(0.03), 0.0, [1.0, 0.0, 0.0]), _gauss([0, 0, 2.0], np.log(0.03), 0.0,
                                                                               [0.0, 1.0, 0.0])]
    _, flag, _ = _check(orc, [x[0] for x in g], [x[1] for x in g], view, 100.0, 32.5, 32.5, 64, 64)
    assert flag[32, 32] == 1
    # equal in FP64 as well: index order on both sides, nothing to excuse
    g = [_gauss([0, 0, 2.0], np.log(0.03), 0.0, [1.0, 0.0, 0.0]), _gauss([0, 0, 2.0], np.log(0.03), 0.0,
                                                                            [0.0, 1.0, 0.0])]
    _, flag, _ = _check(orc, [x[0] for x in g], [x[1] for x in g], VIEW, 100.0, 32.5, 32.5, 64, 64)
    assert not flag.any()


def test_flag_tile_rectangle_edge(orc):
    # footprint radius ceil(3 sqrt(lambda_max)) with lambda_max = sigma^2 + sqrt(0.1) (the discriminant floor of an
    # isotropic footprint) and sigma^2 = (f s / z)^2 + 0.3 chosen so that 3 sqrt(lambda_max) = 11.99: radius 12;
    # centre u = 32 - 12 puts the rectangle's right edge exactly on the boundary of tile 2, whose first pixel
    # (12.5 px away) still sees alpha = 0.993 exp(-12.5^2 / (2 sigma^2)) = 0.0068 > 1/255
    f, z = 100.0, 2.0
    sig2 = (11.99 / 3) ** 2 - np.sqrt(0.1)
    s = np.sqrt(sig2 - 0.3) * z / f
    p, a = _gauss([0, 0, z], np.log(s), 5.0, [1.0, 1.0, 1.0])
    _, flag, _ = _check(orc, [p], [a], VIEW, f, 32.0 - 12.0, 8.0, 64, 16)
    assert flag[7, 32] == 1 and flag[7, 31] == 0
    _, flag, _ = _check(orc, [p], [a], VIEW, f, 32.0 - 15.0, 8.0, 64, 16)  # edge inside tile 1: nothing flagged
    assert not flag.any()
