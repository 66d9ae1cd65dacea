"""Whole-frame pins of the oracle codec: lossless geometry (the decoded voxel
set is exactly the distinct voxel set, Sec. 2.3), positions at voxel centres
(Sec. 2.1), Parseval between coefficient and attribute error (RAHT is
orthonormal, Sec. 3.1), the uniform-quantiser error bound (Sec. 3.4), the
edge cases, and rejection of corrupt streams."""
import numpy as np
import pytest

from paper_2606_05650_gb300 import synthetic as syn


def _enc(orc, pos, attr, J, C=None, **kw):
    if attr is not None and attr.shape[1] == 56:
        groups, steps = syn.gs_channel_groups(), syn.GS_BASE_STEPS
    else:
        C = 0 if attr is None else attr.shape[1]
        groups, steps = np.zeros(C, np.uint8), np.array([0.05])
    return orc.encode_frame(pos, attr, J, groups, steps, with_coeffs=True, **kw)


def test_frame_roundtrip_static_gs(orc):
    pos, attr = syn.static_gs_frame(0, 4000)
    J = 10
    r = _enc(orc, pos, attr, J)
    d = orc.decode_frame(r["bitstream"])
    codes, A, cnt, lo, ext = orc.voxelize(pos, attr, J)
    np.testing.assert_array_equal(d["codes"], codes)                 # exact voxel set
    np.testing.assert_array_equal(d["codes"], r["codes"])
    np.testing.assert_array_equal(d["q"], r["q"])                    # lossless entropy stages
    np.testing.assert_array_equal(d["pos"], orc.voxel_centres(codes, J, lo, ext))
    # Parseval: attribute-domain error energy equals coefficient-domain error energy
    steps = syn.GS_BASE_STEPS[syn.gs_channel_groups()]
    Yhat = d["q"] * steps
    e_coef = ((Yhat - r["coeffs"]) ** 2).sum(0)
    e_attr = ((d["attr"] - A) ** 2).sum(0)
    np.testing.assert_allclose(e_attr, e_coef, rtol=1e-9, atol=1e-12)
    # uniform quantiser (tau = 1/2): every coefficient within half a step
    assert np.all(np.abs(Yhat - r["coeffs"]) <= steps / 2 + 1e-12)


def test_point_cloud_psnr_high_rate_estimate(orc):
    # Sec. 5.4: point clouds at J = 10 with colour step 0.1; the uniform
    # quantiser's high-rate error is step^2 / 12, PSNR 10 log10(12 / step^2) ~ 30.8 dB
    pos, attr = syn.capsule_humanoids_frame(2, 0, 20_000)
    r = orc.encode_frame(pos, attr, 10, np.zeros(3, np.uint8), np.array([0.1]), with_coeffs=True)
    d = orc.decode_frame(r["bitstream"])
    _, A, _, _, _ = orc.voxelize(pos, attr, 10)
    mse = ((d["attr"] - A) ** 2).mean(0)
    psnr = 10 * np.log10(1.0 / mse)
    assert (psnr >= 30.0).all() and (psnr < 40).all()


@pytest.mark.parametrize("J", [1, 2, 21])
def test_frame_extreme_depths(orc, J):
    pos, attr = syn.static_gs_frame(J, 700)
    r = _enc(orc, pos, attr, J)
    d = orc.decode_frame(r["bitstream"])
    np.testing.assert_array_equal(d["codes"], r["codes"])
    assert d["codes"].size <= min(700, 8 ** J)


def test_frame_empty_single_and_one_voxel(orc):
    z = orc.encode_frame(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32), 8,
                         np.zeros(3, np.uint8), np.array([0.1]))
    d = orc.decode_frame(z["bitstream"])
    assert z["nv"] == 0 and d["pos"].shape == (0, 3)
    one = orc.encode_frame(np.array([[0.3, 0.2, 0.1]], np.float32), np.array([[1.0, 2.0, 3.0]], np.float32),
                           8, np.zeros(3, np.uint8), np.array([0.1]), with_coeffs=True)
    d = orc.decode_frame(one["bitstream"])
    assert one["nv"] == 1 and d["attr"].shape == (1, 3)
    np.testing.assert_allclose(d["attr"][0], [1.0, 2.0, 3.0], atol=0.05)
    # all Gaussians in one voxel: the merged attribute is the mean
    pos = np.full((50, 3), 0.5, np.float32)
    attr = np.random.default_rng(1).normal(size=(50, 3)).astype(np.float32)
    r = orc.encode_frame(pos, attr, 6, np.zeros(3, np.uint8), np.array([1e-4]), with_coeffs=True)
    d = orc.decode_frame(r["bitstream"])
    assert r["nv"] == 1
    np.testing.assert_allclose(d["attr"][0], attr.astype(np.float64).mean(0), atol=1e-4)


def test_geometry_only_frame(orc):
    pos, _ = syn.static_gs_frame(4, 3000)
    r = orc.encode_frame(pos, None, 12, np.zeros(0, np.uint8), np.array([1.0]))
    d = orc.decode_frame(r["bitstream"])
    np.testing.assert_array_equal(d["codes"], r["codes"])
    assert d["attr"].shape[1] == 0


def test_corrupt_streams_are_rejected(orc):
    pos, attr = syn.static_gs_frame(5, 2000)
    bs = _enc(orc, pos, attr, 10)["bitstream"]
    for cut in (10, 100, bs.size // 2, bs.size - 9):
        with pytest.raises(RuntimeError):
            orc.decode_frame(bs[:cut])
    bad = bs.copy()
    bad[0] ^= 0xFF
    with pytest.raises(RuntimeError):
        orc.decode_frame(bad)
