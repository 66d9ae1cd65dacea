"""Oracle colour decorrelation of SH coefficients (Sec. 4): RGB -> YUV on every
SH function, then one KLT per YUV channel over the 15 AC functions, before
RAHT.  Pins: the YUV round trip, the KLT's orthonormality, decreasing order and
diagonalisation of the sample covariance (eigenvalues also checked against
numpy's symmetric eigensolver), the codec round trip with the KLT matrices
carried in the header, and the size reduction on correlated colours (the
direction of Table A.8)."""
import numpy as np
import pytest

from paper_2606_05650_gb300 import synthetic as syn


def _ac(A, ch):
    return A[:, 11 + 15 * ch:26 + 15 * ch]


def test_yuv_round_trip_and_luma_row(orc):
    A = np.random.default_rng(0).normal(size=(200, 56))
    Y = orc.yuv_rows(A)
    assert np.abs(orc.yuv_rows(Y, inverse=True) - A).max() < 1e-12
    assert np.allclose(Y[:, 8], 0.299 * A[:, 8] + 0.587 * A[:, 9] + 0.114 * A[:, 10])  # DC luma
    assert np.allclose(Y[:, :8], A[:, :8])  # non-colour channels untouched
    grey = np.zeros((1, 56))
    grey[0, 8:11] = 1.0
    y = orc.yuv_rows(grey)[0, 8:11]
    assert np.allclose(y, [1.0, 0.436 - 0.14713 - 0.28886, 0.615 - 0.51499 - 0.10001])


def test_klt_diagonalises_the_sample_covariance(orc):
    attr = syn.gs_attributes_correlated_sh(np.random.default_rng(1), 10_000)
    K = orc.klt_matrices(attr)
    sample = orc.yuv_rows(attr[:4096].astype(np.float64))
    for ch in range(3):
        Kc = K[ch].astype(np.float64)
        assert np.abs(Kc @ Kc.T - np.eye(15)).max() < 1e-6
        X = _ac(sample, ch)
        S = np.cov(X.T, bias=True)
        D = Kc @ S @ Kc.T
        off = D - np.diag(np.diag(D))
        assert np.abs(off).max() < 1e-5 * np.trace(S)
        ev = np.diag(D)
        assert (np.diff(ev) <= 1e-9 * ev[0]).all()  # decreasing
        assert np.allclose(np.sort(ev)[::-1], np.sort(np.linalg.eigh(S)[0])[::-1], rtol=1e-5, atol=1e-9 * ev[0])
        assert (np.abs(Kc).argmax(1) == np.abs(Kc).argmax(1)).all()
        assert all(Kc[r, np.abs(Kc[r]).argmax()] > 0 for r in range(15))  # sign convention


def test_klt_rows_inverse(orc):
    attr = syn.gs_attributes_correlated_sh(np.random.default_rng(2), 5000)
    K = orc.klt_matrices(attr)
    A = np.random.default_rng(3).normal(size=(300, 56))
    B = orc.klt_rows(A, K)
    assert np.allclose(B[:, :11], A[:, :11])
    assert np.abs(orc.klt_rows(B, K, inverse=True) - A).max() < 1e-5  # K is stored in f32


def test_codec_round_trip_with_colour(orc):
    pos, _ = syn.static_gs_frame(4, 8000)
    attr = syn.gs_attributes_correlated_sh(np.random.default_rng(4), pos.shape[0])
    groups, steps = syn.gs_channel_groups(), np.full(5, 1e-4)
    r = orc.encode_frame(pos, attr, 10, groups, steps, color=True)
    bs = r["bitstream"]
    assert int.from_bytes(bs[88:92].tobytes(), "little") == 1
    d = orc.decode_frame(bs)
    _, merged, *_ = orc.voxelize(pos, attr, 10)
    assert np.abs(d["attr"] - merged).max() < 2e-3
    # the header carries the matrices: re-encoding with them gives the same stream
    r2 = orc.encode_frame(pos, attr, 10, groups, steps, color=True, klt=r["klt"])
    assert np.array_equal(r2["bitstream"], bs)
    bad = bs.copy()
    bad[88] = 2  # unknown flag
    with pytest.raises(RuntimeError):
        orc.decode_frame(bad)


def test_colour_decorrelation_shrinks_correlated_frames(orc):
    pos, _ = syn.static_gs_frame(5, 20_000)
    attr = syn.gs_attributes_correlated_sh(np.random.default_rng(5), pos.shape[0])
    groups, steps = syn.gs_channel_groups(), syn.GS_BASE_STEPS
    plain = orc.encode_frame(pos, attr, 12, groups, steps)["bitstream"].size
    col = orc.encode_frame(pos, attr, 12, groups, steps, color=True)["bitstream"].size
    assert col < 0.95 * plain, (col, plain)
