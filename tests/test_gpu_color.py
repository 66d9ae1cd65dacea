"""SH colour decorrelation on the GPU (gsnfs_quant.color, Sec. 4): streams
decode in the oracle decoder, the oracle encoder given the stream's KLT
matrices reproduces header, occupancy and (outside the rounding zone) every
quantisation index, the GPU's KLT diagonalises the sample covariance, batched
equals plain, the encoder's reconstruction equals the decoder's output, and
correlated colours compress markedly better (the direction of Table A.8)."""
import numpy as np
import pytest

from paper_2606_05650_gb300 import synthetic as syn
from parity import compare_stream, stream_klt

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_05650_gb300 import gsnfs
    return gsnfs


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _frame(seed, n):
    pos, _ = syn.DynamicScene(seed).frame(0, n=n)
    return pos, syn.gs_attributes_correlated_sh(np.random.default_rng(seed), n)


@pytest.mark.parametrize("n,J", [(20_000, 12), (150_000, 16)])
def test_colour_stream_parity(G, orc, n, J):
    pos, attr = _frame(70 + J, n)
    qp = G.QuantParams(syn.gs_channel_groups(), syn.GS_BASE_STEPS, color=True)
    bs, nv, rp, ra = G.encode_frame(_dev(pos), _dev(attr), J, qp, recon=True)
    gp, ga = G.decode_frame(bs)
    host = bs.cpu().numpy()
    res = compare_stream(orc, host, pos, attr, J, qp.groups, qp.steps, qp.tau, qp.rlgr_block, qp.rans_chunk,
                         (gp.cpu().numpy(), ga.cpu().numpy()))
    assert res["nv"] == nv
    ga = ga.cpu().numpy()
    assert np.abs(ra.cpu().numpy() - ga).max() <= 1e-5 * (1 + np.abs(ga).max())
    # the GPU's KLT (FP32 in the stream) diagonalises the sample covariance of the YUV AC vectors
    K = stream_klt(host).astype(np.float64)
    sample = orc.yuv_rows(attr[:4096].astype(np.float64))
    for ch in range(3):
        S = np.cov(sample[:, 11 + 15 * ch:26 + 15 * ch].T, bias=True)
        D = K[ch] @ S @ K[ch].T
        assert np.abs(D - np.diag(np.diag(D))).max() < 1e-5 * np.trace(S)
        assert np.abs(K[ch] - orc.klt_matrices(attr)[ch]).max() < 1e-3  # same basis as the oracle's KLT


def test_colour_batch_equals_plain_and_shrinks(G, orc):
    frames = [_frame(80 + t, n) for t, n in enumerate([40_000, 9_000, 25_000])]
    Js = [16, 13, 15]
    qpc = G.QuantParams(syn.gs_channel_groups(), syn.GS_BASE_STEPS, color=True)
    qp0 = G.QuantParams(syn.gs_channel_groups(), syn.GS_BASE_STEPS)
    out, offs = G.encode_batch([_dev(p) for p, _ in frames], [_dev(a) for _, a in frames], Js, [1.0, 4.0], qpc)
    host = out[: int(offs[-1])].cpu().numpy()
    for f, ((pos, attr), J) in enumerate(zip(frames, Js)):
        plain, *_ = G.encode_frame(_dev(pos), _dev(attr), J, qpc)
        assert np.array_equal(host[int(offs[2 * f]):int(offs[2 * f + 1])], plain.cpu().numpy()), f
        nocol, *_ = G.encode_frame(_dev(pos), _dev(attr), J, qp0)
        assert plain.numel() < 0.8 * nocol.numel(), (plain.numel(), nocol.numel())
    # batched decoding of colour streams equals one-by-one decoding
    pos, attr, rows = G.decode_batch(out, offs, 56, sum(p.shape[0] for p, _ in frames) * 2)
    for k in range(len(offs) - 1):
        p1, a1 = G.decode_frame(out[int(offs[k]):int(offs[k + 1])].clone())
        r0, r1 = int(rows[k]), int(rows[k + 1])
        assert torch.equal(pos[r0:r1], p1) and torch.equal(attr[r0:r1], a1), k
