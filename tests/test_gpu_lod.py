"""Level-of-detail decoding (gsnfs_decode_frame_lod) against the oracle: node
centres at depth Jp bit-exact, node mean attributes equal to the oracle's
means of its own decode of the same stream, full depth equal to the plain
decoder, errors on bad depths."""
import numpy as np
import pytest

from paper_2606_05650_gb300 import synthetic as syn

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


@pytest.mark.parametrize("J,color", [(12, False), (16, False), (13, True)])
def test_lod_matches_oracle(G, orc, J, color):
    pos, attr = syn.DynamicScene(60).frame(0, n=60_000)
    if color:  # SH rows with correlated colour channels, coded with YUV + KLT
        attr = syn.gs_attributes_correlated_sh(np.random.default_rng(61), pos.shape[0])
    qp = G.QuantParams(syn.gs_channel_groups(), syn.GS_BASE_STEPS, color=color)
    bs, nv, _, _ = G.encode_frame(torch.from_numpy(pos).cuda(), torch.from_numpy(attr).cuda(), J, qp)
    host = bs.cpu().numpy()
    dec = orc.decode_frame(host)
    lo = np.frombuffer(host[32:56].tobytes(), dtype=np.float64)
    ext = float(np.frombuffer(host[56:64].tobytes(), dtype=np.float64)[0])
    for Jp in sorted({J, J - 1, J - 4, J // 2, 1, 0}, reverse=True):
        gp, ga = G.decode_frame_lod(bs, Jp)
        nc, npos, na, nw = orc.lod(dec["codes"], dec["attr"], J, Jp, lo, ext)
        assert gp.shape[0] == nc.size, Jp
        assert np.array_equal(gp.cpu().numpy(), npos), Jp
        scale = np.sqrt((na ** 2).mean(0)) + 1e-3
        assert (np.abs(ga.cpu().numpy() - na) / scale).max() < 1e-4, Jp
    p1, a1 = G.decode_frame(bs)
    gp, ga = G.decode_frame_lod(bs, J)
    assert torch.equal(gp, p1) and torch.equal(ga, a1)


def test_lod_rejects_depth_beyond_J(G):
    pos, attr = syn.static_gs_frame(61, 2000)
    qp = G.QuantParams(syn.gs_channel_groups(), syn.GS_BASE_STEPS)
    bs, *_ = G.encode_frame(torch.from_numpy(pos).cuda(), torch.from_numpy(attr).cuda(), 10, qp)
    with pytest.raises(G.GsnfsError):
        G.decode_frame_lod(bs, 11)
