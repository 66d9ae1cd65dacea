"""CUDA-graph replay of the encoder: streams from replayed graphs are
byte-identical to direct launches while the frames' contents, pointers, steps
and rung scales change between replays; a new request shape is captured
anew; the launch counter counts the replayed kernels."""
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
    yield gsnfs
    gsnfs.set_graphs(False)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _qp(G, scale=1.0):
    return G.QuantParams(syn.gs_channel_groups(), np.array(syn.GS_BASE_STEPS) * scale)


def test_replayed_frames_equal_direct_launches(G, orc):
    n, J = 20_000, 14
    frames = [syn.DynamicScene(21).frame(t, n=n) for t in range(4)]
    qp0 = _qp(G)
    buf = torch.empty(G.max_bitstream_bytes(n, J, qp0), dtype=torch.uint8, device="cuda")
    direct = []
    G.set_graphs(False)
    for t, (p, a) in enumerate(frames):
        bs, *_ = G.encode_frame(_dev(p), _dev(a), J, _qp(G, 1 + t), out=buf)
        direct.append(bs.cpu().numpy())
    G.set_graphs(True)
    s0 = G.graph_stats()
    l0 = G.launch_count()
    for t, (p, a) in enumerate(frames):
        bs, *_ = G.encode_frame(_dev(p), _dev(a), J, _qp(G, 1 + t), out=buf)
        assert np.array_equal(bs.cpu().numpy(), direct[t]), t
    s1 = G.graph_stats()
    assert s1[1] - s0[1] == 1 and s1[0] - s0[0] == 3 and s1[2] == s0[2]  # one capture, three replays
    assert G.launch_count() - l0 > 4 * 20  # replays count their kernels
    # another shape: captured anew, still identical
    p, a = frames[0]
    G.set_graphs(False)
    ref, *_ = G.encode_frame(_dev(p[:5000]), _dev(a[:5000]), J, qp0, out=buf)
    ref = ref.cpu().numpy()
    G.set_graphs(True)
    for _ in range(2):
        got, *_ = G.encode_frame(_dev(p[:5000]), _dev(a[:5000]), J, qp0, out=buf)
        assert np.array_equal(got.cpu().numpy(), ref)
    s2 = G.graph_stats()
    assert s2[1] - s1[1] == 1 and s2[0] - s1[0] == 1
    assert orc.decode_frame(ref)["pos"].shape[0] > 0


def test_replayed_batches_equal_direct_launches(G):
    sizes, Js = [30_000, 7_000, 12_345], [16, 17, 18]
    scales = [1.0, 2.0, 4.0, 8.0, 16.0]
    qp = _qp(G)
    outs = {}
    for graphs in (False, True):
        G.set_graphs(graphs)
        out = None
        for t in range(3):
            frames = [syn.DynamicScene(30 + t).frame(f, n=n) for f, n in enumerate(sizes)]
            out, offs = G.encode_batch([_dev(p) for p, _ in frames], [_dev(a) for _, a in frames], Js,
                                       [s * (1 + t) for s in scales], qp, out=out)
            outs[(graphs, t)] = out[: int(offs[-1])].cpu().numpy()
    for t in range(3):
        assert np.array_equal(outs[(False, t)], outs[(True, t)]), t
    assert G.graph_stats()[2] == 0
