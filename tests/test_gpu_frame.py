"""Whole-frame parity through gsnfs_encode_frame / gsnfs_decode_frame:
GPU streams decode in the oracle decoder with the oracle's exact voxel set,
occupancy bytes and positions; quantised indices equal the oracle's except
at rounding boundaries (counted, < 1e-6 of all coefficients); GPU decoding of
any stream matches the oracle's decoding of it; edge cases and corrupt
streams; the batched frames x rungs path is byte-identical to the plain path.
"""
import numpy as np
import pytest

from paper_2606_05650_gb300 import synthetic as syn
from parity import compare_stream

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


def _qp(G, C, steps=None, **kw):
    if C == 56:
        return G.QuantParams(syn.gs_channel_groups(), syn.GS_BASE_STEPS if steps is None else steps, **kw)
    return G.QuantParams(np.zeros(C, np.uint8), [0.05] if steps is None else steps, **kw)


def check_frame(G, orc, pos, attr, J, qp):
    """Encodes on the GPU and checks the stream against the oracle (tests/parity.py)."""
    C = qp.C
    bs, nv, rpos, rattr = G.encode_frame(_dev(pos), _dev(attr) if C else None, J, qp, recon=True)
    gpos, gattr = G.decode_frame(bs)
    res = compare_stream(orc, bs.cpu().numpy(), pos, attr if C else None, J, qp.groups, qp.steps, qp.tau,
                         qp.rlgr_block, qp.rans_chunk,
                         (gpos.cpu().numpy(), gattr.cpu().numpy() if gattr is not None else None))
    assert nv == res["nv"]
    assert np.array_equal(rpos.cpu().numpy(), res["dec"]["pos"])
    if C and nv:
        # the encoder's reconstruction is the decoder's output
        ga = gattr.cpu().numpy()
        assert np.abs(rattr.cpu().numpy() - ga).max() <= 1e-6 * (1 + np.abs(ga).max())
    return res


@pytest.mark.parametrize("n,J,seed", [(10_000, 10, 0), (3001, 10, 1), (25_000, 16, 2), (999, 21, 3), (500, 1, 4),
                                      (4000, 2, 5)])
def test_static_frames(G, orc, n, J, seed):
    pos, attr = syn.static_gs_frame(seed, n)
    check_frame(G, orc, pos, attr, J, _qp(G, 56))


def test_dynamic_frame_depth16(G, orc):
    pos, attr = syn.DynamicScene(1).frame(3, n=250_000)
    out = check_frame(G, orc, pos, attr, 16, _qp(G, 56))
    assert out["nv"] > 200_000


def test_point_cloud_frame_with_duplicates(G, orc):
    pos, attr = syn.capsule_humanoids_frame(2, 1, 200_000)
    out = check_frame(G, orc, pos, attr, 10, _qp(G, 3, [0.1]))
    assert out["nv"] < 200_000  # duplicates merged


@pytest.mark.parametrize("C", [1, 3, 11, 35])
def test_channel_counts(G, orc, C):
    pos, _ = syn.static_gs_frame(40 + C, 6000)
    attr = np.random.default_rng(C).normal(0, 1, (6000, C)).astype(np.float32)
    check_frame(G, orc, pos, attr, 12, _qp(G, C, [0.07]))


@pytest.mark.parametrize("B,tau,chunk", [(32, 0.5, 32), (256, 1 / 3, 4096), (4096, 0.5, 16384),
                                         (65536, 0.25, 1 << 20)])
def test_block_sizes_deadzone_chunks(G, orc, B, tau, chunk):
    pos, attr = syn.static_gs_frame(50, 9000)
    check_frame(G, orc, pos, attr, 11, _qp(G, 56, tau=tau, rlgr_block=B, rans_chunk=chunk))


def test_edge_cases(G, orc):
    qp = _qp(G, 3, [0.1])
    # empty frame
    e, nv, _, _ = G.encode_frame(torch.zeros((0, 3), device="cuda"), torch.zeros((0, 3), device="cuda"), 8, qp)
    assert nv == 0
    d = orc.decode_frame(e.cpu().numpy())
    assert d["pos"].shape[0] == 0
    p, a = G.decode_frame(e)
    assert p.shape[0] == 0
    # one point; all points in one voxel
    check_frame(G, orc, np.array([[0.1, 0.2, 0.3]], np.float32), np.array([[1, 2, 3]], np.float32), 8, qp)
    pos = np.full((300, 3), 0.5, np.float32)
    attr = np.random.default_rng(0).normal(size=(300, 3)).astype(np.float32)
    check_frame(G, orc, pos, attr, 9, qp)
    # two points that only merge at the last binary level (z siblings)
    check_frame(G, orc, np.array([[0, 0, 0], [0, 0, 1]], np.float32), np.array([[1, 0, 0], [3, 0, 0]], np.float32),
                1, qp)


def test_geometry_only(G, orc):
    pos, _ = syn.static_gs_frame(60, 20_000)
    qp = G.geometry_only()
    bs, nv, rpos, _ = G.encode_frame(_dev(pos), None, 14, qp, recon=True)
    ref = orc.encode_frame(pos, None, 14, np.zeros(0, np.uint8), np.array([1.0]))
    assert np.array_equal(bs.cpu().numpy(), ref["bitstream"])
    p, a = G.decode_frame(bs)
    assert a is None and np.array_equal(p.cpu().numpy(), orc.decode_frame(ref["bitstream"])["pos"])


def test_oracle_streams_decode_on_gpu(G, orc):
    pos, attr = syn.static_gs_frame(70, 7000)
    ref = orc.encode_frame(pos, attr, 10, syn.gs_channel_groups(), syn.GS_BASE_STEPS, with_coeffs=True)
    p, a = G.decode_frame(_dev(ref["bitstream"]))
    d = orc.decode_frame(ref["bitstream"])
    assert np.array_equal(p.cpu().numpy(), d["pos"])
    scale = np.sqrt((d["attr"] ** 2).mean(0)) + 0.02
    assert (np.abs(a.cpu().numpy() - d["attr"]) / scale).max() < 1e-4


def test_corrupt_streams_fail_cleanly(G, orc):
    pos, attr = syn.static_gs_frame(80, 5000)
    bs, *_ = G.encode_frame(_dev(pos), _dev(attr), 10, _qp(G, 56))
    host = bs.cpu().numpy()
    for cut in (50, 100, 700, host.size // 2, host.size - 8):
        with pytest.raises(G.GsnfsError):
            G.decode_frame(_dev(host[:cut].copy()))
    rng = np.random.default_rng(0)
    for _ in range(20):  # random byte flips: error or a valid decode, never a fault
        bad = host.copy()
        k = int(rng.integers(96, host.size))
        bad[k] ^= np.uint8(1 << int(rng.integers(0, 8)))
        try:
            G.decode_frame(_dev(bad))
        except G.GsnfsError:
            pass
    torch.cuda.synchronize()
    # the context still works afterwards
    check_frame(G, orc, pos[:1000], attr[:1000], 10, _qp(G, 56))


def test_batched_ladder_equals_plain(G, orc):
    sizes = [5000, 120_000, 777, 33_333]
    Js = [16, 17, 18, 16]
    frames = [syn.DynamicScene(9).frame(t, n=n) for t, n in enumerate(sizes)]
    scales = [1.0, 2.0, 4.0]
    qp = _qp(G, 56)
    out, offs = G.encode_batch([_dev(p) for p, _ in frames], [_dev(a) for _, a in frames], Js, scales, qp)
    host = out.cpu().numpy()
    for f, ((pos, attr), J) in enumerate(zip(frames, Js)):
        for r, s in enumerate(scales):
            k = f * len(scales) + r
            got = host[int(offs[k]):int(offs[k + 1])]
            qps = _qp(G, 56, syn.GS_BASE_STEPS * s)
            plain, *_ = G.encode_frame(_dev(pos), _dev(attr), J, qps)
            assert np.array_equal(got, plain.cpu().numpy()), (f, r)
    d = orc.decode_frame(host[int(offs[0]):int(offs[1])])
    assert d["codes"].size > 0


def test_batched_segments_with_empty_and_single_point_frames(G, orc):
    """The batched encoder sorts each frame as its own segment: frames that are
    empty, hold one point, fit one sort CTA or span many still give the streams
    of one-frame calls."""
    sizes = [0, 1, 70_000, 2, 0, 4096, 300_001]
    Js = [10, 16, 17, 5, 12, 16, 18]
    frames = [syn.DynamicScene(13).frame(t, n=n) if n else (np.zeros((0, 3), np.float32), np.zeros((0, 56), np.float32))
              for t, n in enumerate(sizes)]
    qp = _qp(G, 56)
    out, offs = G.encode_batch([_dev(p) for p, _ in frames], [_dev(a) for _, a in frames], Js, [1.0], qp)
    host = out.cpu().numpy()
    for f, ((pos, attr), J) in enumerate(zip(frames, Js)):
        plain, *_ = G.encode_frame(_dev(pos), _dev(attr), J, qp)
        assert np.array_equal(host[int(offs[f]):int(offs[f + 1])], plain.cpu().numpy()), f


def test_batched_decoder_equals_per_frame_decoding(G, orc):
    # frames of uneven size and depth (one empty, one tiny) decoded in one batch
    frames = [syn.DynamicScene(11).frame(t, n=n) for t, n in enumerate([40_000, 3, 150_000, 0, 9_000])]
    Js = [16, 9, 18, 12, 17]
    qp = _qp(G, 56)
    streams = []
    for (pos, attr), J in zip(frames, Js):
        bs, *_ = G.encode_frame(_dev(pos), _dev(attr), J, qp)
        streams.append(bs.cpu().numpy())
    offs = np.zeros(len(streams) + 1, np.uint64)
    for i, b in enumerate(streams):
        offs[i + 1] = offs[i] + ((b.size + 7) // 8) * 8
    buf = np.zeros(int(offs[-1]), np.uint8)
    for i, b in enumerate(streams):
        buf[int(offs[i]):int(offs[i]) + b.size] = b
    # each stream's true length
    ends = [int(offs[i]) + streams[i].size for i in range(len(streams))]
    bounds = np.array([int(o) for o in offs[:-1]] + [ends[-1]], np.uint64)
    pos, attr, rows = G.decode_batch(_dev(buf), bounds, 56, sum(p.shape[0] for p, _ in frames) + 8)
    pos, attr = pos.cpu().numpy(), attr.cpu().numpy()
    for i, b in enumerate(streams):
        p1, a1 = G.decode_frame(_dev(b))
        r0, r1 = int(rows[i]), int(rows[i + 1])
        assert r1 - r0 == p1.shape[0]
        assert np.array_equal(pos[r0:r1], p1.cpu().numpy())
        if a1 is not None and r1 > r0:
            assert np.array_equal(attr[r0:r1], a1.cpu().numpy())
        assert np.array_equal(pos[r0:r1], orc.decode_frame(b)["pos"])


def test_batched_decoder_corrupt_streams_fail_cleanly(G, orc):
    """The batched decoder reads every frame's header record out of the streams on the device: truncated
    streams, a bad magic, a header size pointing past the stream and flipped bytes give an error or a valid
    decode, never a fault, and the context decodes a good batch afterwards."""
    frames = [syn.DynamicScene(21).frame(t, n=n) for t, n in enumerate([20_000, 7_000, 30_000])]
    streams = []
    for pos, attr in frames:
        bs, *_ = G.encode_frame(_dev(pos), _dev(attr), 14, _qp(G, 56))
        streams.append(bs.cpu().numpy())

    def batch(parts):
        offs = np.zeros(len(parts) + 1, np.uint64)
        for i, b in enumerate(parts):
            offs[i + 1] = offs[i] + ((b.size + 7) // 8) * 8
        buf = np.zeros(max(int(offs[-1]), 8), np.uint8)
        for i, b in enumerate(parts):
            buf[int(offs[i]):int(offs[i]) + b.size] = b
        bounds = np.array([int(o) for o in offs[:-1]] + [int(offs[-2]) + parts[-1].size], np.uint64)
        return _dev(buf), bounds

    cap = sum(p.shape[0] for p, _ in frames) + 8
    bad_cases = []
    for cut in (40, 96, 200, streams[1].size // 2):  # a truncated middle stream
        bad_cases.append([streams[0], streams[1][:cut].copy(), streams[2]])
    s = streams[1].copy()
    s[0] ^= 0xFF  # magic
    bad_cases.append([streams[0], s, streams[2]])
    s = streams[2].copy()
    s[8:12] = np.frombuffer(np.uint32(1 << 30).tobytes(), np.uint8)  # header size far past the stream
    bad_cases.append([streams[0], streams[1], s])
    for parts in bad_cases:
        buf, bounds = batch(parts)
        with pytest.raises(G.GsnfsError):
            G.decode_batch(buf, bounds, 56, cap)
    rng = np.random.default_rng(5)
    for _ in range(12):  # flipped bytes past the fixed header: an error or a valid decode
        parts = [x.copy() for x in streams]
        f = int(rng.integers(0, 3))
        k = int(rng.integers(96, parts[f].size))
        parts[f][k] ^= np.uint8(1 << int(rng.integers(0, 8)))
        buf, bounds = batch(parts)
        try:
            G.decode_batch(buf, bounds, 56, cap)
        except G.GsnfsError:
            pass
    torch.cuda.synchronize()
    buf, bounds = batch(streams)
    pos, attr, rows = G.decode_batch(buf, bounds, 56, cap)
    for i, b in enumerate(streams):
        r0, r1 = int(rows[i]), int(rows[i + 1])
        assert np.array_equal(pos[r0:r1].cpu().numpy(), orc.decode_frame(b)["pos"])


def test_peek_reads_host_and_device_headers(G, orc):
    """gsnfs_peek_frame takes the header in device memory as well as in host memory, and agrees with the
    oracle's decoding of the same stream."""
    qp = _qp(G, 56)
    p, a = syn.DynamicScene(7).frame(0, n=20_000)
    bs, nv, _, _ = G.encode_frame(_dev(p), _dev(a), 14, qp)
    want = (nv, 56, 14)
    assert G.peek_frame(bs) == want  # device tensor
    assert G.peek_frame(bs[:96].contiguous()) == want
    assert G.peek_frame(bs.cpu()) == want  # host tensor
    assert G.peek_frame(bs.cpu().numpy()) == want
    assert orc.decode_frame(bs.cpu().numpy())["pos"].shape[0] == nv
    with pytest.raises(G.GsnfsError):
        G.peek_frame(bs[:95].contiguous())  # fewer than 96 bytes
    bad = bs[:96].clone()
    bad[0] ^= 0xFF  # magic
    with pytest.raises(G.GsnfsError):
        G.peek_frame(bad)
