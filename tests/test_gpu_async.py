"""Header records and the asynchronous batched decoder: gsnfs_encode_batch_headers returns, with the offsets, each
stream's header record (its header tables, the head of its occupancy section and of its attribute section, as the
decoder reads them); gsnfs_decode_batch_async, given those records, decodes without reading anything back and
reports its status in a word written in stream order.  Outputs equal the synchronous decoder's bit for bit."""
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


def _frames(sizes, seed=300):
    scene = syn.DynamicScene(seed)
    out = []
    for t, n in enumerate(sizes):
        p, a = scene.frame(t, n=n)
        out.append((torch.from_numpy(p).cuda(), torch.from_numpy(a).cuda()))
    return out


def _record_from_stream(host, off, end, R):
    """The header record as the decoder would read it from the stream bytes (independent of the library)."""
    b = host[off:end]
    hb = int.from_bytes(b[8:12].tobytes(), "little")
    occ = int.from_bytes(b[72:80].tobytes(), "little")
    attr = int.from_bytes(b[80:88].tobytes(), "little")
    r = np.zeros(R, dtype=np.uint8)
    r[:hb] = b[:hb]
    k = min(24, occ + attr)
    r[4096:4096 + k] = b[hb:hb + k]
    if attr >= 8:
        r[4160:4168] = b[hb + occ:hb + occ + 8]
    return r


@pytest.mark.parametrize("rungs,color", [([1.0], False), ([1.0, 4.0], False), ([1.0, 2.0], True)])
def test_async_decode_equals_sync_decode(G, rungs, color):
    frames = _frames([30_000, 5_000, 1, 60_000, 0, 12_000])
    Js = [16, 12, 10, 17, 9, 14]
    qp = G.QuantParams(syn.gs_channel_groups(), syn.GS_BASE_STEPS, color=color)
    out, offs, hdr = G.encode_batch([p for p, _ in frames], [a for _, a in frames], Js, rungs, qp, headers=True)
    out2, offs2 = G.encode_batch([p for p, _ in frames], [a for _, a in frames], Js, rungs, qp)
    assert np.array_equal(offs, offs2) and torch.equal(out[:int(offs[-1])], out2[:int(offs[-1])])
    host = out[:int(offs[-1])].cpu().numpy()
    for i in range(len(offs) - 1):
        assert np.array_equal(hdr[i], _record_from_stream(host, int(offs[i]), int(offs[i + 1]), G.HEADER_RECORD_BYTES)), i
    rows_cap = sum(int(p.shape[0]) for p, _ in frames) * len(rungs)
    pos0, attr0, rows0 = G.decode_batch(out, offs, 56, rows_cap)
    pos1 = torch.full((max(rows_cap, 1), 3), -7.0, device="cuda")
    attr1 = torch.full((max(rows_cap, 1), 56), -7.0, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    rows1 = G.decode_batch_async(out, offs, hdr, 56, rows_cap, pos1, attr1, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    n = int(rows0[-1])
    assert np.array_equal(rows0, rows1)
    assert torch.equal(pos0, pos1[:n]) and torch.equal(attr0, attr1[:n])


def test_async_decode_back_to_back_calls_reuse_staging(G):
    """Six asynchronous decodes in a row on one stream (more than the four staging slots), statuses in pinned host
    memory, each equal to the synchronous decode of its own streams."""
    qp = G.QuantParams(syn.gs_channel_groups(), syn.GS_BASE_STEPS)
    batches = []
    for k in range(3):
        frames = _frames([20_000 + 7_000 * k, 9_000], seed=310 + k)
        out, offs, hdr = G.encode_batch([p for p, _ in frames], [a for _, a in frames], [15, 13], [1.0], qp,
                                        headers=True)
        batches.append((out, offs, hdr, sum(int(p.shape[0]) for p, _ in frames)))
    status = torch.full((6,), -1, dtype=torch.int32).pin_memory()
    results = []
    for k in range(6):
        out, offs, hdr, cap = batches[k % 3]
        pos = torch.empty((cap, 3), device="cuda")
        attr = torch.empty((cap, 56), device="cuda")
        rows = G.decode_batch_async(out, offs, hdr, 56, cap, pos, attr, status[k:k + 1])
        results.append((pos, attr, rows))
    torch.cuda.synchronize()
    assert status.tolist() == [0] * 6
    for k, (pos, attr, rows) in enumerate(results):
        out, offs, hdr, cap = batches[k % 3]
        p0, a0, r0 = G.decode_batch(out, offs, 56, cap)
        n = int(r0[-1])
        assert torch.equal(p0, pos[:n]) and torch.equal(a0, attr[:n]), k


def test_async_decode_rejects_bad_records(G):
    frames = _frames([8_000])
    qp = G.QuantParams(syn.gs_channel_groups(), syn.GS_BASE_STEPS)
    out, offs, hdr = G.encode_batch([frames[0][0]], [frames[0][1]], [12], [1.0], qp, headers=True)
    bad = hdr.copy()
    bad[0, 0] ^= 0xFF  # magic
    pos = torch.empty((8_000, 3), device="cuda")
    attr = torch.empty((8_000, 56), device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(G.GsnfsError):
        G.decode_batch_async(out, offs, bad, 56, 8_000, pos, attr, status)
    bad = hdr.copy()
    bad[0, 12:16] = np.frombuffer(np.uint32(30).tobytes(), dtype=np.uint8)  # depth beyond the supported range
    with pytest.raises(G.GsnfsError):
        G.decode_batch_async(out, offs, bad, 56, 8_000, pos, attr, status)
