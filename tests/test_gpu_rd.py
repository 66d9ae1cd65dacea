"""Distortion returned by the batched encoder (gsnfs_encode_batch_rd): equal
to the oracle's FP64 sum of squared coefficient errors, equal (Parseval) to
the squared error of the GPU-decoded attributes against the voxel means, and
no effect on the bitstreams; the R-D hull of a ladder is increasing."""
import numpy as np
import pytest

from paper_2606_05650_gb300 import rd, synthetic as syn

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


def test_distortion_matches_oracle_and_decoded_error(G, orc):
    frames = [syn.DynamicScene(50).frame(t, n=n) for t, n in enumerate([30_000, 12_000])]
    Js = [13, 12]
    scales = [1.0, 4.0, 16.0]
    qp = G.QuantParams(syn.gs_channel_groups(), syn.GS_BASE_STEPS)
    P, A = [_dev(p) for p, _ in frames], [_dev(a) for _, a in frames]
    out, offs, dist = G.encode_batch(P, A, Js, scales, qp, distortion=True)
    out2, offs2 = G.encode_batch(P, A, Js, scales, qp)
    assert np.array_equal(offs, offs2)
    assert torch.equal(out[: int(offs[-1])], out2[: int(offs2[-1])])
    R = len(scales)
    for f, ((pos, attr), J) in enumerate(zip(frames, Js)):
        codes, merged, *_ = orc.voxelize(pos, attr, J)
        for r, sc in enumerate(scales):
            steps = qp.steps * sc
            ref = orc.encode_frame(pos, attr, J, qp.groups, steps, qp.tau, qp.rlgr_block, qp.rans_chunk,
                                   with_coeffs=True)
            st = steps[qp.groups]
            e64 = ((ref["coeffs"] - ref["q"] * st) ** 2).sum(0)
            assert np.allclose(dist[f, r], e64, rtol=2e-3, atol=1e-9), (f, r)
            # Parseval: decoded attributes against the voxel means
            k = f * R + r
            gp, ga = G.decode_frame(out[int(offs[k]):int(offs[k + 1])].clone())
            dec_err = ((ga.cpu().numpy().astype(np.float64) - merged) ** 2).sum(0)
            assert np.allclose(dist[f, r], dec_err, rtol=2e-3, atol=1e-6), (f, r)


def test_ladder_hull_and_selection(G):
    frames = [syn.DynamicScene(51).frame(t, n=40_000) for t in range(3)]
    scales = [1.0, 2.0, 4.0, 8.0, 16.0]
    qp = G.QuantParams(syn.gs_channel_groups(), syn.GS_BASE_STEPS)
    out, offs, dist = G.encode_batch([_dev(p) for p, _ in frames], [_dev(a) for _, a in frames], [16] * 3,
                                     scales, qp, distortion=True)
    rate = np.diff(offs.astype(np.int64)).reshape(3, len(scales))
    nv = [G.peek_frame(out[int(offs[k]):int(offs[k + 1])].cpu().numpy())[0] for k in range(0, 15, 5)]
    q = rd.psnr(dist, nv)
    for f in range(3):
        assert (np.diff(rate[f]) < 0).all() and (np.diff(q[f]) < 0).all()  # coarser: smaller and worse
        assert rd.upper_hull(rate[f], q[f])  # non-empty, increasing by construction
    sel = rd.select(rate, q, rate[:, 2])
    assert (rate[np.arange(3), sel] <= rate[:, 2]).all()


def test_rendered_psnr_ladder_and_selection(G):
    """Rendered-view PSNR (Sec. 5.1's measure) per rung of a ladder: decoded
    frames rendered by the GPU rasteriser against the original Gaussians fall
    in quality as the steps grow, the hull keeps the best rung, and a budget
    picks the best hull rung that fits."""
    pos, attr = syn.static_gs_frame(7, n=40_000)
    scales = [0.5, 2.0, 8.0, 32.0]
    qp = G.QuantParams(syn.gs_channel_groups(), syn.GS_BASE_STEPS)
    P, A = [_dev(pos)], [_dev(attr)]
    out, offs = G.encode_batch(P, A, [14], scales, qp)
    views = syn.orbit_views(2, radius=1.6)

    def render(p, a, v):
        return G.render(p, a.contiguous(), v, 300.0, 300.0, 160, 120, 320, 240)
    q = []
    for r in range(len(scales)):
        dp, da = G.decode_frame(out[int(offs[r]):int(offs[r + 1])])
        q.append(rd.rendered_psnr(render, (P[0], A[0]), (dp, da), views))
    rate = np.diff(offs.astype(np.int64))
    assert all(q[r] > q[r + 1] for r in range(len(q) - 1)), q
    assert all(rate[r] > rate[r + 1] for r in range(len(rate) - 1)), rate
    assert q[0] > 30.0
    hull = rd.upper_hull(rate, q)
    assert 0 in hull and (len(scales) - 1) in hull
    sel = rd.select(rate[None], np.array(q)[None], [rate[1] + 1])
    assert sel[0] in hull and rate[sel[0]] <= rate[1] + 1 and q[sel[0]] >= q[1]
