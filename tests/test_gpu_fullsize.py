"""Parity at the benchmark's full sizes and launch configuration: frames of
1M Gaussians coded by the batched call exactly as bench.py runs it, the 1M
point dynamic point cloud (depth 10, YCbCr, every quantisation step of its
ladder) with attribute PSNR against the oracle, and the largest frame of a
bandwidth ladder (2M Gaussians at depth 18, 5 rungs).  Each sampled stream is
checked against the oracle (tests/parity.py); the other streams of a batch
must decode on the GPU to the same frames as when decoded one by one."""
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


def test_headline_batch_at_full_size(G, orc):
    # bench.py's step: 8 frames of 1M Gaussians, depth 16, one batched encode and one batched decode
    F, J = 8, 16
    scene = syn.DynamicScene(1000)
    frames = [scene.frame(t, n=1_000_000) for t in range(F)]
    qp = G.QuantParams(syn.gs_channel_groups(), syn.GS_BASE_STEPS)
    out, offs = G.encode_batch([_dev(p) for p, _ in frames], [_dev(a) for _, a in frames], [J] * F, [1.0], qp)
    pos, attr, rows = G.decode_batch(out, offs, 56, F * 1_000_000)
    host = out[: int(offs[-1])].cpu().numpy()
    for f in (0, F - 1):  # sampled frames against the oracle
        s = host[int(offs[f]):int(offs[f + 1])]
        r0, r1 = int(rows[f]), int(rows[f + 1])
        res = compare_stream(orc, s, frames[f][0], frames[f][1], J, qp.groups, qp.steps, qp.tau, qp.rlgr_block,
                             qp.rans_chunk, (pos[r0:r1].cpu().numpy(), attr[r0:r1].cpu().numpy()))
        assert res["nv"] > 900_000
    # every frame: batched decode equals the one-frame decoder
    for f in range(F):
        s = out[int(offs[f]):int(offs[f + 1])]
        p1, a1 = G.decode_frame(s.clone())
        r0, r1 = int(rows[f]), int(rows[f + 1])
        assert torch.equal(pos[r0:r1], p1) and torch.equal(attr[r0:r1], a1), f


@pytest.mark.parametrize("step", [0.025, 0.05, 0.1, 0.2, 0.4])
def test_point_cloud_frame_psnr_matches_oracle(G, orc, step):
    pos, attr = syn.capsule_humanoids_frame(7, 3, 1_000_000)
    qp = G.QuantParams(np.zeros(3, np.uint8), [step])
    bs, nv, _, _ = G.encode_frame(_dev(pos), _dev(attr), 10, qp)
    gp, ga = G.decode_frame(bs)
    res = compare_stream(orc, bs.cpu().numpy(), pos, attr, 10, qp.groups, qp.steps, qp.tau, qp.rlgr_block,
                         qp.rans_chunk, (gp.cpu().numpy(), ga.cpu().numpy()))
    assert nv < 1_000_000  # duplicates merged at 10 bits per axis
    # attribute PSNR (peak 1) of the GPU decode and of the oracle's decode, against the oracle's voxel means
    codes, merged, *_ = orc.voxelize(pos, attr, 10)
    psnr = lambda a: 10 * np.log10(1.0 / ((a - merged) ** 2).mean(0))
    p_gpu, p_orc = psnr(ga.cpu().numpy().astype(np.float64)), psnr(res["dec"]["attr"])
    assert np.abs(p_gpu - p_orc).max() < 0.01, (p_gpu, p_orc)
    # orthonormal transform and |y - y_hat| <= step / 2: MSE <= step^2 / 4
    assert (p_gpu >= 10 * np.log10(4 / step ** 2) - 0.01).all(), p_gpu


def test_ladder_largest_frame(G, orc):
    sizes = [2_000_000, 50_000, 700_000]
    Js = [18, 16, 17]
    scales = [1.0, 2.0, 4.0, 8.0, 16.0]
    scene = syn.DynamicScene(3000)
    frames = [scene.frame(t, n=n) for t, n in enumerate(sizes)]
    qp = G.QuantParams(syn.gs_channel_groups(), syn.GS_BASE_STEPS)
    out, offs = G.encode_batch([_dev(p) for p, _ in frames], [_dev(a) for _, a in frames], Js, scales, qp)
    host = out[: int(offs[-1])].cpu().numpy()
    R = len(scales)
    for r in (0, R - 1):
        k = 0 * R + r
        s = host[int(offs[k]):int(offs[k + 1])]
        compare_stream(orc, s, frames[0][0], frames[0][1], 18, qp.groups, qp.steps * scales[r], qp.tau,
                       qp.rlgr_block, qp.rans_chunk)
    sz = np.diff(offs.astype(np.int64))[:R]
    assert (np.diff(sz) < 0).all(), sz  # coarser rungs, smaller streams
