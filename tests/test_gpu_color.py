"""SH colour decorrelation on the GPU (gsnfs_quant.color, Sec. 4): streams
decode in the oracle decoder; the oracle encoder, given the stream's KLT
matrices or deriving its own, reproduces header, occupancy and (outside the
rounding zone) every quantisation index; the GPU's KLT rows are eigenvectors
of the FP64 sample covariance and equal the oracle's FP64 Jacobi row by row
to FP32 rounding; batched equals plain, the encoder's reconstruction equals
the decoder's output, and correlated colours compress markedly better (the
direction of Table A.8)."""
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
    _check_klt(orc, stream_klt(host), attr)


U32 = 2.0 ** -24  # unit roundoff of FP32


def _check_klt(orc, K32, attr):
    """The stream's KLT (FP64 on the GPU, rounded to FP32) against the sample covariance S of the YUV AC vectors
    of the first 4096 input rows, computed here in FP64 from the definition (Sec. 4):
      - every row is an eigenvector of S up to the FP32 rounding of K: |S k - rho k| <= 8 u |S| (u = 2^-24);
      - rows are orthonormal to FP32 rounding and ordered by decreasing Rayleigh quotient;
      - row by row, K equals the oracle's FP64 Jacobi rounded to FP32, within 2 u plus the perturbation bound of
        an eigenvector, 1e-12 |S| / gap (gap: the row's distance to the other eigenvalues), sign included
        (largest component positive) unless the two largest components are too close to tell."""
    K = K32.astype(np.float64)
    Kor = orc.klt_matrices(attr).astype(np.float64)
    sample = orc.yuv_rows(attr[:4096].astype(np.float64))
    for ch in range(3):
        a = sample[:, 11 + 15 * ch:26 + 15 * ch]
        d = a - a.mean(0)
        S = d.T @ d / a.shape[0]
        nS = np.linalg.norm(S, 2)
        lam = np.linalg.eigvalsh(S)[::-1]
        rho = np.einsum("rk,kl,rl->r", K[ch], S, K[ch])
        res = np.linalg.norm(K[ch] @ S - rho[:, None] * K[ch], axis=1)
        assert res.max() <= 8 * U32 * nS, (ch, res.max() / nS)
        assert np.abs(K[ch] @ K[ch].T - np.eye(15)).max() <= 16 * U32
        assert np.all(np.diff(rho) <= 16 * U32 * nS)
        for r in range(15):
            gap = np.min(np.abs(np.delete(lam, r) - lam[r]))
            tol = 2 * U32 + 1e-12 * nS / max(gap, 1e-300)
            top = np.sort(np.abs(Kor[ch, r]))[-2:]
            sign_clear = top[1] - top[0] > 1e-9
            diff = np.abs(K[ch, r] - Kor[ch, r]).max()
            if not sign_clear:
                diff = min(diff, np.abs(K[ch, r] + Kor[ch, r]).max())
            assert diff <= tol, (ch, r, diff, tol)


@pytest.mark.parametrize("n,J", [(20_000, 12), (150_000, 16)])
def test_colour_stream_parity_with_own_klt(G, orc, n, J):
    """Both sides derive the KLT themselves: the oracle's stream (its own FP64 K) and the GPU's agree on header,
    occupancy and every index, except where the difference of the two K (FP32 rounding) can move a coefficient
    across a rounding boundary."""
    pos, attr = _frame(170 + J, n)
    qp = G.QuantParams(syn.gs_channel_groups(), syn.GS_BASE_STEPS, color=True)
    bs, nv, _, _ = G.encode_frame(_dev(pos), _dev(attr), J, qp)
    gp, ga = G.decode_frame(bs)
    host = bs.cpu().numpy()
    res = compare_stream(orc, host, pos, attr, J, qp.groups, qp.steps, qp.tau, qp.rlgr_block, qp.rans_chunk,
                         (gp.cpu().numpy(), ga.cpu().numpy()), own_klt=True)
    assert res["nv"] == nv
    _check_klt(orc, stream_klt(host), attr)


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
