"""GPU parity of each stage of the path against the FP64 oracle, through the
C ABI: voxel set and Morton codes (bit-exact), occupancy bytes and header
(bit-exact, Algorithm 1), octree decoding (Algorithms 2-3), the occupancy
rANS section (byte-identical), RAHT forward / inverse (FP32 within the
tolerance derived from Eq. 1), and block RLGR (byte-identical)."""
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


CASES = [  # (name, n, J): spans several tiles, ragged tails, extreme depths
    ("tiny", 37, 4), ("small", 3000, 10), ("cfg0", 10_000, 10), ("deep", 20_000, 21), ("shallow", 5000, 2),
    ("d16", 60_000, 16),
]


@pytest.mark.parametrize("name,n,J", CASES)
def test_voxel_set_and_codes_bit_exact(G, orc, name, n, J):
    pos, _ = syn.static_gs_frame(11, n)
    codes, lo, ext = G.voxelize(_dev(pos), J)
    ref, _, _, rlo, rext = orc.voxelize(pos, np.zeros((n, 1), np.float32), J)
    assert np.array_equal(codes.cpu().numpy().astype(np.uint64), ref)
    assert np.array_equal(lo, rlo) and ext == rext


def test_voxel_grid_edge_cases(G, orc):
    # identical points, a flat slab, negative coordinates, exact bbox corners
    for pos in (np.full((100, 3), 0.25, np.float32),
                np.c_[np.random.default_rng(0).random((500, 2)), np.zeros(500)].astype(np.float32),
                np.random.default_rng(1).uniform(-50, -49, (800, 3)).astype(np.float32),
                np.array([[0, 0, 0], [1, 1, 1], [0.5, 0.5, 0.5]], np.float32)):
        for J in (1, 7, 21):
            codes, lo, ext = G.voxelize(_dev(pos), J)
            ref, _, _, rlo, rext = orc.voxelize(pos, np.zeros((len(pos), 1), np.float32), J)
            assert np.array_equal(codes.cpu().numpy().astype(np.uint64), ref)


def test_voxel_faces_and_far_offsets(G, orc):
    """Coordinates exactly on voxel faces (lattices of the grid spacing) and
    grids far from the origin: the cases where the fast double-float voxel
    index must defer to the FP64 definition."""
    rng = np.random.default_rng(3)
    for J, off, span in ((4, 0.0, 1.0), (10, 0.0, 1.0), (16, 0.0, 1.0), (21, 0.0, 1.0), (10, 1000.0, 1.0),
                         (21, 1000.0, 1.0), (21, -3.0e5, 7.0), (16, 12345.678, 0.001)):
        k = rng.integers(0, 1 << min(J, 20), (4000, 3))
        pos = (off + span * k / float(1 << min(J, 20))).astype(np.float32)
        pos = np.r_[pos, np.float32([[off, off, off], [off + span, off + span, off + span]])]
        pos = np.r_[pos, (pos[:500] + np.float32(span) * rng.uniform(-1e-6, 1e-6, (500, 3))).astype(np.float32)]
        codes, lo, ext = G.voxelize(_dev(pos), J)
        ref, _, _, rlo, rext = orc.voxelize(pos, np.zeros((len(pos), 1), np.float32), J)
        assert np.array_equal(codes.cpu().numpy().astype(np.uint64), ref), (J, off, span)


@pytest.mark.parametrize("name,n,J", CASES)
def test_occupancy_bytes_bit_exact(G, orc, name, n, J):
    pos, _ = syn.static_gs_frame(12, n)
    codes, _, _, _, _ = orc.voxelize(pos, np.zeros((n, 1), np.float32), J)
    occ, lsz = G.octree_encode(_dev(codes.astype(np.int64)), J)
    vox = np.array([orc.morton_decode(c, J) for c in codes], np.uint32) if codes.size < 30000 else None
    if vox is None:
        lo, ext = orc.bbox(pos)
        vox = np.unique(orc.voxel_coords(pos, J, lo, ext), axis=0)
    ref_occ, ref_lsz = orc.octree_encode(vox, J)
    assert np.array_equal(lsz, ref_lsz)
    assert np.array_equal(occ.cpu().numpy(), ref_occ)
    dec = G.octree_decode(occ, J, lsz)
    assert np.array_equal(dec.cpu().numpy().astype(np.uint64), codes)


def test_octree_paper_example(G, orc):
    # Sec. 2.1: root byte 00011000, then 11111111 for the fully occupied child
    vox = np.array([[2, 2, 0], [3, 2, 0], [2, 3, 0], [3, 3, 0], [2, 2, 1], [3, 2, 1], [2, 3, 1], [3, 3, 1],
                    [1, 0, 2], [1, 1, 2]], np.uint32)
    codes = np.sort(orc.morton_codes(vox, 2)).astype(np.int64)
    occ, lsz = G.octree_encode(_dev(codes), 2)
    assert occ.cpu().numpy().tolist() == [0b00011000, 0b11111111, 0b00001010]
    assert lsz.tolist() == [1, 2, 10]


def test_octree_decode_rejects_corrupt(G, orc):
    pos, _ = syn.static_gs_frame(13, 2000)
    codes, *_ = orc.voxelize(pos, np.zeros((2000, 1), np.float32), 8)
    occ, lsz = G.octree_encode(_dev(codes.astype(np.int64)), 8)
    bad = occ.clone()
    bad[3] = 0
    with pytest.raises(G.GsnfsError):
        G.octree_decode(bad, 8, lsz)
    bad2 = occ.clone()
    bad2[5] ^= 1  # changes the popcount of one byte: the level sizes no longer add up
    with pytest.raises(G.GsnfsError):
        G.octree_decode(bad2, 8, lsz)


@pytest.mark.parametrize("n,kind,chunk", [(0, "u", 16384), (1, "u", 32), (31, "u", 32), (5000, "const", 4096),
                                          (100_000, "skew", 16384), (70_001, "u", 32), (300_000, "skew", 4096),
                                          (50_000, "two", 16384)])
def test_occupancy_section_byte_identical(G, orc, n, kind, chunk):
    rng = np.random.default_rng(n + 7)
    if kind == "u":
        d = rng.integers(0, 256, n).astype(np.uint8)
    elif kind == "const":
        d = np.full(n, 0x42, np.uint8)
    elif kind == "two":
        d = rng.choice(np.array([0x18, 0xFF], np.uint8), n)
    else:
        p = np.exp(-np.arange(256) / 6.0)
        d = rng.choice(256, n, p=p / p.sum()).astype(np.uint8)
    sec = G.occupancy_section_encode(_dev(d), chunk)
    ref = orc.occ_section_encode(d, chunk)
    assert np.array_equal(sec.cpu().numpy(), ref)
    back = G.occupancy_section_decode(_dev(ref), n)
    assert np.array_equal(back.cpu().numpy(), d)


def _raht_tol(orc, codes, A, J, Y64):
    w = orc.raht_node_weights(codes, J).astype(np.float64)
    rms = np.sqrt((A.astype(np.float64) ** 2).mean(0))
    # FP32 error scale of a weighted sum of w inputs (the reading of "1e-5 relative")
    return 1e-5 * (np.abs(Y64) + np.sqrt(w)[:, None] * rms[None, :])


@pytest.mark.parametrize("n,J,C", [(1, 5, 4), (2, 1, 3), (700, 6, 56), (10_000, 10, 56), (30_000, 16, 56),
                                   (50_000, 10, 3), (20_000, 12, 11), (8_000, 21, 35), (4000, 16, 256)])
def test_raht_forward_inverse(G, orc, n, J, C):
    pos, _ = syn.static_gs_frame(20 + C, n)
    codes, _, _, _, _ = orc.voxelize(pos, np.zeros((n, 1), np.float32), J)
    rng = np.random.default_rng(C)
    A = (rng.normal(size=(codes.size, C)) + rng.normal(size=C) * 3).astype(np.float32)
    plan = G.RahtPlan(_dev(codes.astype(np.int64)), J, C)
    Y = plan.forward(_dev(A)).cpu().numpy().astype(np.float64)
    Y64 = orc.raht_forward(codes, A.astype(np.float64), J)
    tol = _raht_tol(orc, codes, A, J, Y64)
    assert (np.abs(Y - Y64) <= tol).all(), np.abs(Y - Y64).max()
    back = plan.inverse(_dev(Y.astype(np.float32))).cpu().numpy()
    np.testing.assert_allclose(back, A, rtol=0, atol=2e-5 * (1 + np.abs(A).max()))
    # in place
    X = _dev(A)
    plan.forward(X, out=X)
    assert np.abs(X.cpu().numpy() - Y).max() == 0.0


def test_raht_energy_and_dc_on_gpu(G, orc):
    pos, _ = syn.DynamicScene(5).frame(0, n=200_000)
    codes, _, _, _, _ = orc.voxelize(pos, np.zeros((len(pos), 1), np.float32), 16)
    A = np.random.default_rng(3).normal(2.0, 1.0, size=(codes.size, 8)).astype(np.float32)
    plan = G.RahtPlan(_dev(codes.astype(np.int64)), 16, 8)
    Y = plan.forward(_dev(A)).cpu().numpy().astype(np.float64)
    np.testing.assert_allclose((Y ** 2).sum(0), (A.astype(np.float64) ** 2).sum(0), rtol=2e-5)
    np.testing.assert_allclose(Y[0], np.sqrt(codes.size) * A.astype(np.float64).mean(0), rtol=2e-5)


def test_raht_inverse_with_quantiser(G, orc):
    # encoder reconstruction: quantise -> dequantise -> inverse (Sec. 3.4, Algorithm 6)
    pos, attr = syn.static_gs_frame(30, 8000)
    J = 10
    codes, A, _, _, _ = orc.voxelize(pos, attr, J)
    qp = G.QuantParams(syn.gs_channel_groups(), syn.GS_BASE_STEPS)
    plan = G.RahtPlan(_dev(codes.astype(np.int64)), J, 56)
    Y = plan.forward(_dev(A.astype(np.float32)))
    R = plan.inverse(Y, qp=qp).cpu().numpy().astype(np.float64)
    # the indices the FP32 path takes: floor(|y| * (1/step) + tau) in FP32, each op rounded
    y32 = Y.cpu().numpy()
    steps = syn.GS_BASE_STEPS[syn.gs_channel_groups()]
    inv32 = (1.0 / steps).astype(np.float32)
    q = np.floor((np.abs(y32) * inv32).astype(np.float32) + np.float32(0.5)) * np.sign(y32)
    # they agree with the FP64 oracle's indices except at rounding boundaries
    Y64 = orc.raht_forward(codes, A, J)
    q64 = orc.quantize(Y64, syn.gs_channel_groups(), syn.GS_BASE_STEPS)
    t = np.abs(Y64) / steps + 0.5
    zone = np.minimum(t - np.floor(t), np.ceil(t) - t) < 1e-4
    assert not ((q != q64) & ~zone).any()
    R64 = orc.raht_inverse(codes, q * steps, J)
    scale = np.sqrt((R64 ** 2).mean(0)) + steps
    assert (np.abs(R - R64) / scale).max() < 1e-4


@pytest.mark.parametrize("nv,C,B", [(1, 1, 32), (1000, 3, 64), (5000, 56, 512), (4097, 7, 4096), (30000, 2, 256)])
def test_rlgr_byte_identical(G, orc, nv, C, B):
    rng = np.random.default_rng(nv + C)
    q = np.round(rng.laplace(0, 2.0, (nv, C)) * (rng.random((nv, C)) < 0.5)).astype(np.int32)
    q[rng.random((nv, C)) < 0.001] = rng.integers(-2 ** 30, 2 ** 30, 1)[0]
    slots, bw = G.rlgr_encode_indices(_dev(q), B)
    slots = slots.cpu().numpy().view(np.uint32)
    bw = bw.cpu().numpy()
    nb = (nv + B - 1) // B
    sw = G.rlgr_slot_words(B)
    for c in range(C):
        for b in range(nb):
            ref = orc.rlgr_encode(q[b * B:(b + 1) * B, c])
            k = b * C + c
            assert bw[k] == ref.size
            assert np.array_equal(slots[k * sw: k * sw + bw[k]], ref)
    back = G.rlgr_decode_indices(_dev(slots.view(np.int32)), _dev(bw), nv, C, B)
    assert np.array_equal(back.cpu().numpy(), q)


def test_rlgr_decode_rejects_truncated_blocks(G):
    q = np.round(np.random.default_rng(0).laplace(0, 5, (2000, 2))).astype(np.int32)
    slots, bw = G.rlgr_encode_indices(_dev(q), 512)
    bw2 = bw.clone()
    bw2[1] = max(int(bw2[1]) // 3, 1)
    with pytest.raises(G.GsnfsError):
        G.rlgr_decode_indices(slots, bw2, 2000, 2, 512)
