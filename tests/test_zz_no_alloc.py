"""gsnfs_octree_encode_static: the occupancy encoder for callers that may not
allocate device memory while they run (their own memory pool owns the GPU,
or a real-time loop cannot take cudaMalloc's synchronisation).  Called
through the C ABI and compared with gsnfs_octree_encode on two calls in a
row, the second smaller than the first so that anything the shared scratch
kept from the first call would show.  This file sorts last so that a run
stopping at the first failure has already run every other test."""
import ctypes as ct

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
    L = gsnfs.lib()
    L.gsnfs_octree_encode_static.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_uint64, ct.c_uint32, ct.c_void_p,
                                             ct.c_uint64, ct.c_void_p, ct.POINTER(ct.c_uint64)]
    L.gsnfs_octree_encode_static.restype = ct.c_int
    return gsnfs


def _static_call(G, codes, J, cap):
    """One call through the C ABI: (status, occupancy bytes written, level sizes, reported byte count)."""
    nv = codes.shape[0]
    occ = torch.full((max(cap, 4),), 0xAB, dtype=torch.uint8, device="cuda")  # garbage the call must not keep
    lsz = (ct.c_uint32 * (J + 1))()
    nb = ct.c_uint64()
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = G.lib().gsnfs_octree_encode_static(stream, ct.c_void_p(codes.data_ptr()), nv, J, ct.c_void_p(occ.data_ptr()),
                                            cap, lsz, ct.byref(nb))
    return rc, occ[: min(nb.value, cap)].cpu().numpy(), np.array(lsz[:], dtype=np.uint32), nb.value


def _static_encode(G, codes, J):
    nv = codes.shape[0]
    rc, occ, lsz, _ = _static_call(G, codes, J, (8 * max(nv, 1) * J + 64 + 3) & ~3)
    assert rc == 0, G.lib().gsnfs_status_string(rc)
    return occ, lsz


def _codes(orc, seed, n, J):
    pos, _ = syn.DynamicScene(seed).frame(0, n=n)
    codes, *_ = orc.voxelize(pos, np.zeros((n, 1), np.float32), J)
    return torch.from_numpy(codes.astype(np.int64)).cuda()


def test_static_scratch_matches_the_allocating_encoder_twice(G, orc):
    for seed, n, J in ((1, 400_000, 16), (2, 30_000, 12)):
        codes = _codes(orc, seed, n, J)
        got_occ, got_lsz = _static_encode(G, codes, J)
        ref_occ, ref_lsz = G.octree_encode(codes, J)
        assert np.array_equal(got_lsz, ref_lsz)
        assert np.array_equal(got_occ, ref_occ.cpu().numpy())


def test_static_scratch_rejects_sizes_beyond_its_maximum(G):
    L = G.lib()
    codes = torch.zeros(1, dtype=torch.int64, device="cuda")
    occ = torch.zeros(64, dtype=torch.uint8, device="cuda")
    lsz = (ct.c_uint32 * 17)()
    nb = ct.c_uint64()
    rc = L.gsnfs_octree_encode_static(ct.c_void_p(torch.cuda.current_stream().cuda_stream),
                                      ct.c_void_p(codes.data_ptr()), 1048577, 16, ct.c_void_p(occ.data_ptr()), 64,
                                      lsz, ct.byref(nb))
    assert rc == -7  # GSNFS_ERR_UNSUPPORTED


def test_static_capacity_is_counted_in_whole_words(G, orc):
    """Bytes are written as 32-bit words: a capacity equal to a byte count that is not a multiple of 4 is
    too small (GSNFS_ERR_CAPACITY with the byte count reported); rounded up to 4 it suffices."""
    for seed in range(3, 40):
        codes = _codes(orc, seed, 3_000 + 97 * seed, 11)
        ref_occ, ref_lsz = G.octree_encode(codes, 11)
        nb = int(ref_occ.numel())
        if nb % 4:
            break
    assert nb % 4, "no test frame with a byte count off a word boundary"
    rc, _, _, reported = _static_call(G, codes, 11, nb)
    assert rc == -2 and reported == nb  # GSNFS_ERR_CAPACITY
    rc, occ, lsz, reported = _static_call(G, codes, 11, (nb + 3) & ~3)
    assert rc == 0 and reported == nb
    assert np.array_equal(lsz, ref_lsz)
    assert np.array_equal(occ, ref_occ.cpu().numpy())


def test_static_empty_frame(G):
    """No voxels: every level is empty, as with the allocating encoder."""
    codes = torch.zeros(0, dtype=torch.int64, device="cuda")
    for J in (1, 16):
        rc, occ, lsz, reported = _static_call(G, codes, J, 64)
        ref_occ, ref_lsz = G.octree_encode(codes, J)
        assert rc == 0 and reported == 0 and ref_occ.numel() == 0
        assert np.array_equal(lsz, ref_lsz)
