"""Pins of the oracle's geometry path (voxelisation, Morton codes, octree)
against what the paper fixes: the Sec. 2.2 Morton examples, the Sec. 2.1
occupancy-byte example, the counting invariants of Algorithm 1's header, the
round trip through Algorithms 2-3, and brute force on tiny frames."""
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _lines(name):
    with open(os.path.join(GOLD, name)) as f:
        return [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]


def test_morton_paper_examples(orc):
    for ln in _lines("morton_examples.txt"):
        t = ln.split()
        if t[0] == "parent":
            J, code, parent = int(t[1]), int(t[2], 2), int(t[3], 2)
            assert code >> 3 == parent
        elif t[0] == "child":
            node, i, child = int(t[1], 2), int(t[2]), int(t[3], 2)
            assert (node << 3) + i == child
        else:
            J, x, y, z, code = int(t[0]), int(t[1]), int(t[2]), int(t[3]), int(t[4], 2)
            assert orc.morton(x, y, z, J) == code
            assert orc.morton_decode(code, J) == (x, y, z)


def _morton_text(x, y, z, J):
    # Sec. 2.2 definition read literally: concatenate z_b y_b x_b from b=J-1 down to 0
    s = "".join(f"{(z >> b) & 1}{(y >> b) & 1}{(x >> b) & 1}" for b in range(J - 1, -1, -1))
    return int(s, 2)


@pytest.mark.parametrize("J", [1, 2, 5, 10, 16, 21])
def test_morton_matches_text_definition_and_roundtrips(orc, J):
    rng = np.random.default_rng(J)
    v = rng.integers(0, 1 << J, size=(200, 3), dtype=np.uint64).astype(np.uint32)
    codes = orc.morton_codes(v, J)
    for (x, y, z), m in zip(v, codes):
        assert int(m) == _morton_text(int(x), int(y), int(z), J)
        assert orc.morton_decode(int(m), J) == (int(x), int(y), int(z))
    assert int(codes.max()) < (1 << (3 * J))          # unused high bits are zero


def test_voxel_grid_corners_and_cells(orc):
    # bbox corners land in the first and last cell; the centre in cell 2^(J-1)
    pos = np.array([[0, 0, 0], [1, 1, 1], [0.5, 0.5, 0.5], [0.25, 0.75, 0.0]], np.float32)
    for J in (1, 3, 10, 21):
        v = orc.voxel_coords(pos, J)
        assert v[0].tolist() == [0, 0, 0]
        assert v[1].tolist() == [(1 << J) - 1] * 3
        assert v[2].tolist() == [1 << (J - 1)] * 3
        if J >= 2:
            assert v[3].tolist() == [1 << (J - 2), 3 << (J - 2), 0]


def test_voxel_grid_is_one_cube_over_longest_axis(orc):
    # reading: one cube of side max extent (voxels are cubes)
    pos = np.array([[0, 0, 0], [2, 1, 0.5]], np.float32)
    lo, ext = orc.bbox(pos)
    assert ext == 2.0 and lo.tolist() == [0, 0, 0]
    v = orc.voxel_coords(pos, 4)
    assert v[1].tolist() == [15, 8, 4]


def test_voxel_centres_within_half_cell(orc):
    from paper_2606_05650_gb300 import synthetic as syn
    pos, _ = syn.static_gs_frame(3, 5000)
    J = 10
    lo, ext = orc.bbox(pos)
    v = orc.voxel_coords(pos, J, lo, ext)
    c = orc.voxel_centres(orc.morton_codes(v, J), J, lo, ext)
    cell = ext / 2 ** J
    assert np.abs(c.astype(np.float64) - pos).max() <= 0.5 * cell * (1 + 1e-5) + 1e-7


def test_merge_is_mean_per_voxel(orc):
    rng = np.random.default_rng(5)
    codes = rng.integers(0, 40, size=500).astype(np.uint64)
    attr = rng.normal(size=(500, 7)).astype(np.float32)
    oc, oa, cnt = orc.merge(codes, attr)
    assert oc.tolist() == sorted(set(codes.tolist()))
    assert cnt.sum() == 500
    for k, c in enumerate(oc):
        sel = codes == c
        np.testing.assert_allclose(oa[k], attr[sel].astype(np.float64).mean(0), rtol=0, atol=1e-12)


def _paper_example():
    d = {}
    for ln in _lines("octree_root_example.txt"):
        k, _, v = ln.partition(" ")
        d[k] = v
    vox = np.array([[int(a) for a in t.split(",")] for t in d["voxels"].split()], np.uint32)
    return int(d["J"]), vox, d


def test_octree_root_byte_paper_example(orc):
    J, vox, d = _paper_example()
    occ, lsz = orc.octree_encode(vox, J)
    assert format(occ[0], "08b") == d["byte0"]
    assert format(occ[1], "08b") == d["byte1"]
    assert format(occ[2], "08b") == d["byte2"]
    assert lsz.tolist() == [int(t) for t in d["level_sizes"].split()]


def _brute_octree(codes, J):
    """Occupancy stream by the nested-set definition: at depth d the nodes are
    the distinct prefixes code >> 3(J-d) in ascending order; each emits the
    OR of (1 << child digit) over its children at depth d+1."""
    codes = sorted(set(int(c) for c in codes))
    out, sizes = [], []
    for d in range(J + 1):
        sizes.append(len(set(c >> (3 * (J - d)) for c in codes)))
    for d in range(J):
        nodes = sorted(set(c >> (3 * (J - d)) for c in codes))
        kids = sorted(set(c >> (3 * (J - d - 1)) for c in codes))
        for p in nodes:
            b = 0
            for k in kids:
                if k >> 3 == p:
                    b |= 1 << (k & 7)
            out.append(b)
    return out, sizes


@pytest.mark.parametrize("seed", range(40))
def test_octree_brute_force_tiny_frames(orc, seed):
    rng = np.random.default_rng(100 + seed)
    J = int(rng.integers(1, 6))
    n = int(rng.integers(2, 17))
    vox = np.unique(rng.integers(0, 1 << J, size=(n, 3)).astype(np.uint32), axis=0)
    occ, lsz = orc.octree_encode(vox, J)
    ref, sizes = _brute_octree(orc.morton_codes(vox, J), J)
    assert occ.tolist() == ref
    assert lsz.tolist() == sizes


@pytest.mark.parametrize("J", [1, 2, 4, 10, 16, 21])
def test_octree_invariants_and_roundtrip(orc, J):
    rng = np.random.default_rng(J)
    vox = np.unique(rng.integers(0, 1 << J, size=(3000, 3)).astype(np.uint32), axis=0)
    occ, lsz = orc.octree_encode(vox, J)
    # one byte per internal node (header of Algorithm 1)
    assert occ.size == int(lsz[:J].sum())
    assert lsz[0] == 1 and lsz[J] == vox.shape[0]
    off = 0
    for d in range(J):
        seg = occ[off:off + lsz[d]]
        assert int(np.unpackbits(seg).sum()) == int(lsz[d + 1])   # popcounts = next level size
        assert (seg != 0).all()
        off += lsz[d]
    leaves = orc.octree_decode(occ, J, lsz)                       # Algorithms 2-3
    assert leaves.tolist() == sorted(orc.morton_codes(vox, J).tolist())


def test_octree_single_voxel_and_empty(orc):
    J = 6
    occ, lsz = orc.octree_encode(np.array([[5, 9, 63]], np.uint32), J)
    assert lsz.tolist() == [1] * (J + 1) and occ.size == J
    assert all(bin(b).count("1") == 1 for b in occ)
    occ0, lsz0 = orc.octree_encode(np.zeros((0, 3), np.uint32), J)
    assert occ0.size == 0 and lsz0.tolist() == [0] * (J + 1)


def test_octree_decoder_rejects_inconsistent_headers(orc):
    J, vox, _ = _paper_example()
    occ, lsz = orc.octree_encode(vox, J)
    bad = lsz.copy()
    bad[2] += 1
    with pytest.raises(RuntimeError):
        orc.octree_decode(occ, J, bad)
    occ2 = occ.copy()
    occ2[1] = 0
    with pytest.raises(RuntimeError):
        orc.octree_decode(occ2, J, lsz)
