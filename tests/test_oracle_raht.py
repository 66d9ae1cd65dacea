"""Pins of the oracle's RAHT (Sec. 3.1 Eq. 1, Sec. 3.2, App. D) against
closed forms: hand-worked coefficients, orthonormality of the dense transform
matrix, energy preservation, DC = sqrt(N_v) * mean, zero high-pass for a
constant signal, N_v - 1 butterflies with root weight N_v, and agreement with
the level-list schedule of Algorithm 4 run over 3J levels."""
import math
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _cases():
    out = []
    with open(os.path.join(GOLD, "raht_small.txt")) as f:
        for ln in f:
            if not ln.strip() or ln.startswith("#"):
                continue
            name, J, codes, vals, exp = [t.strip() for t in ln.split("|")]
            ev = [eval(e, {"sqrt": math.sqrt}) for e in exp.split()]
            out.append((name, int(J), [int(c) for c in codes.split()], [float(v) for v in vals.split()], ev))
    return out


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_raht_hand_worked(orc, case):
    name, J, codes, vals, exp = case
    Y = orc.raht_forward(np.array(codes, np.uint64), np.array(vals)[:, None], J)
    np.testing.assert_allclose(Y[:, 0], exp, rtol=0, atol=1e-14)
    A = orc.raht_inverse(np.array(codes, np.uint64), Y, J)
    np.testing.assert_allclose(A[:, 0], vals, rtol=0, atol=1e-14)


def _frame(seed, n, J):
    rng = np.random.default_rng(seed)
    v = np.unique(rng.integers(0, 1 << J, size=(n, 3)).astype(np.uint32), axis=0)
    return v


def _codes(orc, seed, n, J):
    return np.sort(orc.morton_codes(_frame(seed, n, J), J))


@pytest.mark.parametrize("seed,n,J", [(1, 300, 4), (2, 1500, 8), (3, 2000, 8), (4, 60, 21)])
def test_raht_dense_matrix_orthogonal(orc, seed, n, J):
    codes = _codes(orc, seed, n, J)
    nv = codes.size
    T = orc.raht_forward(codes, np.eye(nv), J)       # column k = transform of e_k
    np.testing.assert_allclose(T.T @ T, np.eye(nv), rtol=0, atol=1e-12)
    np.testing.assert_allclose(T @ T.T, np.eye(nv), rtol=0, atol=1e-12)
    # the inverse routine is the transpose
    Ti = orc.raht_inverse(codes, np.eye(nv), J)
    np.testing.assert_allclose(Ti, T.T, rtol=0, atol=1e-12)


@pytest.mark.parametrize("J", [2, 10, 16, 21])
def test_raht_energy_roundtrip_dc(orc, J):
    codes = _codes(orc, 10 + J, 5000, J)
    rng = np.random.default_rng(J)
    A = rng.normal(size=(codes.size, 5)) + np.array([3.0, -1.0, 0.0, 10.0, 0.1])
    Y = orc.raht_forward(codes, A, J)
    np.testing.assert_allclose((Y ** 2).sum(0), (A ** 2).sum(0), rtol=1e-12)
    np.testing.assert_allclose(orc.raht_inverse(codes, Y, J), A, rtol=0, atol=1e-12)
    np.testing.assert_allclose(Y[0], math.sqrt(codes.size) * A.mean(0), rtol=1e-12)


def test_raht_constant_signal_has_no_high_pass(orc):
    codes = _codes(orc, 7, 4000, 12)
    A = np.full((codes.size, 2), 2.5)
    Y = orc.raht_forward(codes, A, 12)
    assert np.abs(Y[1:]).max() < 1e-11
    assert abs(Y[0, 0] - 2.5 * math.sqrt(codes.size)) < 1e-10


def test_raht_single_voxel_identity(orc):
    Y = orc.raht_forward(np.array([123], np.uint64), np.array([[4.0, -2.0]]), 5)
    assert Y.tolist() == [[4.0, -2.0]]


def test_raht_node_weights(orc):
    codes = _codes(orc, 8, 1000, 6)
    w = orc.raht_node_weights(codes, 6)
    assert w[0] == codes.size            # root weight = N_v
    assert (w[1:] >= 2).all()            # every other slot holds a butterfly's high pass


def _schedule_transform(codes, A, J, levels, i0, i1, w0, w1):
    # apply the butterflies of the Algorithm 4 level lists bottom-up (App. D's
    # forward rotation a*y0 + b*y1, -b*y0 + a*y1)
    Y = A.copy()
    order = np.argsort(levels, kind="stable")
    for k in order:
        a = math.sqrt(w0[k] / (w0[k] + w1[k]))
        b = math.sqrt(w1[k] / (w0[k] + w1[k]))
        y0, y1 = Y[i0[k]].copy(), Y[i1[k]].copy()
        Y[i0[k]] = a * y0 + b * y1
        Y[i1[k]] = -b * y0 + a * y1
    return Y


@pytest.mark.parametrize("seed,J", [(1, 3), (2, 6), (3, 10), (4, 16)])
def test_praht_schedule_matches_recursive_definition(orc, seed, J):
    codes = _codes(orc, 50 + seed, 1200, J)
    lv, i0, i1, w0, w1 = orc.praht_schedule(codes, J)
    assert lv.size == codes.size - 1                 # N_v - 1 butterflies
    assert sorted(i1.tolist()) == list(range(1, codes.size))   # every high pass has one slot
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(codes.size, 3))
    np.testing.assert_allclose(_schedule_transform(codes, A, J, lv, i0, i1, w0, w1),
                               orc.raht_forward(codes, A, J), rtol=0, atol=1e-12)
    # weights of the top butterfly add up to N_v
    top = int(np.argmax(lv))
    assert w0[top] + w1[top] == codes.size


def test_stopping_at_3J_minus_1_leaves_root_unmerged(orc):
    # codes 0 and 4 (J=1) differ only in z_0: they meet at binary level 3J = 3
    codes = np.array([0, 4], np.uint64)
    lv, *_ = orc.praht_schedule(codes, 1)
    assert lv.tolist() == [3]


# --- level of detail (decoding to a coarser octree depth) ---------------------
def test_lod_mean_is_lowpass_over_sqrt_weight(orc):
    # Eq. (1) by induction: a node's low-pass coefficient is sqrt(w) times the mean of its values
    rng = np.random.default_rng(7)
    J = 8
    v = np.unique(rng.integers(0, 2 ** J, size=(3000, 3)), axis=0)
    codes = np.sort(orc.morton_codes(v, J))
    A = rng.normal(size=(codes.size, 4))
    for Jp in (0, 1, 3, 5, 7, 8):
        nc, npos, na, nw = orc.lod(codes, A, J, Jp, np.zeros(3), 1.0)
        L, w = orc.raht_lowpass(codes, A, J, 3 * (J - Jp))
        assert np.array_equal(w, nw)
        assert np.abs(L / np.sqrt(w)[:, None] - na).max() < 1e-12
        assert nw.sum() == codes.size and np.array_equal(nc, np.unique(codes >> np.uint64(3 * (J - Jp))))


def test_lod_extremes(orc):
    rng = np.random.default_rng(8)
    J = 6
    codes = np.sort(orc.morton_codes(np.unique(rng.integers(0, 64, size=(500, 3)), axis=0), J))
    A = rng.normal(size=(codes.size, 2))
    nc, npos, na, nw = orc.lod(codes, A, J, J, np.zeros(3), 1.0)  # full depth: the voxels themselves
    assert np.array_equal(nc, codes) and np.allclose(na, A, rtol=0, atol=0)
    nc, npos, na, nw = orc.lod(codes, A, J, 0, np.array([1.0, 2.0, 3.0]), 4.0)  # the root
    assert nw.tolist() == [codes.size] and np.allclose(na[0], A.mean(0))
    assert np.allclose(npos[0], [3.0, 4.0, 5.0])  # centre of the whole cube
    Y = orc.raht_forward(codes, A, J)
    assert np.allclose(na[0] * np.sqrt(codes.size), Y[0], atol=1e-12)  # the DC
