"""Pins of the oracle's quantiser (Sec. 3.4), block RLGR (Sec. 3.4, App. H)
and occupancy rANS stage (Sec. 2.2): hand-derived bit patterns of the codec's
RLGR reading, lossless round trips, the quantiser's error bound and dead zone,
the block-size overhead trend of Table A.5, and the rANS size bound."""
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                a, b = ln.split("|")
                rows.append((a.split(), b.split()))
    return rows


@pytest.mark.parametrize("row", _golden("rlgr_small.txt"), ids=lambda r: " ".join(r[0]))
def test_rlgr_hand_derived_bits(orc, row):
    q = np.array([int(t) for t in row[0]], np.int32)
    assert orc.rlgr_encode(q).tolist() == [int(t) for t in row[1]]
    np.testing.assert_array_equal(orc.rlgr_decode(orc.rlgr_encode(q), q.size), q)


def _streams():
    rng = np.random.default_rng(0)
    yield "zeros", np.zeros(4096, np.int32)
    yield "one", np.array([7], np.int32)
    yield "laplace", np.round(rng.laplace(0, 3, 5000)).astype(np.int32)
    yield "sparse", (rng.random(6000) < 0.02) * rng.integers(-50, 50, 6000).astype(np.int32)
    yield "huge", rng.integers(-2 ** 30, 2 ** 30, 500).astype(np.int32)
    yield "extremes", np.array([2 ** 30, -2 ** 30, 0, 0, 1, -1, 2 ** 30 - 1] * 50, np.int32)
    yield "runs", np.repeat(rng.integers(-3, 4, 300), rng.integers(1, 70, 300)).astype(np.int32)
    yield "tail_run", np.concatenate([rng.integers(-5, 5, 100), np.zeros(33, int)]).astype(np.int32)
    yield "odd_len", np.round(rng.normal(0, 1, 1237)).astype(np.int32)


@pytest.mark.parametrize("name,q", list(_streams()), ids=lambda x: x if isinstance(x, str) else "")
def test_rlgr_lossless(orc, name, q):
    w = orc.rlgr_encode(q)
    np.testing.assert_array_equal(orc.rlgr_decode(w, q.size), q)
    assert w.size * 32 <= 78 * q.size + 32        # worst-case bound used for slot sizing


def test_rlgr_block_overhead_trend(orc):
    # Table A.5: smaller blocks cost a little more (monotone, a few percent at 256)
    rng = np.random.default_rng(1)
    q = np.round(rng.laplace(0, 1.2, 2 ** 16) * (rng.random(2 ** 16) < 0.4)).astype(np.int32)
    sizes = {}
    for B in (256, 512, 1024, 2048, 4096, 8192, 2 ** 16):
        sizes[B] = sum(orc.rlgr_encode(q[s:s + B]).size for s in range(0, q.size, B))
    order = [sizes[B] for B in (256, 512, 1024, 2048, 4096, 8192, 2 ** 16)]
    assert all(a >= b for a, b in zip(order, order[1:]))
    assert sizes[256] / sizes[2 ** 16] < 1.10


def test_rlgr_rejects_truncated(orc):
    q = np.round(np.random.default_rng(2).laplace(0, 5, 2000)).astype(np.int32)
    w = orc.rlgr_encode(q)
    with pytest.raises(RuntimeError):
        orc.rlgr_decode(w[: w.size // 2], q.size)


def test_quantiser_bounds_and_deadzone(orc):
    rng = np.random.default_rng(3)
    Y = rng.normal(0, 2, size=(4000, 3))
    groups = np.array([0, 1, 1], np.uint8)
    steps = np.array([0.1, 0.37])
    Q = orc.quantize(Y, groups, steps, 0.5)
    R = Q * steps[groups]
    assert np.all(np.abs(Y - R) <= steps[groups] / 2 + 1e-15)
    np.testing.assert_array_equal(orc.quantize(-Y, groups, steps, 0.5), -Q)   # sign symmetry
    Qd = orc.quantize(Y, groups, steps, 1 / 3)
    z = np.abs(Y) < (2 / 3) * steps[groups] * (1 - 1e-12)
    assert (Qd[z] == 0).all()                        # dead zone of half-width (1 - tau) * step
    assert (np.abs(Qd) <= np.abs(Q)).all()


@pytest.mark.parametrize("row", _golden("rans_freqs.txt"), ids=lambda r: " ".join(r[0]))
def test_rans_frequency_normalisation(orc, row):
    data = []
    for t in row[0]:
        s, c = t.split(":")
        data += [int(s)] * int(c)
    f = orc.rans_freqs(np.array(data, np.uint8))
    exp = {int(t.split(":")[0]): int(t.split(":")[1]) for t in row[1]}
    assert {int(i): int(f[i]) for i in np.nonzero(f)[0]} == exp
    assert int(f.sum()) == 1 << 15


@pytest.mark.parametrize("n,kind", [(1, "u"), (31, "u"), (32, "u"), (1000, "skew"), (100_000, "skew"),
                                    (70_000, "u"), (50_001, "two"), (5000, "const")])
def test_rans_section_roundtrip_and_bound(orc, n, kind):
    rng = np.random.default_rng(n)
    if kind == "u":
        d = rng.integers(0, 256, n).astype(np.uint8)
    elif kind == "two":
        d = rng.choice(np.array([0x18, 0xFF], np.uint8), n)
    elif kind == "const":
        d = np.full(n, 0x81, np.uint8)
    else:
        p = np.exp(-np.arange(256) / 8.0)
        d = rng.choice(256, n, p=p / p.sum()).astype(np.uint8)
    for chunk in (32, 4096, 16384):
        sec = orc.occ_section_encode(d, chunk)
        np.testing.assert_array_equal(orc.occ_section_decode(sec, n), d)
        cnt = np.bincount(d, minlength=256)
        pr = cnt[cnt > 0] / n
        H0 = float(-(pr * np.log2(pr)).sum())
        nch = -(-n // chunk)
        assert sec.size <= min(16 + ((n + 7) & ~7), n * H0 / 8 * 1.005 + 24 + 512 + 4 * nch + 132 * nch + 8)


def test_rans_handles_empty(orc):
    sec = orc.occ_section_encode(np.zeros(0, np.uint8))
    assert orc.occ_section_decode(sec, 0).size == 0
