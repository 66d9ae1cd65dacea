"""The error bound behind the fast voxel index (double-float evaluation of
(p - lo) * scale, floor taken when the estimate is farther than a margin from
every integer, else the FP64 definition): replayed in numpy float32 on random,
face-aligned and far-offset coordinates, the fast floor always equals the FP64
definition's floor wherever the fast path is taken, and the fallback is rare.
The FMA of the exact product is emulated exactly (float32 products are exact in
float64)."""
import numpy as np

f32 = np.float32


def _fast(p, lo, scale):
    lo_hi = f32(lo)
    lo_lo = f32(lo - np.float64(lo_hi))
    sc_hi = f32(scale)
    sc_lo = f32(scale - np.float64(sc_hi))
    m = 9.5367431640625e-07 + 8.0 * abs(lo) * scale * 3.552713678800501e-15
    margin = f32(m * 1.0000002) if m < 0.25 else f32(2.0)
    s = (p - lo_hi).astype(f32)
    bv = (s - p).astype(f32)
    e1 = ((p - (s - bv).astype(f32)).astype(f32) + (-lo_hi - bv).astype(f32)).astype(f32)
    t_lo = (e1 - lo_lo).astype(f32)
    hi = (s * sc_hi).astype(f32)
    perr = (s.astype(np.float64) * np.float64(sc_hi) - hi.astype(np.float64)).astype(f32)  # exact fma(s, sc_hi, -hi)
    lo_ = (perr + ((s * sc_lo).astype(f32) + (t_lo * sc_hi).astype(f32)).astype(f32)).astype(f32)
    fh = np.floor(hi).astype(f32)
    f = ((hi - fh).astype(f32) + lo_).astype(f32)
    fast = (hi >= 1) & (hi < 8388608) & (f >= margin) & (f <= f32(1) - margin)
    return fast, fh.astype(np.int64)


def _fp64(p, lo, scale):
    return np.floor((p.astype(np.float64) - lo) * scale).astype(np.int64)


def test_fast_floor_equals_fp64_definition():
    rng = np.random.default_rng(7)
    total_fast = total = 0
    # (J, offset, span, typical): typical grids have voxels coarser than float32's spacing of the coordinates;
    # in the others most coordinates sit exactly on voxel faces and take the FP64 definition
    for J, off, span, typical in ((10, 0.0, 1.0, True), (16, 0.0, 1.0, True), (21, 0.0, 1.0, False),
                                  (16, 1000.0, 1.0, False), (21, 1000.0, 1.0, False), (21, -3.0e5, 7.0, False),
                                  (16, 12345.678, 0.001, False), (18, 3.5, 250.0, True)):
        lo = np.float64(f32(off))
        scale = np.float64(1 << J) / np.float64(f32(span))
        k = rng.integers(0, 1 << min(J, 20), 200_000)
        faces = (off + span * k / float(1 << min(J, 20))).astype(f32)
        rand = (off + span * rng.random(200_000)).astype(f32)
        near = (faces + np.float32(span) * rng.uniform(-1e-6, 1e-6, faces.size)).astype(f32)
        for name, p in (("faces", faces), ("random", rand), ("near", near)):
            p = p[p >= f32(lo)]
            fast, q = _fast(p, lo, scale)
            ref = _fp64(p, lo, scale)
            assert np.array_equal(q[fast], ref[fast]), (J, off, span, name)
            if name == "random" and typical:
                total_fast += int(fast.sum())
                total += p.size
    # on typical grids random coordinates almost never fall back (the first voxel layer always does)
    assert total_fast > 0.97 * total, total_fast / total
