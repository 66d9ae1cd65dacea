"""Comparison of one GPU-written stream with the oracle, shared by the GPU
parity tests: header and occupancy section byte-identical to the oracle
encoder's; the oracle decoder reads the GPU stream back to the oracle's exact
voxel set; quantisation indices equal the oracle's except inside the rounding
zone (|y|/step + tau within 1e-4 of an integer), counted and below 1e-6 of all
coefficients; the GPU decoder's output (if given) equals the oracle decoder's
reading of the same stream within FP32 tolerance."""
import numpy as np


def stream_klt(stream):
    """The colour-mode KLT matrices [3, 15, 15] carried in a stream's header (None without colour)."""
    h = np.ascontiguousarray(stream)
    if int.from_bytes(h[88:92].tobytes(), "little") & 1 == 0:
        return None
    J = int.from_bytes(h[12:16].tobytes(), "little")
    C = int.from_bytes(h[16:20].tobytes(), "little")
    G = int.from_bytes(h[20:24].tobytes(), "little")
    so = (96 + 4 * (J + 1) + C + 7) // 8 * 8 + 8 * G
    return np.frombuffer(h[so:so + 2700].tobytes(), dtype=np.float32).reshape(3, 15, 15)


def compare_stream(orc, stream, pos, attr, J, groups, steps, tau, block, chunk, gpu_decoded=None, own_klt=False):
    """own_klt (colour mode): the oracle derives its own KLT matrices instead of taking the stream's; indices may
    then also differ where the difference of the two K can move a coefficient across a rounding boundary."""
    host = np.ascontiguousarray(stream)
    C = 0 if attr is None else attr.shape[1]
    klt = stream_klt(host)  # colour mode: by default the oracle encodes with the stream's own KLT matrices
    ref = orc.encode_frame(pos, attr if C else None, J, groups, steps, tau, block, chunk, with_coeffs=True,
                           color=klt is not None, klt=None if own_klt else klt)
    refbs = ref["bitstream"]
    hb = int.from_bytes(refbs[8:12].tobytes(), "little")
    occb = int.from_bytes(refbs[72:80].tobytes(), "little")
    assert np.array_equal(host[:72], refbs[:72]), "fixed header"
    if own_klt and klt is not None:  # the K tables may differ: compare the rest of the header around them
        kb = int(klt.nbytes)
        assert np.array_equal(host[88:hb - kb], refbs[88:hb - kb]), "header tables"
        assert np.array_equal(host[hb:hb + occb], refbs[hb:hb + occb]), "occupancy section"
    else:
        assert np.array_equal(host[88:hb + occb], refbs[88:hb + occb]), "header tables and occupancy section"
    dec = orc.decode_frame(host)
    assert np.array_equal(dec["codes"], ref["codes"]), "voxel set"
    out = {"nv": int(ref["nv"]), "bytes": int(host.size), "disagree": 0, "dec": dec}
    if C and ref["nv"]:
        q_ref, y64 = ref["q"], ref["coeffs"]
        st = np.asarray(steps, dtype=np.float64)[np.asarray(groups)]
        dis = dec["q"] != q_ref
        t = np.abs(y64) / st + tau
        frac = t - np.floor(t)
        zone = np.minimum(frac, 1 - frac) < 1e-4
        if own_klt and klt is not None:
            # |(K_gpu - K_oracle) a|_r <= sqrt(15) max|dK| |a|_2 per YUV channel, |a|_2 = |y|_2 (K orthonormal)
            kd = np.abs(klt.astype(np.float64) - stream_klt(refbs).astype(np.float64)).reshape(3, -1).max(1)
            for ch in range(3):
                cols = slice(11 + 15 * ch, 26 + 15 * ch)
                bound = np.sqrt(15) * kd[ch] * np.linalg.norm(y64[:, cols], axis=1, keepdims=True) / st[cols]
                zone[:, cols] |= np.minimum(frac[:, cols], 1 - frac[:, cols]) < 1e-4 + bound
        assert not (dis & ~zone).any(), "index disagreement outside the rounding-boundary zone"
        out["disagree"] = int(dis.sum())
        assert dis.sum() <= 1e-6 * dis.size + (1 if dis.size < 1e6 else 0), dis.sum()
    if gpu_decoded is not None:
        gpos, gattr = gpu_decoded
        assert np.array_equal(gpos, dec["pos"]), "decoded positions"
        if C and ref["nv"]:
            st = np.asarray(steps, dtype=np.float64)[np.asarray(groups)]
            scale = np.sqrt((dec["attr"] ** 2).mean(0)) + st
            err = np.abs(gattr.astype(np.float64) - dec["attr"]) / scale
            assert err.max() < 1e-4, err.max()
    return out
