"""ctypes binding of the FP64 CPU oracle (gsnfs_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
CPU-baseline leg of the benchmark.  The product library never imports it.
Arrays are numpy; every function mirrors one C entry point and cites the same
passage of the paper.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gsnfs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ERR = {-1: "invalid argument", -2: "capacity", -3: "corrupt stream", -6: "out of memory"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ct.CDLL(_LIB_PATH)
            p = ct.c_void_p
            i64, i32, u32, f64 = ct.c_int64, ct.c_int, ct.c_uint32, ct.c_double
            L.orc_bbox.argtypes = [p, i64, p, p]
            L.orc_voxel_coords.argtypes = [p, i64, i32, p, f64, p]
            L.orc_morton.argtypes = [u32, u32, u32, i32]
            L.orc_morton.restype = ct.c_uint64
            L.orc_morton_decode.argtypes = [ct.c_uint64, i32, p, p, p]
            L.orc_morton_codes.argtypes = [p, i64, i32, p]
            L.orc_voxel_centres.argtypes = [p, i64, i32, p, f64, p]
            L.orc_merge.argtypes = [p, p, i64, i32, p, p, p]
            L.orc_merge.restype = i64
            L.orc_octree_encode.argtypes = [p, i64, i32, p, p]
            L.orc_octree_encode.restype = i64
            L.orc_octree_decode.argtypes = [p, i64, i32, p, p, i64]
            L.orc_octree_decode.restype = i64
            L.orc_raht_forward.argtypes = [p, i64, i32, i32, p, p]
            L.orc_raht_inverse.argtypes = [p, i64, i32, i32, p, p]
            L.orc_raht_node_weights.argtypes = [p, i64, i32, p]
            L.orc_render.argtypes = [p, p, i64, p, f64, f64, f64, f64, i32, i32, f64, p, p]
            L.orc_sh_basis.argtypes = [p, p]
            L.orc_render.restype = i32
            L.orc_render_check.argtypes = [p, p, i64, p, f64, f64, f64, f64, i32, i32, f64, p, p, p, p]
            L.orc_render_check.restype = i32
            L.orc_lod.argtypes = [p, i64, i32, i32, i32, p, p, f64, p, p, p, p]
            L.orc_lod.restype = i64
            L.orc_raht_lowpass.argtypes = [p, i64, i32, i32, p, i32, p, p]
            L.orc_raht_lowpass.restype = i64
            L.orc_praht_schedule.argtypes = [p, i64, i32, p, p, p, p, p]
            L.orc_praht_schedule.restype = i64
            L.orc_quantize.argtypes = [p, i64, i32, p, p, f64, p]
            L.orc_rlgr_encode.argtypes = [p, i64, i64, p, i64]
            L.orc_rlgr_encode.restype = i64
            L.orc_rlgr_decode.argtypes = [p, i64, i64, i64, p]
            L.orc_rlgr_decode.restype = i32
            L.orc_rans_freqs.argtypes = [p, i64, p]
            L.orc_occ_section_encode.argtypes = [p, i64, u32, p, i64]
            L.orc_occ_section_encode.restype = i64
            L.orc_occ_section_decode.argtypes = [p, i64, p, i64]
            L.orc_occ_section_decode.restype = i64
            L.orc_encode_frame.argtypes = [p, p, i64, i32, i32, i32, p, p, f64, u32, u32, p, i64,
                                           p, p, p, p, i32, p, p]
            L.orc_yuv_rows.argtypes = [p, i64, i32]
            L.orc_klt_rows.argtypes = [p, i64, p, i32]
            L.orc_klt_matrices.argtypes = [p, i64, p]
            L.orc_encode_frame.restype = i64
            L.orc_peek_frame.argtypes = [p, i64, p, p, p]
            L.orc_peek_frame.restype = i32
            L.orc_decode_frame.argtypes = [p, i64, i64, p, p, p, p]
            L.orc_decode_frame.restype = i64
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ct.c_void_p)


def _check(r):
    if r < 0:
        raise RuntimeError(f"oracle error {r}: {ERR.get(int(r), '?')}")
    return r


# --- voxelisation and Morton codes (Sec. 2.1, Sec. 2.2) --------------------
def bbox(pos):
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    lo = np.zeros(3)
    ext = np.zeros(1)
    lib().orc_bbox(_p(pos), pos.shape[0], _p(lo), _p(ext))
    return lo, float(ext[0])


def voxel_coords(pos, J, lo=None, ext=None):
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    if lo is None:
        lo, ext = bbox(pos)
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    v = np.zeros((pos.shape[0], 3), dtype=np.uint32)
    lib().orc_voxel_coords(_p(pos), pos.shape[0], J, _p(lo), float(ext), _p(v))
    return v


def morton(x, y, z, J):
    return int(lib().orc_morton(int(x), int(y), int(z), int(J)))


def morton_codes(vox, J):
    vox = np.ascontiguousarray(vox, dtype=np.uint32).reshape(-1, 3)
    out = np.zeros(vox.shape[0], dtype=np.uint64)
    lib().orc_morton_codes(_p(vox), vox.shape[0], J, _p(out))
    return out


def morton_decode(m, J):
    x, y, z = (ct.c_uint32(), ct.c_uint32(), ct.c_uint32())
    lib().orc_morton_decode(ct.c_uint64(int(m)), J, ct.byref(x), ct.byref(y), ct.byref(z))
    return x.value, y.value, z.value


def voxel_centres(codes, J, lo, ext):
    codes = np.ascontiguousarray(codes, dtype=np.uint64)
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    out = np.zeros((codes.shape[0], 3), dtype=np.float32)
    lib().orc_voxel_centres(_p(codes), codes.shape[0], J, _p(lo), float(ext), _p(out))
    return out


def merge(codes, attr):
    codes = np.ascontiguousarray(codes, dtype=np.uint64)
    attr = np.ascontiguousarray(attr, dtype=np.float32)
    n = codes.shape[0]
    C = attr.shape[1] if attr.ndim == 2 else 0
    oc = np.zeros(max(n, 1), dtype=np.uint64)
    oa = np.zeros((max(n, 1), max(C, 1)), dtype=np.float64)
    cnt = np.zeros(max(n, 1), dtype=np.int64)
    nv = _check(lib().orc_merge(_p(codes), _p(attr), n, C, _p(oc), _p(oa), _p(cnt)))
    return oc[:nv], oa[:nv, :C], cnt[:nv]


def voxelize(pos, attr, J):
    """Full voxelisation: returns (codes sorted, merged attributes FP64, counts, lo, ext)."""
    lo, ext = bbox(pos)
    v = voxel_coords(pos, J, lo, ext)
    codes = morton_codes(v, J)
    oc, oa, cnt = merge(codes, attr)
    return oc, oa, cnt, lo, ext


# --- octree (Sec. 2.1, Sec. 2.3) -------------------------------------------
def octree_encode(vox, J):
    vox = np.ascontiguousarray(vox, dtype=np.uint32)
    nv = vox.shape[0]
    occ = np.zeros(max(nv, 1) * (J + 1), dtype=np.uint8)
    lsz = np.zeros(J + 1, dtype=np.uint32)
    nb = _check(lib().orc_octree_encode(_p(vox), nv, J, _p(occ), _p(lsz)))
    return occ[:nb].copy(), lsz


def octree_decode(occ, J, level_sizes):
    occ = np.ascontiguousarray(occ, dtype=np.uint8)
    lsz = np.ascontiguousarray(level_sizes, dtype=np.uint32)
    cap = int(lsz[J])
    out = np.zeros(max(cap, 1), dtype=np.uint64)
    n = _check(lib().orc_octree_decode(_p(occ), occ.shape[0], J, _p(lsz), _p(out), cap))
    return out[:n]


# --- RAHT (Sec. 3.1 Eq. 1; Sec. 3.2 Algorithm 4) ----------------------------
def raht_forward(codes, A, J):
    codes = np.ascontiguousarray(codes, dtype=np.uint64)
    A = np.ascontiguousarray(A, dtype=np.float64)
    if A.ndim == 1:
        A = A[:, None]
    Y = np.zeros_like(A)
    lib().orc_raht_forward(_p(codes), codes.shape[0], J, A.shape[1], _p(A), _p(Y))
    return Y


def raht_inverse(codes, Y, J):
    codes = np.ascontiguousarray(codes, dtype=np.uint64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    if Y.ndim == 1:
        Y = Y[:, None]
    A = np.zeros_like(Y)
    lib().orc_raht_inverse(_p(codes), codes.shape[0], J, Y.shape[1], _p(Y), _p(A))
    return A


def lod(codes, A, J, Jp, lo, ext):
    """Nodes at octree depth Jp: (node codes, centres f32, mean attributes f64, voxel counts)."""
    codes = np.ascontiguousarray(codes, dtype=np.uint64)
    A = np.ascontiguousarray(A, dtype=np.float64)
    if A.ndim == 1:
        A = A[:, None]
    nv, C = codes.shape[0], A.shape[1]
    m = max(nv, 1)
    nc = np.zeros(m, dtype=np.uint64)
    npos = np.zeros((m, 3), dtype=np.float32)
    na = np.zeros((m, max(C, 1)), dtype=np.float64)
    nw = np.zeros(m, dtype=np.int64)
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    k = _check(lib().orc_lod(_p(codes), nv, J, Jp, C, _p(A), _p(lo), float(ext), _p(nc), _p(npos), _p(na), _p(nw)))
    return nc[:k], npos[:k], na[:k, :C], nw[:k]


def raht_lowpass(codes, A, J, level):
    """Low-pass coefficient (Eq. 1 applied inside each node) of every node at binary level `level`."""
    codes = np.ascontiguousarray(codes, dtype=np.uint64)
    A = np.ascontiguousarray(A, dtype=np.float64)
    if A.ndim == 1:
        A = A[:, None]
    nv, C = codes.shape[0], A.shape[1]
    out = np.zeros((max(nv, 1), max(C, 1)), dtype=np.float64)
    w = np.zeros(max(nv, 1), dtype=np.int64)
    k = _check(lib().orc_raht_lowpass(_p(codes), nv, J, C, _p(A), level, _p(out), _p(w)))
    return out[:k, :C], w[:k]


def sh_basis(d):
    d = np.ascontiguousarray(d, dtype=np.float64)
    Y = np.zeros(16)
    lib().orc_sh_basis(_p(d), _p(Y))
    return Y


def render(pos, attr, view, fx, fy, cx, cy, width, height, znear=0.01, bg=(0.0, 0.0, 0.0), check=False):
    """FP64 splat rasteriser (image [H, W, 3]) of 56-channel Gaussians; view = 3 x 4 world-to-camera [R | t].
    With check=True also returns, per pixel, the threshold flag (uint8 [H, W]: the pixel depends on a decision
    within rounding of its threshold) and the first-order error bound of an FP32 evaluation (float64 [H, W])."""
    pos = np.ascontiguousarray(pos, dtype=np.float32).reshape(-1, 3)
    attr = np.ascontiguousarray(attr, dtype=np.float32).reshape(-1, 56)
    view = np.ascontiguousarray(view, dtype=np.float64).reshape(3, 4)
    bg = np.ascontiguousarray(bg, dtype=np.float64)
    img = np.zeros((height, width, 3), dtype=np.float64)
    if not check:
        _check(lib().orc_render(_p(pos), _p(attr), pos.shape[0], _p(view), float(fx), float(fy), float(cx),
                                float(cy), width, height, float(znear), _p(bg), _p(img)))
        return img
    flag = np.zeros((height, width), dtype=np.uint8)
    tol = np.zeros((height, width), dtype=np.float64)
    _check(lib().orc_render_check(_p(pos), _p(attr), pos.shape[0], _p(view), float(fx), float(fy), float(cx),
                                  float(cy), width, height, float(znear), _p(bg), _p(img), _p(flag), _p(tol)))
    return img, flag, tol


def raht_node_weights(codes, J):
    codes = np.ascontiguousarray(codes, dtype=np.uint64)
    w = np.zeros(codes.shape[0], dtype=np.int64)
    lib().orc_raht_node_weights(_p(codes), codes.shape[0], J, _p(w))
    return w


def praht_schedule(codes, J):
    codes = np.ascontiguousarray(codes, dtype=np.uint64)
    nv = codes.shape[0]
    m = max(nv, 1)
    lv = np.zeros(m, dtype=np.int32)
    i0, i1, w0, w1 = (np.zeros(m, dtype=np.int64) for _ in range(4))
    k = _check(lib().orc_praht_schedule(_p(codes), nv, J, _p(lv), _p(i0), _p(i1), _p(w0), _p(w1)))
    return lv[:k], i0[:k], i1[:k], w0[:k], w1[:k]


# --- quantiser and entropy coders (Sec. 3.4; Sec. 2.2) ----------------------
def quantize(Y, groups, steps, tau=0.5):
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    groups = np.ascontiguousarray(groups, dtype=np.uint8)
    steps = np.ascontiguousarray(steps, dtype=np.float64)
    Q = np.zeros(Y.shape, dtype=np.int32)
    lib().orc_quantize(_p(Y), Y.shape[0], Y.shape[1], _p(groups), _p(steps), float(tau), _p(Q))
    return Q


def rlgr_encode(q):
    q = np.ascontiguousarray(q, dtype=np.int32)
    cap = (q.shape[0] * 78 + 31) // 32 + 2
    w = np.zeros(cap, dtype=np.uint32)
    n = _check(lib().orc_rlgr_encode(_p(q), q.shape[0], 1, _p(w), cap))
    return w[:n].copy()


def rlgr_decode(words, n):
    words = np.ascontiguousarray(words, dtype=np.uint32)
    q = np.zeros(max(n, 1), dtype=np.int32)
    _check(lib().orc_rlgr_decode(_p(words), words.shape[0], n, 1, _p(q)))
    return q[:n]


def rans_freqs(data):
    data = np.ascontiguousarray(data, dtype=np.uint8)
    f = np.zeros(256, dtype=np.uint16)
    lib().orc_rans_freqs(_p(data), data.shape[0], _p(f))
    return f


def occ_section_encode(occ, chunk_syms=4096):
    occ = np.ascontiguousarray(occ, dtype=np.uint8)
    n = occ.shape[0]
    cap = 64 + 2 * n + 1024 + (n // 32 + 1) * 256
    out = np.zeros(cap, dtype=np.uint8)
    k = _check(lib().orc_occ_section_encode(_p(occ), n, chunk_syms, _p(out), cap))
    return out[:k].copy()


def occ_section_decode(sec, n):
    sec = np.ascontiguousarray(sec, dtype=np.uint8)
    out = np.zeros(max(n, 1), dtype=np.uint8)
    k = _check(lib().orc_occ_section_decode(_p(sec), sec.shape[0], _p(out), n))
    return out[:k]


# --- whole frame -------------------------------------------------------------
def encode_frame(pos, attr, J, groups=None, steps=None, tau=0.5, block=512, chunk_syms=4096,
                 with_coeffs=False, color=False, klt=None):
    """Oracle encoder.  Returns dict(bitstream, nv, codes[, coeffs, q][, klt]).  color: the SH colour
    decorrelation of Sec. 4 (56-channel 3DGS rows), with the given KLT matrices [3, 15, 15] or its own."""
    pos = np.ascontiguousarray(pos, dtype=np.float32).reshape(-1, 3)
    n = pos.shape[0]
    if attr is None:
        attr = np.zeros((n, 0), dtype=np.float32)
    attr = np.ascontiguousarray(attr, dtype=np.float32).reshape(n, -1) if n else \
        np.zeros((0, attr.shape[1] if attr.ndim == 2 else 0), dtype=np.float32)
    C = attr.shape[1]
    if groups is None:
        groups = np.zeros(C, dtype=np.uint8)
    groups = np.ascontiguousarray(groups, dtype=np.uint8)
    steps = np.ascontiguousarray(np.atleast_1d(steps if steps is not None else [1.0]), dtype=np.float64)
    G = int(steps.shape[0])
    cap = 4096 + 8 * (J + 1) + 16 * n + 2 * n * J + 12 * n * C + 64 * C * (n // max(block, 1) + 1)
    out = np.zeros(cap, dtype=np.uint8)
    nv = np.zeros(1, dtype=np.int64)
    codes = np.zeros(max(n, 1), dtype=np.uint64)
    coeff = np.zeros((max(n, 1), max(C, 1)), dtype=np.float64) if with_coeffs else None
    q = np.zeros((max(n, 1), max(C, 1)), dtype=np.int32) if with_coeffs else None
    if with_coeffs and C > 0:
        coeff = np.zeros((max(n, 1), C), dtype=np.float64)
        q = np.zeros((max(n, 1), C), dtype=np.int32)
    kin = None if klt is None else np.ascontiguousarray(klt, dtype=np.float32).reshape(3, 15, 15)
    kout = np.zeros((3, 15, 15), dtype=np.float32)
    k = _check(lib().orc_encode_frame(_p(pos), _p(attr), n, C, J, G, _p(groups), _p(steps), float(tau),
                                      block, chunk_syms, _p(out), cap, _p(nv), _p(codes),
                                      _p(coeff) if with_coeffs and C > 0 else None,
                                      _p(q) if with_coeffs and C > 0 else None, 1 if color else 0,
                                      _p(kin), _p(kout)))
    m = int(nv[0])
    res = {"bitstream": out[:k].copy(), "nv": m, "codes": codes[:m].copy()}
    if color:
        res["klt"] = kout
    if with_coeffs and C > 0:
        res["coeffs"] = coeff[:m].copy()
        res["q"] = q[:m].copy()
    return res


def yuv_rows(A, inverse=False):
    """BT.601 YUV of every SH function of 56-channel rows (Sec. 4), in place on a copy."""
    A = np.array(A, dtype=np.float64, order="C")
    lib().orc_yuv_rows(_p(A), A.shape[0], 1 if inverse else 0)
    return A


def klt_rows(A, K, inverse=False):
    A = np.array(A, dtype=np.float64, order="C")
    K = np.ascontiguousarray(K, dtype=np.float32)
    lib().orc_klt_rows(_p(A), A.shape[0], _p(K), 1 if inverse else 0)
    return A


def klt_matrices(attr):
    """KLT matrices [3, 15, 15] (rows = eigenvectors) from the first 4096 rows of a frame's points."""
    attr = np.ascontiguousarray(attr, dtype=np.float32)
    K = np.zeros((3, 15, 15), dtype=np.float32)
    lib().orc_klt_matrices(_p(attr), attr.shape[0], _p(K))
    return K


def peek_frame(bs):
    bs = np.ascontiguousarray(bs, dtype=np.uint8)
    nv, C, J = ct.c_int64(), ct.c_int(), ct.c_int()
    _check(lib().orc_peek_frame(_p(bs), bs.shape[0], ct.byref(nv), ct.byref(C), ct.byref(J)))
    return nv.value, C.value, J.value


def decode_frame(bs):
    """Oracle decoder.  Returns dict(pos f32, attr f64, codes, q)."""
    bs = np.ascontiguousarray(bs, dtype=np.uint8)
    nv, C, J = peek_frame(bs)
    pos = np.zeros((max(nv, 1), 3), dtype=np.float32)
    attr = np.zeros((max(nv, 1), max(C, 1)), dtype=np.float64)
    codes = np.zeros(max(nv, 1), dtype=np.uint64)
    q = np.zeros((max(nv, 1), max(C, 1)), dtype=np.int32)
    k = _check(lib().orc_decode_frame(_p(bs), bs.shape[0], nv, _p(pos), _p(attr), _p(codes), _p(q)))
    return {"pos": pos[:k], "attr": attr[:k, :C], "codes": codes[:k], "q": q[:k, :C], "J": J}
