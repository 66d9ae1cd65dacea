"""Python binding of libgsnfs.so (include/gsnfs.h).

Argument marshalling only: every step of the codec runs in the CUDA library.
Tensors are torch CUDA tensors (PyTorch provides device memory and streams);
calls are enqueued on torch's current stream of the tensor's device.  The
library is loaded on first use and a missing or unloadable library raises
immediately (there is no fallback implementation).
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgsnfs.so")

GSNFS_OK = 0
STATUS = {0: "ok", -1: "invalid argument", -2: "capacity", -3: "corrupt bitstream", -4: "cuda error",
          -5: "timeout", -6: "out of memory", -7: "unsupported"}


class GsnfsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code}: {STATUS.get(code, '?')})")
        self.code = code


class Quant(ct.Structure):
    _fields_ = [("num_channels", ct.c_uint32), ("num_groups", ct.c_uint32),
                ("channel_group", ct.POINTER(ct.c_uint8)), ("steps", ct.POINTER(ct.c_double)),
                ("tau", ct.c_double), ("rlgr_block", ct.c_uint32), ("rans_chunk", ct.c_uint32),
                ("color", ct.c_uint32)]


_lock = threading.Lock()
_lib = None
_ctx = {}


def lib():
    """Loads libgsnfs.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libgsnfs.so not built ({LIB_PATH}); run paper_2606_05650_gb300/build.py")
            L = ct.CDLL(LIB_PATH)
            p, u32, u64, i32 = ct.c_void_p, ct.c_uint32, ct.c_uint64, ct.c_int
            P64 = ct.POINTER(ct.c_uint64)
            Q = ct.POINTER(Quant)
            sig = {
                "gsnfs_create": ([ct.POINTER(p), i32], i32),
                "gsnfs_destroy": ([p], None),
                "gsnfs_status_string": ([i32], ct.c_char_p),
                "gsnfs_reserve": ([p, u64, u32, u32, Q], i32),
                "gsnfs_max_bitstream_bytes": ([u64, u32, Q, P64], i32),
                "gsnfs_encode_frame": ([p, p, p, p, u64, u32, Q, p, u64, P64, p, p, P64], i32),
                "gsnfs_peek_frame": ([p, u64, P64, ct.POINTER(u32), ct.POINTER(u32)], i32),
                "gsnfs_decode_frame": ([p, p, p, u64, p, p, u64, P64], i32),
                "gsnfs_encode_batch": ([p, p, u32, p, p, p, p, u32, p, Q, p, u64, p], i32),
                "gsnfs_encode_batch_rd": ([p, p, u32, p, p, p, p, u32, p, Q, p, u64, p, p], i32),
                "gsnfs_decode_batch": ([p, p, u32, p, p, p, p, u64, p], i32),
                "gsnfs_encode_batch_headers": ([p, p, u32, p, p, p, p, u32, p, Q, p, u64, p, p], i32),
                "gsnfs_decode_batch_async": ([p, p, u32, p, p, p, p, p, u64, p, p], i32),
                "gsnfs_decode_frame_lod": ([p, p, p, u64, u32, p, p, u64, P64], i32),
                "gsnfs_render": ([p, p, p, p, u64, ct.POINTER(Camera), p], i32),
                "gsnfs_voxelize": ([p, p, p, u64, u32, p, p, P64], i32),
                "gsnfs_octree_encode": ([p, p, p, u64, u32, p, u64, p, P64], i32),
                "gsnfs_octree_decode": ([p, p, p, u64, u32, p, p], i32),
                "gsnfs_occupancy_section_encode": ([p, p, p, u64, u32, p, u64, P64], i32),
                "gsnfs_occupancy_section_decode": ([p, p, p, u64, p, u64], i32),
                "gsnfs_raht_plan_create": ([p, p, p, u64, u32, u32, ct.POINTER(p)], i32),
                "gsnfs_raht_plan_destroy": ([p], None),
                "gsnfs_raht_forward": ([p, p, p, p], i32),
                "gsnfs_raht_inverse": ([p, p, p, p, Q], i32),
                "gsnfs_raht_forward_f64": ([p, p, p, p], i32),
                "gsnfs_raht_inverse_f64": ([p, p, p, p, Q], i32),
                "gsnfs_rlgr_slot_words": ([u32], u32),
                "gsnfs_rlgr_encode_indices": ([p, p, p, u64, u32, u32, p, p], i32),
                "gsnfs_rlgr_decode_indices": ([p, p, p, p, u64, u32, u32, p], i32),
                "gsnfs_set_graphs": ([p, i32], i32),
                "gsnfs_tune_set": ([p, i32, u32], i32),
                "gsnfs_tune_get": ([p, i32, ct.POINTER(u32)], i32),
                "gsnfs_graph_stats": ([p, P64], i32),
                "gsnfs_launch_count": ([], u64),
                "gsnfs_profile_enable": ([i32], i32),
                "gsnfs_profile_stage_names": ([ct.POINTER(ct.c_char_p), i32], i32),
                "gsnfs_profile_read": ([ct.POINTER(ct.c_double), ct.POINTER(ct.c_uint64), i32], i32),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _check(code, what):
    if code != GSNFS_OK:
        raise GsnfsError(code, f"{what}: {lib().gsnfs_status_string(code).decode()}")


def context(device=None):
    """One library context per CUDA device."""
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else
                       (device.index if isinstance(device, torch.device) else int(device)))
    with _lock:
        c = _ctx.get(dev.index)
    if c is None:
        h = ct.c_void_p()
        _check(lib().gsnfs_create(ct.byref(h), dev.index), "gsnfs_create")
        with _lock:
            _ctx[dev.index] = h
        c = h
    return c


def set_graphs(enable: bool, device=None):
    """Turns CUDA-graph capture / replay of the encoder on or off."""
    _check(lib().gsnfs_set_graphs(context(device), 1 if enable else 0), "gsnfs_set_graphs")


TUNABLES = {"raht_tile": 0, "raht_grid": 1, "prelude_grid": 2, "raht_pipe": 3}


def tune_set(name: str, value: int, device=None):
    """Sets a launch-shape tunable (0 = built-in default); outputs do not change."""
    _check(lib().gsnfs_tune_set(context(device), TUNABLES[name], int(value)), "gsnfs_tune_set")


def tune_get(name: str, device=None) -> int:
    v = ct.c_uint32()
    _check(lib().gsnfs_tune_get(context(device), TUNABLES[name], ct.byref(v)), "gsnfs_tune_get")
    return int(v.value)


def graph_stats(device=None):
    """(replays, captures, failed captures, graphs cached) of the encoder graphs."""
    out = (ct.c_uint64 * 4)()
    _check(lib().gsnfs_graph_stats(context(device), out), "gsnfs_graph_stats")
    return tuple(int(v) for v in out)


def _stream(t: torch.Tensor):
    return ct.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def _ptr(t):
    return ct.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else ct.c_void_p(0)


def _cuda_f32(t, cols):
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.dim() == 2 and t.shape[1] == cols):
        raise ValueError(f"expected a contiguous CUDA float32 tensor of shape [N, {cols}]")
    return t


class QuantParams:
    """Quantisation / entropy parameters (Sec. 3.4): group id per channel, one
    step per group, rounding offset tau, RLGR block size, rANS chunk size."""

    def __init__(self, groups, steps, tau=0.5, rlgr_block=512, rans_chunk=4096, color=False):
        self.groups = np.ascontiguousarray(np.asarray(groups, dtype=np.uint8).reshape(-1))
        self.steps = np.ascontiguousarray(np.asarray(steps, dtype=np.float64).reshape(-1))
        self.tau = float(tau)
        self.rlgr_block = int(rlgr_block)
        self.rans_chunk = int(rans_chunk)
        self.color = bool(color)

    @property
    def C(self):
        return int(self.groups.shape[0])

    def struct(self, C=None):
        C = self.C if C is None else C
        q = Quant()
        q.num_channels = C
        q.num_groups = int(self.steps.shape[0])
        q.channel_group = self.groups.ctypes.data_as(ct.POINTER(ct.c_uint8))
        q.steps = self.steps.ctypes.data_as(ct.POINTER(ct.c_double))
        q.tau = self.tau
        q.rlgr_block = self.rlgr_block
        q.rans_chunk = self.rans_chunk
        q.color = 1 if self.color else 0
        return q


def geometry_only(rans_chunk=4096):
    return QuantParams(np.zeros(0, np.uint8), [1.0], rans_chunk=rans_chunk)


def max_bitstream_bytes(n, J, qp: QuantParams):
    out = ct.c_uint64()
    q = qp.struct()
    _check(lib().gsnfs_max_bitstream_bytes(n, J, ct.byref(q), ct.byref(out)), "gsnfs_max_bitstream_bytes")
    return out.value


def reserve(n, J, qp: QuantParams, device=None):
    q = qp.struct()
    _check(lib().gsnfs_reserve(context(device), n, qp.C, J, ct.byref(q)), "gsnfs_reserve")


def encode_frame(pos: torch.Tensor, attr, J: int, qp: QuantParams, recon=False, out=None):
    """gsnfs_encode_frame.  Returns (bitstream uint8 tensor view, nv, recon_pos, recon_attr)."""
    _cuda_f32(pos, 3)
    n = pos.shape[0]
    C = qp.C
    if C:
        _cuda_f32(attr, C)
        if attr.shape[0] != n:
            raise ValueError("pos and attr rows differ")
    cap = max_bitstream_bytes(n, J, qp)
    if out is None or out.numel() < cap:
        out = torch.empty(cap, dtype=torch.uint8, device=pos.device)
    rp = torch.empty((max(n, 1), 3), dtype=torch.float32, device=pos.device) if recon else None
    ra = torch.empty((max(n, 1), max(C, 1)), dtype=torch.float32, device=pos.device) if recon and C else None
    q = qp.struct()
    nbytes, nv = ct.c_uint64(), ct.c_uint64()
    _check(lib().gsnfs_encode_frame(context(pos.device), _stream(pos), _ptr(pos), _ptr(attr) if C else None, n, J,
                                    ct.byref(q), _ptr(out), out.numel(), ct.byref(nbytes), _ptr(rp), _ptr(ra),
                                    ct.byref(nv)), "gsnfs_encode_frame")
    m = nv.value
    return (out[: nbytes.value], m, rp[:m] if rp is not None else None,
            ra[:m, :C] if ra is not None else None)


def peek_frame(header):
    """gsnfs_peek_frame on host bytes, a numpy array or a uint8 tensor (host or CUDA).  Returns (N_v, C, J)."""
    nv, C, J = ct.c_uint64(), ct.c_uint32(), ct.c_uint32()
    if isinstance(header, torch.Tensor):
        if header.dtype != torch.uint8 or not header.is_contiguous():
            raise ValueError("header must be a contiguous uint8 tensor")
        ptr, n = ct.c_void_p(header.data_ptr()), header.numel()
    else:
        h = np.frombuffer(bytes(header), dtype=np.uint8) if not isinstance(header, np.ndarray) else header
        h = np.ascontiguousarray(h, dtype=np.uint8)
        ptr, n = h.ctypes.data_as(ct.c_void_p), h.shape[0]
    _check(lib().gsnfs_peek_frame(ptr, n, ct.byref(nv), ct.byref(C), ct.byref(J)), "gsnfs_peek_frame")
    return nv.value, C.value, J.value


def decode_frame(bitstream: torch.Tensor, with_attr=True):
    """gsnfs_decode_frame.  Returns (pos [N_v,3], attr [N_v,C] or None)."""
    if not (bitstream.is_cuda and bitstream.dtype == torch.uint8):
        raise ValueError("bitstream must be a CUDA uint8 tensor")
    head = bitstream[:96].cpu().numpy()
    nv, C, J = peek_frame(head)
    pos = torch.empty((max(nv, 1), 3), dtype=torch.float32, device=bitstream.device)
    attr = torch.empty((max(nv, 1), max(C, 1)), dtype=torch.float32, device=bitstream.device) if with_attr and C else None
    got = ct.c_uint64()
    _check(lib().gsnfs_decode_frame(context(bitstream.device), _stream(bitstream), _ptr(bitstream), bitstream.numel(),
                                    _ptr(pos), _ptr(attr), max(nv, 1), ct.byref(got)), "gsnfs_decode_frame")
    m = got.value
    return pos[:m], (attr[:m, :C] if attr is not None else None)


HEADER_RECORD_BYTES = 4224  # GSNFS_HEADER_RECORD_BYTES


def encode_batch(pos_list, attr_list, J_list, rung_scales, qp: QuantParams, out=None, distortion=False,
                 headers=False):
    """gsnfs_encode_batch: frames x rungs.  Returns (out uint8 tensor, offsets np.uint64[F*R+1]); with
    distortion=True (gsnfs_encode_batch_rd) also the squared-error sums np.float64[F, R, C]; with headers=True
    (gsnfs_encode_batch_headers) also the streams' header records np.uint8[F*R, HEADER_RECORD_BYTES] for
    decode_batch_async."""
    if distortion and headers:
        raise ValueError("distortion and headers are separate calls")
    F = len(pos_list)
    R = len(rung_scales)
    dev = pos_list[0].device
    C = qp.C
    for p in pos_list:
        _cuda_f32(p, 3)
    if C:
        for a, p in zip(attr_list, pos_list):
            _cuda_f32(a, C)
    if out is None:  # worst-case size; a smaller caller buffer is grown on demand below
        cap = 0
        for p, J in zip(pos_list, J_list):
            cap += max_bitstream_bytes(p.shape[0], int(J), qp) * R
        out = torch.empty(cap, dtype=torch.uint8, device=dev)
    hp = (ct.c_void_p * F)(*[p.data_ptr() for p in pos_list])
    ha = (ct.c_void_p * F)(*[(a.data_ptr() if C else 0) for a in (attr_list if C else pos_list)])
    hn = (ct.c_uint64 * F)(*[p.shape[0] for p in pos_list])
    hJ = (ct.c_uint32 * F)(*[int(j) for j in J_list])
    hs = (ct.c_double * R)(*[float(s) for s in rung_scales])
    offs = (ct.c_uint64 * (F * R + 1))()
    q = qp.struct()
    dist = np.zeros((F, R, max(C, 1)), dtype=np.float64) if distortion else None
    hdr = np.zeros((F * R, HEADER_RECORD_BYTES), dtype=np.uint8) if headers else None

    def call(buf):
        if headers:
            return lib().gsnfs_encode_batch_headers(context(dev), _stream(buf), F, hp, ha, hn, hJ, R, hs, ct.byref(q),
                                                    _ptr(buf), buf.numel(), offs, hdr.ctypes.data_as(ct.c_void_p))
        if distortion:
            return lib().gsnfs_encode_batch_rd(context(dev), _stream(buf), F, hp, ha, hn, hJ, R, hs, ct.byref(q),
                                               _ptr(buf), buf.numel(), offs,
                                               dist.ctypes.data_as(ct.c_void_p))
        return lib().gsnfs_encode_batch(context(dev), _stream(buf), F, hp, ha, hn, hJ, R, hs, ct.byref(q), _ptr(buf),
                                        buf.numel(), offs)

    rc = call(out)
    if rc == -2:  # GSNFS_ERR_CAPACITY: offs[F*R] holds the size needed
        out = torch.empty(int(offs[F * R]) + 4096, dtype=torch.uint8, device=dev)
        rc = call(out)
    _check(rc, "gsnfs_encode_batch")
    if distortion:
        return out, np.array(offs[:], dtype=np.uint64), dist[:, :, :C]
    if headers:
        return out, np.array(offs[:], dtype=np.uint64), hdr
    return out, np.array(offs[:], dtype=np.uint64)


def decode_frame_lod(bitstream: torch.Tensor, depth: int):
    """gsnfs_decode_frame_lod: (node centres [n, 3], node mean attributes [n, C] or None) at octree depth `depth`."""
    host = bitstream[:96].cpu().numpy()
    nv, C, J = peek_frame(host)
    dev = bitstream.device
    pos = torch.empty((max(nv, 1), 3), dtype=torch.float32, device=dev)
    attr = torch.empty((max(nv, 1), max(C, 1)), dtype=torch.float32, device=dev) if C else None
    n = ct.c_uint64()
    _check(lib().gsnfs_decode_frame_lod(context(dev), _stream(bitstream), _ptr(bitstream), bitstream.numel(), depth,
                                        _ptr(pos), _ptr(attr), max(nv, 1), ct.byref(n)), "gsnfs_decode_frame_lod")
    k = n.value
    return pos[:k], (attr[:k, :C] if attr is not None else None)


class Camera(ct.Structure):
    """gsnfs_camera: 3 x 4 world-to-camera [R | t] (row major), pinhole intrinsics, image size, near plane, background."""
    _fields_ = [("view", ct.c_double * 12), ("fx", ct.c_double), ("fy", ct.c_double), ("cx", ct.c_double),
                ("cy", ct.c_double), ("width", ct.c_uint32), ("height", ct.c_uint32), ("znear", ct.c_double),
                ("background", ct.c_double * 3)]


def render(pos: torch.Tensor, attr: torch.Tensor, view, fx, fy, cx, cy, width: int, height: int, znear=0.01,
           background=(0.0, 0.0, 0.0), out: torch.Tensor | None = None):
    """gsnfs_render: splat-rasterised image [height, width, 3] (float32) of n 56-channel Gaussians."""
    _cuda_f32(pos, 3)
    _cuda_f32(attr, 56)
    if pos.shape[0] != attr.shape[0]:
        raise ValueError("pos and attr row counts differ")
    cam = Camera()
    v = np.asarray(view, dtype=np.float64).reshape(12)
    cam.view[:] = [float(x) for x in v]
    cam.fx, cam.fy, cam.cx, cam.cy = float(fx), float(fy), float(cx), float(cy)
    cam.width, cam.height, cam.znear = int(width), int(height), float(znear)
    cam.background[:] = [float(x) for x in background]
    if out is None:
        out = torch.empty((height, width, 3), dtype=torch.float32, device=pos.device)
    elif out.shape != (height, width, 3) or out.dtype != torch.float32 or not out.is_contiguous():
        raise ValueError("out must be a contiguous float32 [height, width, 3] tensor")
    _check(lib().gsnfs_render(context(pos.device), _stream(pos), _ptr(pos), _ptr(attr), pos.shape[0], ct.byref(cam),
                              _ptr(out)), "gsnfs_render")
    return out


def decode_batch(data: torch.Tensor, offsets, C: int, rows_cap: int, pos_out: torch.Tensor | None = None,
                 attr_out: torch.Tensor | None = None):
    """gsnfs_decode_batch over streams data[offsets[f]:offsets[f+1]].
    Returns (pos, attr, row offsets).  pos_out [rows_cap, 3] and attr_out
    [rows_cap, C] (contiguous float32 on the same device) receive the rows
    when given, else new tensors are allocated."""
    F = len(offsets) - 1
    hin = (ct.c_uint64 * (F + 1))(*[int(o) for o in offsets])
    rows = (ct.c_uint64 * (F + 1))()
    if pos_out is not None:
        if (pos_out.dtype != torch.float32 or not pos_out.is_contiguous() or pos_out.device != data.device
                or tuple(pos_out.shape) != (max(rows_cap, 1), 3)):
            raise ValueError("pos_out must be a contiguous float32 [rows_cap, 3] tensor on the data's device")
        pos = pos_out
    else:
        pos = torch.empty((max(rows_cap, 1), 3), dtype=torch.float32, device=data.device)
    if C and attr_out is not None:
        if (attr_out.dtype != torch.float32 or not attr_out.is_contiguous() or attr_out.device != data.device
                or tuple(attr_out.shape) != (max(rows_cap, 1), C)):
            raise ValueError("attr_out must be a contiguous float32 [rows_cap, C] tensor on the data's device")
        attr = attr_out
    else:
        attr = torch.empty((max(rows_cap, 1), max(C, 1)), dtype=torch.float32, device=data.device) if C else None
    _check(lib().gsnfs_decode_batch(context(data.device), _stream(data), F, _ptr(data), hin, _ptr(pos), _ptr(attr),
                                    rows_cap, rows), "gsnfs_decode_batch")
    r = np.array(rows[:], dtype=np.uint64)
    n = int(r[-1])
    return pos[:n], (attr[:n, :C] if attr is not None else None), r


def decode_batch_async(data: torch.Tensor, offsets, headers, C: int, rows_cap: int, pos_out: torch.Tensor,
                       attr_out: torch.Tensor | None, status: torch.Tensor):
    """gsnfs_decode_batch_async: decode_batch given the streams' header records (np.uint8[F, HEADER_RECORD_BYTES]
    from encode_batch(..., headers=True)); enqueues the decode on the current stream and returns at once.
    status: an int32 tensor of one element (device, or pinned host memory) receiving the device status once the
    stream reaches the end of the decode (0 = ok).  Returns the row offsets (np.uint64[F+1])."""
    F = len(offsets) - 1
    hin = (ct.c_uint64 * (F + 1))(*[int(o) for o in offsets])
    rows = (ct.c_uint64 * (F + 1))()
    hdr = np.ascontiguousarray(headers, dtype=np.uint8)
    if hdr.shape != (F, HEADER_RECORD_BYTES):
        raise ValueError("headers must be uint8 [frames, HEADER_RECORD_BYTES]")
    for t, cols in ((pos_out, 3), (attr_out, C)):
        if t is not None and (t.dtype != torch.float32 or not t.is_contiguous() or tuple(t.shape) != (max(rows_cap, 1),
                                                                                                      cols)):
            raise ValueError("outputs must be contiguous float32 [rows_cap, 3] and [rows_cap, C] tensors")
    if status.dtype != torch.int32 or status.numel() != 1:
        raise ValueError("status must be a one-element int32 tensor")
    _check(lib().gsnfs_decode_batch_async(context(data.device), _stream(data), F, _ptr(data), hin,
                                          hdr.ctypes.data_as(ct.c_void_p), _ptr(pos_out),
                                          _ptr(attr_out) if C else ct.c_void_p(0), rows_cap, rows,
                                          ct.c_void_p(status.data_ptr())), "gsnfs_decode_batch_async")
    return np.array(rows[:], dtype=np.uint64)


# ---- stage entry points ---------------------------------------------------
def voxelize(pos: torch.Tensor, J: int):
    """gsnfs_voxelize: ascending distinct Morton codes and (lo, ext)."""
    _cuda_f32(pos, 3)
    n = pos.shape[0]
    codes = torch.empty(max(n, 1), dtype=torch.int64, device=pos.device)
    grid = (ct.c_double * 4)()
    nv = ct.c_uint64()
    _check(lib().gsnfs_voxelize(context(pos.device), _stream(pos), _ptr(pos), n, J, _ptr(codes), grid, ct.byref(nv)),
           "gsnfs_voxelize")
    return codes[: nv.value], np.array(grid[:3]), float(grid[3])


def octree_encode(codes: torch.Tensor, J: int):
    """gsnfs_octree_encode: breadth-first occupancy bytes and level sizes."""
    nv = codes.shape[0]
    cap = 8 * max(nv, 1) * J + 64
    occ = torch.empty(cap, dtype=torch.uint8, device=codes.device)
    lsz = (ct.c_uint32 * (J + 1))()
    nb = ct.c_uint64()
    _check(lib().gsnfs_octree_encode(context(codes.device), _stream(codes), _ptr(codes), nv, J, _ptr(occ), cap, lsz,
                                     ct.byref(nb)), "gsnfs_octree_encode")
    return occ[: nb.value], np.array(lsz[:], dtype=np.uint32)


def octree_decode(occ: torch.Tensor, J: int, level_sizes):
    lsz = (ct.c_uint32 * (J + 1))(*[int(x) for x in level_sizes])
    nv = int(level_sizes[J])
    codes = torch.empty(max(nv, 1), dtype=torch.int64, device=occ.device)
    _check(lib().gsnfs_octree_decode(context(occ.device), _stream(occ), _ptr(occ), occ.numel(), J, lsz, _ptr(codes)),
           "gsnfs_octree_decode")
    return codes[:nv]


def occupancy_section_encode(data: torch.Tensor, rans_chunk=4096):
    n = data.numel()
    cap = 64 + 2 * n + 1024 + (n // 32 + 1) * 256
    out = torch.empty(cap, dtype=torch.uint8, device=data.device)
    nb = ct.c_uint64()
    _check(lib().gsnfs_occupancy_section_encode(context(data.device), _stream(data), _ptr(data), n, rans_chunk,
                                                _ptr(out), cap, ct.byref(nb)), "gsnfs_occupancy_section_encode")
    return out[: nb.value]


def occupancy_section_decode(sec: torch.Tensor, n: int):
    out = torch.empty(max(n, 1), dtype=torch.uint8, device=sec.device)
    _check(lib().gsnfs_occupancy_section_decode(context(sec.device), _stream(sec), _ptr(sec), sec.numel(), _ptr(out),
                                                n), "gsnfs_occupancy_section_decode")
    return out[:n]


class RahtPlan:
    """gsnfs_raht_plan_*: the butterfly schedule of a voxel set (Sec. 3.2
    prelude) with forward / inverse transforms (Algorithm 6)."""

    def __init__(self, codes: torch.Tensor, J: int, C: int):
        self.device = codes.device
        self.nv = codes.shape[0]
        self.C = C
        self.J = J
        h = ct.c_void_p()
        _check(lib().gsnfs_raht_plan_create(context(codes.device), _stream(codes), _ptr(codes), self.nv, J, C,
                                            ct.byref(h)), "gsnfs_raht_plan_create")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.gsnfs_raht_plan_destroy(h)
            self._h = None

    def _io(self, x):
        if not (x.is_cuda and x.dtype in (torch.float32, torch.float64) and x.is_contiguous() and x.dim() == 2
                and x.shape[1] == self.C):
            raise ValueError(f"expected a contiguous CUDA float32 or float64 tensor of shape [nv, {self.C}]")
        if x.shape[0] != self.nv:
            raise ValueError("row count differs from the plan's voxel count")

    def forward(self, A: torch.Tensor, out=None):
        """Forward RAHT (FP32, or FP64 for float64 tensors)."""
        self._io(A)
        out = torch.empty_like(A) if out is None else out
        f = lib().gsnfs_raht_forward_f64 if A.dtype == torch.float64 else lib().gsnfs_raht_forward
        _check(f(self._h, _stream(A), _ptr(A), _ptr(out)), "gsnfs_raht_forward")
        return out

    def inverse(self, Y: torch.Tensor, out=None, qp: QuantParams | None = None):
        """Inverse RAHT; with qp, each coefficient is quantised and dequantised first."""
        self._io(Y)
        out = torch.empty_like(Y) if out is None else out
        q = qp.struct() if qp is not None else None
        f = lib().gsnfs_raht_inverse_f64 if Y.dtype == torch.float64 else lib().gsnfs_raht_inverse
        _check(f(self._h, _stream(Y), _ptr(Y), _ptr(out), ct.byref(q) if q is not None else None),
               "gsnfs_raht_inverse")
        return out


# ---- differentiable attribute codec ------------------------------------------
# RAHT is orthonormal (Sec. 3.2: every butterfly of Eq. (1) is a rotation), so
# the transpose of the forward transform is the inverse transform and the
# transpose of the inverse is the forward: each backward pass is the other
# kernel.  A plan's survivor pool is shared by its calls: use one plan from one
# stream at a time.

class RahtForwardFn(torch.autograd.Function):
    """Y = T A; dL/dA = T^T dL/dY = inverse RAHT of dL/dY."""

    @staticmethod
    def forward(ctx, A, plan):
        ctx.plan = plan
        return plan.forward(A.contiguous())

    @staticmethod
    def backward(ctx, g):
        return ctx.plan.inverse(g.contiguous()), None


class RahtInverseFn(torch.autograd.Function):
    """A = T^T Y; dL/dY = T dL/dA = forward RAHT of dL/dA."""

    @staticmethod
    def forward(ctx, Y, plan):
        ctx.plan = plan
        return plan.inverse(Y.contiguous())

    @staticmethod
    def backward(ctx, g):
        return ctx.plan.forward(g.contiguous()), None


class AttrCodecFn(torch.autograd.Function):
    """The attribute codec as a differentiable layer (Sec. 3.2 with the
    quantiser of Sec. 3.4): forward A_hat = T^T (step * q(T A)), the encoder's
    reconstruction; the quantiser's gradient is taken as the identity
    (straight-through), so dL/dA = T^T T dL/dA_hat, evaluated by the forward
    kernel followed by the inverse kernel."""

    @staticmethod
    def forward(ctx, A, plan, qp):
        ctx.plan = plan
        return plan.inverse(plan.forward(A.contiguous()), qp=qp)

    @staticmethod
    def backward(ctx, g):
        return ctx.plan.inverse(ctx.plan.forward(g.contiguous())), None, None


def rlgr_slot_words(B: int) -> int:
    return int(lib().gsnfs_rlgr_slot_words(B))


def rlgr_encode_indices(q: torch.Tensor, B: int):
    """Block RLGR of int32 indices [nv, C]; returns (slots, block_words)."""
    nv, C = q.shape
    nb = (nv + B - 1) // B
    sw = rlgr_slot_words(B)
    slots = torch.zeros(max(C * nb * sw, 1), dtype=torch.int32, device=q.device)
    bw = torch.zeros(max(C * nb, 1), dtype=torch.int32, device=q.device)
    _check(lib().gsnfs_rlgr_encode_indices(context(q.device), _stream(q), _ptr(q), nv, C, B, _ptr(slots), _ptr(bw)),
           "gsnfs_rlgr_encode_indices")
    return slots, bw[: C * nb]


def rlgr_decode_indices(slots: torch.Tensor, block_words: torch.Tensor, nv: int, C: int, B: int):
    q = torch.empty((max(nv, 1), C), dtype=torch.int32, device=slots.device)
    _check(lib().gsnfs_rlgr_decode_indices(context(slots.device), _stream(slots), _ptr(slots), _ptr(block_words), nv,
                                           C, B, _ptr(q)), "gsnfs_rlgr_decode_indices")
    return q[:nv]


# ---- instrumentation ----------------------------------------------------------
def launch_count() -> int:
    """Kernels enqueued by the library since it was loaded."""
    return int(lib().gsnfs_launch_count())


def profile_enable(on: bool = True):
    _check(lib().gsnfs_profile_enable(1 if on else 0), "gsnfs_profile_enable")


def profile_read():
    """{stage: (total ms, intervals)} since the last read (synchronises)."""
    n = lib().gsnfs_profile_stage_names(None, 0) if False else 32
    names = (ct.c_char_p * n)()
    k = lib().gsnfs_profile_stage_names(names, n)
    ms = (ct.c_double * k)()
    cnt = (ct.c_uint64 * k)()
    _check(lib().gsnfs_profile_read(ms, cnt, k), "gsnfs_profile_read")
    return {names[i].decode(): (ms[i], int(cnt[i])) for i in range(k)}
