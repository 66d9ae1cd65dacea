"""The C ABI library builds, loads without a GPU, and exports every entry
point that include/gsnfs.h declares; the binding refuses to run without it."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2606_05650_gb300 import build
    return build.build()


def _declared():
    src = open(os.path.join(ROOT, "include", "gsnfs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gsnfs_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_codec_calls():
    names = _declared()
    for must in ("gsnfs_encode_frame", "gsnfs_decode_frame", "gsnfs_encode_batch", "gsnfs_decode_batch",
                 "gsnfs_raht_forward", "gsnfs_raht_inverse", "gsnfs_octree_encode", "gsnfs_octree_decode"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_exports_are_c_symbols(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (gsnfs_[a-z0-9_]+)$", out, flags=re.M))
    assert set(_declared()) <= exported


def test_build_targets_sm_103a_only():
    from paper_2606_05650_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_status_strings_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.gsnfs_status_string.restype = ctypes.c_char_p
    assert lib.gsnfs_status_string(-3) == b"corrupt bitstream"
    assert lib.gsnfs_status_string(0) == b"ok"


def test_host_side_bounds_and_validation(libpath):
    from paper_2606_05650_gb300 import gsnfs
    qp = gsnfs.QuantParams([0, 0, 1], [0.1, 0.2])
    assert gsnfs.max_bitstream_bytes(1000, 10, qp) > 1000 * 3
    bad = gsnfs.QuantParams([0, 3, 1], [0.1, 0.2])  # group id beyond G
    with pytest.raises(gsnfs.GsnfsError):
        gsnfs.max_bitstream_bytes(10, 10, bad)
    with pytest.raises(gsnfs.GsnfsError):
        gsnfs.max_bitstream_bytes(10, 22, qp)  # J > 21
    with pytest.raises(gsnfs.GsnfsError):
        gsnfs.peek_frame(bytes(96))  # no magic
    # a hand-built header in host memory: magic "GSN1", version 1, J at byte 12, C at 16, N_v at 24
    import struct
    h = bytearray(96)
    struct.pack_into("<II", h, 0, 0x314E5347, 1)
    struct.pack_into("<II", h, 12, 16, 56)
    struct.pack_into("<Q", h, 24, 999_999)
    assert gsnfs.peek_frame(bytes(h)) == (999_999, 56, 16)
    import torch
    assert gsnfs.peek_frame(torch.frombuffer(bytearray(h), dtype=torch.uint8)) == (999_999, 56, 16)
    with pytest.raises(gsnfs.GsnfsError):
        gsnfs.peek_frame(bytes(h[:95]))  # fewer than 96 bytes
    struct.pack_into("<I", h, 12, 22)  # J beyond 21
    with pytest.raises(gsnfs.GsnfsError):
        gsnfs.peek_frame(bytes(h))
