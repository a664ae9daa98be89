"""Index-file header checks run before any device call: a missing file, a
file of another format and a header whose offsets disagree with its leaf
counts are refused on a machine without a GPU."""
import ctypes as C

import numpy as np
import pytest

from paper_2603_24920_gb300 import build_ext
from paper_2603_24920_gb300 import detlsh as D


class Header(C.Structure):
    """Mirror of the index file's fixed header (672 bytes, include/detlsh.h)."""
    _fields_ = ([("magic", C.c_char * 8), ("version", C.c_uint32), ("bom", C.c_uint32),
                 ("header_bytes", C.c_uint32), ("nsections", C.c_uint32), ("n", C.c_int64)]
                + [(f, C.c_int32) for f in ("d", "L", "K", "N_r", "bbits", "M", "box_mode",
                                            "encoding", "tree_group", "has_bf16", "has_proj",
                                            "bf16_exact")]
                + [("seed", C.c_uint64), ("frac", C.c_double), ("eps2", C.c_double)]
                + [(f, C.c_int64) for f in ("m_sample", "max_leaf", "max_leaves", "fb_total")]
                + [("nleaves", C.c_int64 * 16), ("leaf_off", C.c_int64 * 17),
                   ("blk_off", C.c_int64 * 17), ("sblk_off", C.c_int64 * 17)])


@pytest.fixture(scope="module")
def lib():
    build_ext.build()
    return D.lib()


def _valid_header():
    h = Header()
    h.magic = b"DETLSHIX"
    h.version, h.bom, h.header_bytes, h.nsections = 1, 0x01020304, C.sizeof(Header), 17
    h.n, h.d, h.L, h.K, h.N_r, h.bbits, h.M = 1000, 8, 2, 4, 16, 4, 64
    h.has_bf16, h.frac, h.eps2, h.m_sample = 1, 0.1, 5.0, 100
    leaves = [40, 70]
    off = blk = sblk = 0
    for t in range(17):
        h.leaf_off[t], h.blk_off[t], h.sblk_off[t] = off, blk, sblk
        if t < 2:
            h.nleaves[t] = leaves[t]
            nb = -(-leaves[t] // 32)
            off, blk, sblk = off + leaves[t], blk + nb, sblk + -(-nb // 32)
    h.max_leaves, h.max_leaf = 70, 60
    return h


def _load_status(lib, path):
    out = C.c_void_p()
    s = lib.detlsh_load(str(path).encode(), None, C.byref(out))
    assert not out.value
    return s


def test_header_size(lib):
    assert C.sizeof(Header) == 672


def test_missing_and_foreign_files(lib, tmp_path):
    assert _load_status(lib, tmp_path / "missing") == -9
    p = tmp_path / "noise"
    p.write_bytes(np.random.default_rng(0).integers(0, 256, 4096, dtype=np.uint8).tobytes())
    assert _load_status(lib, p) == -10
    p.write_bytes(b"DETLSHIX")  # shorter than a header
    assert _load_status(lib, p) == -10


@pytest.mark.parametrize("field,value", [("version", 2), ("bom", 0x04030201), ("N_r", 24),
                                         ("bbits", 5), ("L", 0), ("m_sample", 1001),
                                         ("max_leaves", 69), ("eps2", -1.0), ("bf16_exact", 2)])
def test_bad_header_fields(lib, tmp_path, field, value):
    h = _valid_header()
    setattr(h, field, value)
    p = tmp_path / "bad"
    p.write_bytes(bytes(h))
    assert _load_status(lib, p) == -10


def test_offsets_must_follow_the_leaf_counts(lib, tmp_path):
    h = _valid_header()
    h.blk_off[1] += 1
    p = tmp_path / "bad"
    p.write_bytes(bytes(h))
    assert _load_status(lib, p) == -10


def test_valid_header_reaches_the_device_check(lib, tmp_path):
    # without a GPU the load stops at NO_DEVICE; with one, at the missing arrays
    p = tmp_path / "hdr"
    p.write_bytes(bytes(_valid_header()))
    assert _load_status(lib, p) in (-6, -10)


def test_null_arguments(lib):
    out = C.c_void_p()
    assert lib.detlsh_load(None, None, C.byref(out)) == -1
    assert lib.detlsh_save(None, b"x", None) == -1
