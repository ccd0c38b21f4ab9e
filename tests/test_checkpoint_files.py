"""lsm_load rejects files that are not checkpoints before any device work
(runs without a GPU: only the library's host code is reached)."""
import struct

import pytest

from paper_2201_04565_gb300 import build, lsm


@pytest.fixture(scope="module")
def L():
    build.build()
    lsm.load_library()
    return lsm


def _load_error(L, path):
    with pytest.raises(L.LsmError) as ei:
        L.lsm_load(str(path))
    assert ei.value.status == L.LSM_EINVAL
    return str(ei.value)


def test_missing_file(L, tmp_path):
    assert "cannot open" in _load_error(L, tmp_path / "absent.lsmckpt")


def test_foreign_file(L, tmp_path):
    p = tmp_path / "foreign.bin"
    p.write_bytes(b"GIF89a" + bytes(200))
    assert "not a checkpoint" in _load_error(L, p)


def test_other_version(L, tmp_path):
    p = tmp_path / "v9.lsmckpt"
    p.write_bytes(b"LSMCKPT\0" + struct.pack("<II", 9, 0x01020304) + bytes(64))
    assert "unsupported" in _load_error(L, p)


def test_truncated_file(L, tmp_path):
    p = tmp_path / "cut.lsmckpt"
    # a valid preamble, then a vector count far beyond the file's length
    body = struct.pack("<iqqddddd", 2, 10, 9, 0.01, 0.1, 0.0, 1.0, 1.0) + struct.pack("<Q", 1 << 40)
    p.write_bytes(b"LSMCKPT\0" + struct.pack("<II", 1, 0x01020304) + body + bytes(8))
    assert "truncated or malformed" in _load_error(L, p)


def test_null_arguments(L):
    import ctypes as C
    lib = L.load_library()
    assert lib.lsm_save(None, b"x") == L.LSM_EINVAL
    out = C.c_void_p()
    assert lib.lsm_load(None, None, C.byref(out)) == L.LSM_EINVAL
