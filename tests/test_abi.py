"""The C-ABI library loads and exports every symbol include/lsm.h declares;
argument checks that need no GPU reject bad input (no compute calls here)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b((?:lsm|lsmb|nn)_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2201_04565_gb300 import build, lsm
    build.build()
    return lsm.load_library()


def test_header_declares_the_five_core_calls():
    names = _declared_symbols()
    for core in ("lsm_build_from_image", "lsm_step", "lsm_apply_strain", "lsm_stress_strain",
                 "lsm_broken_mask"):
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2201_04565_gb300 import lsm
    bound = {name for name, _, _ in lsm.SIGNATURES}
    extra = set()
    try:
        from paper_2201_04565_gb300 import batch
        extra = {name for name, _, _ in batch.SIGNATURES}
    except ImportError:
        pass
    try:
        from paper_2201_04565_gb300 import nn
        extra |= {name for name, _, _ in nn.SIGNATURES}
    except ImportError:
        pass
    assert _declared_symbols() <= bound | extra


def test_bad_descriptors_rejected_before_any_device_work(lib):
    from paper_2201_04565_gb300 import lsm
    k, e = [[1.0]], [[0.1]]
    with pytest.raises(lsm.LsmError) as ei:
        lsm.lsm_build_from_image(np.ones((4, 1), np.uint8), k, e)  # nx < 2
    assert ei.value.status == lsm.LSM_EINVAL
    with pytest.raises(lsm.LsmError):
        lsm.lsm_build_from_image(np.full((3, 3), 2, np.uint8), k, e)  # phase > nphase
    with pytest.raises(lsm.LsmError):
        lsm.lsm_build_from_image(np.zeros((3, 3), np.uint8), k, e)  # no particles
    with pytest.raises(lsm.LsmError):
        lsm.lsm_build_from_image(np.ones((3, 3), np.uint8), k, e, dt=-1.0)
    with pytest.raises(lsm.LsmError):
        lsm.lsm_build_from_image(np.ones((3, 3), np.uint8), k, e, precision=7)
    X = np.zeros((2, 3))
    with pytest.raises(lsm.LsmError):  # not canonical order
        lsm.lsm_build_network(X, [1, 0], [2, 1], [1, 1], [1, 1], [2, 2])
    with pytest.raises(lsm.LsmError):  # si >= sj
        lsm.lsm_build_network(X, [1], [1], [1], [1], [2])
    msg = lib.lsm_last_error(None)
    assert msg and b"sj" in msg


def test_null_arguments(lib):
    assert lib.lsm_step(None, 1) == -1
    assert lib.lsm_apply_strain(None, 0.1) == -1
    assert lib.lsm_build_from_image(None, None) == -1
    lib.lsm_destroy(None)


def test_product_package_does_not_reference_the_oracle():
    pkg = os.path.join(ROOT, "paper_2201_04565_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cpp", ".h")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "lsm_oracle" not in text, fn
