"""GPU path vs the FP64 oracle at the full workload sizes, in the launch
configuration the benchmark times (tile kernels, lsm_step(20) per load
increment), element by element over every particle.

  - 2D 2048 x 2048 two-phase composite (4,194,304 particles, 16,764,930
    springs): exact64 bit-identical positions and velocities; df64 positions
    within 1e-10 relative (normwise) and the stress sample within 1e-6; f32
    displacement error stated and bounded;
  - 3D 256^3 foam (5.9M particles, 47.5M springs) under compression: df64 and
    f32 against the oracle, same bars;
  - the paper's triangular packing of the 2048 x 2048 image (4,840,290
    particles, 14,512,048 springs) on the strip kernel: df64 positions
    within 1e-10 relative, identical broken set, stress within 1e-6.

Two increments of 20 time steps each: the oracle (threaded, bit-identical to
its sequential form) finishes them in seconds at these sizes.
"""
import os

import numpy as np
import pytest

from gen.images import foam_volume, inclusion_image, one_phase_materials, two_phase_materials

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_04565_gb300 import build, lsm
    build.build()
    lsm.load_library()
    return lsm


@pytest.fixture(scope="module")
def img2d():
    return inclusion_image(2048, 2048, 10.0, 60.0, 0.30, 1)


@pytest.fixture(scope="module")
def img3d():
    return foam_volume(256, 4.0, 0.35, seed=2)


def _oracle_run(oracle_mod, img, mats, eps_inc, incs=2, steps=20, lattice=0):
    k, e, m = mats
    o = oracle_mod.Oracle.from_image(img, k, e, m, lattice=lattice)
    o.set_threads(os.cpu_count() or 1)
    samples = []
    for i in range(1, incs + 1):
        o.apply_strain(i * eps_inc)
        o.step(steps)
        samples.append(o.observe())
    x, v, _ = o.state()
    X = o.topology()["X"]
    return o, x, v, X, samples


def _gpu_run(L, img, mats, precision, eps_inc, incs=2, steps=20, lattice=0):
    k, e, m = mats
    g = L.Specimen.from_image(img, k, e, m, precision=precision, path=0, lattice=lattice)
    for i in range(1, incs + 1):
        g.apply_strain(i * eps_inc)
        g.step(steps)
    x, v = g.state()
    s = g.samples()
    mask, first = g.broken()
    g.close()
    return x, v, s, mask, first


@pytest.fixture(scope="module")
def ref2d(oracle_mod, img2d):
    o, x, v, X, s = _oracle_run(oracle_mod, img2d, two_phase_materials(), 1e-3)
    mask, _, first = o.broken()
    return dict(x=x, v=v, X=X, s=s, mask=mask, first=first, n=o.n, m=o.m)


@pytest.mark.parametrize("precision", ["exact64", "df64", "f32"])
def test_2d_2048_full_size(L, img2d, ref2d, precision):
    x, v, s, mask, first = _gpu_run(L, img2d, two_phase_materials(), precision, 1e-3)
    r = ref2d
    assert x.shape == r["x"].shape == (2, 4194304)
    assert np.array_equal(mask, r["mask"]) and first == r["first"]
    if precision == "exact64":
        assert np.array_equal(x, r["x"]) and np.array_equal(v, r["v"])
        for a, b in zip(s, r["s"]):
            assert a["sigma_vir"] == pytest.approx(b["sigma_vir"], rel=1e-12)
        return
    dx = np.abs(x - r["x"]).max()
    rel_x = dx / np.abs(r["x"]).max()
    rel_u = dx / np.abs(r["x"] - r["X"]).max()
    print("2048^2 %s: position error %.3e relative, displacement error %.3e relative" % (precision, rel_x, rel_u))
    if precision == "df64":
        assert rel_x <= 1e-10
        for a, b in zip(s, r["s"]):
            assert a["sigma_vir"] == pytest.approx(b["sigma_vir"], rel=1e-6)
    else:
        assert rel_u < 1e-4
        for a, b in zip(s, r["s"]):
            assert a["sigma_vir"] == pytest.approx(b["sigma_vir"], rel=1e-3)


@pytest.fixture(scope="module")
def ref3d(oracle_mod, img3d):
    o, x, v, X, s = _oracle_run(oracle_mod, img3d, one_phase_materials(), -1e-3)
    mask, _, first = o.broken()
    return dict(x=x, v=v, X=X, s=s, mask=mask, first=first)


@pytest.mark.parametrize("precision", ["df64", "f32"])
def test_3d_foam256_full_size(L, img3d, ref3d, precision):
    x, v, s, mask, first = _gpu_run(L, img3d, one_phase_materials(), precision, -1e-3)
    r = ref3d
    assert x.shape == r["x"].shape and x.shape[0] == 3
    assert np.array_equal(mask, r["mask"]) and first == r["first"]
    dx = np.abs(x - r["x"]).max()
    rel_x = dx / np.abs(r["x"]).max()
    rel_u = dx / np.abs(r["x"] - r["X"]).max()
    print("foam 256^3 %s: position error %.3e relative, displacement error %.3e relative" % (precision, rel_x, rel_u))
    if precision == "df64":
        assert rel_x <= 1e-10
        for a, b in zip(s, r["s"]):
            assert a["sigma_vir"] == pytest.approx(b["sigma_vir"], rel=1e-6)
    else:
        assert rel_u < 1e-4
        for a, b in zip(s, r["s"]):
            assert a["sigma_vir"] == pytest.approx(b["sigma_vir"], rel=1e-3)


def test_2d_2048_triangular_full_size(oracle_mod, L, img2d):
    """The triangular packing at full size, in the strip kernel's launch
    configuration for it (one wave of strips over the site grid)."""
    mats = two_phase_materials()
    o, xo, vo, X, so = _oracle_run(oracle_mod, img2d, mats, 1e-3, lattice=1)
    mo, _, fo = o.broken()
    n = o.n
    x, v, s, mask, first = _gpu_run(L, img2d, mats, "df64", 1e-3, lattice=1)
    assert x.shape == xo.shape == (2, n) and n == 4840290
    assert np.array_equal(mask, mo) and first == fo
    dx = np.abs(x - xo).max()
    rel_x = dx / np.abs(xo).max()
    print("2048^2 triangular df64: position error %.3e relative, displacement error %.3e relative"
          % (rel_x, dx / np.abs(xo - X).max()))
    assert rel_x <= 1e-10
    for a, b in zip(s, so):
        assert a["sigma_vir"] == pytest.approx(b["sigma_vir"], rel=1e-6)
