"""Pipelined readback (lsm_readback_async / lsm_readback_wait): every
increment's broken-spring mask and sample, copied out on the context's
second stream while later increments run, equal what the synchronising calls
(lsm_broken_mask, lsm_sample_last) return for that increment, on the tile and
strip kernels and on the spring-list kernels; the two device snapshots are
reused while copies are in flight, the sample buffer may grow under them, and
bad arguments are refused."""
import numpy as np
import pytest

from gen.images import foam_volume, inclusion_image, one_phase_materials, two_phase_materials

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_04565_gb300 import build, lsm
    build.build()
    lsm.load_library()
    return torch, lsm


def _spec(lsm, path, prec="df64", kind="2d"):
    if kind == "3d":
        img = foam_volume(14, 1.5, 0.6, seed=21)
        k, e, m = one_phase_materials(1.0, 0.02)
        return lsm.Specimen.from_image(img, k, e, m, precision=prec, path=path)
    img = inclusion_image(48, 40, 3.0, 6.0, 0.3, 11)
    k, e, m = two_phase_materials()
    return lsm.Specimen.from_image(img, k, e, m, precision=prec, path=path, lattice=1 if kind == "tri" else 0)


@pytest.mark.parametrize("path,prec,kind", [(0, "df64", "2d"), (0, "exact64", "2d"), (1, "df64", "2d"),
                                            (3, "f32", "2d"), (0, "df64", "tri"), (0, "df64", "3d")])
def test_readback_matches_synchronous_calls(env, path, prec, kind):
    """2D tile kernel (df64, exact64), spring-list kernels, strip kernel,
    triangular packing (strip kernel on its site grid), 3D voxel tile kernel."""
    torch, lsm = env
    a, b = _spec(lsm, path, prec, kind), _spec(lsm, path, prec, kind)  # pipelined / synchronous twins
    n_inc, nst, deps = 12, 20, 0.01  # large increments: springs break within the run
    masks = [torch.empty(max(a.m, 1), dtype=torch.uint8, pin_memory=True).numpy() for _ in range(n_inc)]
    samples = [torch.empty(64, dtype=torch.uint8, pin_memory=True).numpy() for _ in range(n_inc)]
    want = []
    for q in range(n_inc):
        for s in (a, b):
            s.apply_strain((q + 1) * deps)
            s.step(nst)
        a.readback_async(masks[q], samples[q])  # no wait: up to n_inc copies queued
        mb, fb = b.broken()
        want.append((mb.copy(), b.last_sample()))
    a.readback_wait()
    assert want[-1][0].sum() > 0, "the run should break springs"
    for q in range(n_inc):
        assert np.array_equal(masks[q][:a.m], want[q][0]), q
        got = lsm.sample_from_buffer(samples[q])
        assert got == want[q][1], q


def test_readback_parts_errors_and_sample_growth(env):
    torch, lsm = env
    s = _spec(lsm, 0)
    buf = torch.empty(64, dtype=torch.uint8, pin_memory=True).numpy()
    with pytest.raises(RuntimeError):
        s.readback_async(None, buf)  # no sample recorded yet
    short = np.zeros(max(s.m - 1, 1), np.uint8)
    with pytest.raises(ValueError):
        s.readback_async(short, None)
    h = s.h
    L = lsm.load_library()
    assert L.lsm_readback_async(h, short.ctypes.data_as(lsm.C.c_void_p), short.size, None) == lsm.LSM_EINVAL
    assert L.lsm_readback_async(h, None, 0, None) == lsm.LSM_EINVAL
    # the mask alone, before any step
    mask = torch.empty(max(s.m, 1), dtype=torch.uint8, pin_memory=True).numpy()
    mask[:] = 7
    s.readback_async(mask, None)
    s.readback_wait()
    assert not mask[:s.m].any()
    # more calls than the initial sample buffer holds (1,024), each followed by
    # a sample readback: the buffer grows while copies are queued
    s.apply_strain(0.01)
    ring = [torch.empty(64, dtype=torch.uint8, pin_memory=True).numpy() for _ in range(2)]
    for q in range(1100):
        s.step(1)
        s.readback_async(None, ring[q % 2])
    s.readback_wait()
    got = lsm.sample_from_buffer(ring[1099 % 2])
    assert got == s.last_sample()
    assert got["step"] == 1100
