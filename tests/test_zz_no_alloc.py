"""lsm_spring_energy_static: the entry point that allocates no device memory.

It serves callers that cannot allocate (code running inside another
framework's memory pool or budget, or code that must not trigger the implicit
device-wide synchronisation of cudaFree). Its result must equal
  - what the allocating path reports through lsm_observe: the potential
    energy and the virial sum of the intact springs (the latter read back as
    sigma_vir * Omega with all velocities set to zero), and
  - the FP64 oracle's energy U and virial sum W (orc_forces) at the same
    positions and broken set, which shares no code with the library.
Checked on two calls in a row, since every call shares the library's static
scratch array, in 2D and in 3D, each case spanning several 4096-spring
partial chunks.

This file is collected last on purpose (see the file name).
"""
import ctypes as C

import numpy as np
import pytest

from gen.images import foam_volume, inclusion_image, one_phase_materials, two_phase_materials

pytestmark = pytest.mark.gpu


def _case(kind):
    """A specimen loaded past its first breaks: (image, materials, build
    keywords, strain increment, increments)."""
    if kind == "2d":
        return inclusion_image(48, 40, 3.0, 6.0, 0.3, 12), two_phase_materials(), {}, 2.5e-3, 30
    # 3D voxel foam: 3,600 particles, 25,342 springs (7 chunks); exact64 runs
    # the spring-list kernels there
    return foam_volume(20, 2.0, 0.45, seed=9), one_phase_materials(1.0, 0.04), {"grip_mode": 1}, 3e-3, 20


@pytest.mark.parametrize("kind", ["2d", "3d"])
def test_static_energy_matches_observe_and_oracle(oracle_mod, kind):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_04565_gb300 import build, lsm
    build.build()
    lsm.load_library()

    img, (k_tab, e_tab, m_tab), kw, deps, incs = _case(kind)
    dim = img.ndim
    g = lsm.Specimen.from_image(img, k_tab, e_tab, m_tab, precision="exact64", **kw)
    o = oracle_mod.Oracle.from_image(img, k_tab, e_tab, m_tab, **kw)
    for i in range(1, incs + 1):  # load past the first breaks
        g.apply_strain(i * deps)
        g.step(20)
        o.apply_strain(i * deps)
        o.step(20)
    x, _ = g.state()
    g.set_state(v=np.zeros_like(x))  # velocities zero: sigma_vir * Omega = virial sum
    ref = g.observe()
    mask, _ = g.broken()
    assert mask.sum() > 0, "the case must include broken springs"
    # exact64 is bit-identical to the oracle, so both hold the same state
    assert np.array_equal(o.broken()[0], mask) and np.array_equal(o.state()[0], x)
    _, U, W = o.forces(x)
    topo = g.topology()
    assert g.m > 4096, "the case must span several partial chunks"
    omega = (img.shape[-1] - 1) * 1.0
    for s in img.shape[:-1]:
        omega *= s * 1.0

    dev = torch.device("cuda:0")
    tx = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    tsi = torch.from_numpy(topo["si"]).to(dev)
    tsj = torch.from_numpy(topo["sj"]).to(dev)
    tk = torch.from_numpy(topo["k"]).to(dev)
    tr0 = torch.from_numpy(topo["r0"]).to(dev)
    tbr = torch.from_numpy(mask.astype(np.uint8)).to(dev)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def ptr(t):
        return C.c_void_p(t.data_ptr())

    results = []
    for _ in range(2):
        out.fill_(float("nan"))
        lsm.lsm_spring_energy_static(dim, g.n, g.m, ptr(tx), ptr(tsi), ptr(tsj), ptr(tk), ptr(tr0),
                                     ptr(tbr), ptr(out), C.c_void_p(stream.cuda_stream))
        torch.cuda.synchronize()
        results.append(out.cpu().numpy().copy())
    for pe, w in results:
        assert pe == pytest.approx(ref["pe"], rel=1e-12)
        assert w == pytest.approx(ref["sigma_vir"] * omega, rel=1e-12)
        assert pe == pytest.approx(U, rel=1e-12)
        assert w == pytest.approx(W, rel=1e-12)
    assert np.array_equal(results[0], results[1])

    # sizes beyond the static buffer are refused with a message, before any launch
    with pytest.raises(lsm.LsmError) as ei:
        lsm.lsm_spring_energy_static(dim, g.n, 4096 * 65536 + 1, ptr(tx), ptr(tsi), ptr(tsj), ptr(tk),
                                     ptr(tr0), None, ptr(out), None)
    assert ei.value.status == lsm.LSM_EINVAL
    assert "static buffer" in str(ei.value)
    g.close()
