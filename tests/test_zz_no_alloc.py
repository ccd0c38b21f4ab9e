"""lsm_spring_energy_static: the entry point that allocates no device memory.

It serves callers that cannot allocate (code running inside another
framework's memory pool or budget, or code that must not trigger the implicit
device-wide synchronisation of cudaFree). Its result must equal what the
allocating path reports through lsm_observe: the potential energy and the
virial sum of the intact springs (the latter read back as sigma_vir * Omega
with all velocities set to zero). Checked on two calls in a row, since every
call shares the library's static scratch array.

This file is collected last on purpose (see the file name).
"""
import ctypes as C

import numpy as np
import pytest

from gen.images import inclusion_image, two_phase_materials

pytestmark = pytest.mark.gpu


def test_static_energy_matches_observe():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_04565_gb300 import build, lsm
    build.build()
    lsm.load_library()

    nx, ny = 48, 40
    img = inclusion_image(nx, ny, 3.0, 6.0, 0.3, 12)
    k_tab, e_tab, m_tab = two_phase_materials()
    g = lsm.Specimen.from_image(img, k_tab, e_tab, m_tab, precision="exact64")
    for i in range(1, 31):  # load past the first breaks
        g.apply_strain(i * 2.5e-3)
        g.step(20)
    x, _ = g.state()
    g.set_state(v=np.zeros_like(x))  # velocities zero: sigma_vir * Omega = virial sum
    ref = g.observe()
    mask, _ = g.broken()
    assert mask.sum() > 0, "the case must include broken springs"
    topo = g.topology()
    omega = (nx - 1) * 1.0 * ny * 1.0

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
        lsm.lsm_spring_energy_static(2, g.n, g.m, ptr(tx), ptr(tsi), ptr(tsj), ptr(tk), ptr(tr0),
                                     ptr(tbr), ptr(out), C.c_void_p(stream.cuda_stream))
        torch.cuda.synchronize()
        results.append(out.cpu().numpy().copy())
    for pe, w in results:
        assert pe == pytest.approx(ref["pe"], rel=1e-12)
        assert w == pytest.approx(ref["sigma_vir"] * omega, rel=1e-12)
    assert np.array_equal(results[0], results[1])

    # sizes beyond the static buffer are refused with a message, before any launch
    with pytest.raises(lsm.LsmError) as ei:
        lsm.lsm_spring_energy_static(2, g.n, 4096 * 65536 + 1, ptr(tx), ptr(tsi), ptr(tsj), ptr(tk),
                                     ptr(tr0), None, ptr(out), None)
    assert ei.value.status == lsm.LSM_EINVAL
    assert "static buffer" in str(ei.value)
    g.close()
