"""Checkpoint and resume through the C ABI (lsm_save / lsm_load): a context
saved after fracture has started and reloaded continues bit for bit like the
original, on every kernel path (2D tile kernel, spring-list kernels, 3D voxel
tile kernel, triangular packing, general networks, constant strain-rate
loading)."""
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


def _build(L, case):
    if case["kind"] == "2d":
        img = inclusion_image(48, 40, 3.0, 6.0, 0.3, 11)
        k, e, m = two_phase_materials()
        return L.Specimen.from_image(img, k, e, m, precision=case["prec"], path=case.get("path", 0),
                                     lattice=case.get("lattice", 0))
    if case["kind"] == "3d":
        img = foam_volume(14, 1.5, 0.6, seed=21)
        k, e, m = one_phase_materials(1.0, 0.02)
        return L.Specimen.from_image(img, k, e, m, precision=case["prec"], path=case.get("path", 0))
    # a general network: a jittered square lattice with first and second
    # neighbours, gripped on its first and last columns
    rng = np.random.default_rng(4)
    nx, ny = 12, 9
    X = np.array([[i + 0.05 * rng.standard_normal() for j in range(ny) for i in range(nx)],
                  [j + 0.05 * rng.standard_normal() for j in range(ny) for i in range(nx)]])
    si, sj = [], []
    for j in range(ny):
        for i in range(nx):
            p = j * nx + i
            for di, dj in ((1, 0), (0, 1), (1, 1), (-1, 1)):
                a, b = i + di, j + dj
                if 0 <= a < nx and b < ny:
                    si.append(p)
                    sj.append(b * nx + a)
    si, sj = np.array(si, np.int32), np.array(sj, np.int32)
    order = np.lexsort((np.maximum(si, sj), np.minimum(si, sj)))
    si, sj = np.minimum(si, sj)[order].astype(np.int32), np.maximum(si, sj)[order].astype(np.int32)
    d = X[:, sj] - X[:, si]
    r0 = np.sqrt((d ** 2).sum(0))
    col = np.array([i for j in range(ny) for i in range(nx)])
    grip = np.where(col == 0, 1, np.where(col == nx - 1, 2, 0)).astype(np.uint8)
    fix = np.zeros((2, nx * ny), np.uint8)
    fix[0, grip > 0] = 1  # the load axis of both grips is prescribed
    return L.Specimen.from_network(X, si, sj, np.ones(len(si)), r0, (r0 * 1.03) ** 2, fix=fix, grip=grip,
                                   damping=0.1, xc=0.5 * (nx - 1), omega=float((nx - 1) * ny),
                                   grip_area=float(ny), precision=case["prec"])


CASES = [
    dict(kind="2d", prec="exact64"),
    dict(kind="2d", prec="df64"),
    dict(kind="2d", prec="f32", path=1),
    dict(kind="2d", prec="fast64", lattice=1),
    dict(kind="2d", prec="df64", lattice=1),
    dict(kind="2d", prec="f32", lattice=1, rate=0.05),
    dict(kind="3d", prec="df64"),
    dict(kind="3d", prec="exact64"),
    dict(kind="net", prec="exact64"),
    dict(kind="2d", prec="df64", rate=0.05),
]


def _drive(g, case, incs, first):
    for i in range(first, first + incs):
        if not case.get("rate"):
            g.apply_strain(i * 7e-3)
        g.step(15)


def _snapshot(g):
    x, v = g.state()
    mask, first = g.broken()
    return dict(x=x, v=v, mask=mask, first=first, brk=g.break_steps(), samples=g.samples(),
                counters=g.counters()[:2])


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(str(v) for v in c.values()))
def test_resume_is_bit_identical(L, tmp_path, case):
    a = _build(L, case)
    if case.get("rate"):
        a.apply_strain(0.01)
        a.set_strain_rate(case["rate"])
    _drive(a, case, 8, 1)
    if case["kind"] != "net":
        assert a.broken()[1] >= 0  # saved after fracture has started
    ck = tmp_path / "ctx.lsmckpt"
    a.save(str(ck))
    _drive(a, case, 6, 9)
    ref = _snapshot(a)
    a.close()

    b = L.Specimen.load(str(ck))
    _drive(b, case, 6, 9)
    got = _snapshot(b)
    b.close()
    assert np.array_equal(got["x"], ref["x"]) and np.array_equal(got["v"], ref["v"])
    assert np.array_equal(got["mask"], ref["mask"]) and got["first"] == ref["first"]
    assert np.array_equal(got["brk"], ref["brk"])
    assert got["counters"] == ref["counters"]
    assert len(got["samples"]) == len(ref["samples"]) == 14
    for p, q in zip(got["samples"], ref["samples"]):
        assert p == q


def test_corrupt_checkpoint_is_rejected(L, tmp_path):
    img = inclusion_image(20, 16, 2.0, 4.0, 0.3, 2)
    k, e, m = two_phase_materials()
    g = L.Specimen.from_image(img, k, e, m, precision="df64")
    g.apply_strain(0.01)
    g.step(5)
    ck = tmp_path / "ok.lsmckpt"
    g.save(str(ck))
    g.close()
    raw = bytearray(ck.read_bytes())
    raw[len(raw) // 2] ^= 0x40  # one flipped bit in the state
    bad = tmp_path / "bad.lsmckpt"
    bad.write_bytes(bytes(raw))
    with pytest.raises(L.LsmError) as ei:
        L.Specimen.load(str(bad))
    assert ei.value.status == L.LSM_EINVAL and "checksum" in str(ei.value)
    short = tmp_path / "short.lsmckpt"
    short.write_bytes(bytes(raw[: len(raw) - 100]))
    with pytest.raises(L.LsmError) as ei:
        L.Specimen.load(str(short))
    assert ei.value.status == L.LSM_EINVAL
