"""Failure detection, with every fault made on the host (no GPU fault, trap or
hang): a non-finite value seeded into the state, a device allocation cap, a
relaxation cap, out-of-range requests. Each must come back as the documented
status and leave the library usable."""
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


def _specimen(L, kind, prec, path=0):
    if kind == "2d":
        img = inclusion_image(40, 32, 3.0, 6.0, 0.3, 7)
        k, e, m = two_phase_materials()
    else:
        img = foam_volume(12, 1.5, 0.6, seed=5)
        k, e, m = one_phase_materials()
    return L.Specimen.from_image(img, k, e, m, precision=prec, path=path)


@pytest.mark.parametrize("kind,prec,path", [("2d", "exact64", 0), ("2d", "df64", 0), ("2d", "fast64", 1),
                                            ("2d", "f32", 1), ("3d", "df64", 0), ("3d", "exact64", 0)])
@pytest.mark.parametrize("where", ["x", "v"])
def test_non_finite_state_is_reported(L, kind, prec, path, where):
    g = _specimen(L, kind, prec, path)
    X = g.state()[0]  # reference positions (nothing has moved yet)
    g.apply_strain(1e-3)
    g.step(4)
    x, v = g.state()
    interior = np.flatnonzero((X[0] > X[0].min()) & (X[0] < X[0].max()))
    p = interior[len(interior) // 2]
    if where == "x":
        x[1, p] = np.nan
    else:
        v[1, p] = np.inf
    g.set_state(x, v)
    g.step(3)
    with pytest.raises(L.LsmError) as ei:
        g.synchronize()
    assert ei.value.status == L.LSM_ENONFINITE
    g.close()
    # the library is still usable: a fresh context steps normally
    h = _specimen(L, kind, prec, path)
    h.apply_strain(1e-3)
    h.step(4)
    h.synchronize()
    assert np.all(np.isfinite(h.state()[0]))
    h.close()


@pytest.mark.parametrize("kind,prec,path", [("2d", "df64", 3), ("2d", "df64", 2), ("2d", "f32", 3),
                                            ("2d", "exact64", 0), ("3d", "df64", 0)])
def test_coincident_particles_are_reported(L, kind, prec, path):
    """Two neighbours moved onto the same point: the spring between them has
    r = 0 and its force is not finite. In the fixed-point modes the force's
    conversion to double makes that a finite value of at least 2^128, so the
    next step's positions leave the fixed-point range; in the FP64 modes the
    velocities become non-finite. Either way the next synchronising call
    returns LSM_ENONFINITE, and the library stays usable."""
    g = _specimen(L, kind, prec, path)
    X = g.state()[0]
    d = X[:, 1:] - X[:, :-1]
    same_line = np.all(d[1:] == 0.0, axis=0)
    cand = np.flatnonzero(same_line & (d[0] > 0) & (X[0, :-1] > X[0].min()) & (X[0, 1:] < X[0].max()))
    p = cand[len(cand) // 2]  # an interior particle whose +x neighbour is the next particle
    x, v = g.state()
    x[:, p] = x[:, p + 1]
    g.set_state(x, v)
    g.step(3)
    with pytest.raises(L.LsmError) as ei:
        g.synchronize()
    assert ei.value.status == L.LSM_ENONFINITE
    g.close()
    h = _specimen(L, kind, prec, path)
    h.step(2)
    h.synchronize()
    assert np.all(np.isfinite(h.state()[0]))
    h.close()


def test_allocation_cap_reports_enomem_without_leaking(L, monkeypatch):
    import torch
    img = inclusion_image(512, 512, 5.0, 20.0, 0.3, 3)
    k, e, m = two_phase_materials()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    monkeypatch.setenv("LSM_MAX_ALLOC_BYTES", str(1 << 20))  # every pixel-grid array is 2-4 MB
    for prec, path in [("df64", 0), ("exact64", 1), ("f32", 1)]:
        for _ in range(5):
            with pytest.raises(L.LsmError) as ei:
                L.Specimen.from_image(img, k, e, m, precision=prec, path=path)
            assert ei.value.status == L.LSM_ENOMEM
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 < (8 << 20)  # the failed builds released what they had allocated
    monkeypatch.delenv("LSM_MAX_ALLOC_BYTES")
    g = L.Specimen.from_image(img, k, e, m, precision="df64")
    g.apply_strain(1e-3)
    g.step(2)
    g.synchronize()
    g.close()


def test_relax_cap_reports_enotconv(L):
    g = _specimen(L, "2d", "df64")
    g.apply_strain(5e-3)
    st, taken = g.relax(1e-14, 40, 10)
    assert st == L.LSM_ENOTCONV and taken == 40
    s = g.samples()[-1]
    assert s["residual"] > 1e-14 and s["step"] == 40
    st, taken = g.relax(1e-3, 100000, 10)  # a reachable tolerance converges afterwards
    assert st == L.LSM_OK and g.samples()[-1]["residual"] <= 1e-3
    g.close()


def test_out_of_range_requests(L):
    g = _specimen(L, "2d", "df64")
    for call in (lambda: g.step(0), lambda: g.step(10 ** 6), lambda: g.apply_strain(float("nan")),
                 lambda: g.apply_strain(-1.0), lambda: g.set_strain_rate(float("inf"))):
        with pytest.raises(L.LsmError) as ei:
            call()
        assert ei.value.status == L.LSM_EINVAL
    g.apply_strain(1e-3)  # nothing above changed the context
    g.step(2)
    g.synchronize()
    assert g.counters()[0] == 2
    g.close()
