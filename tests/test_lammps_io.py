"""LAMMPS data / dump interop (the paper's solver reads bond-style data files
and writes dump files): a lattice written as a data file and read back gives
the same network, and a network build from it runs the same dynamics as the
image build in the oracle, bit for bit."""
import numpy as np
import pytest

from gen.images import inclusion_image, two_phase_materials
from paper_2201_04565_gb300 import lammps_io as lio


def _bond_classes(t):
    """One bond type per distinct (k, r0, rc2) triple."""
    keys = sorted(set(zip(t["k"].tolist(), t["r0"].tolist(), t["rc2"].tolist())))
    idx = {kk: q + 1 for q, kk in enumerate(keys)}
    types = np.array([idx[kk] for kk in zip(t["k"].tolist(), t["r0"].tolist(), t["rc2"].tolist())])
    params = {idx[kk]: (kk[0], kk[1], float(np.sqrt(kk[2]))) for kk in keys}
    return types, params


def test_data_round_trip_and_dynamics(oracle_mod, tmp_path):
    img = inclusion_image(14, 11, 1.5, 3.0, 0.3, 7)
    img[4, 3:7] = 0
    k, e, m = two_phase_materials()
    o = oracle_mod.Oracle.from_image(img, k, e, m)
    t = o.topology()
    btypes, params = _bond_classes(t)
    path = tmp_path / "lattice.data"
    # write the bonds in a shuffled order and reversed direction: the reader
    # restores the canonical order
    rng = np.random.default_rng(0)
    perm = rng.permutation(o.m)
    bonds = np.stack([t["sj"], t["si"]], axis=1)[perm]
    lio.write_data(path, t["X"], np.ones(o.n, dtype=np.int64), bonds, bond_types=btypes[perm], masses={1: 1.0})
    d = lio.read_data(path)
    net = lio.network_from_data(d, params, dim=2)
    assert np.array_equal(net["si"], t["si"]) and np.array_equal(net["sj"], t["sj"])
    assert np.array_equal(net["X"], t["X"])
    assert np.array_equal(net["k"], t["k"]) and np.array_equal(net["r0"], t["r0"])
    assert np.allclose(net["rc2"], t["rc2"], rtol=1e-15, atol=0)
    ny, nx = img.shape
    o2 = oracle_mod.Oracle.from_network(net["X"], net["si"], net["sj"], net["k"], net["r0"], t["rc2"],
                                        mass=net["mass"], fix=t["fix"], grip=t["grip"], dt=0.01, damping=0.1,
                                        xc=0.5 * (nx - 1), omega=(nx - 1) * ny, grip_area=ny)
    for i in range(1, 6):
        o.apply_strain(i * 1e-2)
        o2.apply_strain(i * 1e-2)
        o.step(20)
        o2.step(20)
    x1, v1, _ = o.state()
    x2, v2, _ = o2.state()
    assert np.array_equal(x1, x2) and np.array_equal(v1, v2)
    assert np.array_equal(o.broken()[0], o2.broken()[0])


def test_dump_round_trip(tmp_path):
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 9))
    ids, types = np.arange(1, 10), np.ones(9, dtype=int)
    box = np.array([[-5.0, 5.0], [-5.0, 5.0], [-0.5, 0.5]])
    path = tmp_path / "run.dump"
    lio.write_dump(path, 0, ids, types, x, box, append=False)
    lio.write_dump(path, 20, ids, types, 2 * x, box)
    fr = lio.read_dump(path)
    assert [f[0] for f in fr] == [0, 20]
    assert np.array_equal(fr[1][3][:2], 2 * x) and np.all(fr[1][3][2] == 0.0)
    assert np.array_equal(fr[0][1], ids)


def test_reader_rejects_bad_files(tmp_path):
    p = tmp_path / "bad.data"
    p.write_text("title\n\n2 atoms\n\nAtoms\n\n1 1 0.0 0.0\n2 1 1.0 0.0\n")
    with pytest.raises(ValueError):
        lio.read_data(p)
    p.write_text("title\n\n2 atoms\n1 bonds\n\nAtoms\n\n1 1 1 0 0 0\n2 1 1 1 0 0\n\nBonds\n\n1 1 1 1\n")
    with pytest.raises(ValueError):
        lio.network_from_data(lio.read_data(p), {1: (1.0, 1.0, None)})
