"""LAMMPS data and dump files for interoperability (Section 3.1: the paper's
solver reads particle geometry from a LAMMPS data file in the "bond" atom
style and writes particle coordinates as LAMMPS dump files, for tools such as
OVITO).

Host-side text I/O only:
  read_data(path)            -> dict: ids, mol, types, X [3][n] (or [2][n]),
                                box, masses, bonds (type, i, j) in file order
  network_from_data(d, bond_params, dim)
                             -> arguments of lsm_build_network (springs in
                                canonical order, endpoints as 0-based indices)
  write_data(path, ...)      -> a data file in the same style
  write_dump(path, step, ids, types, x, box, append=True)
                             -> one "ITEM: TIMESTEP" frame (id type x y z)
"""
from __future__ import annotations

import numpy as np


def _sections(lines):
    """Split a data file into its header lines and named sections."""
    names = ("Atoms", "Bonds", "Masses", "Velocities", "Bond Coeffs", "Pair Coeffs", "Angles")
    header, sections, cur = [], {}, None
    for raw in lines:
        line = raw.split("#", 1)[0].strip()
        if not line:
            continue
        word = next((nm for nm in names if line == nm or line.startswith(nm + " ")), None)
        if word is not None:
            cur = word
            sections[cur] = []
            continue
        if cur is None:
            header.append(line)
        else:
            sections[cur].append(line.split())
    return header, sections


def read_data(path):
    with open(path) as f:
        header, sec = _sections(f.readlines())
    box = np.zeros((3, 2))
    for line in header:
        w = line.split()
        for k, ax in (("xlo", 0), ("ylo", 1), ("zlo", 2)):
            if len(w) >= 4 and w[2] == k:
                box[ax] = [float(w[0]), float(w[1])]
    atoms = sec.get("Atoms", [])
    if not atoms:
        raise ValueError("no Atoms section in %s" % path)
    if len(atoms[0]) < 6:
        raise ValueError("Atoms must be in the bond style: id mol type x y z")
    order = np.argsort([int(a[0]) for a in atoms], kind="stable")
    atoms = [atoms[q] for q in order]
    ids = np.array([int(a[0]) for a in atoms], dtype=np.int64)
    mol = np.array([int(a[1]) for a in atoms], dtype=np.int64)
    types = np.array([int(a[2]) for a in atoms], dtype=np.int32)
    X = np.array([[float(a[3]) for a in atoms], [float(a[4]) for a in atoms], [float(a[5]) for a in atoms]])
    masses = {int(r[0]): float(r[1]) for r in sec.get("Masses", [])}
    bonds = np.array([[int(b[1]), int(b[2]), int(b[3])] for b in sec.get("Bonds", [])], dtype=np.int64)
    return dict(ids=ids, mol=mol, types=types, X=X, box=box, masses=masses, bonds=bonds.reshape(-1, 3))


def network_from_data(d, bond_params, dim=2):
    """Spring arrays for lsm_build_network from a data file's atoms and bonds.
    bond_params: {bond type: (k, r0, rc)} (rc = None: unbreakable). Springs
    are returned in canonical order (si < sj, sorted); a bond listed twice is
    an error."""
    index = {int(i): q for q, i in enumerate(d["ids"])}
    rows = []
    for bt, a1, a2 in d["bonds"]:
        i, j = index[int(a1)], index[int(a2)]
        if i == j:
            raise ValueError("bond from atom %d to itself" % a1)
        k, r0, rc = bond_params[int(bt)]
        rows.append((min(i, j), max(i, j), float(k), float(r0), np.inf if rc is None else float(rc) ** 2))
    rows.sort(key=lambda r: (r[0], r[1]))
    for a, b in zip(rows, rows[1:]):
        if (a[0], a[1]) == (b[0], b[1]):
            raise ValueError("atoms %d and %d are bonded twice" % (a[0], a[1]))
    si = np.array([r[0] for r in rows], dtype=np.int32)
    sj = np.array([r[1] for r in rows], dtype=np.int32)
    k = np.array([r[2] for r in rows])
    r0 = np.array([r[3] for r in rows])
    rc2 = np.array([r[4] for r in rows])
    mass = np.array([d["masses"].get(int(t), 1.0) for t in d["types"]])
    return dict(X=np.ascontiguousarray(d["X"][:dim]), si=si, sj=sj, k=k, r0=r0, rc2=rc2, mass=mass)


def write_data(path, X, types, bonds, bond_types=None, masses=None, box=None, title="lattice spring model"):
    """A data file in the bond atom style. X [dim][n]; types [n]; bonds
    (i, j) 0-based pairs; bond_types [m] (default 1)."""
    X = np.asarray(X, dtype=np.float64)
    dim, n = X.shape
    X3 = np.zeros((3, n))
    X3[:dim] = X
    bonds = np.asarray(bonds, dtype=np.int64).reshape(-1, 2)
    bt = np.ones(len(bonds), dtype=np.int64) if bond_types is None else np.asarray(bond_types)
    types = np.asarray(types)
    if box is None:
        lo, hi = X3.min(axis=1) - 0.5, X3.max(axis=1) + 0.5
        box = np.stack([lo, hi], axis=1)
    with open(path, "w") as f:
        f.write("%s\n\n%d atoms\n%d bonds\n%d atom types\n%d bond types\n\n" %
                (title, n, len(bonds), int(types.max()) if n else 0, int(bt.max()) if len(bt) else 0))
        for ax, nm in enumerate("xyz"):
            f.write("%.17g %.17g %slo %shi\n" % (box[ax][0], box[ax][1], nm, nm))
        if masses:
            f.write("\nMasses\n\n")
            for t in sorted(masses):
                f.write("%d %.17g\n" % (t, masses[t]))
        f.write("\nAtoms # bond\n\n")
        for q in range(n):
            f.write("%d 1 %d %.17g %.17g %.17g\n" % (q + 1, types[q], X3[0, q], X3[1, q], X3[2, q]))
        f.write("\nBonds\n\n")
        for q, (i, j) in enumerate(bonds):
            f.write("%d %d %d %d\n" % (q + 1, bt[q], i + 1, j + 1))


def write_dump(path, step, ids, types, x, box, append=True):
    """One dump frame: ITEM: TIMESTEP / NUMBER OF ATOMS / BOX BOUNDS /
    ATOMS id type x y z. x [dim][n]."""
    x = np.asarray(x, dtype=np.float64)
    dim, n = x.shape
    with open(path, "a" if append else "w") as f:
        f.write("ITEM: TIMESTEP\n%d\nITEM: NUMBER OF ATOMS\n%d\nITEM: BOX BOUNDS pp pp pp\n" % (step, n))
        for ax in range(3):
            f.write("%.17g %.17g\n" % (box[ax][0], box[ax][1]))
        f.write("ITEM: ATOMS id type x y z\n")
        for q in range(n):
            z = x[2, q] if dim == 3 else 0.0
            f.write("%d %d %.17g %.17g %.17g\n" % (ids[q], types[q], x[0, q], x[1, q], z))


def read_dump(path):
    """All frames of a dump file: list of (step, ids, types, x [3][n])."""
    frames = []
    with open(path) as f:
        lines = [ln.strip() for ln in f]
    q = 0
    while q < len(lines):
        if lines[q] != "ITEM: TIMESTEP":
            q += 1
            continue
        step = int(lines[q + 1])
        n = int(lines[q + 3])
        rows = [lines[q + 9 + r].split() for r in range(n)]
        ids = np.array([int(r[0]) for r in rows])
        types = np.array([int(r[1]) for r in rows])
        x = np.array([[float(r[c]) for r in rows] for c in (2, 3, 4)])
        frames.append((step, ids, types, x))
        q += 9 + n
    return frames
