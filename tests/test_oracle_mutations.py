"""The oracle's pins catch plausible mistakes.

Each case plants one slip in a private copy of the oracle's C source (on the
CPU, never in the repository copy), rebuilds it, and runs every pin of
test_oracle_pins against the mutant: at least one pin must fail.
"""
import importlib.util
import inspect
import os
import shutil
import sys

import pytest

import test_oracle_pins as pins

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = {
    "drop half in half-kick": ("const double dt = o->dt, hdt = 0.5 * o->dt;",
                               "const double dt = o->dt, hdt = o->dt;"),
    "reaction sign on j": ("            o->F[c * n + j] -= f;", "            o->F[c * n + j] += f;"),
    "damping sign": ("o->a[e] = (o->F[e] - o->gamma * vh) / o->mass[p];",
                     "o->a[e] = (o->F[e] + o->gamma * vh) / o->mass[p];"),
    "diagonal rest length": ("const double r0_2 = a * sqrt(2.0);", "const double r0_2 = a * 2.0;"),
    "non-strict break test": ("if (r2 > o->rc2[s]) { /* Heaviside", "if (r2 >= o->rc2[s]) { /* Heaviside"),
    "rc not squared": ("o->rc2[s] = rc * rc;", "o->rc2[s] = rc;"),
    "kinetic virial sign": ("out[1] = (W - mvv) / o->omega;", "out[1] = (W + mvv) / o->omega;"),
    "stretch uses r0 twice": ("double c_s = o->k[s] * (r - o->r0[s]) / r;\n        for (int c = 0; c < dim; c++) {\n            double f = c_s * d[c];\n            o->F",
                              "double c_s = o->k[s] * (r - o->r0[s]) / o->r0[s];\n        for (int c = 0; c < dim; c++) {\n            double f = c_s * d[c];\n            o->F"),
    "energy missing half": ("u += 0.5 * o->k[s] * st * st;", "u += o->k[s] * st * st;"),
    "transposed k table": ("double kk = k_tab[(ph - 1) * nphase + (pq - 1)];",
                           "double kk = k_tab[(pq - 1) * nphase + (ph - 1)] * (ph == pq ? 1.0 : 0.9);"),
    "affine remap sign": ("o->x[p] = o->xc + (o->x[p] - o->xc) * s;", "o->x[p] = o->xc - (o->x[p] - o->xc) * s;"),
    "grip set without eps": ("o->x[p] = o->X[p] + eps_new * (o->X[p] - o->xc);",
                             "o->x[p] = o->X[p] + eps_new * o->X[p];"),
    "field stress missing half": ("double t = 0.5 * (d[pairs[q][0]] * (c_s * d[pairs[q][1]]));",
                                  "double t = d[pairs[q][0]] * (c_s * d[pairs[q][1]]);"),
    "field strain J J^T": ("for (int c = 0; c < dim; c++) t += J[c * 3 + a] * J[c * 3 + b];",
                           "for (int c = 0; c < dim; c++) t += J[a * 3 + c] * J[b * 3 + c];"),
    "field kinetic sign": ("stress[q * n + p] = (stress[q * n + p] - vv) / cell;",
                           "stress[q * n + p] = (stress[q * n + p] + vv) / cell;"),
    "triangular row height": ("const double h = a * sqrt(3.0) * 0.5;", "const double h = a * sqrt(2.0) * 0.5;"),
    "triangular neighbour parity": ("jx = (ix) + ((iy) & 1 ? 0 : -1) + ((t) == 2);",
                                    "jx = (ix) + ((iy) & 1 ? -1 : 0) + ((t) == 2);"),
    "strain-rate step index": ("const double eps = o->rate_eps0 + (double)(o->step + 1 - o->rate_step0) * o->rate_dt;",
                               "const double eps = o->rate_eps0 + (double)(o->step - o->rate_step0) * o->rate_dt;"),
    "dropped z term": ("if (dim == 3) r2 = r2 + d[2] * d[2];\n        double r = sqrt(r2);\n        double c_s",
                       "double r = sqrt(r2);\n        double c_s"),
}


def _mutant(tmp_path, name, old, new):
    dst = tmp_path / ("oracle_" + str(abs(hash(name))))
    shutil.copytree(os.path.join(ROOT, "oracle"), dst,
                    ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    src = dst / "lsm_oracle.c"
    text = src.read_text()
    assert text.count(old) >= 1, name
    src.write_text(text.replace(old, new, 1))
    spec = importlib.util.spec_from_file_location(
        "oracle_mut_%d" % abs(hash(name)), dst / "__init__.py", submodule_search_locations=[str(dst)])
    mod = importlib.util.module_from_spec(spec)
    sys.modules[spec.name] = mod
    spec.loader.exec_module(mod)
    mod.oracle._lib = None
    mod.build_oracle(force=True)
    return mod


def _pin_calls():
    calls = []
    for name, fn in inspect.getmembers(pins, inspect.isfunction):
        if not name.startswith("test_"):
            continue
        marks = getattr(fn, "pytestmark", [])
        params = [m for m in marks if m.name == "parametrize"]
        if params:
            argnames, values = params[0].args
            names = [q.strip() for q in argnames.split(",")]
            for val in values:
                kw = dict(zip(names, val if len(names) > 1 else (val,)))
                calls.append((name, fn, kw))
        else:
            calls.append((name, fn, {}))
    return calls


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(tmp_path, name):
    old, new = MUTATIONS[name]
    mod = _mutant(tmp_path, name, old, new)
    failed = []
    slow = ("relax", "modulus", "poisson", "energy_not_above")
    calls = sorted(_pin_calls(), key=lambda c: any(q in c[0] for q in slow))
    for pin_name, fn, kw in calls:  # cheap pins first; stop at the first catch
        try:
            fn(mod, **kw)
        except Exception:  # an assertion, or the mutant rejecting its input
            failed.append(pin_name)
            break
    assert failed, "no pin caught mutation %r" % name
