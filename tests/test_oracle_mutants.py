"""The oracle's pins catch plausible mistakes: each test below plants one
mistake in a private copy of the oracle's C source (on the CPU), builds it, and
checks that at least one pin of test_oracle_pins fails on it while the real
oracle passes them all.  CPU only.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2209_11287_gb300 import workloads

SRC = os.path.join(os.path.dirname(oracle.__file__), "sj_oracle.c")

MUTANTS = {
    "strict_less": ("if (s <= e2) ++c;", "if (s < e2) ++c;"),
    "dropped_last_dim": ("for (int32_t k = 0; k < d; ++k) {\n        double t = a[k] - b[k];",
                         "for (int32_t k = 0; k < d - 1; ++k) {\n        double t = a[k] - b[k];"),
    "wrong_sign": ("double t = a[k] - b[k];", "double t = a[k] + b[k];"),
    "wrong_index": ("double t = a[k] - b[k];", "double t = a[k] - b[(k + 1) % d];"),
    "single_precision": ("double t = a[k] - b[k];\n        double t2 = t * t;",
                         "float t = (float)(a[k] - b[k]);\n        double t2 = (double)(t * t);"),
    "no_self_pairs": ("if (s <= e2) ++c;", "if (s <= e2 && j != i) ++c;"),
    "eps_not_squared": ("const double e2 = eps * eps;\n    int nt = set_threads(nthreads);\n    int64_t total = 0;\n#pragma omp parallel for schedule(dynamic, 16) reduction",
                        "const double e2 = eps;\n    int nt = set_threads(nthreads);\n    int64_t total = 0;\n#pragma omp parallel for schedule(dynamic, 16) reduction"),
}


def _build_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    src = src.replace(old, new)
    c = tmp_path / f"{name}.c"
    c.write_text(src)
    so = tmp_path / f"{name}.so"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so), str(c), "-lm"],
                   check=True)
    return oracle._configure(ctypes.CDLL(str(so)))


def _pins_pass(lib) -> bool:
    """A compact run of the pins: the hand-enumerated fixture, the dyadic lattice
    against integer arithmetic, and the count on the unit-square closed form."""
    from tests.test_oracle_pins import _read_tiny
    x, cases = _read_tiny()
    for eps, expected in cases.items():
        got = {tuple(int(v) for v in p) for p in oracle.keys_to_pairs(oracle.join(x, eps, lib=lib))}
        if got != expected:
            return False
    g = np.random.Generator(np.random.PCG64(100))
    k = g.integers(0, 40, size=(200, 3))
    xl = k / 64.0
    for r in (5, 9):
        s = ((k[:, None, :] - k[None, :, :]) ** 2).sum(-1)
        want = int((s <= r * r).sum())
        if oracle.join(xl, r / 64.0, lib=lib).size != want:
            return False
    from tests.test_oracle_pins import exact_in, near_tie_points
    xt, eps = near_tie_points(npairs=100)
    keys = set(int(v) for v in oracle.join(xt, eps, lib=lib))
    for p in range(xt.shape[0] // 2):
        i, j = 2 * p, 2 * p + 1
        if (((i << 32) | j) in keys) != exact_in(xt, i, j, eps):
            return False
    return True


def test_real_oracle_passes():
    assert _pins_pass(oracle._load())


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    lib = _build_mutant(tmp_path, name)
    assert not _pins_pass(lib), f"planted mistake {name} was not caught"


def test_row_offset_mutant_is_caught(tmp_path):
    """A mistake in the row function alone (the query row taken at q instead of
    q d) is caught by the lattice row pin, which the real oracle passes."""
    src = open(SRC).read()
    old = "const double* a = x + q * (int64_t)d;"
    assert src.count(old) == 1
    c = tmp_path / "row_offset.c"
    c.write_text(src.replace(old, "const double* a = x + q;"))
    so = tmp_path / "row_offset.so"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so), str(c), "-lm"],
                   check=True)
    lib = oracle._configure(ctypes.CDLL(str(so)))

    def row(x, q):
        x = np.ascontiguousarray(x, dtype=np.float64)
        out = np.empty(x.shape[0], dtype=np.float64)
        lib.sjo_sqdist_row(x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), x.shape[0], x.shape[1], int(q),
                           out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return out

    from tests.test_oracle_pins import lattice_row_ok
    assert lattice_row_ok(oracle.sqdist_row)
    assert not lattice_row_ok(row), "planted mistake in the row function was not caught"
