"""Pins of the oracle's set comparator, ``oracle.compare_pair_sets``.

Most single-join GPU parity tests decide through it, so it gets pinned on its
own: key sets built by hand that differ by a known pair, on points where the
exact distance of that pair is known to be far from eps or within the 1e-9
band around it (the band of the parity contract: a mismatch is allowed only
for a pair whose exact distance lies within a relative 1e-9 of eps, Sec. II-A,
Eq. 1 being the set that must result).  Planted mistakes in a private copy of
the comparator (arguments swapped, band ignored, band misread, always zero,
set difference in the wrong direction) each fail at least one pin.  CPU only.
"""
import inspect

import numpy as np
import pytest

import oracle


def _key(i, j):
    return (int(i) << 32) | int(j)


def _line(offsets):
    """1-D points at the given coordinates."""
    return np.asarray(offsets, dtype=np.float64).reshape(-1, 1)


EPS = 0.25  # a power of two: eps^2 and every coordinate below are exact


def _cases():
    """(points, eps, ref keys, got keys, expected (only_ref, only_got, bad))."""
    out = []
    # three points: 0 and 1 at distance 0.125 (far inside), 2 far outside
    x = _line([0.0, 0.125, 10.0])
    full = np.array(sorted([_key(0, 0), _key(0, 1), _key(1, 0), _key(1, 1), _key(2, 2)]), dtype=np.int64)
    # identical sets
    out.append(("identical", x, EPS, full, full.copy(), (0, 0, 0)))
    # a pair far inside eps missing from got: a real mismatch
    got = full[full != _key(0, 1)]
    out.append(("missing_inside", x, EPS, full, got, (1, 0, 1)))
    # a pair far outside eps present in got only: a real mismatch
    got = np.sort(np.append(full, _key(0, 2)))
    out.append(("extra_outside", x, EPS, full, got, (0, 1, 1)))
    # a self pair (distance 0) missing: a real mismatch
    got = full[full != _key(2, 2)]
    out.append(("missing_self", x, EPS, full, got, (1, 0, 1)))
    # a borderline pair: distance eps (1 + 1e-10), inside the 1e-9 band, so
    # either answer is allowed
    xb = _line([0.0, EPS * (1.0 + 1e-10)])
    ref_b = np.array([_key(0, 0), _key(1, 1)], dtype=np.int64)
    got_b = np.array([_key(0, 0), _key(0, 1), _key(1, 1)], dtype=np.int64)
    out.append(("borderline_extra", xb, EPS, ref_b, got_b, (0, 1, 0)))
    out.append(("borderline_missing", xb, EPS, got_b, ref_b, (1, 0, 0)))
    # just outside the band: distance eps (1 + 1e-7) is a real mismatch
    xo = _line([0.0, EPS * (1.0 + 1e-7)])
    out.append(("outside_band", xo, EPS, ref_b, got_b, (0, 1, 1)))
    # inside eps by 1e-7 relative: also outside the band
    xi = _line([0.0, EPS * (1.0 - 1e-7)])
    out.append(("inside_band_edge", xi, EPS, got_b, ref_b, (1, 0, 1)))
    # several mismatches at once, one of them borderline: counts add up
    xm = _line([0.0, 0.125, 10.0, 10.0 + EPS * (1.0 - 1e-11)])
    ref_m = np.array(sorted([_key(0, 0), _key(0, 1), _key(1, 0), _key(1, 1), _key(2, 2), _key(3, 3),
                             _key(2, 3), _key(3, 2)]), dtype=np.int64)
    got_m = np.array(sorted([_key(0, 0), _key(0, 1), _key(1, 1), _key(2, 2), _key(3, 3), _key(2, 3),
                             _key(0, 3)]), dtype=np.int64)
    # only in ref: (1,0) real, (3,2) borderline; only in got: (0,3) real
    out.append(("mixed", xm, EPS, ref_m, got_m, (2, 1, 2)))
    return out


def _pins_pass(compare) -> bool:
    for name, x, eps, ref, got, want in _cases():
        if tuple(compare(x, eps, ref, got)) != want:
            return False
    return True


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_comparator_case(case):
    name, x, eps, ref, got, want = case
    assert oracle.compare_pair_sets(x, eps, ref, got) == want, name


def test_band_rel_is_honoured():
    """A pair at eps (1 + 1e-7) is borderline under a 1e-6 band, not under 1e-9."""
    x = _line([0.0, EPS * (1.0 + 1e-7)])
    ref = np.array([_key(0, 0), _key(1, 1)], dtype=np.int64)
    got = np.array([_key(0, 0), _key(0, 1), _key(1, 1)], dtype=np.int64)
    assert oracle.compare_pair_sets(x, EPS, ref, got, rel=1e-6) == (0, 1, 0)
    assert oracle.compare_pair_sets(x, EPS, ref, got, rel=1e-9) == (0, 1, 1)


def test_borderline_points_are_what_the_cases_claim():
    """The fixtures' distances, checked in exact rational arithmetic."""
    from fractions import Fraction
    for off, rel_border in ((EPS * (1.0 + 1e-10), True), (EPS * (1.0 + 1e-7), False),
                            (EPS * (1.0 - 1e-7), False), (EPS * (1.0 - 1e-11), True)):
        r = Fraction(off) / Fraction(EPS)
        lo, hi = Fraction(1) - Fraction(1, 10**9), Fraction(1) + Fraction(1, 10**9)
        assert (lo <= r <= hi) == rel_border, off


# ---- planted mistakes in a private copy of the comparator -------------------

MUTANTS = {
    "arguments_swapped": ("only_ref = np.setdiff1d(ref, got, assume_unique=False)\n"
                          "    only_got = np.setdiff1d(got, ref, assume_unique=False)",
                          "only_ref = np.setdiff1d(got, ref, assume_unique=False)\n"
                          "    only_got = np.setdiff1d(ref, got, assume_unique=False)"),
    "band_ignored": ("if not is_borderline(x, int(k) >> 32, int(k) & 0xFFFFFFFF, eps, rel):",
                     "if False:"),
    "everything_bad": ("if not is_borderline(x, int(k) >> 32, int(k) & 0xFFFFFFFF, eps, rel):",
                       "if True:"),
    "wide_band": ("if not is_borderline(x, int(k) >> 32, int(k) & 0xFFFFFFFF, eps, rel):",
                  "if not is_borderline(x, int(k) >> 32, int(k) & 0xFFFFFFFF, eps, 1e-3):"),
    "transposed_key": ("if not is_borderline(x, int(k) >> 32, int(k) & 0xFFFFFFFF, eps, rel):",
                       "if not is_borderline(x, int(k) & 0xFFFFFFFF, int(k) & 0xFFFFFFFF, eps, rel):"),
    "one_side_only": ("for k in np.concatenate([only_ref, only_got]):", "for k in only_ref:"),
    "always_zero": ("return int(only_ref.size), int(only_got.size), bad", "return 0, 0, 0"),
}


def _mutant(name):
    old, new = MUTANTS[name]
    src = inspect.getsource(oracle.compare_pair_sets)
    assert src.count(old) == 1, name
    ns = dict(vars(oracle))
    exec(compile(src.replace(old, new), f"<mutant {name}>", "exec"), ns)
    return ns["compare_pair_sets"]


def test_real_comparator_passes():
    assert _pins_pass(oracle.compare_pair_sets)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_comparator_mutant_is_caught(name):
    assert not _pins_pass(_mutant(name)), f"planted mistake {name} was not caught"
