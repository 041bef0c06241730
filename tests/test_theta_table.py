"""The truncated-Taylor admissible norms theta_m used by the exponential action
(Section 2 `expmvtay2`, which follows Al-Mohy & Higham, "Computing the action of
the matrix exponential", SIAM J. Sci. Comput. 33 (2011)) against the values that
paper prints in its Table 3.1 to two significant digits, for the unit roundoffs
u = 2^-53 and u = 2^-24 at m = 5, 10, ..., 55.

The CUDA library's table (`theta_tables.h`, double row at 2^-53, float row at the
chosen 2^-20) is generated by `gen_theta.py` from the backward-error series; the
double row is compared with the published row directly, the generator with the
published single-precision row, and the header's rows with the generator."""
import os
import re
import sys

import mpmath as mp
import pytest

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2207_09776_b300", "csrc")
sys.path.insert(0, CSRC)
import gen_theta  # noqa: E402

MS = list(range(5, 60, 5))
# Al-Mohy & Higham (2011), Table 3.1: theta_m for m = 5, 10, ..., 55
PUBLISHED = {
    53: [2.4e-3, 1.4e-1, 6.4e-1, 1.4e0, 2.4e0, 3.5e0, 4.7e0, 6.0e0, 7.2e0, 8.5e0, 9.9e0],
    24: [1.3e-1, 1.0e0, 2.2e0, 3.6e0, 4.9e0, 6.3e0, 7.7e0, 9.1e0, 1.1e1, 1.2e1, 1.3e1],
}


def _header_rows():
    src = open(os.path.join(CSRC, "theta_tables.h")).read()
    rows = {}
    for name in ("msk_theta_f64", "msk_theta_f32"):
        body = re.search(name + r"\[[^\]]*\] = \{([^}]*)\}", src).group(1)
        rows[name] = [float(x) for x in body.split(",") if x.strip()]
    return rows


def _agrees_to_two_digits(value, printed):
    """|value - printed| within half a unit of the printed second digit (plus 1 %
    of that unit, for values that sit on a rounding boundary)."""
    unit = 10.0 ** (mp.floor(mp.log10(printed)) - 1)
    return abs(value - printed) <= 0.51 * float(unit)


def test_double_row_of_the_header_is_the_published_one():
    f64 = _header_rows()["msk_theta_f64"]
    for m, want in zip(MS, PUBLISHED[53]):
        assert _agrees_to_two_digits(f64[m - 1], want), (m, f64[m - 1], want)


def test_generator_reproduces_the_published_single_precision_row():
    for m, want in zip(MS, PUBLISHED[24]):
        got = float(gen_theta.theta(m, mp.mpf(2) ** -24))
        assert _agrees_to_two_digits(got, want), (m, got, want)


@pytest.mark.parametrize("name,exp", [("msk_theta_f64", gen_theta.TOL64_EXP), ("msk_theta_f32", gen_theta.TOL32_EXP)])
def test_header_rows_are_the_generator_output(name, exp):
    row = _header_rows()[name]
    for m in (1, 2, 7, 30, len(row)):
        got = float(gen_theta.theta(m, mp.mpf(2) ** -exp))
        assert row[m - 1] == pytest.approx(got, rel=1e-15), (name, m)


def test_theta_increases_with_the_degree_and_the_tolerance():
    rows = _header_rows()
    for name in rows:
        r = rows[name]
        assert all(b > a for a, b in zip(r, r[1:])), name
    f64, f32 = rows["msk_theta_f64"], rows["msk_theta_f32"]
    assert all(b > a for a, b in zip(f64, f32))      # looser tolerance, larger admissible norm
