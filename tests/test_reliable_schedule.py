"""Host logic of the mixed-precision solves: the reliable-update schedule
(csrc/reliable.h, compiled here with the host C++ compiler, no GPU).  The
way from the starting residual r0 to the target is split into the fewest
equal reductions no larger than dmax; checked against that definition
written out (k = the smallest integer with dmax^k <= target/r0, reduction
(target/r0)^(1/k)) and against the schedules quoted for the solver."""
import math
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CASES = [
    # r0, target, dmax
    (1.0, 5e-11, 5e-6),     # FP32 at tol 1e-10: one update, at sqrt(5e-11)
    (1.0, 5e-11, 1e-4),     # three segments of 3.7e-4
    (1.0, 5e-11, 0.1),      # FP16 inner steps: eleven segments
    (1.0, 1e-8, 1e-4),      # an exact power: two segments of exactly 1e-4
    (3.0, 2.0, 1e-4),       # less than one segment: the whole way at once
    (661.9, 3.3e-8, 5e-6),  # the chi_L solve at 24^3x64x24
    (1.0, 1.0, 1e-4),       # at the target already: dmax
    (0.0, 1e-8, 1e-4),      # zero residual: dmax
    (1e-12, 1e-8, 1e-4),    # below the target: dmax
]


def _definition(r0, target, dmax):
    if not (r0 > 0 and target > 0 and target < r0):
        return dmax
    ratio = target / r0
    k = 1
    while dmax ** k > ratio * (1 + 1e-12):
        k += 1
    return ratio ** (1.0 / k)


@pytest.fixture(scope="module")
def schedule(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("rel")
    src = d / "sched.cpp"
    body = "\n".join(f'    std::printf("%.17g\\n", equal_segment_reduction({r0!r}, {t!r}, {m!r}));' for r0, t, m in CASES)
    src.write_text('#include <cstdio>\n#include "reliable.h"\nint main() {\n' + body + "\n    return 0;\n}\n")
    exe = d / "sched"
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_1611_00298_gb300", "csrc"), str(src),
                    "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    return [float(v) for v in out]


def test_schedule_matches_its_definition(schedule):
    for (r0, t, m), got in zip(CASES, schedule):
        want = _definition(r0, t, m)
        assert math.isclose(got, want, rel_tol=1e-12), (r0, t, m, got, want)


def test_schedule_properties(schedule):
    for (r0, t, m), got in zip(CASES, schedule):
        assert got >= m * (1 - 1e-12)  # never a larger step than dmax
        if r0 > 0 and 0 < t < r0:
            k = round(math.log(t / r0) / math.log(got))
            assert math.isclose(got ** k, t / r0, rel_tol=1e-9)  # k equal segments reach the target
            assert m ** (k - 1) > t / r0  # and fewer segments of at most dmax would not


def test_quoted_schedules(schedule):
    assert math.isclose(schedule[0], math.sqrt(5e-11), rel_tol=1e-12)
    assert math.isclose(schedule[1], 5e-11 ** (1 / 3), rel_tol=1e-12)
    assert math.isclose(schedule[3], 1e-4, rel_tol=1e-9)
    assert math.isclose(schedule[4], 2.0 / 3.0, rel_tol=1e-12)
    assert schedule[6] == schedule[7] == schedule[8] == 1e-4
