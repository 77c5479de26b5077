"""The FP64 sweep's integer forms (csrc/lap_int.cuh) against the FP64 evaluation order they stand in for, on the host:
wherever one of the two Laplacian paths (exact sum, rounded sum) accepts a sextuple, or 2c - prev a pair, its bits
must equal the plain FP64 order (each difference, partial sum and the leapfrog's 2c - prev rounded, no contraction),
over seeded random inputs of many kinds -- smooth, flat, rough, steep tails, exact ties and zeros, sign changes,
neighbours a few ulps apart (rounding ties), differences near the 2^50-unit limit, |prev| near 2|c| and values in
every binade."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("lap") / "lap_int_check")
    subprocess.run([cxx, "-O2", "-ffp-contract=off", "-std=c++17", "-o", exe,
                    os.path.join(HERE, "native", "lap_int_check.cpp")], check=True)
    return exe


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_integer_laplacian_equals_fp64_order(checker, seed):
    out = subprocess.run([checker, "4000000", str(seed)], check=True, capture_output=True, text=True)
    cases, accepted, mismatches = map(int, out.stdout.split())
    assert mismatches == 0, out.stderr
    assert cases == 3 * 4000000  # sextuples through both Laplacian paths, pairs for 2c - prev
    assert accepted > cases // 2  # most inputs take an integer path
