"""The integer-pipe binary64 sum and product of the FP64 form (lbm_fp64emu.cuh),
compiled for the host, against the host's own IEEE 754 binary64 arithmetic bit for
bit: tests/fp64emu_check.cpp draws operand families that reach every path of the
routines (random bit patterns with zeros, subnormals, infinities and NaNs; every
exponent distance; cancelling sums; exact ties of the sum and of the product;
products at the edges of the normal range; the lattice's magnitudes; zeros of both
signs, subnormals, infinities and NaNs against normal values and against each other)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2602_21242_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("fp64emu") / "fp64emu_check")
    cmd = [cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-I", CSRC,
           os.path.join(HERE, "fp64emu_check.cpp"), "-o", exe]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    return exe


@pytest.mark.parametrize("seed", [1, 2602])
def test_integer_pipe_arithmetic_matches_ieee(checker, seed):
    res = subprocess.run([checker, "400000", str(seed)], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stdout + res.stderr
    lines = [l for l in res.stdout.splitlines() if l.strip()]
    assert len(lines) == 10 and all(l.endswith("all equal") for l in lines), res.stdout
