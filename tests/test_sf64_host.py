"""The integer-pipe float64 routines (csrc/sf64.cuh) compiled for the host
and checked against the host's IEEE arithmetic: division and square root
(and multiply, add, subtract, the comparisons and the integer-to-unit
conversion of RANDOM) must be bit-identical (correctly rounded), exp and
log within 1 ulp of a
long-double reference, over millions of operands including near-1 ratios,
exact quotients, perfect squares and the whole exponent range (operands
outside the fast path take the native operation). The single-precision
seeds are perturbed by up to 2 ulp, so the Newton steps are exercised with a
seed no better than the hardware's."""
import os
import subprocess

import pytest

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sf64")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("sf64") / "check")
    r = subprocess.run(["g++", "-O2", "-std=c++17", os.path.join(HERE, "check.cpp"), "-o", exe],
                       stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    assert r.returncode == 0, r.stdout.decode()
    return exe


@pytest.mark.parametrize("op,n", [("div", 2_000_000), ("sqrt", 2_000_000), ("exp", 1_000_000), ("log", 1_000_000),
                                  ("mul", 2_000_000), ("mulk", 2_000_000), ("add", 2_000_000), ("sub", 2_000_000), ("cmp", 500_000),
                                  ("u53", 500_000)])
def test_sf64_against_host_ieee(checker, op, n):
    for seed in (1, 2):
        r = subprocess.run([checker, op, str(n), str(seed)], stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        out = r.stdout.decode()
        assert r.returncode == 0, out
        assert "mismatches=0" in out, out
