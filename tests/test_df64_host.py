"""Host pins of the double-word arithmetic (lbm_df64.cuh) that the LBM_DF64 policy runs on
the FP32 pipes, and of its D2Q9 weights (lbm_lattice.cuh): tests/df64_host_check.cpp is
compiled with the CUDA rounding intrinsics replaced by their IEEE definitions and checked
against long-double references.  Bounds, with u = 2^-24 (the published bounds of the
algorithms of Joldes, Muller and Popescu, ACM TOMS 2017, with some slack for the
unnormalised products):
  conversion of a double: 2^-48 relative;
  sum: 4u^2 (|x| + |y|) (the sloppy sum is bounded relative to the operands);
  product: 5u^2 relative; product with a float: 3u^2; product then sum: 8u^2 (|xy| + |z|);
  quotient: 16u^2; reciprocal square root (from a 2^-22 first approximation): 16u^2,
  and finite, within 1e-6, for arguments below FP32's normal range;
  the comparison operators agree with the exact values; the nine weights are within 1e-15
  of 4/9, 1/9, 1/36 and sum to exactly 1."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
U2 = 2.0 ** -48


@pytest.fixture(scope="module")
def measured(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("df64") / "df64_host_check")
    subprocess.run([cxx, "-std=c++17", "-O2", "-ffp-contract=off", "-o", exe,
                    os.path.join(HERE, "df64_host_check.cpp")], check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return {k: float(v) for k, v in (line.split() for line in out.splitlines())}


def test_conversion_and_sum(measured):
    assert measured["conv"] <= 2.0 ** -48
    assert measured["add"] <= 4 * U2


def test_products(measured):
    assert measured["mul"] <= 5 * U2
    assert measured["mulf"] <= 3 * U2
    assert measured["chain"] <= 8 * U2


def test_quotient_and_rsqrt(measured):
    assert measured["div"] <= 16 * U2
    assert measured["rsqrt"] <= 16 * U2
    assert measured["nonfinite"] == 0
    assert measured["tiny_rsqrt"] <= 1e-6


def test_comparisons_and_weights(measured):
    assert measured["bad_cmp"] == 0
    assert measured["weight_sum_minus_1"] == 0.0
    assert measured["weight_dev"] <= 1e-15
