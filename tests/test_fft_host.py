"""The device FFT core (csrc/sfac_fft.cuh) compiled for the host and run by one
host thread per GPU thread, meeting at a barrier wherever the CTA synchronises
(tests/host_fft/check_fft.cpp). Every line length 4..4096 of the FP64 passes,
forward and inverse, with complex twiddles and with the ratio twiddles of the
FP64 plan passes (radix 8/4/2, radix 16 at 4096), and the FP32 radix-16
structure of lengths 32..4096 on the packed two-lane FP32 forms the kernels use (emulated lane by
lane), against a long-double DFT.

Bound: the error of a radix-2-based FFT grows like log2 N roundings, so the
max error relative to the largest exact value must stay below 4 log2(N) u
with u = 2^-53 (FP64) or 2^-24 (FP32). The ratio-twiddle table is followed by
poison values: a record read past its end would break the bound."""
import math
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2209_08437_gb300", "csrc")
HERE = os.path.join(ROOT, "tests", "host_fft")


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("fft") / "check_fft")
    cmd = [cxx, "-std=c++20", "-O2", "-ffp-contract=off", "-I", os.path.join(HERE, "shim"), "-I", CSRC,
           "-I", os.path.join(ROOT, "include"),
           "-x", "c++", os.path.join(CSRC, "sfac_host.cu"), os.path.join(HERE, "check_fft.cpp"),
           "-o", exe, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and ("barrier" in r.stderr and "No such file" in r.stderr):
        pytest.skip("host C++ library without <barrier>")
    assert r.returncode == 0, r.stderr[-4000:]
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    rows = []
    for line in out.stdout.splitlines():
        kind, n, e, inv, err = line.split()
        rows.append((kind, int(n), int(e), int(inv), float(err)))
    return rows


def test_every_length_and_direction_is_covered(results):
    kinds = {(k, n, inv) for k, n, _, inv, _ in results}
    for n in (4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096):
        for inv in (0, 1):
            assert ("complex64b", n, inv) in kinds
            assert ("ratio64", n, inv) in kinds
            if n >= 32:
                assert ("complex32b", n, inv) in kinds


def test_twiddle_rows_equal_the_table_bit_for_bit(results):
    """The FP32 passes read their twiddles from per-thread rows (TwRows); the
    rows hold the table's values, so every line equals the table-indexed FFT
    exactly, for every FP32 shape (16, 8, 4 and 2 values per thread)."""
    same = [(n, e, inv, v) for k, n, e, inv, v in results if k == "rows32same"]
    shapes = {(n, e) for n, e, _, _ in same}
    assert {(256, 16), (512, 16), (128, 8), (64, 2), (32, 16)} <= shapes
    assert all(v == 1 for *_, v in same), [s for s in same if s[3] != 1]


def test_errors_within_the_rounding_bound(results):
    for kind, n, e, inv, err in results:
        if kind == "rows32same":
            continue
        u = 2.0 ** -24 if kind == "complex32b" else 2.0 ** -53
        bound = 4 * max(1, math.log2(n)) * u
        print(f"{kind:10s} N={n:5d} E={e:2d} inv={inv} err={err:.2e} bound={bound:.1e}")
        assert err <= bound, (kind, n, inv, err, bound)


def test_ratio_twiddles_no_less_accurate_than_complex(results):
    by = {(k, n, inv): err for k, n, _, inv, err in results}
    for (k, n, inv), err in by.items():
        if k == "ratio64":
            assert err <= 2 * by[("complex64b", n, inv)] + 2.0 ** -53, (n, inv)
