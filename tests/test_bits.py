"""The integer-pipe FP64 <-> FP32 conversions of the mixed-precision Gram-Schmidt sweeps
(csrc/dg_bits.cuh), compiled for the host and checked on the CPU against IEEE-754 semantics:
truncation toward zero within 2^-23, exact round trips of FP32 values, flush of magnitudes under
2^-126, overflow to Inf, and Inf / NaN (whatever the NaN payload) carried through."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2306_01085_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <cstdint>
#include <cstring>
#include "dg_bits.cuh"
int main() {
  uint64_t b;
  while (scanf("%llx", (unsigned long long*)&b) == 1) {
    double d; memcpy(&d, &b, 8);
    float f = dg::to_f32(d);
    uint32_t fb; memcpy(&fb, &f, 4);
    double back = dg::to_f64(f);
    uint64_t bb; memcpy(&bb, &back, 8);
    printf("%08x %016llx\n", fb, (unsigned long long)bb);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def conv(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if not cxx or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("needs a host C++ compiler and the CUDA headers")
    d = tmp_path_factory.mktemp("bits")
    src, exe = d / "bits.cpp", d / "bits"
    src.write_text(PROGRAM)
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", CSRC, "-I", cuda_inc, str(src), "-o", str(exe)], check=True,
                   capture_output=True)

    def run(values):
        bits = np.asarray(values, dtype=np.float64).view(np.uint64)
        return run_bits(bits)

    def run_bits(bits):
        inp = "\n".join(f"{int(x):x}" for x in bits) + "\n"
        out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout.split()
        f = np.array([int(x, 16) for x in out[0::2]], dtype=np.uint32).view(np.float32)
        back = np.array([int(x, 16) for x in out[1::2]], dtype=np.uint64).view(np.float64)
        return f, back

    run.bits = run_bits
    return run


def test_truncates_toward_zero_within_2_pow_minus_23(conv):
    rng = np.random.default_rng(5)
    x = rng.standard_normal(4000) * np.exp(rng.uniform(-80, 80, 4000))
    f, _ = conv(x)
    f = f.astype(np.float64)
    assert np.all(np.sign(f) == np.sign(x))
    assert np.all(np.abs(f) <= np.abs(x))
    assert np.all(np.abs(f - x) <= 2.0 ** -23 * np.abs(x))


def test_fp32_values_round_trip_exactly(conv):
    rng = np.random.default_rng(6)
    x32 = (rng.standard_normal(2000) * np.exp(rng.uniform(-80, 80, 2000))).astype(np.float32)
    f, back = conv(x32.astype(np.float64))
    assert np.array_equal(f, x32)
    assert np.array_equal(back, x32.astype(np.float64))


def test_range_ends(conv):
    big = float(np.finfo(np.float32).max)
    tiny = float(np.finfo(np.float32).tiny)          # 2^-126
    x = np.array([big, -big, 2.0 ** 128, -2.0 ** 200, 1e300, tiny, tiny / 2, -1e-300, 0.0, -0.0])
    f, _ = conv(x)
    assert f[0] == np.float32(big) and f[1] == -np.float32(big)
    assert np.isposinf(f[2]) and np.isneginf(f[3]) and np.isposinf(f[4])
    assert f[5] == np.float32(tiny)
    assert f[6] == 0.0 and f[7] == 0.0
    assert np.signbit(f[9]) and not np.signbit(f[8])


def test_inf_and_nan_are_carried(conv):
    payload_low = np.uint64(0x7FF0000000000001)      # NaN whose payload sits below the kept bits
    neg_nan = np.uint64(0xFFF8000000000000)
    bits = np.array([np.float64(np.inf).view(np.uint64), np.float64(-np.inf).view(np.uint64), payload_low,
                     neg_nan, np.float64(np.nan).view(np.uint64)], dtype=np.uint64)
    f, back = conv.bits(bits)
    assert np.isposinf(f[0]) and np.isneginf(f[1])
    assert np.all(np.isnan(f[2:]))
    assert np.isposinf(back[0]) and np.isneginf(back[1]) and np.all(np.isnan(back[2:]))
