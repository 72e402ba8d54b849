"""Host logic of the exact reciprocals the general kernels and the diagnostics
use in place of a division by the cell size.  x / d and x * (1/d) give the same
bits only when 1/d is exact (d a power of two) and neither d nor 1/d, nor d^2
and its reciprocal, leaves the normal range; otherwise the view must hold 0 so
that the kernels divide.  Compiled here with the host compiler against the
library's own header."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"

SRC = r"""
#include <cmath>
#include <cstdio>
#include <cstring>
#include "axp_internal.h"
using namespace axp;
template <typename T> void show(const char *tag, T d) {
    View<T> v;
    std::memset(&v, 0, sizeof(v));
    for (int a = 0; a < 3; a++) v.d[a] = d;
    set_reciprocals(v);
    std::printf("%s %a %a %a\n", tag, (double)v.rd[1], (double)v.rd2[1], (double)v.rdd[1]);
}
int main() {
    show<double>("d32", 1.0 / 32);
    show<double>("d05", 0.05);
    show<double>("d4", 4.0);
    show<double>("dtiny", std::ldexp(1.0, -540));
    show<double>("dzero", 0.0);
    show<float>("f16", 1.0f / 16);
    show<float>("f07", 0.07f);
    show<float>("ftiny", std::ldexp(1.0f, -70));
    return 0;
}
"""


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("recip")
    src, exe = d / "t.cpp", d / "t"
    src.write_text(SRC)
    subprocess.run([cxx, "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I",
                    os.path.join(ROOT, "paper_2406_16796_gb300", "csrc"), "-I", CUDA_INC, str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {line.split()[0]: [float.fromhex(x) for x in line.split()[1:]] for line in out.splitlines()}


def test_power_of_two_cell_sizes_get_exact_reciprocals(results):
    assert results["d32"] == [32.0, 16.0, 1024.0]
    assert results["d4"] == [0.25, 0.125, 0.0625]
    assert results["f16"] == [16.0, 8.0, 256.0]


def test_other_cell_sizes_keep_the_division(results):
    assert results["d05"] == [0.0, 0.0, 0.0]
    assert results["f07"] == [0.0, 0.0, 0.0]
    assert results["dzero"] == [0.0, 0.0, 0.0]


def test_a_square_below_the_normal_range_keeps_its_division(results):
    # 2^-540 squared is 2^-1080, below FP64's normal range; 2^-70 squared is
    # below FP32's: the reciprocals of d and 2d stay exact, that of d^2 is dropped
    assert results["dtiny"] == [2.0 ** 540, 2.0 ** 539, 0.0]
    assert results["ftiny"] == [2.0 ** 70, 2.0 ** 69, 0.0]
