"""Host-side preparation of the launch parameters (no GPU): fill_coef_sets in
csrc/gadi_params.h derives the FP32/FP64 coefficient sets the kernels read and
the exponent k with which the FP64 residual forms a_d x as an exponent shift
when A's centre coefficient a_d is 2^k.  Compiled here with the host C++
compiler (the header is plain C++)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2512_21164_gb300", "csrc")

PROG = r"""
#include <cstddef>
#include <cstdint>
#include "gadi_params.h"
#include <cstdio>
#include <cstdlib>
using namespace gadi;
int main(int argc, char **argv)
{
    // argv: a_d, then 7 values for H (d, c0..c5), S (d, c0..c5, e): printed back
    Params P{};
    P.co.a_d = std::strtod(argv[1], nullptr);
    P.co.h_d = std::strtod(argv[2], nullptr);
    for (int k = 0; k < 6; k++) P.co.h_c[k] = std::strtod(argv[3 + k], nullptr);
    P.co.s_d = std::strtod(argv[9], nullptr);
    for (int k = 0; k < 6; k++) P.co.s_c[k] = std::strtod(argv[10 + k], nullptr);
    P.co.s_e = std::strtod(argv[16], nullptr);
    P.co.t_d = P.co.s_d;
    for (int k = 0; k < 6; k++) P.co.t_c[k] = -P.co.s_c[k];
    P.co.t_e = -P.co.s_e;
    fill_coef_sets(P);
    std::printf("%d\n", P.ad_pow2 == kNoPow2 ? 9999 : P.ad_pow2);
    const Coef7<float> *f[3] = {&P.hf, &P.sf, &P.tf};
    const Coef7<double> *d[3] = {&P.hd, &P.sd, &P.td};
    for (int i = 0; i < 3; i++) {
        std::printf("%a %a", (double)f[i]->d, d[i]->d);
        for (int k = 0; k < 6; k++) std::printf(" %a %a", (double)f[i]->c[k], d[i]->c[k]);
        std::printf(" %a %a\n", (double)f[i]->e, d[i]->e);
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("params")
    src, exe = d / "p.cpp", d / "p"
    src.write_text(PROG)
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return str(exe)


def _run(exe, a_d, h=None, s=None):
    h = h if h is not None else [4.5] + [-1.0] * 6
    s = s if s is not None else [0.5] + [0.25, -0.25, 0.125, -0.125, 0.0, 0.0] + [0.0]
    out = subprocess.run([exe, repr(a_d)] + [repr(v) for v in h + s], check=True, capture_output=True,
                         text=True).stdout.split("\n")
    k = int(out[0])
    sets = [[float.fromhex(t) for t in line.split()] for line in out[1:4]]
    return k, sets


@pytest.mark.parametrize("a_d,k", [(4.0, 2), (1.0, 0), (0.5, -1), (2.0 ** 300, 300), (2.0 ** -1000, -1000),
                                   (6.0, None), (4.0 + 2.0 ** -50, None), (3.0, None), (-4.0, None),
                                   (0.0, None), (5e-324, None), (float("inf"), None)])
def test_centre_power_of_two_exponent(prog, a_d, k):
    """ad_pow2 is k exactly for a positive normal 2^k (then a_d x is x with
    k added to its exponent), and 'none' for everything else: other values,
    negative, zero, subnormal, infinite."""
    got, _ = _run(prog, a_d)
    assert got == (k if k is not None else 9999)


def test_coefficient_sets_round_to_nearest(prog):
    """The FP32 sets are the FP64 coefficients rounded to nearest (what a
    device conversion gives), the FP64 sets the coefficients themselves, S^T
    the negated off-diagonal of S, and H's e is zero."""
    rng = np.random.default_rng(7)
    h = [float(v) for v in rng.normal(size=7)]
    s = [float(v) for v in rng.normal(size=8)]
    _, sets = _run(prog, 4.0, h, s)
    hs, ss, ts = sets
    # each line: d (f32, f64), c0..c5 (f32, f64), e (f32, f64)
    def split(line):
        return line[0::2], line[1::2]
    hf, hd = split(hs)
    sf, sd = split(ss)
    tf, td = split(ts)
    assert hd[:7] == h and hd[7] == 0.0
    assert sd == s[:7] + [s[7]]
    assert td[0] == s[0] and td[1:7] == [-v for v in s[1:7]] and td[7] == -s[7]
    for f, d in ((hf, hd), (sf, sd), (tf, td)):
        assert f == [float(np.float32(v)) for v in d]
