"""The pins catch plausible mistakes in the oracle.

Each case plants one slip in a copy of oracle/fdk_oracle.c -- a dropped or
wrong weight, a swapped row, axis or tap, a sign, an off-by-one -- compiles
it, and runs the pin suite (tests/test_oracle_pins.py) against that build in
a separate process.  Every mutant must fail at least one pin; the unmutated
copy, built the same way, must pass them all.  The mistakes are planted in
the oracle on the CPU only, and each keeps every memory access in bounds.
"""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "fdk_oracle.c")

MUTANTS = {
    "u from the v row": ("double u = up / w;", "double u = vp / w;"),
    "x and y swapped in u'": ("double up = P[0] * X + P[1] * Y", "double up = P[0] * Y + P[1] * X"),
    "truncation for u": ("double fu = literal_trunc ? trunc(u) : floor(u);", "double fu = trunc(u);"),
    "fraction sign": ("*a = u - fu;", "*a = fu - u;"),
    "1/w instead of 1/w^2": ("*inv_w2 = 1.0 / (w * w);", "*inv_w2 = 1.0 / w;"),
    "last column dropped": ("if (m < 0 || m >= W || n < 0 || n >= H) return 0.0;",
                            "if (m < 0 || m >= W - 1 || n < 0 || n >= H) return 0.0;"),
    "image read transposed": ("return (double)img[n * W + m];", "return (double)img[m * H + n];"),
    "tap (i+1, j) read as (i, j+1)": ("double p10 = oracle_tap(img, jb->W, jb->H, i + 1, j);",
                                      "double p10 = oracle_tap(img, jb->W, jb->H, i, j + 1);"),
    "lerp weights swapped": ("double lo = (1.0 - a) * p00 + a * p10;", "double lo = a * p00 + (1.0 - a) * p10;"),
    "origin off by one voxel in x": ("double X = jb->org[0] + (double)x * jb->vs[0];",
                                     "double X = jb->org[0] + (double)(x + 1) * jb->vs[0];"),
    "voxels behind the source kept": ("if (!(w > 0.0)) return 0;", "if (w == 0.0) return 0;"),
    "adjoint taps swapped": ("double ws[4] = {(1.0 - b) * (1.0 - a), (1.0 - b) * a, b * (1.0 - a), b * a};",
                             "double ws[4] = {(1.0 - b) * (1.0 - a), b * (1.0 - a), (1.0 - b) * a, b * a};"),
    "adjoint without 1/w^2": ("double g = (double)row[x] * iw2;", "double g = (double)row[x];"),
    "ramp kernel sign": ("-1.0 / (pi * pi * (double)d * (double)d)", "1.0 / (pi * pi * (double)d * (double)d)"),
    "cosine weight centres swapped": ("const double du = (double)m - u0, dv = (double)n - v0;",
                                      "const double du = (double)m - v0, dv = (double)n - u0;"),
    "focal length without the u0 term": ("const double f2 = G[0][0] / s2 - u0 * u0;",
                                         "const double f2 = G[0][0] / s2;"),
    "v from the u row": ("double v = vp / w;", "double v = up / w;"),
    "z step with the y voxel size": ("double Z = jb->org[2] + (double)z * jb->vs[2];",
                                     "double Z = jb->org[2] + (double)z * jb->vs[1];"),
    "ramp kernel centre tap 1/2": ("h[d] = (d == 0) ? 0.25 :", "h[d] = (d == 0) ? 0.5 :"),
    "even ramp taps nonzero": ("((d % 2) ? -1.0 / (pi * pi * (double)d * (double)d) : 0.0)",
                               "(-1.0 / (pi * pi * (double)d * (double)d))"),
    "cosine weight squared": ("f / sqrt(f * f + du * du + dv * dv)", "f * f / (f * f + du * du + dv * dv)"),
    "views overwrite instead of accumulate": ("row[x] += val * iw2;", "row[x] = val * iw2;"),
    "last detector row dropped": ("n < 0 || n >= H) return 0.0;", "n < 0 || n >= H - 1) return 0.0;"),
    "filter scale dropped": ("o[m] = scale * acc;", "o[m] = acc;"),
    "count keeps pairs behind the source": ("if (!(w > 0.0)) continue;", "if (w == 0.0) continue;"),
    "count on [0, W) x [0, H)": ("if (u > -1.0 && u < Wd && v > -1.0 && v < Hd) ++count;",
                                 "if (u >= 0.0 && u < Wd && v >= 0.0 && v < Hd) ++count;"),
    "v fraction sign": ("*b = v - fv;", "*b = fv - v;"),
    "tap (i+1, j+1) read as (i, j+1)": ("double p11 = oracle_tap(img, jb->W, jb->H, i + 1, j + 1);",
                                        "double p11 = oracle_tap(img, jb->W, jb->H, i, j + 1);"),
    "adjoint drops the last column": ("if (ms[t] < 0 || ms[t] >= jb->W ||", "if (ms[t] < 0 || ms[t] >= jb->W - 1 ||"),
    "filter convolution one-sided": ("for (int64_t mp = 0; mp < W; ++mp) {", "for (int64_t mp = 0; mp <= m; ++mp) {"),
    "voxel list reads row j for row j+1": ("(1.0 - a) * oracle_tap(img, W, H, i, j + 1)",
                                           "(1.0 - a) * oracle_tap(img, W, H, i, j)"),
}


def _build(tmp_path, name, text):
    src = tmp_path / f"{name}.c"
    src.write_text(text)
    lib = tmp_path / f"{name}.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-pthread",
                    str(src), "-o", str(lib), "-lm"], check=True)
    return str(lib)


def _pins(lib):
    env = dict(os.environ, FDK_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(HERE, "test_oracle_pins.py"),
                        "-x", "-q", "-p", "no:cacheprovider"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout


def test_unmutated_copy_passes(tmp_path):
    rc, out = _pins(_build(tmp_path, "clean", open(SRC).read()))
    assert rc == 0, out[-2000:]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) >= 1, f"mutation site not found: {old}"
    rc, out = _pins(_build(tmp_path, "mutant", text.replace(old, new)))
    assert rc != 0, f"no pin caught the mutant '{name}'"
    assert " failed" in out, f"the mutant '{name}' did not fail a pin cleanly:\n{out[-2000:]}"
