"""Mutation check of the oracle's pins: plant one plausible mistake at a time (a wrong
coefficient, sign, index or transposed operand) in a temporary copy of the oracle, rebuild it,
and require that the pin suite fails against every mutant.  Mistakes are planted only in the
CPU oracle copy under a temporary directory; nothing here touches the GPU library."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "zm_oracle.c")

MUTANTS = [
    ("stencil coefficient", "+ 8.0 * fp1 - 8.0 * fm1 + fm2", "+ 8.0 * fp1 - 7.0 * fm1 + fm2"),
    ("stencil outer sign", "(-fp2 + 8.0 * fp1 - 8.0 * fm1 + fm2)", "(fp2 + 8.0 * fp1 - 8.0 * fm1 - fm2)"),
    ("second-difference centre", "- 30.0 * f0", "- 32.0 * f0"),
    ("free-edge mirror instead of extrapolation",
     "return 2.0 * f[(size_t)0 * n2 + j] - f[(size_t)(-i) * n2 + j];",
     "return f[(size_t)(-i) * n2 + j];"),
    ("seam shift sign", "if (i < 0) { i += n1; s -= shift1; }", "if (i < 0) { i += n1; s += shift1; }"),
    ("normal cross-product component", "double cy = w1 * x2 - x1 * w2;", "double cy = x1 * w2 - w1 * x2;"),
    ("sheet strength transposed",
     "w[p] * a2[c * N + p] - w[N + p] * a1[c * N + p]", "w[p] * a1[c * N + p] - w[N + p] * a2[c * N + p]"),
    ("BR prefactor", "-weight / (4.0 * ZMO_PI)", "-weight / (2.0 * ZMO_PI)"),
    ("BR sign", "double pref = -weight", "double pref = weight"),
    ("BR kernel exponent", "1.0 / (r2 * sqrt(r2))", "1.0 / (r2 * r2)"),
    ("BR cross index", "(rz * gx - rx * gz)", "(rz * gx - ry * gz)"),
    ("BR core size", "rz * rz + d2;", "rz * rz + delta;"),
    ("Riesz sign", "si = -(c1 * r1[p] + c2 * r2[p]);", "si = (c1 * r1[p] + c2 * r2[p]);"),
    ("Riesz components swapped", "sr = c1 * i1[p] + c2 * i2[p];", "sr = c2 * i1[p] + c1 * i2[p];"),
    ("Riesz normalisation", "r1[p] / (double)N", "r1[p] / (double)n1"),
    ("FFT twiddle sign", "double ang = sign * 2.0", "double ang = -2.0"),
    ("Nyquist not removed", "2 * a != n1 && 2 * b != n2", "1"),
    ("jump term weight", "0.125 * jump", "0.25 * jump"),
    ("jump term metric transposed", "(h22 * w1 * w1 - 2.0 * h12 * w1 * w2 + h11 * w2 * w2)",
     "(h11 * w1 * w1 - 2.0 * h12 * w1 * w2 + h22 * w2 * w2)"),
    ("kinetic term weight", "0.5 * uu", "uu"),
    ("gravity term", "g * z[2 * N + p]", "g * z[N + p]"),
    ("Atwood factor", "*= -2.0 * atwood", "*= -atwood"),
    ("viscosity sign", "+= mu * tmp[p]", "-= mu * tmp[p]"),
    ("low-order velocity sign", "-0.5 * s[p] * nrm", "0.5 * s[p] * nrm"),
    ("RK3 weight", "{1.0, 0.25, 2.0 / 3.0}", "{1.0, 0.5, 2.0 / 3.0}"),
    ("cutoff test reversed", "return dist2 <= cutoff * cutoff;", "return dist2 >= cutoff * cutoff;"),
    ("cutoff boundary exclusive", "return dist2 <= cutoff * cutoff;", "return dist2 < cutoff * cutoff;"),
    ("cutoff decided in FP32", "return dist2 <= cutoff * cutoff;",
     "return (float)dist2 <= (float)(cutoff * cutoff);"),
    ("cutoff against the unsquared distance", "return dist2 <= cutoff * cutoff;", "return dist2 <= cutoff;"),
    ("cutoff distance drops a component", "for (int c = 0; c < 3; c++) {\n        double d = zi",
     "for (int c = 0; c < 2; c++) {\n        double d = zi"),
    ("medium order takes the wrong velocity for Phi", "zmo_phi(N, z, w, h, u_low ? u_low : u, prm->g, phi);",
     "zmo_phi(N, z, w, h, u, prm->g, phi);"),
    ("RK3 stage uses old state", "b[stage] * (y[k] + dt * ydot[k])", "b[stage] * (y0[k] + dt * ydot[k])"),
    # the general-length FFT (sides that are not powers of two)
    ("prime-length DFT root index", "(size_t)((long long)t * k % n) * scale", "(size_t)((long long)t * (k + 1) % n) * scale"),
    ("Cooley-Tukey twiddle index", "(size_t)((long long)q * k % n) * scale", "(size_t)((long long)q * k % m) * scale"),
    ("Cooley-Tukey sub-transform index", "sub[(size_t)q * m + k % m], ai", "sub[(size_t)q * m + k / p], ai"),
    ("general-length roots without the sign", "const double ang = sign * 2.0 * ZMO_PI * t / n;",
     "const double ang = -2.0 * ZMO_PI * t / n;"),
    ("signed frequency of odd sides", "return 2 * idx < n ? idx : idx - n;", "return idx < n / 2 ? idx : idx - n;"),
]


def _run_mutant(tmp, k, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    d = os.path.join(tmp, f"m{k}")
    os.makedirs(d)
    shutil.copy(os.path.join(ROOT, "oracle", "zm_oracle.h"), d)
    with open(os.path.join(d, "zm_oracle.c"), "w") as f:
        f.write(src.replace(old, new, 1))
    lib = os.path.join(d, "liboracle.so")
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-o", lib,
                    os.path.join(d, "zm_oracle.c"), "-lm"], check=True, capture_output=True)
    env = dict(os.environ, ZM_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "not slow",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode


def test_every_planted_mistake_fails_a_pin():
    with tempfile.TemporaryDirectory() as tmp:
        with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
            futs = {ex.submit(_run_mutant, tmp, k, old, new): name
                    for k, (name, old, new) in enumerate(MUTANTS)}
            survivors = [futs[f] for f in cf.as_completed(futs) if f.result() == 0]
    assert not survivors, f"pins did not catch: {survivors}"
