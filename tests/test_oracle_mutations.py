"""The oracle's pins must catch plausible mistakes.  Each case plants one
mistake (a dropped term, a wrong sign, a shifted index, a transposed operand)
in a private copy of the oracle source, builds it with gcc on the host and
runs the pin suite against that build, which must fail."""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sscg_oracle.c")

MUTANTS = {
    "sw-alpha-index": ("rhs[s - 1 + j - 1] * alpha[s - i + j - 1]", "rhs[s - 1 + j - 1] * alpha[s - i + j]"),
    "sw-b1-sign": ("= -rhs[i + j - 1 - 1];", "= rhs[i + j - 1 - 1];"),
    "sw-W-sign": ("t -= b1[i + (size_t)k * s] * beta[k + (size_t)j * s];", "t += b1[i + (size_t)k * s] * beta[k + (size_t)j * s];"),
    "sw-rhs-divisor": ("rhs[s - 1 + i - 1] = -t / as;", "rhs[s - 1 + i - 1] = -t / alpha[0];"),
    "update-beta-transposed": ("t += Pold[i + (size_t)(half * s + l) * n] * beta[l + (size_t)j * s];",
                               "t += Pold[i + (size_t)(half * s + l) * n] * beta[j + (size_t)l * s];"),
    "cvm-wrong-column": ("vm[s + j] = orc_dot(n, COL(P, n, j), COL(P, n, 2 * s - 1));",
                         "vm[s + j] = orc_dot(n, COL(P, n, j), COL(P, n, 2 * s - 2));"),
    "pmpk-pout": ("pout = ptemp + 1;", "pout = ptemp;"),
    "pcg-beta-inverted": ("double beta = rho_new / rho;", "double beta = rho / rho_new;"),
    "pcg-residual-sign": ("x[i] += alpha * p[i]; r[i] -= alpha * sv[i];", "x[i] += alpha * p[i]; r[i] += alpha * sv[i];"),
    "gram-C-without-A": ("C[l + (size_t)j * s] = -orc_dot(n, COL(APo, n, l), COL(U, n, j));",
                         "C[l + (size_t)j * s] = -orc_dot(n, COL(Po, n, l), COL(U, n, j));"),
    "gram-G-transposed-triangle": ("G[i + (size_t)j * s] = orc_dot(n, COL(U, n, i), COL(AU, n, j));",
                                   "G[i + (size_t)j * s] = orc_dot(n, COL(U, n, i), COL(AU, n, i));"),
    "newton-shift-sign": ("un[i] = (w[i] - theta[j] * uj[i]) / sigma;", "un[i] = (w[i] + theta[j] * uj[i]) / sigma;"),
    "newton-leja-first-point": ("v = fabs(t[k]);", "v = -fabs(t[k]);"),
    "cheb-basis-dropped-term": ("un[i] = 2.0 * (w[i] - c * uj[i]) / delta - um[i];", "un[i] = 2.0 * (w[i] - c * uj[i]) / delta;"),
    "cheb-prec-rho": ("double rho_new = 1.0 / (2.0 * theta / delta - rho);", "double rho_new = 1.0 / (2.0 * theta / delta + rho);"),
    "lanczos-diag-term": ("d[j] = 1.0 / a[j] + (j > 0 ? bb[j - 1] / a[j - 1] : 0.0);", "d[j] = 1.0 / a[j];"),
    "chol-back-substitution": ("t -= L[k + (size_t)i * n] * x[k];", "t -= L[i + (size_t)k * n] * x[k];"),
    "mlp-tanh-derivative": ("d2[j] = t * (1.0 - h2[j] * h2[j]);", "d2[j] = t * (1.0 - h2[j]);"),
    "features-coupling-scale": ("double lc = log(a / sqrt(d[i] * d[j]));", "double lc = log(a / sqrt(d[i] * d[i]));"),
    "features-std-mean": ("double e = log(d[i]) - mean;", "double e = log(d[i]);"),
    "adam-bias-correction": ("theta[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);",
                             "theta[i] -= lr * m[i] / (sqrt(v[i] / c2) + eps);"),
    "adam-moment-weights": ("v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];", "v[i] = b1 * v[i] + (1.0 - b1) * g[i] * g[i];"),
    "pfcg-gamma-sign": ("p[i] = u[i] - c * p[i];", "p[i] = u[i] + c * p[i];"),
    "spmv-dropped-diagonal": ("for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++) t += A->val[k] * x[A->col[k]];\n        y[i] = t;",
                              "for (int32_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++) if (A->col[k] != i) t += A->val[k] * x[A->col[k]];\n        y[i] = t;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "mutant.c")
        so = os.path.join(d, "mutant.so")
        open(c, "w").write(src.replace(old, new))
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", "-I",
                        os.path.join(ROOT, "oracle"), c, "-o", so, "-lm"], check=True)
        env = dict(os.environ, SSCG_ORACLE_LIB=so, OMP_NUM_THREADS="2")
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not slow",
                            os.path.join(ROOT, "tests", "test_oracle_pins.py")], env=env, cwd=ROOT,
                           capture_output=True, text=True, timeout=600)
        assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
