"""The oracle pins catch plausible mistakes: each case plants one slip in a
copy of the oracle's C source (on the CPU), builds it, and runs the pin suite
against it, which must fail."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "cswgs_oracle.c")

MUTATIONS = {
    "forward sign flipped": ("double d = phi[k] - oracle_spot_phase(P, xyz, n, m);",
                             "double d = oracle_spot_phase(P, xyz, n, m) - phi[k];"),
    "x and y swapped": ("double xp = (double)(m % P) - 0.5 * P;\n    double yp = (double)(m / P) - 0.5 * P;",
                        "double xp = (double)(m / P) - 0.5 * P;\n    double yp = (double)(m % P) - 0.5 * P;"),
    "theta dropped from Eq. 1": ("double ph = oracle_spot_phase(P, xyz, n, m) + theta[n];",
                                 "double ph = oracle_spot_phase(P, xyz, n, m);"),
    "defocus normalised by P^2": ("/ (half * half));", "/ ((double)P * P));"),
    "pixel origin off by one": ("double xp = (double)(m % P) - 0.5 * P;",
                                "double xp = (double)(m % P) - 0.5 * P + 1.0;"),
    "mean of |V| not divided by N": ("mean /= (double)N;", "mean /= 1.0;"),
    "update uses intensities": ("mean += hypot(V[2 * n], V[2 * n + 1]);",
                                "mean += V[2 * n] * V[2 * n] + V[2 * n + 1] * V[2 * n + 1];"),
    "efficiency from amplitudes": ("sum += in;", "sum += sqrt(in);"),
    "uniformity without 1 -": ("1.0 - (imax - imin) / (imax + imin)", "(imax - imin) / (imax + imin)"),
    "weights ignored in Eq. 1": ("sr += amp[n] * cos(ph);\n            si += amp[n] * sin(ph);",
                                 "sr += cos(ph);\n            si += sin(ph);"),
    "theta0 scaled to [0, 1)": ("theta[n] = ORACLE_TWO_PI * ((double)(x >> 11) * 0x1.0p-53);",
                                "theta[n] = ((double)(x >> 11) * 0x1.0p-53);"),
    "Feistel not a bijection": ("uint64_t nr = (L + F) % p;", "uint64_t nr = (L + F) % p | 1u;"),
    "Feistel moduli not alternated": ("            p = q;\n            q = t;", "            (void)t;"),
    "no cycle walking": ("} while (y >= D);", "} while (0);"),
    "round aperture edge excluded": ("return xp * xp + yp * yp <= (int64_t)(P / 2) * (P / 2);",
                                     "return xp * xp + yp * yp < (int64_t)(P / 2) * (P / 2);"),
    "beam radius at 1/e intensity": ("return exp(-(xp * xp + yp * yp) / (waist * waist));",
                                     "return exp(-(xp * xp + yp * yp) / (2.0 * waist * waist));"),
    "pupil amplitude applied twice": ("double a = A ? A[k] : 1.0;", "double a = A ? A[k] * A[k] : 1.0;"),
    "metrics normalised by pixel count": ("norm += A[k];", "norm += 1.0;"),
    "window offset from j": ("off = (((int64_t)(j - 1) % D)", "off = (((int64_t)j % D)"),
    "phase outside the pupil kept": ("for (int64_t m = 0; m < M; ++m) phi[m] = 0.0;", "(void)0;"),
    "full iterations not applied": ("int full = it >= I - n_full;", "int full = 0;"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor not found: %s" % name
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", str(mut), "-o", str(so), "-lm"],
                   check=True)
    env = dict(os.environ, CSWGS_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "the pins did not catch: %s" % name
    assert "failed" in r.stdout
