"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of ``oracle/lya_oracle.c`` (on the
CPU), builds it, and runs the pin suite against that build in a subprocess.
The suite must fail for every mutant: a pin set that a dropped term, a flipped
sign or a swapped index slips through would not be pinning anything.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lya_oracle.c")

MUTANTS = [
    ("peculiar velocity sign", "double u_j = (double)j * du + (double)vpec[j];",
     "double u_j = (double)j * du - (double)vpec[j];"),
    ("velocity of the wrong pixel", "double u_j = (double)j * du + (double)vpec[j];",
     "double u_j = (double)j * du + (double)vpec[i];"),
    ("no periodic image", "double d = nearest_image(vh_i - u_j, V);", "double d = vh_i - u_j;"),
    ("b left in km/s in the prefactor", "acc += nhi[j] / (b[j] * ORC_KMS_CMS) * shape;",
     "acc += nhi[j] / b[j] * shape;"),
    ("Gaussian width off by sqrt 2", "double x = d / b[j];", "double x = d / (b[j] * 1.41421356237);"),
    ("temperature exponent sign", "pow(T / 1.0e4, -0.7)", "pow(T / 1.0e4, 0.7)"),
    ("density to the first power", "* rho * rho * zf * zf * zf;", "* rho * zf * zf * zf;"),
    ("missing 1/sqrt(pi)", "ORC_SIGMA_A * dR / sqrt(ORC_PI);", "ORC_SIGMA_A * dR;"),
    ("comoving pixel width", "double mpc = p->box / (p->h * (1.0 + p->z) * (double)n_pix);\n    return mpc * ORC_MPC_CM;",
     "double mpc = p->box / (p->h * (double)n_pix);\n    return mpc * ORC_MPC_CM;"),
    ("no temperature pivot", "double r = rho < p->delta_pivot ? rho : p->delta_pivot;", "double r = rho;"),
    ("baryon instead of hydrogen density", "return (1.0 - p->y_he) * p->omega_b", "return p->omega_b"),
    ("Newton step sign", "double An = (gp < 0.0) ? A - g / gp : NAN;", "double An = (gp < 0.0) ? A + g / gp : NAN;"),
    ("PDF bins not centred", "double k = floor((40.0 * F + 1.0) / 2.0);", "double k = floor((40.0 * F) / 2.0);"),
    ("averaged profile: cell half-width du", "double ax = fabs(x), hw = 0.5 * du / b[j];",
     "double ax = fabs(x), hw = du / b[j];"),
    ("averaged profile: b dropped from the cell mean", "shape = sqrt(ORC_PI) * b[j] / (2.0 * du)",
     "shape = sqrt(ORC_PI) / (2.0 * du)"),
    ("averaged profile: erfc sum", "(erfc(ax - hw) - erfc(ax + hw))", "(erfc(ax - hw) + erfc(ax + hw))"),
    ("sample variance", "*var = sum_get(&v) / (double)n;\n    *tau_eff = -log(m);\n    return 0;\n}\n\n/* The same",
     "*var = sum_get(&v) / (double)(n - 1);\n    *tau_eff = -log(m);\n    return 0;\n}\n\n/* The same"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for '{name}' not found"
    mutated = src.replace(old, new, 1)
    c = tmp_path / "mutant.c"
    c.write_text(mutated)
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", str(c), "-o", str(so), "-lm"],
                   check=True)
    env = dict(os.environ, LYA_ORACLE_LIB=str(so), OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_profile.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch mutant '{name}':\n{r.stdout[-2000:]}"
