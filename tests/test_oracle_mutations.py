"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (a sign, an
index, a time sheet, a factor, a grid offset, a misplaced link), on the CPU,
and runs tests/test_oracle_pins.py against the mutated copy: at least one pin
must fail.  The unmutated oracle passes the same pins in the main suite.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (what the mistake is, exact text in dirac_oracle.c, replacement)
MUTATIONS = [
    ("sign of the y difference (c_y)", "coeff[1] = pb ? I : -I;", "coeff[1] = pb ? -I : I;"),
    ("z difference without its sign class", "coeff[2] = pb ? -1.0 : 1.0;", "coeff[2] = 1.0;"),
    ("same sign of m on both sheets", "double beta = upper ? 1.0 : -1.0;", "double beta = 1.0;"),
    ("lower half-step on the upper time sheet", "half_step(p, &g, psi, V_fine, 0, t + p->dt / 2);",
     "half_step(p, &g, psi, V_fine, 0, t);"),
    ("sign of the Peierls phase of the up link", "up = up * cexp(-I * phi_p);", "up = up * cexp(I * phi_p);"),
    ("link midpoint at the far end", "yp[a] += h / 2.0;", "yp[a] += h;"),
    ("down neighbour taken on the wrong side", "Cm[a] = wrap(C[a] - 1, g->M[a]);",
     "Cm[a] = wrap(C[a] + 1 - 2 * (a == 0), g->M[a]);"),
    ("sign of the difference part", "psi[f] = ((1.0 - I * th) * psi[f] - S) / (1.0 + I * th);",
     "psi[f] = ((1.0 - I * th) * psi[f] + S) / (1.0 + I * th);"),
    ("Cayley denominator conjugated", "psi[f] = ((1.0 - I * th) * psi[f] - S) / (1.0 + I * th);",
     "psi[f] = ((1.0 - I * th) * psi[f] - S) / (1.0 - I * th);"),
    ("theta without the factor 1/2", "cplx th = p->dt * (beta * p->m + potential(p, V_fine, f, x, t)) / 2.0;",
     "cplx th = p->dt * (beta * p->m + potential(p, V_fine, f, x, t));"),
    ("B0 and B1 grid offsets swapped", "{1, 0, 1}, /* B0 */ {0, 1, 1}, /* B1 */",
     "{0, 1, 1}, /* B0 */ {1, 0, 1}, /* B1 */"),
    ("sign of the imaginary potential", "return V + I * potential_imag(p, x);",
     "return V - I * potential_imag(p, x);"),
    ("plane-wave link integral without its sinc factor", "double sinc = u == 0.0 ? 1.0 : sin(u) / u;",
     "double sinc = 1.0;"),
    ("down link read at the value's own point",
     "phi_m += p->q * mod * g->link[a][fine_index(g, Cm[0], Cm[1], Cm[2])];",
     "phi_m += p->q * mod * g->link[a][fine_index(g, C[0], C[1], C[2])];"),
    ("sign of the cross term of the functional", "out[0] = naive + cross_lower;",
     "out[0] = naive - cross_lower;"),
    ("modulated potential taken half a step late",
     "if (V_fine) V += V_fine[f] * (1.0 + p->Vmod_amp * cos(p->Vmod_omega * t));",
     "if (V_fine) V += V_fine[f] * (1.0 + p->Vmod_amp * cos(p->Vmod_omega * (t + p->dt / 2)));"),
    ("link integrals not modulated in time", "double mod = 1.0 + p->Alink_amp * cos(p->Alink_omega * t);",
     "double mod = 1.0 + p->Alink_amp;"),
    ("Klein step applied on the step itself", "x[p->step_axis] > p->step_x0", "x[p->step_axis] >= p->step_x0"),
    ("soft core with a instead of a^2", "V -= p->sc_Z / sqrt(r2 + p->sc_a * p->sc_a);",
     "V -= p->sc_Z / sqrt(r2 + p->sc_a);"),
    ("absorbing layer only at the lower face", "double d = x[a] < L - x[a] ? x[a] : L - x[a];",
     "double d = x[a];"),
]


def copy_tree(dst):
    skip = shutil.ignore_patterns("_build", "__pycache__", "*.so", "csrc", "*.o")
    for d in ("oracle", "tests", "paper_1309_3452_gb300"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(dst, d), ignore=skip)


@pytest.mark.parametrize("what,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_the_mistake(tmp_path, what, old, new):
    copy_tree(str(tmp_path))
    src = os.path.join(str(tmp_path), "oracle", "dirac_oracle.c")
    text = open(src).read()
    assert text.count(old) == 1, f"mutation site not found once: {old}"
    open(src, "w").write(text.replace(old, new))
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    # the mutated copy compiles ...
    b = subprocess.run([sys.executable, "-c", "from oracle import oracle as O; O.build()"], cwd=str(tmp_path),
                       capture_output=True, text=True, timeout=300, env=env)
    assert b.returncode == 0, b.stderr[-2000:]
    # ... and fails at least one pin (exit status 1: tests failed, not a collection error)
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-x", "-q",
                        "-p", "no:cacheprovider"], cwd=str(tmp_path), capture_output=True, text=True,
                       timeout=600, env=env)
    assert r.returncode == 1 and " failed" in r.stdout, (what, r.stdout[-2000:])
