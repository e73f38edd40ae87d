"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source or of its
Python helpers (a sign, an index, a dropped term, a transposed operand, a
wrong constant, a too narrow light-cone window) and runs the
oracle pin tests against the mutated copy in a subprocess: at least one pin
must fail. This shows that the pins constrain every part of the oracle, not
only that the oracle passes them.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = [
    ("Liouvillian sign", "v *= -I / ORC_HBAR;", "v *= I / ORC_HBAR;"),
    ("H0 index transposed", "if (j == l) v -= H[m * N + k];", "if (j == l) v -= H[k * N + m];"),
    ("interaction sign", "arg[i] = I * ops->mu[i]", "arg[i] = -I * ops->mu[i]"),
    ("V^+ not transposed", "Vh[i * N + j] = conj(V[j * N + i]);", "Vh[i * N + j] = conj(V[i * N + j]);"),
    ("relaxation dropped", "if (p->G) {", "if (0) {"),
    ("trace transposed", "s += mu[j * N + k] * X[k * N + j];", "s += mu[j * N + k] * X[j * N + k];"),
    ("H stencil sign", "H[i] += ch * (E[(i + 1) % n] - E[i]);", "H[i] += ch * (E[i] - E[(i + 1) % n]);"),
    ("dP/dt sign", "cb * ((H[i] - H[im1]) / p->dx - dP[i]);", "cb * ((H[i] - H[im1]) / p->dx + dP[i]);"),
    ("Mur sign", "En[n - 1] = E[n - 2] + kappa * (En[n - 2] - E[n - 1]);",
     "En[n - 1] = E[n - 2] - kappa * (En[n - 2] - E[n - 1]);"),
    ("full step instead of half", "Ls[i] = ops->L[i] * (0.5 * p->dt);", "Ls[i] = ops->L[i] * p->dt;"),
    ("Pade coefficient", "((double)k * (double)(2 * m - k + 1));", "((double)k * (double)(2 * m - k + 2));"),
    ("too few squarings", "while (ldexp(nrm, -s) > 0.5)", "while (ldexp(nrm, -s) > 64.0)"),
    ("dP/dt from the wrong state", "superop_apply(NN, ops->L, rho, r1);", "superop_apply(NN, ops->L, r2, r1);"),
    ("H coefficient", "const double ch = p->dt / (muu * p->dx);", "const double ch = p->dt / (muu * p->dx * 1.0000001);"),
    ("V instead of V^+", "mat_mul(N, T, Vh, r2);", "mat_mul(N, T, V, r2);"),
    ("PSTD shift of dE/dx", "spectral_kernel(n, p->dx, 0.5, cp);", "spectral_kernel(n, p->dx, -0.5, cp);"),
    ("PSTD derivative sign", "I * k * cexpl(", "-I * k * cexpl("),
    ("PSTD wavenumber not folded", "(m <= n / 2) ? m : m - n;", "m;"),
    ("PSTD dP/dt sign", "cb * (dv[i] - dP[i]);", "cb * (dv[i] + dP[i]);"),
    ("PSTD H coefficient", "H[i] += (p->dt / muu) * dv[i];", "H[i] += (p->dt / muu) * 1.0000001 * dv[i];"),
    # the light-cone window of run_window: one cell inside the light cone on each side
    ("window inside the light cone", "half = n_steps + 1", "half = n_steps - 1", "__init__.py"),
]


@pytest.mark.slow
@pytest.mark.parametrize("mutation", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_mutation_is_caught(tmp_path, mutation):
    name, old, new = mutation[:3]
    target = mutation[3] if len(mutation) > 3 else "mln_oracle.c"
    for d in ("oracle", "workloads", "tests"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d,
                        ignore=shutil.ignore_patterns("_build", "__pycache__"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), tmp_path / "pytest.ini")
    src = tmp_path / "oracle" / target
    text = src.read_text()
    assert text.count(old) == 1, name
    src.write_text(text.replace(old, new))
    files = [f"tests/{f}" for f in ("test_oracle_expm.py", "test_oracle_liouville.py", "test_oracle_fdtd.py",
                                            "test_oracle_pstd.py", "test_oracle_window.py")]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "not gpu", *files],
                       cwd=tmp_path, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutation '{name}' was not caught:\n{r.stdout[-2000:]}"
