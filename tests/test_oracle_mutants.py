"""The pins catch plausible mistakes: each case plants one mistake in a copy of an oracle's C source (a dropped
term, a wrong sign, coefficient or index, a transposed operand), rebuilds that copy, and requires the oracle's pin
tests to fail on it.  CPU only; the product library is not involved."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

GRAVITY = "hg_oracle.c"
HYDRO = "hydro_oracle.c"
PINS = {GRAVITY: "tests/test_oracle_pins.py", HYDRO: "tests/test_hydro_pins.py"}

MUTANTS = [
    # the wave-equation oracle
    (GRAVITY, "source sign", "- src * (rho[iidx(g, i, j, k)] - rho_bar);", "+ src * (rho[iidx(g, i, j, k)] - rho_bar);"),
    (GRAVITY, "2 pi for 4 pi", "* 4.0 * OG_PI * g->G; }", "* 2.0 * OG_PI * g->G; }"),
    (GRAVITY, "leapfrog coefficient", "2.0 * phi[q] - phi_prev[q] + nu2 * L", "1.0 * phi[q] - phi_prev[q] + nu2 * L"),
    (GRAVITY, "wrong +y neighbour", "s += phi[gidx(g, i, j + 1, k)] - c;", "s += phi[gidx(g, i, j - 1, k)] - c;"),
    (GRAVITY, "periodic wrap off by one", "src[axis] = hi ? 0 : n[axis] - 1;", "src[axis] = hi ? 1 : n[axis] - 1;"),
    (GRAVITY, "multipole weight", "4.0 * OG_PI / (2.0 * l + 1.0) * s * rp", "4.0 * OG_PI / (2.0 * l + 3.0) * s * rp"),
    (GRAVITY, "Robin update coefficient", "ug - robin_coef(g, f, gc) * (ug - ui)", "ug - 0.5 * robin_coef(g, f, gc) * (ug - ui)"),
    (GRAVITY, "gradient neighbour", "ay[q] = -(phi[gidx(g, i, j + 1, k)] - phi[gidx(g, i, j - 1, k)]) * inv2h;",
     "ay[q] = -(phi[gidx(g, i, j + 1, k)] - phi[gidx(g, i - 1, j, k)]) * inv2h;"),
    (GRAVITY, "adjoint source sign", "grad[iidx(g, i, j, k)] -= src * l;", "grad[iidx(g, i, j, k)] += src * l;"),
    (GRAVITY, "adjoint Robin ratio", "+= a_ * ri / rg * lg;", "+= a_ * rg / ri * lg;"),
    (GRAVITY, "Legendre seed", "pmm *= -(2.0 * q - 1.0) * st;", "pmm *= -(2.0 * q + 1.0) * st;"),
    # the hydrodynamics oracle
    (HYDRO, "no energy source", "r[4] = r[4] + ((u[1] * ax + u[2] * ay) + u[3] * az);", "r[4] = r[4];"),
    (HYDRO, "momentum source sign", "r[1] = r[1] + u[0] * ax;", "r[1] = r[1] - u[0] * ax;"),
    (HYDRO, "flux difference sign", "r[q] = d == 0 ? lo[q] - hi[q] : r[q] + (lo[q] - hi[q]);",
     "r[q] = d == 0 ? hi[q] - lo[q] : r[q] + (hi[q] - lo[q]);"),
    (HYDRO, "slope factor 1", "wl[q] = w0[q] + 0.5 * mc(", "wl[q] = w0[q] + 1.0 * mc("),
    (HYDRO, "HLL instead of HLLC", "us[1 + d] = fac * ss;", "us[1 + d] = fac * w[1 + d];"),
    (HYDRO, "Heun second stage", "u[q] = 0.5 * (U[q * n + c] + (U1[q * n + c] + dt * L[q * n + c]));",
     "u[q] = U1[q * n + c] + dt * L[q * n + c];"),
    (HYDRO, "virial half", "const double W = 0.5 * srp * h3;", "const double W = srp * h3;"),
    (HYDRO, "kinetic half", "return 0.5 * ((u[1] * *vx + u[2] * *vy) + u[3] * *vz);",
     "return ((u[1] * *vx + u[2] * *vy) + u[3] * *vz);"),
    (HYDRO, "Davis S_L as a max", "const double sl = a1 < a2 ? a1 : a2;", "const double sl = a1 > a2 ? a1 : a2;"),
    (HYDRO, "y-neighbour along x", "    else if (d == 1) j += t;", "    else if (d == 1) i += t;"),
    (HYDRO, "MC central weight", "const double c = 0.5 * (a + b), a2 = 2.0 * a, b2 = 2.0 * b;",
     "const double c = 1.0 * (a + b), a2 = 2.0 * a, b2 = 2.0 * b;"),
    (HYDRO, "high boundary not clamped", "if (i > g->nx - 1) i = g->nx - 1;", "if (i > g->nx - 1) i = 0;"),
]


def _run_pins(tmp_path, src, old=None, new=None):
    for d in ("oracle", "tests", "paper_1602_05700_gb300"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d,
                        ignore=shutil.ignore_patterns("_build", "__pycache__", "*.so", "*.o"))
    for f in ("pytest.ini", "bench.py"):  # bench.py: the pinned Poisson references of the studies live there
        shutil.copy(os.path.join(ROOT, f), tmp_path)
    if old is not None:
        path = tmp_path / "oracle" / src
        text = path.read_text()
        assert text.count(old) == 1, f"mutation anchor not found exactly once: {old}"
        path.write_text(text.replace(old, new))
    env = dict(os.environ, PYTHONPATH=str(tmp_path))
    return subprocess.run([sys.executable, "-m", "pytest", PINS[src], "-x", "-q", "-p", "no:cacheprovider"],
                          cwd=tmp_path, env=env, capture_output=True, text=True, timeout=600)


@pytest.mark.parametrize("src", [GRAVITY, HYDRO])
def test_unmutated_copy_passes_its_pins(tmp_path, src):
    """The control: the same copy-and-rebuild procedure without a mutation passes, so a failure below is the
    mutation's."""
    r = _run_pins(tmp_path, src)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("src,name,old,new", MUTANTS, ids=[f"{m[0].split('_')[0]}: {m[1]}" for m in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path, src, name, old, new):
    r = _run_pins(tmp_path, src, old, new)
    assert r.returncode != 0, f"no pin caught the planted mistake '{name}':\n{r.stdout[-2000:]}"
    assert "failed" in r.stdout, r.stdout[-2000:]  # a failing pin, not a collection or build error
