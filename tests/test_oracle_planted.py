"""Planted mistakes: each case copies the oracle into a temporary directory, plants one plausible
mistake in its C source, rebuilds it there and runs the pin that must catch it, which has to
fail.  The repository's own oracle is never touched.  Several of these mistakes passed every
pin that existed before the named one was written; they record why those pins are there."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, text in oracle/aw_oracle.c, replacement, pin that must fail)
PLANTED = [
    ("coarse polynomial at the centre of each fine face",
     "xiC[tb] = (ijk[tb] - r * cm[tb] + S->T.x[gi]) / r;", "xiC[tb] = (ijk[tb] - r * cm[tb] + 0.5) / r;",
     "tests/test_oracle_scheme.py::test_coarse_fine_patch_design_order[3-3.6-1.0]"),
    ("coarse sub-step time taken at the sub-step's start",
     "eval_st(S, qC, xiC, (sub + S->T.x[gs]) / r, qc);", "eval_st(S, qC, xiC, S->T.x[gs] / r, qc);",
     "tests/test_oracle_scheme.py::test_coarse_fine_patch_design_order[2-2.7-1.0]"),
    ("update divides by dx for every axis",
     "u[v] -= dt / dx[a] * (F", "u[v] -= dt / dx[0] * (F",
     "tests/test_oracle_scheme.py::test_coarse_fine_patch_design_order[3-3.6-2.0]"),
    ("3D coarse side sums the memory of one slab of children",
     "\n  int rz = d == 3 ? r : 1;\n  double s[MAXV] = {0};", "\n  int rz = 1;\n  double s[MAXV] = {0};",
     "tests/test_oracle_scheme.py::test_coarse_fine_patch_3d"),
    ("level-0 step without the r^l factor of local time stepping",
     "double dt = rl * S->c.cfl / den;", "double dt = S->c.cfl / den;",
     "tests/test_oracle_scheme.py::test_lts_level0_step_not_limited_by_refinement"),
    ("inflow ghosts on the opposite face",
     "return S->c.bc[2 * a + (c < 0 ? 0 : 1)] == BC_INFLOW;", "return S->c.bc[2 * a + (c < 0 ? 1 : 0)] == BC_INFLOW;",
     "tests/test_oracle_inflow.py::test_boundary_reconstruction_sees_the_ghost_states"),
    ("z momentum not negated beyond a wall",
     "    for (int a = 0; a < S->d; a++)\n      if (reflected(S, lv, a, c[a]))",
     "    for (int a = 0; a < 2; a++)\n      if (reflected(S, lv, a, c[a]))",
     "tests/test_oracle_reflective.py::test_octant_with_walls_equals_full_domain_3d"),
    ("GLM: psi flux c_h B_n instead of c_h^2 B_n",
     "f[8] = P->c_h * P->c_h * B[n];", "f[8] = P->c_h * B[n];",
     "tests/test_oracle_mhd.py::test_glm_cleaning_wave[2-2.7]"),
    ("energy flux v (E + 0.9 p)",
     "f[d + 1] = vn * (E + p);", "f[d + 1] = vn * (E + 0.9 * p);",
     "tests/test_oracle_riemann.py::test_sod_converges_to_exact_solution[2]"),
    ("time step from the largest axis term instead of the sum over axes",
     "for (int a = 0; a < S->d; a++) den += max_speed(&S->P, u, a) / dx[a];",
     "for (int a = 0; a < S->d; a++) { double t_ = max_speed(&S->P, u, a) / dx[a]; if (t_ > den) den = t_; }",
     "tests/test_oracle_dt.py::test_dt_euler_2d_constant_state"),
    ("time step from the smallest spacing over the sum of speeds",
     "for (int a = 0; a < S->d; a++) den += max_speed(&S->P, u, a) / dx[a];",
     "for (int a = 0; a < S->d; a++) den += max_speed(&S->P, u, a) / (dx[0] < dx[1] ? dx[0] : dx[1]);",
     "tests/test_oracle_dt.py::test_dt_euler_3d_constant_state"),
    ("MHD Jacobian: energy flux without the work of the normal field on v.B",
     "  A[4][5 + n] -= vB;\n", "\n",
     "tests/test_oracle_osher.py::test_mhd_jacobian_spectrum_and_abs_jacobian_match_numpy"),
    ("MHD Jacobian: total pressure without the magnetic pressure",
     "  for (int a = 0; a < 3; a++) dpt[5 + a] += B[a];\n", "\n",
     "tests/test_oracle_osher.py::test_mhd_jacobian_spectrum_and_abs_jacobian_match_numpy"),
    ("indicator without its cross terms",
     "    for (int l = 0; l < d; l++) {\n      double D2, G, A;", "    for (int l = k; l <= k; l++) {\n      double D2, G, A;",
     "tests/test_oracle_indicator.py::test_mixed_derivative_counts"),
]


@pytest.mark.slow
@pytest.mark.parametrize("name,old,new,pin", PLANTED, ids=[p[0] for p in PLANTED])
def test_planted_mistake_fails_its_pin(tmp_path, name, old, new, pin):
    shutil.copytree(os.path.join(ROOT, "oracle"), tmp_path / "oracle",
                    ignore=shutil.ignore_patterns("*.so", "*.tmp", "__pycache__"))
    shutil.copytree(os.path.join(ROOT, "tests"), tmp_path / "tests", ignore=shutil.ignore_patterns("__pycache__"))
    shutil.copy(os.path.join(ROOT, "aw_inputs.py"), tmp_path / "aw_inputs.py")
    src = tmp_path / "oracle" / "aw_oracle.c"
    text = src.read_text()
    assert text.count(old) == 1, f"the text to change must occur once in the oracle: {old!r}"
    src.write_text(text.replace(old, new))
    env = {k: v for k, v in os.environ.items() if k != "PYTHONPATH"}
    p = subprocess.run([sys.executable, "-m", "pytest", pin, "-q", "-x", "-p", "no:cacheprovider"], cwd=tmp_path,
                       env=env, capture_output=True, text=True, timeout=600)
    # exit code 1: tests ran and failed (2-5 would be an interrupted run, a usage or collection error)
    assert p.returncode == 1, f"{name}: the pin did not fail\n{p.stdout[-2000:]}\n{p.stderr[-2000:]}"
    assert " failed" in p.stdout
