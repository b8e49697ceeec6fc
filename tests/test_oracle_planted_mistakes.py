"""The pins of the corrector-step oracle catch plausible mistakes.

Each case copies the oracle (and the input generator) to a scratch
directory, plants one mistake in the copy -- a flipped or dropped term,
swapped operands, a wrong index or weight, the literal reading of a garbled
formula -- and runs the pins against the copy in a fresh interpreter: at
least one pin must fail.  Only the scratch copy is changed; everything runs
on the CPU."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CP2 = "test_oracle_cp2.py"
CP1 = "test_oracle_cp1.py"

MISTAKES = [
    # CP2 step (Eq. flux_k_+_2/3, Eq. Cs2_6 / App. C, Eq. RT0, Eq. grad_PSI)
    ("ep_estimate_sign", "cps_oracle.c", CP2,
     "sum += est;\n                    ++count;\n                }\n            }\n            if (count",
     "sum -= est;\n                    ++count;\n                }\n            }\n            if (count"),
    ("conormal_components_swapped", "cps_oracle.c", CP2,
     "double c1 = (dtau[0] * n2y - dtau[1] * n2x) / det;",
     "double c1 = (n1x * dtau[1] - n1y * dtau[0]) / det;"),
    ("literal_projection_reading", "cps_oracle.c", CP2,
     "double c1 = (dtau[0] * n2y - dtau[1] * n2x) / det;\n    double c2 = (n1x * dtau[1] - n1y * dtau[0]) / det;",
     "double c1 = fabs(dtau[0] * n1x + dtau[1] * n1y) + 0 * det;\n    double c2 = fabs(dtau[0] * n2x + dtau[1] * n2y);"),
    ("distances_swapped", "cps_oracle.c", CP2,
     "*est = c1 * (e1 - eta[c]) / dist[s1] + c2 * (e2 - eta[c]) / dist[s2];",
     "*est = c1 * (e1 - eta[c]) / dist[s2] + c2 * (e2 - eta[c]) / dist[s1];"),
    ("averaging_weight", "cps_oracle.c", CP2,
     "if (count > 0) tau[s] = len[s] * sum / count;",
     "if (count > 0) tau[s] = len[s] * sum / 2;"),
    ("area_weights_swapped", "cps_oracle.c", CP2,
     "fbar[s] = (une * area[ep] - unp * area[e])",
     "fbar[s] = (une * area[e] - unp * area[ep])"),
    ("dirichlet_mean_flux_dropped", "cps_oracle.c", CP2,
     "fbar[s] = une * len[s];", "fbar[s] = 0.0 * une * len[s];"),
    ("tangential_flux_left_out_of_Q", "cps_oracle.c", CP2,
     "if (ep >= 0) q = fbar[s] - T[s] * (eta[e] - eta[ep]) + tau[s];",
     "if (ep >= 0) q = fbar[s] - T[s] * (eta[e] - eta[ep]);"),
    ("rt0_wrong_node", "cps_oracle.c", CP2,
     "ux += q * (gx - p[j][0]) / a2;", "ux += q * (gx - p[(j + 1) % 3][0]) / a2;"),
    ("mbar_offdiagonal_sign", "cps_oracle.c", CP2,
     "g_next[e] = g_k[e] + m00 * du + m01 * dv;", "g_next[e] = g_k[e] + m00 * du - m01 * dv;"),
    # CP1 step (Eq. cs1_sys2, Eq. CS1_sys_coeff, App. B)
    ("cp1_rhs_sign_as_printed", "__init__.py", CP1,
     "lap = np.stack([-cp1_laplacian(T, nbr, isd, du_breve[0]),\n                    -cp1_laplacian(T, nbr, isd, du_breve[1])])",
     "lap = np.stack([cp1_laplacian(T, nbr, isd, du_breve[0]),\n                    cp1_laplacian(T, nbr, isd, du_breve[1])])"),
    ("cp1_coupling_sign", "__init__.py", CP1,
     "un = solve(Ax, Dx, lap[0] - mass[:, 1] * v, u)",
     "un = solve(Ax, Dx, lap[0] + mass[:, 1] * v, u)"),
    ("cp1_coupled_component", "__init__.py", CP1,
     "vn = solve(Ay, Dy, lap[1] - mass[:, 1] * u, v)",
     "vn = solve(Ay, Dy, lap[1] - mass[:, 1] * v, v)"),
    ("cp1_laplacian_drops_dirichlet", "__init__.py", CP1,
     "open_side = (nbr >= 0) | (is_dirichlet != 0)", "open_side = (nbr >= 0)"),
    ("cp1_mbar12_sign_vertex_fields", "cps_oracle.c", CP1,
     "m01 += cf * kinv[3 * v + 1] / dt;", "m01 -= cf * kinv[3 * v + 1] / dt;"),
    ("cp1_mbar12_sign_cell_fields", "cps_oracle.c", CP1,
     "m01 = cf * kinv[3 * e + 1] / dt;\n            m11 = (1.0 + cf * kinv[3 * e + 2]) / dt;\n        }\n        out",
     "m01 = -cf * kinv[3 * e + 1] / dt;\n            m11 = (1.0 + cf * kinv[3 * e + 2]) / dt;\n        }\n        out"),
    ("cp1_cell_area_doubled", "cps_oracle.c", CP1,
     "double area = 0.5 * ((b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]));",
     "double area = 1.0 * ((b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]));"),
    ("cp1_first_sweep_dropped", "__init__.py", CP1,
     "    u = solve(Ax, Dx, lap[0], None)\n    v = solve(Ay, Dy, lap[1], None)",
     "    u = 0 * solve(Ax, Dx, lap[0], None)\n    v = 0 * solve(Ay, Dy, lap[1], None)"),
]


def _copy(work, pins):
    shutil.copytree(os.path.join(ROOT, "oracle"), work / "oracle",
                    ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    shutil.copytree(os.path.join(ROOT, "synth"), work / "synth",
                    ignore=shutil.ignore_patterns("__pycache__"))
    (work / "tests").mkdir()
    shutil.copy(os.path.join(ROOT, "tests", "conftest.py"), work / "tests")
    shutil.copy(os.path.join(ROOT, "tests", pins), work / "tests")


def _run_pins(work, pins):
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider",
                           os.path.join("tests", pins)], cwd=work, capture_output=True,
                          text=True, timeout=600)


@pytest.mark.slow
@pytest.mark.parametrize("pins", [CP2, CP1])
def test_unplanted_copy_passes_its_pins(tmp_path, pins):
    """Control: the copy itself, with nothing planted, passes every pin."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc not installed")
    work = tmp_path / "control"
    _copy(work, pins)
    r = _run_pins(work, pins)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-2000:])


@pytest.mark.slow
@pytest.mark.parametrize("name,fname,pins,old,new", MISTAKES, ids=[m[0] for m in MISTAKES])
def test_pins_catch_planted_mistake(tmp_path, name, fname, pins, old, new):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not installed")
    work = tmp_path / name
    _copy(work, pins)
    target = work / "oracle" / fname
    text = target.read_text()
    assert text.count(old) == 1, f"the planted line is not unique or missing in {fname}"
    target.write_text(text.replace(old, new))
    r = _run_pins(work, pins)
    assert r.returncode == 1 and " failed" in r.stdout, (name, r.stdout[-2000:], r.stderr[-2000:])
