"""The pins of the oracle catch plausible mistakes.

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
GEO = "test_oracle_geometry.py"
ASM = "test_oracle_assembly.py"
SOL = "test_oracle_solve.py"
ADJ = "test_oracle_adjoint.py"

MISTAKES = [
    # geometry (Sec. 3.1, Eq. cs1_discr)
    ("circumcentre_sign", "cps_oracle.c", GEO,
     "cc[2 * e + 0] = a[0] + (cy * b2 - by * c2) / (2.0 * cross);",
     "cc[2 * e + 0] = a[0] + (by * c2 - cy * b2) / (2.0 * cross);"),
    ("inward_normals", "cps_oracle.c", GEO,
     "double nx = ty / l, ny = -tx / l; /* outward for a CCW triangle */",
     "double nx = -ty / l, ny = tx / l; /* outward for a CCW triangle */"),
    ("boundary_distance_halved", "cps_oracle.c", GEO,
     "d = (mx - cc[2 * e]) * nx + (my - cc[2 * e + 1]) * ny;",
     "d = 0.5 * ((mx - cc[2 * e]) * nx + (my - cc[2 * e + 1]) * ny);"),
    # Xi (Eq. Cs2_4) and assembly (Eq. CS2_sys_coeff, Eq. CS1_sys_coeff)
    ("xi_determinant_sign", "cps_oracle.c", ASM,
     "double det = m00 * m11 - m01 * m01;", "double det = m00 * m11 + m01 * m01;"),
    ("xi_offdiagonal_sign", "cps_oracle.c", ASM,
     "xi[1] = -s * m01;", "xi[1] = s * m01;"),
    ("transmissibility_times_distance", "cps_oracle.c", ASM,
     "T[s] = len[s] * dn / d;", "T[s] = len[s] * dn * d;"),
    ("side_tensor_from_one_node", "cps_oracle.c", ASM,
     "for (int c = 0; c < 3; ++c) xs[c] = 0.5 * (xa[c] + xb[c]);\n                } else if (ep >= 0) {",
     "for (int c = 0; c < 3; ++c) xs[c] = xa[c];\n                } else if (ep >= 0) {"),
    ("cp1_mass_mean_over_two_nodes", "cps_oracle.c", ASM,
     "mkk /= 3.0;", "mkk /= 2.0;"),
    ("dirichlet_side_ignored", "cps_oracle.c", ASM,
     "if (ep < 0 && !is_dirichlet[s]) continue; /* no-flux side */",
     "if (ep < 0) continue; /* no-flux side */"),
    # solves (Sec. 3.2.2: PCG with incomplete Cholesky)
    ("cg_beta_inverted", "cps_oracle.c", SOL,
     "double beta = rho_new / rho;", "double beta = rho / rho_new;"),
    ("ic0_pivot_not_square_rooted", "cps_oracle.c", SOL,
     "f->v[dpos] = sqrt(s);", "f->v[dpos] = s;"),
    ("ic0_offdiagonal_not_scaled", "cps_oracle.c", SOL,
     "f->v[p] = s / f->v[f->rp[kk + 1] - 1];", "f->v[p] = s;"),
    ("dense_cholesky_diagonal", "cps_oracle.c", SOL,
     "double ljj = sqrt(s);", "double ljj = s;"),
    # adjoint (derived from Eq. CS2_sys_coeff)
    ("side_gradient_sign", "cps_oracle.c", ADJ,
     "if (ep >= 0) dT[s] = -(lambda[e] - lambda[ep]) * (x[e] - x[ep]);",
     "if (ep >= 0) dT[s] = (lambda[e] - lambda[ep]) * (x[e] - x[ep]);"),
    ("theta_chain_factor", "cps_oracle.c", ADJ,
     "double dxi = xi * s / (1.0 + s);", "double dxi = xi / (1.0 + s);"),
    ("interior_side_half_weight_dropped", "cps_oracle.c", ADJ,
     "if (nbr[k] >= 0) g += dT[k] * len[k] / (2.0 * dist[k]);",
     "if (nbr[k] >= 0) g += dT[k] * len[k] / dist[k];"),
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


def _run_pins(work, pins, first_failure=False):
    args = [sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider"]
    if first_failure:
        args.append("-x")                     # one failing pin is enough
    return subprocess.run(args + [os.path.join("tests", pins)], cwd=work, capture_output=True,
                          text=True, timeout=600)


@pytest.mark.slow
@pytest.mark.parametrize("pins", [CP2, CP1, GEO, ASM, SOL, ADJ])
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
    r = _run_pins(work, pins, first_failure=True)
    assert r.returncode == 1 and " failed" in r.stdout, (name, r.stdout[-2000:], r.stderr[-2000:])
