"""The oracle's pins catch plausible mistakes.

Each case plants one mistake (a dropped factor, a flipped sign, a wrong index
or convention) into a temporary copy of the oracle and runs the pin suite and
the hand-derived golden values against that copy in a subprocess; at least one
of them must fail.  The real
oracle is never modified.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = {
    "green_U2_coefficient": ("c2 = (lam0 + mu0) / (mu0 * (lam0 + 2.0 * mu0))",
                             "c2 = (lam0 + mu0) / (mu0 * (lam0 + 1.0 * mu0))"),
    "green_U1_sign": ("u1 = u1 - delta * pp", "u1 = u1 + delta * pp"),
    "nyquist_kept": ("k[n // 2] = 0.0                            # Nyquist index -> 0", "pass"),
    "g0_sign": ("return np.stack([(v_hat[i] - c * xi[i] * xv * iq) * iq / mu0 for i in range(3)])",
                "return np.stack([-(v_hat[i] - c * xi[i] * xv * iq) * iq / mu0 for i in range(3)])"),
    "g0_coefficient": ("c = (lam0 + mu0) / (lam0 + 2.0 * mu0)\n    xv", "c = (lam0 + mu0) / (lam0 + 1.0 * mu0)\n    xv"),
    "sym_grad_sign": ("out[a] = 0.5j * (xi[j] * u_hat[i] + xi[i] * u_hat[j])",
                      "out[a] = -0.5j * (xi[j] * u_hat[i] + xi[i] * u_hat[j])"),
    "mean_strain_dft_scale": ("eb0_hat[:, 0, 0, 0] = n * np.asarray(mean_strain, dtype=float)   # reading R3\n    table1",
                              "eb0_hat[:, 0, 0, 0] = np.asarray(mean_strain, dtype=float)   # reading R3\n    table1"),
    "cd_mean_strain_dft_scale": ("eb0_hat[:, 0, 0, 0] = n * np.asarray(mean_strain, dtype=float)   # reading R3\n    eb0",
                                 "eb0_hat[:, 0, 0, 0] = np.asarray(mean_strain, dtype=float)   # reading R3\n    eb0"),
    "displacement_scale": ('return _real(-1j * g0_apply(v, xi, lam0, mu0), "displacement")',
                           'return _real(-2j * g0_apply(v, xi, lam0, mu0), "displacement")'),
    "translation_direction": ("np.roll(field, (sz, sy, sx)", "np.roll(field, (-sz, -sy, -sx)"),
    "lame_trace_term": ("out[:3] += lam * tr", "out[:3] += 0.5 * lam * tr"),
    "shear_counted_once": ("acc = acc + (c1 * u1 + c2 * u2) * t[k][l]",
                           "acc = acc + (c1 * u1 + c2 * u2) * t[k][l] * (1.0 if k <= l else 0.0)"),
    "green_U2_dropped": ("u2 = P[i][j] * P[k][l]", "u2 = 0.0"),
    "average_normalisation": ("return acc / m, hits, infos", "return acc / (m + 1), hits, infos"),
    "body_force_sign": ("-6.0 * x * s * s / (a * a)", "6.0 * x * s * s / (a * a)"),
    "body_force_power": ("-6.0 * x * s * s / (a * a)", "-6.0 * x * s / (a * a)"),
    "body_force_without_minimum_image": ("        return d - n * np.round(d / n)", "        return d"),
    "green_U1_coefficient": ("c1 = 1.0 / (4.0 * mu0)", "c1 = 1.0 / (2.0 * mu0)"),
    "residual_normaliser_shear_once": ("\n    s0n = np.sqrt(np.sum(np.abs(s0[:3]) ** 2) + 2.0 * np.sum(np.abs(s0[3:]) ** 2))",
                                       "\n    s0n = np.sqrt(np.sum(np.abs(s0[:3]) ** 2) + np.sum(np.abs(s0[3:]) ** 2))"),
    "cd_residual_normaliser_shear_once": ("        s0n = np.sqrt(np.sum(np.abs(s0[:3]) ** 2) + 2.0 * np.sum(np.abs(s0[3:]) ** 2))",
                                          "        s0n = np.sqrt(np.sum(np.abs(s0[:3]) ** 2) + np.sum(np.abs(s0[3:]) ** 2))"),
    "residual_xi_min_of_shortest_edge": ("\n    den = np.sqrt(np.sum(np.abs(b_hat[:, act]) ** 2)) + 2.0 * np.pi / max(dims) * s0n",
                                         "\n    den = np.sqrt(np.sum(np.abs(b_hat[:, act]) ** 2)) + 2.0 * np.pi / min(dims) * s0n"),
    "wavevector_of_the_x_edge": ("        out.append(2.0 * np.pi * k / n)", "        out.append(2.0 * np.pi * k / dims[0])"),
    "phase_map_without_minimum_image": ("        return np.where(d >= n, d - 2 * n, d)", "        return d"),
    "initial_strain_zero": ('        eps = _real(eb0_hat, "eps0")', '        eps = np.zeros_like(_real(eb0_hat, "eps0"))'),
    "kernel_gradient_without_tikhonov": ("grad = 2.0 * (G @ c - g + lam * c)", "grad = 2.0 * (G @ c - g)"),
    "kernel_loss_without_constant": ("J = float(c @ G @ c - 2 * g @ c + s + lam * c @ c)",
                                     "J = float(c @ G @ c - 2 * g @ c + lam * c @ c)"),
    "kernel_radius_unscaled": ("K = coef @ bernstein(coef.size - 1, d / delta)", "K = coef @ bernstein(coef.size - 1, d)"),
    "concentration_over_matrix": ('As[:, J] = res["eps"][:, incl].mean(axis=1)',
                                  'As[:, J] = res["eps"][:, ~incl].mean(axis=1)'),
    "adam_second_moment_without_bias_correction": ("vh = v / (1 - betas[1] ** t)", "vh = v"),
    "displacement_without_lame_term": ("lam_tr = lam0 * (eps[0] + eps[1] + eps[2])",
                                       "lam_tr = 0.0 * (eps[0] + eps[1] + eps[2])"),
    "g0_projection_sign": ("(v_hat[i] - c * xi[i] * xv * iq) * iq / mu0", "(v_hat[i] + c * xi[i] * xv * iq) * iq / mu0"),
    "reference_strain_sign": ("return sym_grad_hat(g0_apply(b_hat, xi, lam0, mu0), xi)",
                              "return -sym_grad_hat(g0_apply(b_hat, xi, lam0, mu0), xi)"),
    "translation_axes_swapped": ("np.roll(field, (sz, sy, sx), axis=(-3, -2, -1))",
                                 "np.roll(field, (sx, sy, sz), axis=(-3, -2, -1))"),
    "residual_over_all_modes": ("act = np.broadcast_to(q > 0, sig_hat.shape[1:])",
                                "act = np.broadcast_to(q >= 0, sig_hat.shape[1:])"),
    "stress_of_the_reference_medium": ("b_hat, xi)\n    sig = apply_local(phase, table, eps)\n    u = displacement",
                                       "b_hat, xi)\n    sig = apply_local(phase, [c0] * len(table), eps)\n    u = displacement"),
    "sphere_boundary_exclusive": ("ph[d2 <= T] = p", "ph[d2 < T] = p"),
    "residual_misses_load": ("div = div_hat(sig_hat, xi) + b_hat", "div = div_hat(sig_hat, xi)"),
    "moduli_engineering_shear": ("    E[J] = 1.0\n", "    E[J] = 1.0 if J < 3 else 0.5\n"),
    "concentration_over_all_voxels": ('As[:, J] = res["eps"][:, incl].mean(axis=1)',
                                      'As[:, J] = res["eps"].reshape(6, -1).mean(axis=1)'),
    "ensemble_indicator_of_first_configuration": ("        v = (ph != 0).astype(float)\n        acc[0:3] += res[\"u\"]\n        acc[3:6] += v * res[\"u\"]\n        acc[6:12] += res[\"eps\"]\n        acc[12:18] += v * res[\"eps\"]\n        acc[18:24] += res[\"sig\"]\n        acc[24:30] += v * res[\"sig\"]\n        hits += (ph != 0)\n        infos.append((res[\"sweeps\"], res[\"resid\"]))\n    return acc / len(configs)",
                                                  "        v = (configs[0] != 0).astype(float)\n        acc[0:3] += res[\"u\"]\n        acc[3:6] += v * res[\"u\"]\n        acc[6:12] += res[\"eps\"]\n        acc[12:18] += v * res[\"eps\"]\n        acc[18:24] += res[\"sig\"]\n        acc[24:30] += v * res[\"sig\"]\n        hits += (ph != 0)\n        infos.append((res[\"sweeps\"], res[\"resid\"]))\n    return acc / len(configs)"),
    "radial_shell_rounded_up": ("shell = np.floor(np.sqrt(D2.astype(np.float64)) / 2.0)",
                                "shell = np.ceil(np.sqrt(D2.astype(np.float64)) / 2.0)"),
    "radial_shear_counted_once": ("w = np.array([1.0, 1.0, 1.0, 2.0, 2.0, 2.0] if ncomp == 6",
                                  "w = np.array([1.0, 1.0, 1.0, 1.0, 1.0, 1.0] if ncomp == 6"),
    "rve_radius_off_by_one": ("rp = 0 if above.size == 0 else int(above[-1]) + 1",
                              "rp = 0 if above.size == 0 else int(above[-1])"),
    "rve_containment_without_annulus": ("ok = r is not None and r + a / 2.0 <= n / 2.0",
                                        "ok = r is not None and r <= n / 2.0"),
    "kernel_operator_sign": ("out += k * (np.roll(u, (-oz, -oy, -ox), axis=(-3, -2, -1)) - u)",
                             "out += k * (u - np.roll(u, (-oz, -oy, -ox), axis=(-3, -2, -1)))"),
    "horizon_inclusive": ("keep = (d > 0) & (d < delta)", "keep = (d > 0) & (d <= delta)"),
    "adam_without_bias_correction": ("mh = m1 / (1 - betas[0] ** t)", "mh = m1"),
    "tikhonov_dropped": ("exact = np.linalg.solve(G + lam * np.eye(n), g)", "exact = np.linalg.solve(G, g)"),
    "stiffness_over_inclusions": ('Ls[:, J] = res["sig"].reshape(6, -1).mean(axis=1)',
                                  'Ls[:, J] = res["sig"][:, incl].mean(axis=1)'),
    "cd_rhs_with_full_stiffness": ("bA = div_hat(fft3(apply_local(phase, table1, eb0)), xi)",
                                   "bA = div_hat(fft3(apply_local(phase, table, eb0)), xi)"),
    "cd_operator_sign": ("    return -div_hat(fft3(apply_local(phase, table, eps)), xi)",
                         "    return div_hat(fft3(apply_local(phase, table, eps)), xi)"),
    "cd_beta_of_old_residual": ("            beta = rz_new / rz                                      # Eq. 5.21",
                                "            beta = rz / rz_new                                      # Eq. 5.21"),
    "cd_residual_update_sign": ("            r = r - alpha * q                                       # Eq. 5.20",
                                "            r = r + alpha * q                                       # Eq. 5.20"),
    "cd_direction_from_unpreconditioned_residual": ("            p = z + beta * p                                        # Eq. 5.22",
                                                    "            p = r + beta * p                                        # Eq. 5.22"),
}


def run_pins(tmp_path, src):
    (tmp_path / "oracle").mkdir()
    (tmp_path / "oracle" / "__init__.py").write_text("")
    (tmp_path / "oracle" / "bfcs_oracle.py").write_text(src)
    (tmp_path / "tests").mkdir()
    shutil.copy(os.path.join(ROOT, "tests", "test_oracle_pins.py"), tmp_path / "tests")
    shutil.copy(os.path.join(ROOT, "tests", "test_golden.py"), tmp_path / "tests")
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), tmp_path / "tests" / "golden")
    # one thread per child: the children run side by side
    env = dict(os.environ, PYTHONPATH=str(tmp_path), OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
               MKL_NUM_THREADS="1")
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                           "-W", "ignore::pytest.PytestUnknownMarkWarning",
                           "tests/test_oracle_pins.py", "tests/test_golden.py"], cwd=tmp_path, env=env,
                          capture_output=True, text=True, timeout=900)


@pytest.fixture(scope="module")
def mutated_runs(tmp_path_factory):
    """Every planted mistake run once, the children concurrently (one per core);
    the parametrised tests below read their outcomes."""
    src = open(os.path.join(ROOT, "oracle", "bfcs_oracle.py")).read()

    def one(name):
        before, after = MUTATIONS[name]
        if src.count(before) != 1:
            return name, None
        return name, run_pins(tmp_path_factory.mktemp(name), src.replace(before, after))

    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        return dict(ex.map(one, sorted(MUTATIONS)))


def test_unmutated_copy_passes(tmp_path):
    """Control: the copied pin suite runs and passes on the real oracle alone."""
    r = run_pins(tmp_path, open(os.path.join(ROOT, "oracle", "bfcs_oracle.py")).read())
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, mutated_runs):
    r = mutated_runs[name]
    assert r is not None, "mutation anchor drifted"
    assert r.returncode != 0, f"planted mistake {name!r} passed every pin:\n{r.stdout[-2000:]}"
    # caught by a failing pin, not by an import or collection error
    assert r.returncode == 1 and " failed" in r.stdout and " error" not in r.stdout, r.stdout[-2000:]
