"""Mutation check of the oracle pins.

Each case plants one plausible mistake in a copy of the oracle source (a
dropped term, a wrong sign, a swapped index, a transposed operand), builds it
on the CPU, and runs the pin suite against it: the pins must fail for every
mutant. The real oracle is never modified.
"""
import concurrent.futures as cf
import os
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "gl_oracle.cpp")

MUTANTS = {
    "rotation_sign": ("yp = -s * dx + c * dy;", "yp = s * dx + c * dy;"),
    "rotate_back_sign": ("ax = c * alx - s * aly;", "ax = c * alx + s * aly;"),
    "series_coefficient": ("(2.0 * n - (2.0 - t)) / (2.0 * n + (2.0 - t))", "(2.0 * n - (2.0 - t)) / (2.0 * n + (2.0 + t))"),
    "series_sign": ("const T cn = -f *", "const T cn = f *"),
    "epl_b_scale": ("const T b = thetaE * sqrt(q);", "const T b = thetaE;"),
    "epl_power": ("pow(b / R, t - 1.0)", "pow(b / R, t)"),
    "phi_half_angle": ("phi = 0.5 * atan2(e2, e1);", "phi = atan2(e2, e1);"),
    "q_of_e": ("q = (1.0 - e) / (1.0 + e);", "q = 1.0 - e;"),
    "shear_sign": ("ay = g2 * x - g1 * y;", "ay = g2 * x + g1 * y;"),
    "shear_swap": ("ax = g1 * x + g2 * y;", "ax = g1 * y + g2 * x;"),
    "sersic_bn": ("1.9992 * l[1] - 0.3271", "1.9992 * l[1] + 0.3271"),
    "sersic_axis_ratio": ("sqrt(q * xl * xl + yl * yl / q)", "sqrt(xl * xl / q + q * yl * yl)"),
    "sersic_index": ("pow(rho / l[0], 1.0 / l[1])", "pow(rho / l[0], l[1])"),
    "lens_light_at_beta": ("return sersic(bx, by, p + 15) + sersic(T(x), T(y), p + 8);",
                           "return sersic(bx, by, p + 15) + sersic(bx, by, p + 8);"),
    "grid_transpose": ("const double x = (j * k + b - cx) * sub;", "const double x = (i * k + a - cx) * sub;"),
    "grid_offset": ("const double cx = (k * W - 1) * 0.5", "const double cx = (k * W) * 0.5"),
    "binning_norm": ("out[i * W + j] = acc / double(k * k);", "out[i * W + j] = acc / double(k);"),
    "pixel_area_dropped": ("pre[i] = pre[i] * area;", "pre[i] = pre[i];"),
    "pixel_area_subpixel": ("const double area = s.dpix * s.dpix;", "const double area = s.dpix * s.dpix / (s.k * s.k);"),
    "conv_no_flip": ("const int ii = i + c - a;", "const int ii = i - c + a;"),
    "conv_transpose": ("acc += psf[a * K + b] * img[ii * W + jj];", "acc += psf[b * K + a] * img[ii * W + jj];"),
    "poisson_term": ("var = var + model[i] / s.gain_exposure;", "var = var + model[i] * s.gain_exposure;"),
    "loglik_norm": ("ll += -0.5 * (c2 + log(2.0 * PI * var));", "ll += -0.5 * (c2 + log(var));"),
    "dual_product_rule": ("r.d[i] = a.d[i] * b.v + a.v * b.d[i];", "r.d[i] = a.d[i] * b.v;"),
    "dual_quotient": ("r.d[i] = (a.d[i] - r.v * b.d[i]) * inv;", "r.d[i] = (a.d[i] + r.v * b.d[i]) * inv;"),
}


def _run_mutant(name, old, new, tmp):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor for %s not unique/present" % name
    path = os.path.join(tmp, name + ".cpp")
    lib = os.path.join(tmp, name + ".so")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    subprocess.run(["g++", "-std=c++17", "-O1", "-fopenmp", "-fPIC", "-shared", path, "-o", lib], check=True)
    env = dict(os.environ, GL_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return name, r.returncode


def test_every_planted_mistake_fails_a_pin():
    with tempfile.TemporaryDirectory() as tmp:
        with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
            futs = [ex.submit(_run_mutant, n, o, w, tmp) for n, (o, w) in MUTANTS.items()]
            results = dict(f.result() for f in futs)
    survivors = [n for n, rc in results.items() if rc == 0]
    assert not survivors, "mutants not caught by any pin: %s" % survivors


MAP_MUTANTS = {
    "prior_sd": ('("normal", 0.0, 0.06), ("normal", 0.0, 0.06),  # x_epl, y_epl',
                 '("normal", 0.0, 0.03), ("normal", 0.0, 0.06),  # x_epl, y_epl'),
    "lognormal_grad": ("g[:, j] = -(np.log(x) - math.log(e[1])) / (e[2] ** 2 * x) - 1.0 / x",
                       "g[:, j] = -(np.log(x) - math.log(e[1])) / (e[2] ** 2 * x)"),
    "sigmoid_jacobian": ("dlj[:, j] = 1.0 - 2.0 * s", "dlj[:, j] = 2.0 * s - 1.0"),
    "objective_drops_logJ": ("f = -(np.asarray(loglik_theta) + lp + lj)", "f = -(np.asarray(loglik_theta) + lp)"),
    "gradient_drops_dlogJ": ("g = -((np.asarray(grad_theta) + glp) * d + dlj)", "g = -((np.asarray(grad_theta) + glp) * d)"),
    "adam_no_bias_correction": ("mhat = m / (1.0 - ADAM_B1 ** t)", "mhat = m"),
    "schedule_reversed": ("return LR_START + (LR_END - LR_START) * frac", "return LR_END + (LR_START - LR_END) * frac"),
    "sigmoid_bounds": ('return ("sigmoid", entry[3], entry[4])', 'return ("sigmoid", entry[4], entry[3])'),
}


def _run_map_mutant(name, old, new, tmp, module="map_oracle.py", test="test_map_oracle.py"):
    import shutil
    dst = os.path.join(tmp, name)
    for part in ("oracle", "tests", "paper_2202_07663_gb300"):   # what the oracle's tests import
        shutil.copytree(os.path.join(ROOT, part), os.path.join(dst, part),
                        ignore=shutil.ignore_patterns("*.so", "_build", "__pycache__", ".pytest_cache"))
    path = os.path.join(dst, "oracle", module)
    src = open(path).read()
    assert src.count(old) == 1, "mutation anchor for %s not unique/present" % name
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    import oracle as real
    env = dict(os.environ, GL_ORACLE_LIB=real.build())
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(dst, "tests", test)],
                       cwd=dst, env=env, capture_output=True, text=True, timeout=600)
    return name, r.returncode


def test_every_planted_map_mistake_fails_a_pin():
    with tempfile.TemporaryDirectory() as tmp:
        with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
            futs = [ex.submit(_run_map_mutant, n, o, w, tmp) for n, (o, w) in MAP_MUTANTS.items()]
            results = dict(f.result() for f in futs)
    survivors = [n for n, rc in results.items() if rc == 0]
    assert not survivors, "MAP mutants not caught by any pin: %s" % survivors


VI_MUTANTS = {
    "diagonal_not_exponentiated": ("L[i, j] = math.exp(phi[k]) if i == j else phi[k]", "L[i, j] = phi[k]"),
    "score_drops_log_q": ("    f = log_q(z, mu, L) - np.asarray(logp, np.float64)\n    return f.mean(), (f[:, None]",
                          "    f = -np.asarray(logp, np.float64)\n    return f.mean(), (f[:, None]"),
    "pathwise_entropy_sign": ("- np.diag(1.0 / np.diag(L))\n    return f.mean(), _to_u",
                              "+ np.diag(1.0 / np.diag(L))\n    return f.mean(), _to_u"),
    "pathwise_mu_sign": ("gmu = -gz.mean(axis=0)", "gmu = gz.mean(axis=0)"),
    "score_factor_order": ("np.outer(a, w)", "np.outer(w, a)"),
    "chain_rule_drops_diagonal": ("            out.append(gL[i, j] * L[i, i] if i == j else gL[i, j])",
                                  "            out.append(gL[i, j])"),
    "log_q_drops_2pi": ("- logdet_L - 0.5 * d * math.log(2.0 * math.pi)", "- logdet_L"),
    "log_q_logdet_sign": ("- logdet_L - 0.5", "+ logdet_L - 0.5"),
    "schedule_linear": ("return LR_PEAK - LR_PEAK * (1.0 - frac) ** 2", "return LR_PEAK * frac"),
    "sigma_init": ("SIGMA_INIT = 1e-6", "SIGMA_INIT = 1e-4"),
    "pathwise_eps_transposed": ("gL = np.tril(-(gz.T @ eps)", "gL = np.tril(-(eps.T @ gz)"),
}


def test_every_planted_vi_mistake_fails_a_pin():
    with tempfile.TemporaryDirectory() as tmp:
        with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
            futs = [ex.submit(_run_map_mutant, n, o, w, tmp, "vi_oracle.py", "test_vi_oracle.py")
                    for n, (o, w) in VI_MUTANTS.items()]
            results = dict(f.result() for f in futs)
    survivors = [n for n, rc in results.items() if rc == 0]
    assert not survivors, "VI mutants not caught by any pin: %s" % survivors


HMC_MUTANTS = {
    "chees_drops_jitter_factor": ("grad += w[cidx] * t * a * c", "grad += w[cidx] * a * c"),
    "chees_velocity_sign": ("c = np.sum((q_prop[cidx] - mp) * v_prop[cidx])",
                            "c = -np.sum((q_prop[cidx] - mp) * v_prop[cidx])"),
    "chees_previous_uncentred": ("np.sum((q_prev[cidx] - m) ** 2)", "np.sum(q_prev[cidx] ** 2)"),
    "chees_criterion_scale": ("crit += w[cidx] * 0.25 * a * a", "crit += w[cidx] * 0.5 * a * a"),
    "chees_unweighted": ("grad += w[cidx] * t * a * c", "grad += t * a * c"),
    "halton_first_digit": ("out, f = 0.0, 1.0 / base", "out, f = 0.0, 0.5 / base"),
}


def test_every_planted_hmc_mistake_fails_a_pin():
    with tempfile.TemporaryDirectory() as tmp:
        with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
            futs = [ex.submit(_run_map_mutant, n, o, w, tmp, "hmc_oracle.py", "test_hmc_oracle.py")
                    for n, (o, w) in HMC_MUTANTS.items()]
            results = dict(f.result() for f in futs)
    survivors = [n for n, rc in results.items() if rc == 0]
    assert not survivors, "HMC mutants not caught by any pin: %s" % survivors


VARIANT_MUTANTS = {
    "variance_not_clipped": ("np.maximum(image, 0.0) / gain_exposure", "image / gain_exposure"),
    "solve_unweighted": ("w = 1.0 / np.asarray(var, np.float64)", "w = np.ones_like(np.asarray(var, np.float64))"),
    "rhs_swapped": ("r = np.array([np.sum(w * A[b, i] * D) for i in range(2)])",
                    "r = np.array([np.sum(w * A[b, 1 - i] * D) for i in range(2)])"),
    "basis_swapped": ("pl[:, I_L], pl[:, I_S] = 1.0, 0.0", "pl[:, I_L], pl[:, I_S] = 0.0, 1.0"),
    "amplitude_gradient_kept": ("        g[:, I_L] = 0.0\n", "        g[:, I_L] = g[:, I_L]\n"),
    "singular_keeps_weaker": ("i = max(live, key=lambda j: G[j, j])", "i = min(range(2), key=lambda j: G[j, j])"),
}


def test_every_planted_variant_mistake_fails_a_pin():
    with tempfile.TemporaryDirectory() as tmp:
        with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
            futs = [ex.submit(_run_map_mutant, n, o, w, tmp, "variant_oracle.py", "test_variant_oracle.py")
                    for n, (o, w) in VARIANT_MUTANTS.items()]
            results = dict(f.result() for f in futs)
    survivors = [n for n, rc in results.items() if rc == 0]
    assert not survivors, "variant mutants not caught by any pin: %s" % survivors
