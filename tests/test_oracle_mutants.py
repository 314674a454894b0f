"""The oracle's pins catch plausible mistakes (no GPU).  Each case plants one
mistake in a copy of oracle/oracle.c: a transposed operand, a wrong
neighbour index, a dropped term, a flipped sign, a wrong normalisation, in
the iteration, its variants (BGS passes, Tikhonov warm start, penalty
adaptation, vectorial TV) and the reverse pass.  It then runs the oracle's
pin suites against the mutated copy (several copies at a time) and expects
them to fail.  The real oracle is never modified."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = ["test_golden.py", "test_oracle_primitives.py", "test_oracle_admm.py", "test_oracle_variants.py",
        "test_oracle_grad.py"]

# (name, original source text, planted mistake); each original occurs once.
MUTANTS = [
    ("convolution_as_correlation",
     "xp[(size_t)(i - p + b) * W + (j - q + b)]", "xp[(size_t)(i + p + b) * W + (j + q + b)]"),
    ("difference_wrong_neighbour",
     "x[(size_t)i * N + wrap(j + 1, N)] - c;", "x[(size_t)i * N + wrap(j - 1, N)] - c;"),
    ("prox_hard_threshold",
     "double g = nrm > tau ? (nrm - tau) / nrm : 0.0;", "double g = nrm > tau ? 1.0 : 0.0;"),
    ("z_update_drops_memory_term",
     "double zn = relax * tmp[i] - (relax - 1.0) * yt[c * P + i];", "double zn = relax * tmp[i];"),
    ("x_step_rhs_sign",
     "for (size_t i = 0; i < P; ++i) rhs[i] += mu * tmp[i];",
     "for (size_t i = 0; i < P; ++i) rhs[i] -= mu * tmp[i];"),
    ("x_step_operator_without_mu",
     "s[i] = a[i] + mu * dd[i];", "s[i] = a[i] + dd[i];"),
    ("dual_update_sign",
     "double dn = a[i] - vn[i];", "double dn = vn[i] - a[i];"),
    ("fill_mean_over_every_pixel",
     "double mean = cnt ? s / (double)cnt : 0.0;", "double mean = s / (double)((size_t)M * N);"),
    ("dft_conjugated_roots",
     "double a = sign * 2.0 * M_PI * (double)k / (double)L;",
     "double a = -sign * 2.0 * M_PI * (double)k / (double)L;"),
    ("tv_separate_per_channel",
     "or_vsoft(a, (int)P, 2 * C, lambda / mu, vn);",
     "for (int c = 0; c < C; ++c) or_vsoft(a + 2 * c * P, (int)P, 2, lambda / mu, vn + 2 * c * P);"),
    ("bgs_passes_ignored",
     "for (int pass = 0; pass < passes; ++pass) {", "for (int pass = 0; pass < 1; ++pass) {"),
    ("tikhonov_tau_doubled",
     "for (size_t i = 0; i < P; ++i) s[i] = a[i] + tau * e[i];",
     "for (size_t i = 0; i < P; ++i) s[i] = a[i] + 2.0 * tau * e[i];"),
    ("penalty_rule_branches_swapped",
     "if (nd > adapt_t * nv) f = 2.0;\n      else if (nv > adapt_t * nd) f = 0.5;",
     "if (nd > adapt_t * nv) f = 0.5;\n      else if (nv > adapt_t * nd) f = 2.0;"),
    ("d_rescaled_the_wrong_way",
     "for (size_t i = 0; i < 2 * C * P; ++i) d[i] /= f;", "for (size_t i = 0; i < 2 * C * P; ++i) d[i] *= f;"),
    ("reverse_pass_drops_relax",
     "tb[c * P + i] = obs ? 0.0 : relax * yv;", "tb[c * P + i] = obs ? 0.0 : yv;"),
    ("fill_uses_the_first_plane_mask",
     "or_init_ytilde(y + c * P, mask + c * P, M, N, K, round_f32, yt + c * P);",
     "or_init_ytilde(y + c * P, mask, M, N, K, round_f32, yt + c * P);"),
    ("objective_fits_unobserved_pixels",
     "if (mask[c * P + i]) fit += (y[c * P + i] - tmp[i]) * (y[c * P + i] - tmp[i]);",
     "fit += (y[c * P + i] - tmp[i]) * (y[c * P + i] - tmp[i]);"),
    ("adapted_solve_keeps_the_old_penalty",
     "        den = solve_denominator(M, N, h, K, mu);\n      }",
     "        den = solve_denominator(M, N, h, K, mu / f);\n      }"),
    ("tikhonov_z_over_relaxed",
     "if (!mask[i]) yt[i] = tmp[i]; /* z = M_z H x */",
     "if (!mask[i]) yt[i] = 2.0 * tmp[i] - yt[i]; /* z = M_z H x */"),
    ("warm_start_v_from_the_padded_observation",
     "or_diff_fwd(x + c * P, M, N, v + 2 * c * P, v + (2 * c + 1) * P); /* v0 = D x0, x0 = warm-start x */",
     "or_diff_fwd(yt + c * P, M, N, v + 2 * c * P, v + (2 * c + 1) * P); /* v0 = D x0, x0 = warm-start x */"),
    ("reverse_pass_z_memory_sign",
     "yb[c * P + i] = obs ? yv : -(relax - 1.0) * yv;", "yb[c * P + i] = obs ? yv : (relax - 1.0) * yv;"),
    ("vertical_difference_adjoint_sign",
     "+ uv[(size_t)wrap(i - 1, M) * N + j] - uv[o];", "- uv[(size_t)wrap(i - 1, M) * N + j] + uv[o];"),
    ("band_clamp_off_by_one",
     "int ic = i < b ? b : (i >= M - b ? M - b - 1 : i);", "int ic = i < b ? b : (i >= M - b ? M - b : i);"),
    ("prox_norm_misses_the_last_plane",
     "for (int c = 0; c < dim; ++c) s += a[(size_t)c * n + j] * a[(size_t)c * n + j];",
     "for (int c = 0; c + 1 < dim; ++c) s += a[(size_t)c * n + j] * a[(size_t)c * n + j];"),
    ("dft_combine_twiddle_drops_the_block_offset",
     "w->tw[(size_t)((r * (k + q * m)) % n) * step]", "w->tw[(size_t)((r * k) % n) * step]"),
]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    """Runs the pin suites against every mutant, several at a time; returns
    {name: (exit status, end of the output)}."""
    src = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    jobs = []
    for name, old, new in MUTANTS:
        assert src.count(old) == 1, name
        d = tmp_path_factory.mktemp(name)
        (d / "oracle").mkdir()
        (d / "oracle" / "oracle.c").write_text(src.replace(old, new))
        shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), d / "oracle" / "__init__.py")
        jobs.append((name, d))
    # cwd = the copy's parent, so `import oracle` finds the mutant first.
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "--rootdir", ROOT,
           "-c", os.path.join(ROOT, "pytest.ini"), *[os.path.join(ROOT, "tests", f) for f in PINS]]
    width = max(2, min(8, (os.cpu_count() or 2) // 2))
    out, running = {}, []
    while jobs or running:
        while jobs and len(running) < width:
            name, d = jobs.pop(0)
            env = dict(os.environ, PYTHONPATH=os.pathsep.join([str(d), ROOT]), OMP_NUM_THREADS="2")
            log = open(d / "log.txt", "w")
            running.append((name, d, log, subprocess.Popen(cmd, cwd=d, env=env, stdout=log,
                                                           stderr=subprocess.STDOUT)))
        name, d, log, proc = running.pop(0)
        proc.wait(timeout=900)
        log.close()
        out[name] = (proc.returncode, (d / "log.txt").read_text()[-2000:])
    return out


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_pins_catch_a_planted_mistake(outcomes, name):
    status, tail = outcomes[name]
    assert status == 1, f"{name}: the pins did not fail (exit status {status})\n{tail}"
