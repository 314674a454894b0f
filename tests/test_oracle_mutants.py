"""The oracle's pins catch plausible mistakes (no GPU).  Each case plants one
mistake in a copy of oracle/oracle.c: a transposed operand, a wrong
neighbour index, a dropped term, a flipped sign, a wrong normalisation, in
the iteration, its variants (BGS passes, Tikhonov warm start, penalty
adaptation, vectorial TV) and the reverse pass.  It then runs the oracle's
pin suites against the mutated copy and expects them to fail.  The real
oracle is never modified."""
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
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_a_planted_mistake(tmp_path, name, old, new):
    src = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert src.count(old) == 1, name
    pkg = tmp_path / "oracle"
    pkg.mkdir()
    (pkg / "oracle.c").write_text(src.replace(old, new))
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), pkg / "__init__.py")
    # cwd = the copy's parent, so `import oracle` finds the mutant first.
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([str(tmp_path), ROOT]))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "--rootdir", ROOT, "-c", os.path.join(ROOT, "pytest.ini"),
                        *[os.path.join(ROOT, "tests", f) for f in PINS]],
                       cwd=tmp_path, env=env, capture_output=True, text=True, timeout=900)
    assert "liboracle" not in r.stderr or r.returncode != 2, r.stderr[-2000:]
    assert r.returncode == 1, f"{name}: the pins did not fail\n{r.stdout[-2000:]}"
