"""The oracle pins have teeth: plausible mistakes planted in copies of the
oracle's C source (CPU only) must each fail at least one pin."""
import importlib.util
import os
import shutil

import pytest

import test_oracle_pins as pins

ORACLE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")

MUTANTS = {
    "y_uses_x_spacing": ("double d2y = (T[p + sy] - c) - (c - T[p - sy]);\n    double d2z",
                         "double d2y = (T[p + sx] - c) - (c - T[p - sx]);\n    double d2z"),
    "dropped_z_term": ("return (d2x * _dx2 + d2y * _dy2) + d2z * _dz2;",
                       "return (d2x * _dx2 + d2y * _dy2);"),
    "wrong_update_sign": ("T2[p] = T[p] + dt * ((lam * Ci[p]) * lap);",
                          "T2[p] = T[p] - dt * ((lam * Ci[p]) * lap);"),
    "ci_index_shift": ("T2[p] = T[p] + dt * ((lam * Ci[p]) * lap);",
                       "T2[p] = T[p] + dt * ((lam * Ci[p + 1]) * lap);"),
    "adjoint_spacing_swapped": ("Tbar[p] = ybar[p] + ((d2x * _dx2 + d2y * _dy2) + d2z * _dz2);",
                                "Tbar[p] = ybar[p] + ((d2x * _dy2 + d2y * _dx2) + d2z * _dz2);"),
    "adjoint_w_not_masked": ("for (int64_t i = 1; i < nx - 1; ++i) {\n                int64_t q = i + nx * (j + ny * k);\n                w[q]",
                             "for (int64_t i = 0; i < nx; ++i) {\n                int64_t q = i + nx * (j + ny * k);\n                w[q]"),
    "cibar_missing_lam": ("Cibar[q] += (dt * lam) * (ybar[q] * lap);",
                          "Cibar[q] += dt * (ybar[q] * lap);"),
    "dt_uses_max_spacing": ("if (dy * dy < m) m = dy * dy;", "if (dy * dy > m) m = dy * dy;"),
}

PIN_CALLS = [
    lambda o: pins.test_golden_constant_field_stays_bitwise(o),
    lambda o: pins.test_eigenmode_decay_factor(o, (17, 12, 9), (2, 1, 3), 0.0),
    lambda o: pins.test_eigenmode_decay_factor(o, (10, 14, 19), (3, 2, 1), 1.7),
    lambda o: pins.test_dense_matrix_forward(o, (5, 7, 6), 7),
    lambda o: pins.test_dense_matrix_adjoint(o, (5, 7, 6)),
    lambda o: pins.test_adjoint_dot_product(o),
    lambda o: pins.test_complex_step_gradient(o),
    lambda o: pins.test_stable_dt_paper_setup_and_max_principle(o),
]


def load_mutant(tmp_path, name, old, new):
    d = tmp_path / f"oracle_{name}"
    shutil.copytree(ORACLE_DIR, d, ignore=shutil.ignore_patterns("_build", "__pycache__"))
    src = d / "diffusion3d_oracle.c"
    text = src.read_text()
    assert old in text, f"mutant {name}: pattern not found"
    src.write_text(text.replace(old, new, 1))
    spec = importlib.util.spec_from_file_location(f"oracle_mutant_{name}", d / "__init__.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build(force=True)
    return mod


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    mod = load_mutant(tmp_path, name, old, new)
    caught = 0
    for call in PIN_CALLS:
        try:
            call(mod)
        except (AssertionError, FloatingPointError, ValueError):
            caught += 1
    assert caught >= 1, f"no pin caught the planted mistake {name}"
