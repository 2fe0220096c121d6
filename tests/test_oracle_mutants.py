"""The oracle's pins catch plausible mistakes: each case builds a copy of the oracle with one
planted mistake (on the CPU, in a temporary directory) and checks that the pin aimed at that
part of the method fails on it, while the same pin passes on the real oracle."""
import importlib.util
import os
import shutil
import sys

import pytest

from conftest import ROOT

import test_oracle_pins as pins

# (what is wrong, exact source text, replacement, pin that must fail, pin arguments)
MUTANTS = [
    ("KPM recurrence adds w_{k-1}",
     "for (int64_t i = 0; i < n; i++) w2[i] = 2.0 * w2[i] - w0[i];\n            mu[k + 1]",
     "for (int64_t i = 0; i < n; i++) w2[i] = 2.0 * w2[i] + w0[i];\n            mu[k + 1]",
     pins.test_kpm_exact_on_diagonal_matrix, ()),
    ("slicer without interpolation between grid points",
     "sli[i] = x[j - 1] + f * (x[j] - x[j - 1]);", "sli[i] = x[j];",
     pins.test_slicer_ends_hit_the_quantiles_of_the_interpolated_count, ()),
    ("quadrature slicer cuts at the node",
     "sli[s] = 0.5 * (prev + t[p]);", "sli[s] = t[p];",
     pins.test_slicer_landos_hand_computed_cuts, ()),
    ("pencil KPM without B in the starting vector",
     "        orc_matvec(&B, u, y0);                                                   /* y_0 = B u */",
     "        memcpy(y0, u, sizeof(double) * n);",
     pins.test_kpm_gen_matches_dense_pencil_formula, ()),
    ("pencil thick restart without locked deflation",
     "        for (int j = 0; j < nlock; j++) {\n            const double h = orc_dot(n, z, U + (size_t)j * n);\n"
     "            for (int64_t r = 0; r < n; r++) z[r] -= h * BU[(size_t)j * n + r];\n        }",
     "",
     pins.test_cheblantr_gen_restarts_against_closed_form, (2.0, 3.0, 40)),
]


def _mutant_oracle(tmp_path, old, new, tag):
    src = os.path.join(ROOT, "oracle")
    dst = tmp_path / f"oracle_{tag}"
    shutil.copytree(src, dst, ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    c = dst / "evsl_oracle.c"
    text = c.read_text()
    assert text.count(old) == 1, "mutation site not found exactly once"
    c.write_text(text.replace(old, new))
    name = f"oracle_mutant_{tag}"
    spec = importlib.util.spec_from_file_location(name, dst / "__init__.py",
                                                  submodule_search_locations=[str(dst)])
    mod = importlib.util.module_from_spec(spec)
    sys.modules[name] = mod
    spec.loader.exec_module(mod)
    mod.build(force=True)
    return mod


@pytest.mark.parametrize("case", range(len(MUTANTS)), ids=[m[0] for m in MUTANTS])
def test_pin_fails_on_planted_mistake(tmp_path, oracle_mod, case):
    what, old, new, pin, args = MUTANTS[case]
    pin(oracle_mod, *args)                      # passes on the oracle itself
    mutant = _mutant_oracle(tmp_path, old, new, str(case))
    with pytest.raises(AssertionError):
        pin(mutant, *args)
