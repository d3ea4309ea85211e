"""Plants typical mistakes in a copy of the oracle (on the CPU) and checks
that the pins catch each one: a dropped term, a wrong sign, a wrong index, a
transposed operand, a missing normalisation.  Each mutant is compiled to a
temporary library and the named pins are run against it in a subprocess."""
import os
import subprocess
import sys

import pytest

from oracle import oracle as o

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PHYS = "tests/test_oracle_physics.py"
PRIM = "tests/test_oracle_primitives.py"
GAUSS = "tests/test_oracle_gauss.py"

MUTANTS = [
    ("drop ln R~ from ln Q (Eq. (2))",
     "log(Qp) - log((double)R) - dbeta", "log(Qp) - dbeta",
     [f"{PHYS}::test_pa_matches_exact_enumeration"]),
    ("drop the E_min shift from ln Q",
     "- dbeta * (double)Emin;", ";",
     [f"{PHYS}::test_pa_matches_exact_enumeration"]),
    ("reweight with the wrong temperature difference (Eq. (1))",
     "double w = or_pexp(-(dbeta * (double)(E[j] - Emin)));",
     "double w = or_pexp(-((dbeta + 1.0) * (double)(E[j] - Emin)));",
     [f"{PHYS}::test_pa_matches_exact_enumeration"]),
    ("no division by Q' in the Poisson mean",
     "double a = ((double)R_target * w) / Qp;", "double a = ((double)R_target * w);",
     [f"{PHYS}::test_population_total_tracks_target"]),
    ("wrong sign of the energy change",
     "int dE = -2 * sig[i] * h;", "int dE = 2 * sig[i] * h;",
     [f"{PHYS}::test_metropolis_sweeps_sample_boltzmann_distribution"]),
    ("wrong threshold index",
     "< thr[dE / 2]) flip = 1;", "< thr[dE / 4 + 1]) flip = 1;",
     [f"{PHYS}::test_metropolis_sweeps_sample_boltzmann_distribution"]),
    ("transposed operands in the Poisson recurrence",
     "P = (P * am) / (double)k;", "P = (P * (double)k) / am;",
     [f"{PRIM}::test_poisson_piece_matches_pmf_on_stratified_grid"]),
    ("ln Omega written as N",
     "r->mbF = (double)N * 0x1.62e42fefa39efp-1;", "r->mbF = (double)N;",
     [f"{PHYS}::test_init_invariants_3d"]),
    ("Taylor polynomial truncated",
     "#define PEXP_DEGREE 13", "#define PEXP_DEGREE 9",
     [f"{PRIM}::test_pexp_within_two_ulp_of_exact"]),
    ("Philox with nine rounds",
     "for (int round = 0; round < 10; round++)", "for (int round = 0; round < 9; round++)",
     [f"{PRIM}::test_philox_matches_triton_reference"]),
    ("R^(r) factor ignored in the weights",
     "double y = x[r] + (Rw ? log(Rw[r]) : 0.0);\n    double e", "double y = x[r];\n    double e",
     [f"{PRIM}::test_weighted_average_closed_forms"]),
    ("1/M dropped from Eq. (7)",
     "*mbFbar = mux + log(Sx) - log((double)M);", "*mbFbar = mux + log(Sx);",
     [f"{PRIM}::test_weighted_average_closed_forms"]),
    ("pair weight from the first run only (Eq. (11))",
     "    double x = x1[r] + x2[r];\n    double y = x;\n    if (R1) y = y + log(R1[r]) + log(R2[r]);\n    double e",
     "    double x = x1[r];\n    double y = x;\n    if (R1) y = y + log(R1[r]) + log(R2[r]);\n    double e",
     [f"{PRIM}::test_pair_weighted_average_closed_forms"]),
    ("second population factor dropped from the pair weight",
     "    if (R1) y = y + log(R1[r]) + log(R2[r]);\n    double e",
     "    if (R1) y = y + log(R1[r]);\n    double e",
     [f"{PRIM}::test_pair_weighted_average_closed_forms"]),
    ("overlap of a replica with itself",
     "dot += a->spins[i * N + k] * b->spins[i * N + k];",
     "dot += a->spins[i * N + k] * a->spins[i * N + k];",
     [f"{PHYS}::test_overlap_exact_cases"]),
    ("sweep counter not advanced between sweeps",
     "uint32_t T = (uint32_t)(T0 + t);", "uint32_t T = (uint32_t)(T0);",
     [f"{PHYS}::test_metropolis_sweeps_sample_boltzmann_distribution"]),
]


GAUSS_MUTANTS = [
    ("Gaussian: E_min shift dropped from ln Q",
     "- dbeta * ((double)Emin * OG_INV_SCALE);", ";",
     [f"{GAUSS}::test_gaussian_pa_matches_exact_enumeration"]),
    ("Gaussian: wrong sign of the energy change",
     "int32_t dE = -2 * sig[i] * h;", "int32_t dE = 2 * sig[i] * h;",
     [f"{GAUSS}::test_gaussian_sweeps_sample_boltzmann_distribution"]),
    ("Gaussian: wrong fixed-point scale in the acceptance",
     "float x = -((bf * ef) * (float)OG_INV_SCALE);", "float x = -((bf * ef) * (float)0x1.0p-14);",
     [f"{GAUSS}::test_acceptance_fraction_is_boltzmann_factor"]),
    ("single-precision exp truncated",
     "#define FEXP_DEGREE 7", "#define FEXP_DEGREE 4",
     [f"{GAUSS}::test_fexp_within_two_float_ulp"]),
    ("Gaussian: Poisson mean without 1/Q'",
     "double a = ((double)R_target * w[j]) / Qp;", "double a = ((double)R_target * w[j]);",
     [f"{GAUSS}::test_gaussian_invariants", f"{GAUSS}::test_gaussian_pa_matches_exact_enumeration"]),
]

ALL = [(m[0], m[1], m[2], m[3], "main") for m in MUTANTS] + [(m[0], m[1], m[2], m[3], "gauss") for m in GAUSS_MUTANTS]


@pytest.mark.parametrize("name,old,new,pins,which", ALL, ids=[m[0] for m in ALL])
def test_pins_catch_planted_mistake(name, old, new, pins, which, tmp_path):
    path = o.SRC if which == "main" else o.SRC_GAUSS
    src = open(path).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    mutant = tmp_path / os.path.basename(path)
    mutant.write_text(src.replace(old, new))
    if which == "main":
        lib = o.build(src=str(mutant), out=str(tmp_path / "libmutant.so"))
    else:
        lib = o.build(src=o.SRC, out=str(tmp_path / "libmutant.so"), src_gauss=str(mutant))
    env = dict(os.environ, PA_ORACLE_LIB=lib)
    p = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        *pins], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert p.returncode != 0, f"pins {pins} did not catch: {name}\n{p.stdout[-800:]}"
    assert "skipped" not in p.stdout.splitlines()[-1], p.stdout[-400:]
