"""The pins reject a broken oracle.

Each case plants one plausible mistake in a copy of oracle/fl_oracle.cpp,
builds it, and runs the oracle pin tests against it (in a subprocess); at
least one pin must fail.  This shows the pins are not circular: a dropped
term, a wrong sign, index or coefficient, or a transposed operand anywhere
in the oracle is caught."""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fl_oracle.cpp")
PINS = ["tests/test_oracle_limiters.py", "tests/test_oracle_bruteforce.py",
        "tests/test_oracle_properties.py", "tests/test_oracle_adjoint.py",
        "tests/test_oracle_distances.py"]

# (name, original text, mutated text)
MUTANTS = [
    ("sign_tie_goes_positive", "return (u > 0.0) ? 1 : -1;", "return (u >= 0.0) ? 1 : -1;"),
    ("upstream_sign_dropped", "e.dU = (e.s > 0) ? acc : -acc;", "e.dU = acc;"),
    ("upstream_from_downwind_cell",
     "for (int64_t q = m.cf_ptr[e.C]; q < m.cf_ptr[e.C + 1]; ++q) {\n    const int64_t j = m.cf_idx[q];\n    if (j == f) continue;\n    const double w",
     "for (int64_t q = m.cf_ptr[e.D]; q < m.cf_ptr[e.D + 1]; ++q) {\n    const int64_t j = m.cf_idx[q];\n    if (j == f) continue;\n    const double w"),
    ("normal_dot_transposed",
     "const double w = m.nx[f] * m.nx[j] + m.ny[f] * m.ny[j] + m.nz[f] * m.nz[j];\n    acc = acc + dist_term(m, w",
     "const double w = m.nx[f] * m.ny[j] + m.ny[f] * m.nx[j] + m.nz[f] * m.nz[j];\n    acc = acc + dist_term(m, w"),
    ("superbee_cap_wrong", "std::fmin(r, 2.0)));", "std::fmin(r, 1.0)));"),
    ("face_value_from_downwind", "e.thf = th[e.C] + 0.5 * e.psi * e.du;",
     "e.thf = th[e.D] + 0.5 * e.psi * e.du;"),
    ("divergence_sign_swapped",
     "const double sigma = (m.c0[f] == c) ? 1.0 : -1.0;\n      // a face whose",
     "const double sigma = (m.c0[f] == c) ? -1.0 : 1.0;\n      // a face whose"),
    ("volume_dropped", "R[c] = -acc / m.vol[c];", "R[c] = -acc;"),
    ("rk3_coefficient", "const double RK3_A[3] = {0.0, 0.75, 1.0 / 3.0};",
     "const double RK3_A[3] = {0.0, 0.25, 1.0 / 3.0};"),
    ("smart_middle_branch", "0.25 + 0.75 * r), 4.0));", "0.25 + 0.5 * r), 4.0));"),
    ("tlm_alpha_sign", "return 0.5 * (e.psi - pr);", "return 0.5 * (e.psi + pr);"),
    ("tlm_infinite_ratio_product", "const double pr = (e.dpsi != 0.0) ? e.dpsi * e.r : 0.0;",
     "const double pr = e.dpsi * e.r;"),
    ("branch_from_rounded_ratio", "e.dpsi = dpsi_exact(lim, e.dU, e.du, e.r);",
     "(void)psi_branch(lim, e.r, &e.dpsi);"),
    ("smart_branch_at_infinite_ratio", "if (std::isinf(r)) { *dpsi = 0.0; return 4.0; }", ""),
    ("central_slope_dropped_on_flat_faces", "e.psi = (lim == L_CENTRAL) ? 1.0 : 0.0;",
     "e.psi = 0.0;"),
    ("adjoint_downwind_to_upwind", "out[e.D] += g * alpha;", "out[e.C] += g * alpha;"),
    ("distance_weight_inverted", "return m.dist.empty() ? term : term / m.dist[j];",
     "return m.dist.empty() ? term : term * m.dist[j];"),
    ("distance_of_face_dropped", "return m.dist.empty() ? acc : acc * m.dist[f];",
     "return acc;"),
]


@pytest.mark.parametrize("name,orig,mut", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_planted_mistake(name, orig, mut):
    src = open(SRC).read()
    # the first occurrence is the forward path (eval_face / rhs); later ones
    # are the tangent-linear copies
    assert src.count(orig) >= 1, "mutation anchor missing: %s" % name
    with tempfile.TemporaryDirectory() as d:
        cpp = os.path.join(d, "fl_oracle_%s.cpp" % name)
        lib = os.path.join(d, "liboracle_%s.so" % name)
        with open(cpp, "w") as fh:
            fh.write(src.replace(orig, mut, 1))
        subprocess.check_call(["g++", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp",
                               "-std=c++17", "-shared", "-fPIC", "-o", lib, cpp])
        env = dict(os.environ, FL_ORACLE_MUTANT_LIB=lib)
        res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"]
                             + PINS, cwd=ROOT, env=env, capture_output=True, text=True)
        assert res.returncode != 0, "mutant %s passed every pin" % name
