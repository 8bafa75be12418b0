"""Runs a fast subset of the oracle pins against the oracle build given on
the command line.  Exit status 0: every pin passed; 1: a pin failed."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import oracle  # noqa: E402

oracle._LIB = oracle.load(sys.argv[1])

import test_oracle_pins as P  # noqa: E402

CHECKS = [
    lambda: [P.test_case_one_golden(r) for r in range(3)],
    lambda: P.test_case_one_printed_formula_random(),
    lambda: [P.test_lq_matches_lapack_householder(k, s) for k in (6, 9) for s in (0, 1)],
    lambda: [P.test_dense_complement_brute_force(kind, n)
             for kind in ("shell", "cube", "far") for n in (3, 5, 17, 40)],
    lambda: [P.test_implicit_passes_match_projector(kind, 33) for kind in ("shell", "cube")],
    lambda: [P.test_tree_matches_real_bisection(kind, n) for kind in ("shell", "cube") for n in (9, 50)],
    lambda: P.test_invariants_large(1000),
    lambda: P.test_table1_orthogonality(500),
    lambda: [P.test_node_assembly_eq_3_5(s) for s in range(3)],
    lambda: P.test_lq_rank_deficient_is_exact_and_valid(),
    lambda: [P.test_lq_badly_scaled_full_rank_matches_lapack(e) for e in (33, 39)],
    lambda: [P.test_singular_T22_flag_marks_exactly_the_collinear_nodes(n) for n in (12, 27)],
]

failed = 0
for c in CHECKS:
    try:
        c()
    except AssertionError:
        failed += 1
sys.exit(1 if failed else 0)
