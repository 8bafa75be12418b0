"""Mutation check of the oracle pins: each plausible mistake below (a
dropped term, a wrong sign, a transposed operand, a swapped index or axis) is
planted in a copy of the oracle source, compiled, and must make at least one
pin fail.  The planted copies live in a temporary directory; the oracle
itself is never modified."""
import os
import subprocess
import sys

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "zq_oracle.c")

MUTANTS = [
    ("up_drop_beta_term", "t[a] = p->alpha * tx[a] + p->beta * ty[a];", "t[a] = p->alpha * tx[a];"),
    ("up_s_sign", "u[k++] = p->beta * tx[a] - p->alpha * ty[a];", "u[k++] = p->beta * tx[a] + p->alpha * ty[a];"),
    ("up_s_swap_weights", "u[k++] = p->beta * tx[a] - p->alpha * ty[a];", "u[k++] = p->alpha * tx[a] - p->beta * ty[a];"),
    ("up_transposed_G", "y[i] += p->G[i * k + j] * u[j];", "y[i] += p->G[j * k + i] * u[j];"),
    ("down_untransposed_G", "y[i] += p->G[j * k + i] * z[j];", "y[i] += p->G[i * k + j] * z[j];"),
    ("down_swap_weights", "Lx[a] = p->alpha * Lp[a] + p->beta * sigma;", "Lx[a] = p->beta * Lp[a] + p->alpha * sigma;"),
    ("down_sigma_sign", "Ly[a] = p->beta * Lp[a] - p->alpha * sigma;", "Ly[a] = p->beta * Lp[a] + p->alpha * sigma;"),
    ("leaf_velocity_rotational", "out[3 * (int64_t)i + a] = Lp[a];", "out[3 * (int64_t)i + a] = Lp[3 + a];"),
    ("centroid_unweighted", "p->c[a] = ((double)nx * cx[a] + (double)ny * cy[a]) / (double)n;", "p->c[a] = 0.5 * (cx[a] + cy[a]);"),
    ("shift_scale_unreduced", "double sk = sqrt((double)nx * (double)ny / (double)n);", "double sk = sqrt((double)nx * (double)n / (double)ny);"),
    ("shift_sign", "double d[3] = {cx[0] - cy[0], cx[1] - cy[1], cx[2] - cy[2]};", "double d[3] = {cy[0] - cx[0], cy[1] - cx[1], cy[2] - cx[2]};"),
    ("cross_matrix_transposed", "double K[9] = {0.0, -d[2], d[1], d[2], 0.0, -d[0], -d[1], d[0], 0.0};", "double K[9] = {0.0, d[2], -d[1], -d[2], 0.0, d[0], d[1], -d[0], 0.0};"),
    ("alpha_beta_swapped", "p->alpha = sqrt((double)nx / (double)n);", "p->alpha = sqrt((double)ny / (double)n);"),
    ("householder_v_scale", "v[j][i] = A[i][j] / (alpha - beta);", "v[j][i] = A[i][j] / (alpha + beta);"),
    ("householder_beta_sign", "double beta = (alpha >= 0.0) ? -norm : norm;", "double beta = (alpha >= 0.0) ? norm : -norm;"),
    ("T22_not_transposed", "L[3 * r + c] = (c <= r) ? A[c][r] : 0.0;", "L[3 * r + c] = (c <= r) ? A[r][c] : 0.0;"),
    ("case_one_g3_sign", "G[6 + a] = -h[a];", "G[6 + a] = h[a];"),
    ("case_one_L_sign", "L[3 * a + 1] = -s * g1[a];", "L[3 * a + 1] = s * g1[a];"),
    ("case_one_g1_sign", "g1[1] = -d[2] / s;\n    g1[2] = d[1] / s;", "g1[1] = d[2] / s;\n    g1[2] = -d[1] / s;"),
    ("qgen_s_row_sign", "C[(row + a) * cols + 3 * (nx + i) + a] = -p->alpha / sqrt((double)ny);", "C[(row + a) * cols + 3 * (nx + i) + a] = p->alpha / sqrt((double)ny);"),
    ("bisect_axis_order_x_first", "int axis = 2 - l % 3; /* z, then y, then x */", "int axis = l % 3;"),
    ("bisect_msb_last", "int bit = QBITS - 1 - l / 3;", "int bit = l / 3;"),
    ("quantise_unnormalised", "double t = (p[a][i] - lo) / (hi - lo);", "double t = (p[a][i] - lo);"),
    ("no_sign_normalisation", "flip[j] = A[j][j] < 0.0;", "flip[j] = 0;"),
    ("sign_flip_R_only", "for (int c = 0; c < k; ++c) G[j * k + c] = -G[j * k + c];", ";"),
    ("rank_flag_last_pivot_only", "for (int j = 0; j < 3; ++j)\n    if (L[4 * j] == 0.0", "for (int j = 2; j < 3; ++j)\n    if (L[4 * j] == 0.0"),
    ("rank_flag_never", "p->degenerate = rank_deficient(M, k, p->L);", "p->degenerate = 0;"),
    ("no_numerical_zero_rule", "    if (noise)\n      for (int i = j; i < k; ++i) A[i][j] = 0.0;", ";"),
    ("zero_rule_per_entry", "if (noise)\n      for (int i = j; i < k; ++i) A[i][j] = 0.0;",
     "for (int i = j; i < k; ++i)\n      if (A[i][j] != 0.0 && ilogb(A[i][j]) < emax - 40) A[i][j] = 0.0;"),
]


def test_probe_passes_on_the_real_oracle():
    r = subprocess.run([sys.executable, os.path.join(HERE, "_mutant_probe.py"), str(oracle.build())],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    mutant = tmp_path / f"{name}.c"
    mutant.write_text(src.replace(old, new))
    lib = oracle.build(force=True, src=mutant, out=tmp_path / f"lib{name}.so")
    r = subprocess.run([sys.executable, os.path.join(HERE, "_mutant_probe.py"), str(lib)],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode != 0, f"planted mistake {name} passed every pin"
