"""The oracle's pins catch plausible mistakes (CPU only).

Each case copies the oracle, the seeded input generator, the pin tests and
their golden files into a temporary directory, plants one mistake in the
copy of oracle.c (the repository's own oracle is never touched) and runs the
pins there: at least one must fail.  The control case plants nothing and
must pass, so that a failure is the mistake's and not the harness's.  A
mutant that passes every pin would name a gap in the pins.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# name -> [(text in oracle.c, replacement)] or [(file of the oracle, text, replacement)],
# each text present exactly once in its file
MUTANTS = {
    "control": [],
    # blocks and the 3x3 inverse
    "matvec_transposed_block": [("acc += a[r * BS + c] * x[c];", "acc += a[c * BS + r] * x[c];")],
    "inverse_without_pivoting": [("if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;", "if (0) piv = r;")],
    # ILU0 (Algorithm 2)
    "ilu0_left_product_with_pivot": [("blk_mul(lu + BS2 * mk, dinv + BS2 * (int64_t)k, lik);",
                                      "blk_mul(dinv + BS2 * (int64_t)k, lu + BS2 * mk, lik);")],
    "ilu0_update_added": [("for (int e = 0; e < BS2; ++e) c[e] -= p[e];",
                           "for (int e = 0; e < BS2; ++e) c[e] += p[e];")],
    "ilu0_diagonal_not_updated": [("if (mkj >= 0) blk_mul_sub(lik, lu + BS2 * mkj, lu + BS2 * mj);",
                                   "if (mkj >= 0 && j != i) blk_mul_sub(lik, lu + BS2 * mkj, lu + BS2 * mj);")],
    # ILU0 application (Algorithm 1)
    "apply_without_inverse_pivot": [("    double zi[BS] = {0.0, 0.0, 0.0};\n    blk_matvec_add(dinv + BS2 * (int64_t)i, acc, zi);\n"
                                     "    for (int c = 0; c < BS; ++c) z[(int64_t)BS * i + c] = zi[c];",
                                     "    for (int c = 0; c < BS; ++c) z[(int64_t)BS * i + c] = acc[c];")],
    "apply_backward_skips_last_upper": [("      if (j <= i) continue;\n      double t[BS] = {0.0, 0.0, 0.0};\n"
                                         "      blk_matvec_add(lu + BS2 * m, z + (int64_t)BS * j, t);",
                                         "      if (j <= i || m == rowptr[i + 1] - 1) continue;\n"
                                         "      double t[BS] = {0.0, 0.0, 0.0};\n"
                                         "      blk_matvec_add(lu + BS2 * m, z + (int64_t)BS * j, t);")],
    # BiCGStab (van der Vorst) and the stopping rule of Section 4.2
    "bicgstab_beta_inverted": [("double beta = (rho / rho_prev) * (alpha / omega);",
                                "double beta = (rho / rho_prev) * (omega / alpha);")],
    "bicgstab_half_step_without_update": [("      for (size_t e = 0; e < n; ++e) x[e] += alpha * ph[e];\n      status = 0;",
                                           "      status = 0;")],
    "bicgstab_residual_sign": [("r[e] = s[e] - omega * t[e];", "r[e] = s[e] + omega * t[e];")],
    "bicgstab_stops_late": [("    if (nr <= tol) {", "    if (nr <= 0.5 * tol) {")],
    "bicgstab_half_step_stops_late": [("    if (ns <= tol) { /* half-step exit */", "    if (ns <= 0.5 * tol) {")],
    "bicgstab_stops_early": [("    if (nr <= tol) {", "    if (nr <= 2.0 * tol) {")],
    # the four breakdown tests: without one, the method divides by an exact zero
    "bicgstab_rho_zero_unchecked": [("if (rho == 0.0) {", "if (rho != rho) {")],
    "bicgstab_rhv_zero_unchecked": [("if (rhv == 0.0) {", "if (rhv != rhv) {")],
    "bicgstab_tt_zero_unchecked": [("if (tt == 0.0) {", "if (tt != tt) {")],
    "bicgstab_omega_zero_unchecked": [("if (omega == 0.0) {", "if (omega != omega) {")],
    # schedules (Section 4.4)
    "levels_not_incremented": [("if (j < i && level[j] + 1 > l) l = level[j] + 1;",
                                "if (j < i && level[j] > l) l = level[j];")],
    "graph_not_symmetrised": [("      deg[i]++;\n      deg[j]++;", "      deg[i]++;"),
                              ("      adj[ptr[i] + fill[i]++] = j;\n      adj[ptr[j] + fill[j]++] = i;",
                               "      adj[ptr[i] + fill[i]++] = j;")],
    "permute_leaves_columns_unsorted": [("while (at > base && pcolidx[at - 1] > nc) {", "while (0) {")],
    # wells (Section 4.6)
    "wells_added": [("y[(int64_t)BS * wcells[p] + c] -= acc;", "y[(int64_t)BS * wcells[p] + c] += acc;")],
    "wells_B_for_C": [("acc += C[12 * (int64_t)p + 3 * r + c] * t2[r];", "acc += B[12 * (int64_t)p + 3 * r + c] * t2[r];")],
    # the FP32-factor variant
    "f32_ilu0_update_added": [("for (int e = 0; e < BS2; ++e) lu[BS2 * mj + e] -= p[e];",
                               "for (int e = 0; e < BS2; ++e) lu[BS2 * mj + e] += p[e];")],
    "f32_apply_without_inverse_pivot": [("t += dinv[BS2 * (int64_t)i + a * BS + c] * acc[c];",
                                         "t += (a == c) ? acc[c] : 0.0f;")],
    # dense Gaussian elimination (brute force)
    "dense_solve_rhs_not_swapped": [("      double t = b[col];\n      b[col] = b[piv];\n      b[piv] = t;\n", "")],
    # smallest-last colouring and the Kempe reduction
    "smallest_last_not_reversed": [("for (int32_t t = cnt - 1; t >= 0; --t) {\n    int32_t v = order[t];",
                                    "for (int32_t t = 0; t < cnt; ++t) {\n    int32_t v = order[t];")],
    "smallest_last_degrees_not_updated": [("        deg[u]--;\n", "")],
    "kempe_chain_may_reach_a_neighbour": [("if (nbr_of[y] == v || qn == kempe_cap) {", "if (qn == kempe_cap) {")],
    "kempe_chain_not_exchanged": [("colour[queue[q]] = colour[queue[q]] == a ? b : a;", "colour[queue[q]] = b;")],
    # order inside a set, and the stable order by key
    "open_rows_first": [("for (int32_t i = 0; i < nb; ++i) out[i] = 2 * key[i];",
                         "for (int32_t i = 0; i < nb; ++i) out[i] = 2 * key[i] + 1;"),
                        ("      if (key[j] > key[i]) out[i] = 2 * key[i] + 1;\n      if (key[i] > key[j]) out[j] = 2 * key[j] + 1;",
                         "      if (key[j] > key[i]) out[i] = 2 * key[i];\n      if (key[i] > key[j]) out[j] = 2 * key[j];")],
    "order_by_key_unstable": [("for (int32_t i = 0; i < nb; ++i) perm[start[key[i]]++] = i;",
                               "for (int32_t i = nb - 1; i >= 0; --i) perm[start[key[i]]++] = i;")],
    # SpMV's gather and the value permutation
    "spmv_reads_the_row_not_the_column": [("blk_matvec_add(vals + BS2 * m, x + (int64_t)BS * colidx[m], yi);",
                                           "blk_matvec_add(vals + BS2 * m, x + (int64_t)BS * i, yi);")],
    "permute_drops_the_blocks_values": [("      memcpy(pvals + BS2 * at, vals + BS2 * m, sizeof(double) * BS2);\n",
                                         "      memcpy(pvals + BS2 * at, vals + BS2 * (rowptr[oi]), sizeof(double) * BS2);\n")],
    # the Chow-Patel initial guess, the Jacobi backward sweep
    "chow_patel_guess_without_pivot_inverse": [
        ("      if (colidx[m] < i) blk_mul(vals + BS2 * m, dinv + BS2 * (int64_t)colidx[m], lu + BS2 * m);\n"
         "      else memcpy(lu + BS2 * m, vals + BS2 * m, sizeof(double) * BS2);",
         "      memcpy(lu + BS2 * m, vals + BS2 * m, sizeof(double) * BS2);")],
    "jacobi_backward_without_inverse_pivot": [
        ("      double zi[BS] = {0.0, 0.0, 0.0};\n      blk_matvec_add(dinv + BS2 * (int64_t)i, acc, zi);\n"
         "      memcpy(z2 + (int64_t)BS * i, zi, sizeof zi);",
         "      memcpy(z2 + (int64_t)BS * i, acc, sizeof acc);")],
    # block-Jacobi pattern (Section 4.5), in the oracle's Python half
    "jacobi_pattern_keeps_cross_blocks": [("__init__.py", "keep = part[rows] == part[colidx]",
                                           "keep = (part[rows] == part[colidx]) | (rows + 1 == colidx)")],
    "schedule_long_rows_first": [("__init__.py", "key3 = 2 * key2 + (lens > common).astype(np.int32)",
                                  "key3 = 2 * key2 + (lens <= common).astype(np.int32)")],
    # restarted GMRES: the end-of-cycle update
    "gmres_rotation_sign": [("H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;", "H[(i + 1) * m + j] = sn[i] * a + cs[i] * c;")],
    "gmres_cycle_update_unpreconditioned": [("    orc_ilu_apply(nb, rowptr, colidx, lu, dinv, w, z);\n    for (size_t e = 0; e < n; ++e) x[e] += z[e];",
                                             "    for (size_t e = 0; e < n; ++e) x[e] += w[e];")],
    # Chow-Patel sweeps and Jacobi triangular sweeps: Gauss-Seidel instead of synchronous
    "chow_patel_in_place": [("          blk_mul(sum, dinv + BS2 * (int64_t)j, lu2 + BS2 * m);",
                             "          blk_mul(sum, dinv + BS2 * (int64_t)j, lu2 + BS2 * m);\n"
                             "          memcpy(lu + BS2 * m, lu2 + BS2 * m, sizeof sum);")],
    "jacobi_forward_in_place": [("        blk_matvec_add(lu + BS2 * m, y + (int64_t)BS * colidx[m], tv);",
                                 "        blk_matvec_add(lu + BS2 * m, y2 + (int64_t)BS * colidx[m], tv);")],
}


def _tree(dst):
    """The pins with what they import, copied into dst."""
    ign = shutil.ignore_patterns("_build", "__pycache__", "*.so", "*.tmp")
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"), ignore=ign)
    os.makedirs(os.path.join(dst, "paper_2309_11488_gb300"))
    open(os.path.join(dst, "paper_2309_11488_gb300", "__init__.py"), "w").close()
    shutil.copy(os.path.join(ROOT, "paper_2309_11488_gb300", "synth.py"), os.path.join(dst, "paper_2309_11488_gb300"))
    os.makedirs(os.path.join(dst, "tests"))
    for f in ("conftest.py", "test_oracle_pins.py", "test_oracle_breakdown.py", "breakdown_fixture.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests"))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(dst, "tests", "golden"))


def _run(name, root):
    """Plant mutant `name` in a fresh copy under root and run the pins there;
    returns (exit code, output tail)."""
    dst = os.path.join(root, name)
    _tree(dst)
    for edit in MUTANTS[name]:
        fname, old, new = edit if len(edit) == 3 else ("oracle.c", *edit)
        path = os.path.join(dst, "oracle", fname)
        with open(path) as f:
            src = f.read()
        if src.count(old) != 1:
            return -1000, f"mutation text not found exactly once: {old!r}"
        with open(path, "w") as f:
            f.write(src.replace(old, new))
    # one thread each: the runs go side by side, so numpy's BLAS must not fan out
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1", OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
               MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                        "test_oracle_pins.py", "test_oracle_breakdown.py"], cwd=os.path.join(dst, "tests"), env=env, capture_output=True,
                       text=True, timeout=900)
    return r.returncode, r.stdout[-3000:]


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    """Every mutant's pin run, the runs side by side (independent processes)."""
    from concurrent.futures import ThreadPoolExecutor
    root = str(tmp_path_factory.mktemp("mutants"))
    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        futs = {name: ex.submit(_run, name, root) for name in MUTANTS}
        return {name: f.result() for name, f in futs.items()}


@pytest.mark.parametrize("name", list(MUTANTS))
def test_pins_catch_a_planted_mistake(name, results):
    rc, out = results[name]
    assert rc != -1000, out
    if name == "control":
        assert rc == 0, out
    else:
        # 1: a pin failed; negative: the mutant crashed the process.  Anything
        # else (collection or usage errors) would be the harness's fault.
        assert rc == 1 or rc < 0, (name, rc, out)
