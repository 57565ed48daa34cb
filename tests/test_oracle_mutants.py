"""The oracle's pins catch plausible mistakes: each one planted in a copy of the oracle fails
at least one pin.

Every mutant below is a copy of oracle/amg_oracle.c with one mistake of the kind a
restatement of the paper could make (a transposed operand, a dropped term, a wrong sign or
index, an off-by-one, the paper's own over-simple claims taken literally). Each copy is
compiled with the oracle's flags and the pin files (tests/test_oracle_*.py) run against it in
a subprocess, through the oracle loader's library override. A pin must fail (pytest exit
status 1: a test failed, not a crash). A build of the unmodified source through the same path
must pass, so the failures come from the mistakes.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

from oracle import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = [os.path.join("tests", f) for f in ("test_oracle_aggregation.py", "test_oracle_galerkin.py",
                                          "test_oracle_smoother.py", "test_oracle_cycle.py",
                                          "test_oracle_disk.py", "test_oracle_octree.py")]

# name -> (text in the oracle, replacement): each text occurs exactly once
MUTANTS = {
    # Sec. 3.2 / 4.2 binning: x and y exchanged in the cell coordinates
    "bin_x_y_exchanged": (
        "        f->t1[j] = cell_index_1d(x[j], h->bbox[0], h->bbox[1], L);\n"
        "        f->t2[j] = cell_index_1d(y[j], h->bbox[2], h->bbox[3], L);",
        "        f->t1[j] = cell_index_1d(y[j], h->bbox[2], h->bbox[3], L);\n"
        "        f->t2[j] = cell_index_1d(x[j], h->bbox[0], h->bbox[1], L);"),
    # eq. subregion: rounding up instead of down (off by one cell)
    "bin_rounds_up": (
        "    return (int)floor(s);",
        "    return (int)ceil(s) < w ? (int)ceil(s) : w - 1;"),
    # Sec. 3.1 depth rule: 4^L < N instead of 4^L <= N
    "depth_strict": (
        "    while (N >= (1LL << (2 * (L + 1)))) L++;",
        "    while (N > (1LL << (2 * (L + 1)))) L++;"),
    # Sec. 4.2 parent cell with t1 and t2 exchanged (the text's transposed form, reading R2)
    "parent_transposed": (
        "            cid[i] = (c3 * w + c2) * w + c1;",
        "            cid[i] = (c3 * w + c1) * w + c2;"),
    # Sec. 2 / Sec. 5: empty cells kept as (empty) aggregates instead of compacted away
    "empty_cells_kept": (
        "        for (long long c = 0; c < ncell; c++) num[c] = num[c] ? nc++ : -1;",
        "        for (long long c = 0; c < ncell; c++) num[c] = nc++;"),
    # eq. acsum: the diagonal entries dropped from the Galerkin sums
    "galerkin_drops_diagonal": (
        "                buf[k].v = f->val[p];",
        "                buf[k].v = f->col[p] == i ? 0.0 : f->val[p];"),
    # eq. acsum: every contribution summed into the row's own aggregate (column index lost)
    "galerkin_wrong_column": (
        "                buf[k].c = f->agg[f->col[p]];",
        "                buf[k].c = f->agg[i];"),
    # Sec. 4.5 taken literally: four colours whatever the span (fails reading R5)
    "four_colours_always": (
        "    lv->m = lv->span + 1 > 2 ? lv->span + 1 : 2;",
        "    lv->m = 2;"),
    # reading R5: the span measured in t1 only
    "span_ignores_t2": (
        "            if (d2 > s) s = d2;",
        "            (void)d2;"),
    # Sec. 6 octree colouring with m instead of m^2 for the third coordinate
    "octree_colour_weight": (
        "        if (lv->t3) lv->color[i] += lv->m * lv->m * (lv->t3[i] % lv->m);",
        "        if (lv->t3) lv->color[i] += lv->m * (lv->t3[i] % lv->m);"),
    # octree span: the third coordinate's offsets left out
    "octree_span_ignores_t3": (
        "                if (d3 > s) s = d3;",
        "                (void)d3;"),
    # octree coarse cells: t3 of a coarse row read as its t2
    "octree_coarse_t3": (
        "                if (dim == 3) cl->t3[num[c]] = (int)(c / ((long long)w * w));",
        "                if (dim == 3) cl->t3[num[c]] = (int)((c / w) % w);"),
    # Sec. 4.5 colour formula with t1 and t2 exchanged
    "colour_transposed": (
        "        lv->color[i] = (lv->t1[i] % lv->m) + lv->m * (lv->t2[i] % lv->m);",
        "        lv->color[i] = (lv->t2[i] % lv->m) + lv->m * (lv->t1[i] % lv->m);"),
    # R_k: the forward sweep run in the reversed order
    "forward_sweep_reversed": (
        "    if (!backward)\n        for (int p = 0; p < lv->n; p++) gs_row(lv, lv->perm[p], f, u);",
        "    if (!backward)\n        for (int p = lv->n - 1; p >= 0; p--) gs_row(lv, lv->perm[p], f, u);"),
    # Gauss-Seidel update with the wrong sign on the off-diagonal terms
    "gs_sign": (
        "        else s -= lv->val[p] * u[j];",
        "        else s += lv->val[p] * u[j];"),
    # reading R14: the post-smoother sweeps in the forward order (not the adjoint R^t)
    "backward_sweep_forward": (
        "        for (int p = lv->n - 1; p >= 0; p--) gs_row(lv, lv->perm[p], f, u);",
        "        for (int p = 0; p < lv->n; p++) gs_row(lv, lv->perm[p], f, u);"),
    # Alg. 2: f restricted instead of the residual f - A u1
    "restricts_f_not_residual": (
        "    for (int i = 0; i < n; i++) r[i] = f[i] - r[i];",
        "    for (int i = 0; i < n; i++) r[i] = f[i];"),
    # Alg. 2: u2 = P e instead of u1 + P e
    "prolongation_overwrites": (
        "    for (int i = 0; i < n; i++) z[i] += e[lv->agg[i]];",
        "    for (int i = 0; i < n; i++) z[i] = e[lv->agg[i]];"),
    # Alg. 2: the post-smoothing step dropped
    "no_post_smoothing": (
        "    for (int s = 0; s < h->opt.nu_post; s++) smooth(lv, 1, f, z);",
        ""),
    # reading R10 as a parameter: the post-smoothing's sweep count taken from nu_pre
    "post_sweeps_from_nu_pre": (
        "    for (int s = 0; s < h->opt.nu_post; s++) smooth(lv, 1, f, z);",
        "    for (int s = 0; s < h->opt.nu_pre; s++) smooth(lv, 1, f, z);"),
    # every pre-smoothing sweep restarted from zero (the sweeps do not compose)
    "pre_sweeps_restart_from_zero": (
        "    for (int s = 0; s < h->opt.nu_pre; s++) smooth(lv, 0, f, z);",
        "    for (int s = 0; s < h->opt.nu_pre; s++) {\n"
        "        for (int i = 0; i < n; i++) z[i] = 0.0;\n        smooth(lv, 0, f, z);\n    }"),
    # Alg. 1: the orthogonalisation coefficient with the wrong sign
    "alg1_beta_sign": (
        "            double beta = -dot(n, z, q + (size_t)j * n) / pAp[j];",
        "            double beta = dot(n, z, q + (size_t)j * n) / pAp[j];"),
    # Alg. 1: alpha from (r, r) instead of (r, p)
    "alg1_alpha": (
        "        double alpha = dot(n, r, pi) / pAp[it];\n"
        "        for (int i = 0; i < n; i++) u[i] += alpha * pi[i];",
        "        double alpha = dot(n, r, r) / pAp[it];\n"
        "        for (int i = 0; i < n; i++) u[i] += alpha * pi[i];"),
    # outer flexible CG: the orthogonalisation coefficient with the wrong sign
    "outer_beta_sign": (
        "            double beta = -dot(n, z, Q[j]) / pAp[j];",
        "            double beta = dot(n, z, Q[j]) / pAp[j];"),
    # reading R13: the outer iteration stops on the absolute residual, not relative to ||b||
    "outer_stop_absolute": (
        "        rel = sqrt(dot(n, r, r)) / bn;\n        if (!isfinite(rel))",
        "        rel = sqrt(dot(n, r, r));\n        if (!isfinite(rel))"),
    # coarsest exact solve: the backward substitution reads L instead of L^t
    "cholesky_transposed": (
        "        for (int k = i + 1; k < n; k++) s -= a[(size_t)k * n + i] * u[k];",
        "        for (int k = i + 1; k < n; k++) s -= a[(size_t)i * n + k] * u[k];"),
    # coarsest factorisation: the diagonal update with the wrong sign
    "cholesky_diagonal_sign": (
        "        for (int k = 0; k < j; k++) d -= a[(size_t)j * n + k] * a[(size_t)j * n + k];",
        "        for (int k = 0; k < j; k++) d += a[(size_t)j * n + k] * a[(size_t)j * n + k];"),
    # Sec. 3.1 eq. ab12: the box's upper x bound taken from y
    "box_upper_x_from_y": (
        "            if (x[j] > b1) b1 = x[j];",
        "            if (y[j] > b1) b1 = y[j];"),
    # octree binning: z measured against the y extent of the box
    "octree_z_in_y_box": (
        "        if (dim == 3) f->t3[j] = cell_index_1d(z[j], h->bbox[4], h->bbox[5], L);",
        "        if (dim == 3) f->t3[j] = cell_index_1d(z[j], h->bbox[2], h->bbox[3], L);"),
    # octree depth: 4^L <= N (the quadtree rule) instead of 8^L <= N
    "octree_depth_rule": (
        "    while (N >= (1LL << (3 * (L + 1)))) L++;",
        "    while (N >= (1LL << (2 * (L + 1)))) L++;"),
    # sweep order pi: rows in index order within a colour, not grouped by block (fine level)
    "sweep_ignores_blocks": (
        "    for (int i = 0; i < n; i++) tmp[cnt[blockkey[i]]++] = i;",
        "    for (int i = 0; i < n; i++) tmp[i] = i;"),
    # Alg. 2 restriction: P^t r summed into the wrong coarse row (off by one aggregate)
    "restriction_shifted": (
        "    for (int i = 0; i < n; i++) fc[lv->agg[i]] += r[i];",
        "    for (int i = 0; i < n; i++) fc[(lv->agg[i] + 1) % cl->n] += r[i];"),
    # readings R6 / R17: Galerkin sums that cancel to exactly zero dropped from the pattern
    "galerkin_drops_exact_zeros": (
        "            c->col[out] = buf[a].c;\n            c->val[out] = s;\n            out++;",
        "            if (s != 0.0) {\n            c->col[out] = buf[a].c;\n"
        "            c->val[out] = s;\n            out++; }"),
    # the coarsest level: coarsening continues while n >= coarsest_max instead of n >
    "coarsest_threshold": (
        "    while (h->lev[h->nlev - 1].n > opt->coarsest_max) {",
        "    while (h->lev[h->nlev - 1].n >= opt->coarsest_max) {"),
    # reading R11: one Alg. 1 step on every level (a V-cycle) whatever kcycle_n says
    "kcycle_one_step": (
        "    int steps = h->opt.kcycle_n;",
        "    int steps = 1;"),
}


def _build(name, text, tmp):
    src = open(oracle.SRC).read()
    if text is not None:
        old, new = text
        assert src.count(old) == 1, f"{name}: the mutated text must occur once in the oracle"
        src = src.replace(old, new)
    c = os.path.join(tmp, f"{name}.c")
    with open(c, "w") as f:
        f.write(src)
    so = os.path.join(tmp, f"lib{name}.so")
    oracle.compile_oracle(c, so)
    return so


def _run_pins(so):
    env = dict(os.environ, **{oracle.LIB_OVERRIDE_ENV: so})
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"  # the runs go in parallel: one BLAS thread each
    r = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-x", "-q", "-m", "not gpu",
                        "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    return r.returncode, r.stdout[-2000:]


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    tmp = str(tmp_path_factory.mktemp("mutants"))
    cases = {"unmodified": None, **MUTANTS}
    with cf.ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        libs = dict(zip(cases, ex.map(lambda kv: _build(kv[0], kv[1], tmp), cases.items())))
        runs = dict(zip(cases, ex.map(_run_pins, [libs[k] for k in cases])))
    return runs


def test_unmodified_oracle_passes_through_the_same_path(results):
    rc, out = results["unmodified"]
    assert rc == 0, out


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(results, name):
    rc, out = results[name]
    assert rc == 1, f"{name}: pins exit status {rc} (1 = a pin failed)\n{out}"
