"""Planted mistakes in the adaptive-grid oracle: its pins (quadtree and
octree) must notice a plausible error in every part of it.

Each case copies oracle/fc_oracle_amr.c, makes one small change (a wrong
weight, index range, loop bound or sign), compiles the copy against the
unaltered fc_oracle.c it includes, and runs the pin named beside the change
against it (through FC_ORACLE_AMR_LIB) in a child process; the pin must
fail.  A control case runs every named pin against an unaltered copy
compiled the same way, and they must pass.  Nothing here calls the CUDA
library, and the oracle files are never modified.

A pin run that the planted mistake crashes (an index taken from a wrong
parent) counts as caught.  The balance call after the coarsening of
Algorithm 1 is left out: replacing
every leaf of the highest level of a 2:1 balanced tree with its parent keeps
the tree balanced, so removing the call changes nothing.
"""
import concurrent.futures as cf
import os
import re
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ODIR = os.path.join(ROOT, "oracle")
SRC = os.path.join(ODIR, "fc_oracle_amr.c")
PINS = "tests/test_oracle_amr_pins.py::"
P3 = "test_oracle_amr3d_pins.py::"  # a pin of the octree file (its name carries the file)

# name, original text, altered text, occurrence, catching pin
MUTANTS = [
    # tree
    ("refinement_stops_early", "for (int l = U; l < R; ++l) {", "for (int l = U; l < R - 1; ++l) {", 0,
     "test_refinement_balance_and_algorithm_1"),
    ("balance_faces_only", "if (T->lev[amr_cell(T, x, y, z)] < l - 1) {",
     "if ((dx == 0 || dy == 0) && T->lev[amr_cell(T, x, y, z)] < l - 1) {", 0,
     "test_refinement_balance_and_algorithm_1"),
    ("coarsen_to_root", "if (T->lev[c] == rmax && rmax > 0) T->lev[c] = (unsigned char)(rmax - 1);",
     "if (T->lev[c] == rmax && rmax > 0) T->lev[c] = 0;", 0, "test_refinement_balance_and_algorithm_1"),
    # hanging nodes
    ("hanging_weight", "w[t] = 1.0 / k;", "w[t] = 0.5 / k;", 0, "test_forms_equal_the_uniform_finest_grid"),
    ("hanging_parent_edge", "N->hp[4 * m + 1] = amr_vid(T, b[0], b[1], dim == 3 ? b[2] : 0);",
     "N->hp[4 * m + 1] = amr_vid(T, a[0], a[1], dim == 3 ? a[2] : 0);", 0, "test_hanging_nodes"),
    # assembly
    ("element_level", "const or_level* U = ul[l];", "const or_level* U = ul[T->R];", 0,
     "test_forms_equal_the_uniform_finest_grid"),
    ("divergence_transpose_dropped", "else if (cc < dim) v = e->B[cc][b][a];", "else if (cc < dim) v = 0.0;", 0,
     "test_uniform_tree_is_the_uniform_grid"),
    ("lift_sign", "L->rhs[r] = L->rhs[r] - L->val[p] * L->wfix[L->col[p]];",
     "L->rhs[r] = L->rhs[r] + L->val[p] * L->wfix[L->col[p]];", 0, "test_uniform_tree_is_the_uniform_grid"),
    # patches
    ("velocity_one_ring", "const long k = adj[j * AMR_ADJ + u];", "const long k = j;", 0,
     "test_uniform_tree_is_the_uniform_grid"),
    ("pressure_not_owned", "if (j == i) own[dim] = n;", "if (j == i) own[dim] = -1;", 0, "test_owner_count_is_one"),
    # prolongation
    ("prolongation_weight", "wa = wa * (((a >> k) & 1) ? t[k] : 1.0 - t[k]);",
     "wa = wa * (((a >> k) & 1) ? 1.0 - t[k] : t[k]);", 0,
     "test_prolongation_exact_on_linear_fields"),
    # octrees (3D pins)
    ("balance_no_z_neighbours", "for (int dz = -rz; dz <= rz; ++dz)", "for (int dz = 0; dz <= 0; ++dz)", 0,
     P3 + "test_octree_refinement_balance_and_algorithm_1"),
    ("cut_samples_one_plane", "const int dim = G->dim, m3 = dim == 3 ? 3 : 1;", "const int dim = G->dim, m3 = 1;", 0,
     P3 + "test_octree_refinement_balance_and_algorithm_1"),
    ("face_centre_parents", "c[w] += (t >> 1) * s;", "c[w] += (t & 1) * s;", 0, P3 + "test_octree_hanging_nodes"),
    ("face_centre_weight", "w[t] = 1.0 / k;", "w[t] = k == 4 ? 0.5 : 1.0 / k;", 0,
     P3 + "test_octree_forms_equal_the_uniform_finest_grid"),
    ("face_centres_on_one_side", "for (int side = 0; side < 2; ++side) {", "for (int side = 0; side < 1; ++side) {", 0,
     P3 + "test_octree_forms_equal_the_uniform_finest_grid"),
    ("inflow_z_profile", "w0 = w0 * 4.0 * sz * (1.0 - sz);", "w0 = w0 * 4.0 * sz;", 0,
     P3 + "test_uniform_octree_is_the_uniform_grid"),
    ("element_cell_z", "(dim == 3 ? Z / s : 0)", "(dim == 3 ? Z / s / 2 : 0)", 0, P3 + "test_uniform_octree_is_the_uniform_grid"),
    ("prolongation_z", "dim == 3 ? (double)(Z - Z0) / s : 0.0", "dim == 3 ? (double)(Z - Z0) / (2 * s) : 0.0", 0,
     P3 + "test_octree_prolongation_exact_on_linear_fields"),
]


def _mutate(src, old, new, occ):
    idx = -1
    for _ in range(occ + 1):
        idx = src.index(old, idx + 1)
    return src[:idx] + new + src[idx + len(old):]


def _node(pin):
    return "tests/" + pin if "::" in pin else PINS + pin


def _run_pins(text, pins, workdir):
    c = os.path.join(workdir, "fc_oracle_amr_variant.c")
    so = os.path.join(workdir, "libfc_oracle_amr_variant.so")
    with open(c, "w") as f:
        f.write(text)
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
                           "-I", ODIR, "-o", so, c, "-lm"])
    env = dict(os.environ, FC_ORACLE_AMR_LIB=so, OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", "-rf"] + [_node(p) for p in pins]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    failed = re.findall(r"FAILED \S+::(\S+)", r.stdout)
    failed = failed + [P3 + f for f in failed]  # octree pins are named with their file
    if r.returncode < 0 or "Fatal Python error" in r.stderr + r.stdout:
        failed = failed + ["<crash>"]  # the pin run died on the planted mistake
    return r.returncode, failed


@pytest.fixture(scope="module")
def outcomes():
    src = open(SRC).read()
    jobs = {"control": (src, sorted({m[4] for m in MUTANTS}))}
    for name, old, new, occ, pin in MUTANTS:
        text = _mutate(src, old, new, occ)
        assert text != src, name
        jobs[name] = (text, [pin])
    with tempfile.TemporaryDirectory() as tmp:
        def one(item):
            name, (text, pins) = item
            d = os.path.join(tmp, name)
            os.makedirs(d)
            return name, _run_pins(text, pins, d)
        with cf.ThreadPoolExecutor(min(8, os.cpu_count() or 1)) as ex:
            return dict(ex.map(one, jobs.items()))


def test_mutant_texts_occur_in_the_oracle():
    src = open(SRC).read()
    for name, old, new, occ, pin in MUTANTS:
        assert src.count(old) > occ, name


def test_unaltered_copy_passes_every_named_pin(outcomes):
    rc, failed = outcomes["control"]
    assert rc == 0 and not failed, failed


@pytest.mark.parametrize("name,pin", [(m[0], m[4]) for m in MUTANTS], ids=[m[0] for m in MUTANTS])
def test_pin_catches_planted_mistake(outcomes, name, pin):
    rc, failed = outcomes[name]
    assert rc != 0 and (pin in failed or "<crash>" in failed), (name, pin, failed)
