"""Planted mistakes in the Q2-Q1 oracle: its pins must notice a plausible
error in every part of it.

Each case copies oracle/fc_oracle_q2.c, makes one small change (a wrong
weight, basis function, sign, index range or dropped factor), compiles the
copy against the unaltered fc_oracle.c it includes, and runs the pin named
beside the change against it (through FC_ORACLE_Q2_LIB) in a child process;
the pin must fail.  A control case runs every named pin against an
unaltered copy compiled the same way, and they must pass.  Nothing here
calls the CUDA library, and the oracle files are never modified.

Like the Q1-Q1 oracle's pivoting, the row-max equilibration of the patch
blocks only moves rounding and is left out.
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
SRC = os.path.join(ODIR, "fc_oracle_q2.c")
PINS = "tests/test_oracle_q2_pins.py::"

# name, original text, altered text, occurrence, catching pin
MUTANTS = [
    # Q2 and Q1 basis
    ("q2_bubble_sign", "v[1] = 4.0 * t * (1.0 - t);", "v[1] = 4.0 * t * (1.0 + t);", 0,
     "test_uncut_element_matrices_closed_form[2]"),
    ("q2_derivative", "d[2] = 4.0 * t - 1.0;", "d[2] = 4.0 * t + 1.0;", 0,
     "test_uncut_element_matrices_closed_form[2]"),
    ("q1_pressure_basis_swapped", "f = f * (((b >> k) & 1) ? t[k] : 1.0 - t[k]);",
     "f = f * (((b >> k) & 1) ? 1.0 - t[k] : t[k]);", 0, "test_uncut_element_matrices_closed_form[2]"),
    # volume rule
    ("gauss_weight", "gw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};", "gw[3] = {5.0 / 18.0, 6.0 / 18.0, 5.0 / 18.0};",
     0, "test_uncut_element_matrices_closed_form[2]"),
    ("gauss_point", "0.5 - 0.5 * sqrt(0.6), 0.5, 0.5 + 0.5 * sqrt(0.6)", "0.5 - 0.5 * sqrt(0.5), 0.5, 0.5 + 0.5 * sqrt(0.5)",
     0, "test_uncut_element_matrices_closed_form[2]"),
    ("split_never", "if (npos != 0 && npos != ns && level < L->qdepth) {", "if (npos != 0 && npos != ns && level < 0) {",
     0, "test_cut_quadrature_area_and_perimeter"),
    ("alpha_dropped_in_a", "e->A[a][b] = e->A[a][b] + w * al * L->eta * g;", "e->A[a][b] = e->A[a][b] + w * L->eta * g;",
     0, "test_q2_nitsche_forms_on_linear_fields[2]"),
    ("divergence_sign", "e->B[c][a][b] = e->B[c][a][b] - w * al * grad[a][c] * pv[b];",
     "e->B[c][a][b] = e->B[c][a][b] + w * al * grad[a][c] * pv[b];", 0, "test_uncut_element_matrices_closed_form[2]"),
    # Nitsche terms
    ("nitsche_consistency_sign", "double t = -L->eta * val[a] * dn[b] - L->eta * dn[a] * val[b] + L->lambda",
     "double t = L->eta * val[a] * dn[b] - L->eta * dn[a] * val[b] + L->lambda", 0,
     "test_q2_nitsche_forms_on_linear_fields[2]"),
    ("nitsche_penalty_dropped", "- L->eta * dn[a] * val[b] + L->lambda * val[a] * val[b];",
     "- L->eta * dn[a] * val[b];", 0, "test_q2_nitsche_forms_on_linear_fields[2]"),
    ("boundary_coupling_sign", "e->B[c][a][b] = e->B[c][a][b] + bp->w * val[a] * bp->n[c] * pv[b];",
     "e->B[c][a][b] = e->B[c][a][b] - bp->w * val[a] * bp->n[c] * pv[b];", 0,
     "test_q2_nitsche_forms_on_linear_fields[2]"),
    # Dirichlet data and elimination
    ("inflow_profile_scale", "double v = 4.0 * L->ubar * s * (1.0 - s);", "double v = L->ubar * s * (1.0 - s);", 0,
     "test_manufactured_2d_channel_rates"),
    ("upper_wall_missing", "(J == 0 || J == Q->nf[1] - 1)", "(J == 0)", 0, "test_manufactured_3d_duct_rate"),
    ("lift_sign", "rhs[r] = rhs[r] - val[p] * wfix[col[p]];", "rhs[r] = rhs[r] + val[p] * wfix[col[p]];", 0,
     "test_manufactured_2d_channel_rates"),
    # patches and ownership
    ("ownership_range", "const int owned = s0 >= 0 && s0 <= 1 &&", "const int owned = s0 >= 0 && s0 <= 2 &&", 0,
     "test_owner_count_is_one[2-1]"),
    ("pressure_not_owned", "if (i == a[0] && j == a[1] && k == a[2]) own[no - 1] = n;", ";", 0,
     "test_owner_count_is_one[2-1]"),
    ("velocity_box_shifted", "const long I = 2 * a[0] - 4 + dx,", "const long I = 2 * a[0] - 3 + dx,", 0,
     "test_q2_patch_sizes[2]"),
    ("pressure_box_shrunk", "const long i = a[0] - 1 + dx,", "const long i = a[0] + dx,", 0, "test_q2_patch_sizes[2]"),
    # local solve and sweep
    ("equilibration_one_sided", "a[(long)r * n + c] = dsc[r] * a[(long)r * n + c] * dsc[c];",
     "a[(long)r * n + c] = dsc[r] * a[(long)r * n + c];", 0, "test_whole_domain_patch_is_the_direct_solve[2]"),
    ("omega_dropped", "xn[pd[o]] = x[pd[o]] + om * s;", "xn[pd[o]] = x[pd[o]] + s;", 0,
     "test_whole_domain_patch_is_the_direct_solve[2]"),
    ("dirichlet_rows_frozen", "if (Q->fixed[k]) xn[k] = x[k] + r[k];", "if (Q->fixed[k]) xn[k] = x[k];", 0,
     "test_whole_domain_patch_is_the_direct_solve[2]"),
    ("residual_sign", "for (long k = 0; k < Q->ndof; ++k) r[k] = b[k] - r[k];",
     "for (long k = 0; k < Q->ndof; ++k) r[k] = r[k] - b[k];", 0, "test_whole_domain_patch_is_the_direct_solve[2]"),
    # transfers
    ("q2_transfer_position", "const double t = (double)(F - 4 * m) / 4.0;", "const double t = (double)(F - 4 * m) / 2.0;",
     0, "test_transfers_exact_and_transposed[2]"),
    ("q1_transfer_weight", "else { *wl = 0.5; *wh = 0.5; }", "else { *wl = 0.25; *wh = 0.75; }", 0,
     "test_transfers_exact_and_transposed[2]"),
    ("restriction_not_transposed", "bc[d] = bc[d] + wt * rv;", "bc[d] = bc[d] + 0.5 * wt * rv;", 0,
     "test_transfers_exact_and_transposed[2]"),
    # V-cycle and FGMRES
    ("coarse_correction_dropped", "  q2_prolong_add(L, C, xc, x);\n", "\n", 0,
     "test_q2_iteration_counts_bounded_under_refinement"),
    ("mgs_sign", "for (long t = 0; t < n; ++t) w[t] = w[t] - hij * V[(long)i * n + t];",
     "for (long t = 0; t < n; ++t) w[t] = w[t] + hij * V[(long)i * n + t];", 0,
     "test_q2_fgmres_reaches_direct_solution[2]"),
    ("fgmres_update_uses_v", "for (long t = 0; t < n; ++t) x[t] = x[t] + y[i] * Z[(long)i * n + t];",
     "for (long t = 0; t < n; ++t) x[t] = x[t] + y[i] * V[(long)i * n + t];", 0,
     "test_q2_fgmres_reaches_direct_solution[2]"),
]


def _mutate(src, old, new, occ):
    idx = -1
    for _ in range(occ + 1):
        idx = src.index(old, idx + 1)
    return src[:idx] + new + src[idx + len(old):]


def _run_pins(text, pins, workdir):
    c = os.path.join(workdir, "fc_oracle_q2_variant.c")
    so = os.path.join(workdir, "libfc_oracle_q2_variant.so")
    with open(c, "w") as f:
        f.write(text)
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
                           "-I", ODIR, "-o", so, c, "-lm"])
    env = dict(os.environ, FC_ORACLE_Q2_LIB=so, OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", "-rf"] + [PINS + p for p in pins]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, re.findall(r"FAILED \S+::(\S+)", r.stdout)


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
    assert rc != 0 and pin in failed, (name, pin, failed)
