"""Planted mistakes: the oracle's pins must notice a plausible error anywhere
in the oracle.

Each case copies oracle/fc_oracle.c, makes one small change of the kind a
slip produces (a dropped term or factor, a flipped sign, a transposed
operand, a wrong weight or index range), compiles the copy and runs the pin
named beside the change against it (through FC_ORACLE_LIB) in a child
process.  The pin must fail.  A control case runs every named pin against an
unaltered copy compiled the same way, and they must pass.  Nothing here calls
the CUDA library, and the oracle file itself is never modified.

One change is known to survive every pin and is left out: taking away the
partial pivoting of the patch LU.  The patch blocks are symmetrically
equilibrated saddle-point matrices with a symmetric positive definite velocity
block and a negative semi-definite stabilised pressure block
(quasi-definite), which LU factors stably without row exchanges; their owned
inverse rows still agree with a 40-digit solve to 1e-12.

Two skips in the Galerkin product are equivalent to their removal for these
boundary presets and are left out too: dropping constrained fine rows and
dropping constrained fine columns.  The constrained fine nodes lie on the box
faces, and the fine nodes a free coarse node interpolates to never do.
"""
import concurrent.futures as cf
import os
import re
import subprocess
import sys
import tempfile

import pytest

from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fc_oracle.c")
PINS = "tests/test_oracle_pins.py::"

# name, original text, altered text, which occurrence (0 = first), catching pin
MUTANTS = [
    # Q1 basis (Sec. 2.2)
    ("basis_swapped", "f1[k] = bit ? xi[k] : 1.0 - xi[k];", "f1[k] = bit ? 1.0 - xi[k] : xi[k];", 0,
     "test_nitsche_forms_on_linear_fields[2]"),
    ("gradient_sign", "d1[k] = (bit ? 1.0 : -1.0) / h[k];", "d1[k] = (bit ? -1.0 : 1.0) / h[k];", 0,
     "test_uncut_element_matrices_closed_form[True-2]"),
    # volume terms of a, b and f (eq. stokes_disc_weak_fcm_2)
    ("alpha_dropped_in_a", "e->A[a][b] = e->A[a][b] + w * al * L->eta * g;",
     "e->A[a][b] = e->A[a][b] + w * L->eta * g;", 0, "test_uncut_element_matrices_closed_form[False-2]"),
    ("eta_dropped_in_a", "e->A[a][b] = e->A[a][b] + w * al * L->eta * g;",
     "e->A[a][b] = e->A[a][b] + w * al * g;", 0, "test_textbook_2d_laplacian_numbers"),
    ("divergence_transposed", "- w * al * grad[a][c] * val[b];", "- w * al * val[a] * grad[b][c];", 0,
     "test_uncut_element_matrices_closed_form[True-2]"),
    ("alpha_dropped_in_b", "- w * al * grad[a][c] * val[b];", "- w * grad[a][c] * val[b];", 0,
     "test_uncut_element_matrices_closed_form[False-2]"),
    ("alpha_dropped_in_f", "e->f[c][a] = e->f[c][a] + w * al * f[c] * val[a];",
     "e->f[c][a] = e->f[c][a] + w * f[c] * val[a];", 0, "test_uncut_element_matrices_closed_form[False-2]"),
    # volume quadrature: Gauss rule and box split
    ("gauss_abscissa", "0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)", "0.5 - 0.5 / 3.0, 0.5 + 0.5 / 3.0", 0,
     "test_textbook_2d_laplacian_numbers"),
    ("leaf_weight", "for (int k = 0; k < dim; ++k) w = w * (hb[k] * 0.5);",
     "for (int k = 0; k < dim; ++k) w = w * hb[k];", 0, "test_fluid_volume_converges_with_depth[2]"),
    ("split_never", "if (cut && level < L->qdepth) {", "if (cut && level < 0) {", 0,
     "test_fluid_volume_converges_with_depth[2]"),
    # Nitsche terms on the obstacle boundary
    ("nitsche_consistency_sign", "double t = -L->eta * val[a] * dn[b] - L->eta * dn[a] * val[b]",
     "double t = -L->eta * val[a] * dn[b] + L->eta * dn[a] * val[b]", 0,
     "test_nitsche_forms_on_linear_fields[2]"),
    ("nitsche_one_sided", "double t = -L->eta * val[a] * dn[b] - L->eta * dn[a] * val[b]",
     "double t = -2.0 * L->eta * val[a] * dn[b]", 0, "test_nitsche_forms_on_linear_fields[2]"),
    ("nitsche_penalty_dropped", " + L->lambda * val[a] * val[b];", ";", 0,
     "test_nitsche_forms_on_linear_fields[2]"),
    ("pressure_boundary_sign", "e->B[c][a][b] = e->B[c][a][b] + bp->w * val[a] * bp->n[c] * val[b];",
     "e->B[c][a][b] = e->B[c][a][b] - bp->w * val[a] * bp->n[c] * val[b];", 0,
     "test_nitsche_forms_on_linear_fields[2]"),
    # boundary rule
    ("sphere_normal_outward", "p->n[k] = -e[k];", "p->n[k] = e[k];", 0,
     "test_boundary_rule_exact_integrals[3-sphere]"),
    ("circle_normal_outward", "n[0] = -ct; n[1] = -st;", "n[0] = ct; n[1] = st;", 0,
     "test_boundary_rule_exact_integrals[2-circle]"),
    ("circle_weight", "w = 0.5 * dt * sh->r[0];", "w = dt * sh->r[0];", 0,
     "test_boundary_rule_exact_integrals[2-circle]"),
    # pressure stabilisation c(q, p)
    ("stabilisation_mean_dropped", "(M[a][b] - m[a] * m[b] / vol)", "(M[a][b])", 0,
     "test_stabilisation_annihilates_constants[2]"),
    ("stabilisation_sign", "double v = -(1.0 / L->eta) * (M[a][b]", "double v = (1.0 / L->eta) * (M[a][b]", 0,
     "test_uncut_element_matrices_closed_form[True-2]"),
    ("stabilisation_eta", "double v = -(1.0 / L->eta) * (M[a][b]", "double v = -(M[a][b]", 0,
     "test_uncut_element_matrices_closed_form[True-2]"),
    # local solves: equilibrated LU (Sec. 3.1.2)
    ("equilibration_one_sided", "a[(long)r * n + c] = dsc[r] * a[(long)r * n + c] * dsc[c];",
     "a[(long)r * n + c] = dsc[r] * a[(long)r * n + c];", 0, "test_whole_domain_patch_is_exact_solve[2]"),
    ("equilibration_unscaled_solution",
     "  lu_solve(n, lu, piv, b);\n  for (int j = 0; j < n; ++j) b[j] = dsc[j] * b[j];",
     "  lu_solve(n, lu, piv, b);", 0, "test_whole_domain_patch_is_exact_solve[2]"),
    ("back_substitution_transposed", "for (int c = r + 1; c < n; ++c) s = s - lu[(long)r * n + c] * b[c];",
     "for (int c = r + 1; c < n; ++c) s = s - lu[(long)c * n + r] * b[c];", 0,
     "test_whole_domain_patch_is_exact_solve[2]"),
    # the RA sweep (Sec. 3.1)
    ("omega_dropped", "xn[i * nd + c] = x[i * nd + c] + L->omega * y[c];", "xn[i * nd + c] = x[i * nd + c] + y[c];",
     0, "test_sweep_order_and_partition_independent[2]"),
    ("dirichlet_rows_frozen", "if (L->fixed[k]) xn[k] = x[k] + r[k];", "if (L->fixed[k]) xn[k] = x[k];", 0,
     "test_sweep_order_and_partition_independent[2]"),
    ("patch_shifted", "long ib[3] = {ia[0] + dx - 2, ia[1] + dy - 2, dim == 3 ? ia[2] + dz - 2 : 0};",
     "long ib[3] = {ia[0] + dx - 1, ia[1] + dy - 2, dim == 3 ? ia[2] + dz - 2 : 0};", 0, "test_patch_sizes"),
    ("pressure_patch_shrunk", "for (int dx = 0; dx < 3; ++dx) {\n        long ib[3] = {ia[0] + dx - 1,",
     "for (int dx = 1; dx < 3; ++dx) {\n        long ib[3] = {ia[0] + dx - 1,", 0, "test_patch_sizes"),
    # transfers (Sec. 3)
    ("prolongation_weight", "wgt = wgt * (lo[k] == hi[k] ? 1.0 : 0.5);", "wgt = wgt * (lo[k] == hi[k] ? 1.0 : 0.25);",
     0, "test_prolongation_exact_on_linear_fields[2]"),
    ("restriction_weight", "wgt = wgt * (lo[k] == hi[k] ? 1.0 : 0.5);", "wgt = wgt * (lo[k] == hi[k] ? 1.0 : 0.25);",
     1, "test_restriction_is_transpose_of_prolongation[2]"),
    ("restriction_keeps_constrained", "if (Cc->fixed[k]) bc[k] = 0.0;", "if (0) bc[k] = 0.0;", 1,
     "test_restriction_with_strong_dirichlet_rows[2-1]"),
    # V-cycle
    ("coarse_correction_dropped", "  or_prolong_add(L, C, xc, x);\n", "\n", 0,
     "test_iteration_counts_h_independent_without_obstacle"),
    ("post_smoothing_dropped", "for (int s = 0; s < M->nu_post; ++s) or_sweep(L, b, x, M->mode, NULL);", "", 0,
     "test_iteration_counts_h_independent_without_obstacle"),
    # FGMRES with modified Gram-Schmidt and Givens rotations
    ("mgs_sign", "w[t] = w[t] - hij * V[(long)i * n + t];", "w[t] = w[t] + hij * V[(long)i * n + t];", 0,
     "test_fgmres_reaches_direct_solution[2]"),
    ("givens_sign", "H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;", "H[(i + 1) * m + j] = sn[i] * a + cs[i] * c;",
     0, "test_fgmres_reaches_direct_solution[2]"),
    ("hessenberg_transposed", "for (int t = i + 1; t < k; ++t) s = s - H[i * m + t] * y[t];",
     "for (int t = i + 1; t < k; ++t) s = s - H[t * m + i] * y[t];", 0, "test_fgmres_reaches_direct_solution[2]"),
    # strong Dirichlet data of the two setups
    ("inflow_profile_scale", "double v = 4.0 * L->ubar * s * (1.0 - s);", "double v = L->ubar * s * (1.0 - s);", 0,
     "test_manufactured_2d_channel_convergence"),
    ("inflow_all_components", "if (!wall && inflow && c == 0) {", "if (!wall && inflow) {", 0,
     "test_manufactured_2d_channel_convergence"),
    ("channel_upper_wall_missing", "int wall = (idx[1] == 0 || idx[1] == L->n[1]);", "int wall = (idx[1] == 0);", 0,
     "test_presets_constrain_the_faces_of_the_setups[2-0]"),
    ("porous_upper_wall_missing", "int wall = (idx[1] == 0 || idx[1] == L->n[1]);", "int wall = (idx[1] == 0);", 1,
     "test_presets_constrain_the_faces_of_the_setups[2-1]"),
    # level set and alpha (Sec. 2)
    ("ellipse_rotation_sign", "double yp = -s->rot[1] * dx + s->rot[0] * dy;",
     "double yp = s->rot[1] * dx + s->rot[0] * dy;", 0, "test_ellipse_area"),
    ("circle_sqrt_dropped", "return s->r[0] - sqrt(q);", "return s->r[0] - q;", 0,
     "test_fluid_volume_converges_with_depth[2]"),
    ("union_as_intersection", "if (s == 0 || q > p) p = q;", "if (s == 0 || q < p) p = q;", 0,
     "test_overlapping_obstacles_form_a_union"),
    ("alpha_swapped", "return phi_all(L, x) > 0.0 ? L->alpha : 1.0;", "return phi_all(L, x) > 0.0 ? 1.0 : L->alpha;",
     0, "test_uncut_element_matrices_closed_form[True-2]"),
    ("sample_points_quarter", "double x[3] = {lo[0] + hb[0] * (0.5 * i), lo[1] + hb[1] * (0.5 * j),",
     "double x[3] = {lo[0] + hb[0] * (0.25 * i), lo[1] + hb[1] * (0.25 * j),", 0,
     "test_fluid_volume_converges_with_depth[3]"),
    ("stabilisation_gauss_weight", "for (int k = 0; k < dim; ++k) w = w * (L->h[k] * 0.5);",
     "for (int k = 0; k < dim; ++k) w = w * L->h[k];", 0, "test_uncut_element_matrices_closed_form[True-2]"),
    # body force
    ("force_cos_as_sin", "f[1] = L->force[1] * cos(pi * x[1]);", "f[1] = L->force[1] * sin(pi * x[1]);", 0,
     "test_load_vector_channel_force"),
    ("force_z_factor_dropped", "if (L->dim == 3) f[0] = f[0] * sin(pi * x[2]);", "", 0,
     "test_manufactured_3d_duct_convergence"),
    # boundary rule, more
    ("sphere_weight_radius", "double w = r * r * (0.5 * dm) * df;", "double w = r * (0.5 * dm) * df;", 0,
     "test_boundary_rule_exact_integrals[3-sphere]"),
    ("ellipse_normal_axes", "double nx = b * ct, ny = a * st;", "double nx = a * ct, ny = b * st;", 0,
     "test_boundary_rule_exact_integrals[2-ellipse]"),
    ("boundary_point_other_shape_kept", "if (!ok || point_in_other_shape(L, s, x)) continue;", "if (!ok) continue;",
     0, "test_overlapping_obstacles_form_a_union"),
    # assembly of the rows of L and of the residual
    ("coupling_transposed", "else if (cb < dim) v = e->B[cb][lb][la];", "else if (cb < dim) v = e->B[cb][la][lb];",
     0, "test_operator_exactly_symmetric[2-0]"),
    ("velocity_components_coupled", "if (ca < dim && cb < dim) v = (ca == cb) ? e->A[la][lb] : 0.0;",
     "if (ca < dim && cb < dim) v = e->A[la][lb];", 0, "test_manufactured_2d_channel_convergence"),
    ("lift_sign", "rhs = rhs - out[nb * nd + cb] * wb;", "rhs = rhs + out[nb * nd + cb] * wb;", 0,
     "test_manufactured_2d_channel_convergence"),
    ("constrained_column_kept", "        rhs = rhs - out[nb * nd + cb] * wb;\n        out[nb * nd + cb] = 0.0;",
     "        rhs = rhs - out[nb * nd + cb] * wb;", 0, "test_operator_exactly_symmetric[2-0]"),
    ("residual_sign", "for (long i = 0; i < L->ndof; ++i) r[i] = b[i] - r[i];",
     "for (long i = 0; i < L->ndof; ++i) r[i] = r[i] - b[i];", 0, "test_fgmres_reaches_direct_solution[2]"),
    ("pressure_not_owned", "if (nb == node) own[dim] = n;", ";", 0, "test_owner_count_is_one[2]"),
    # coarse solve and FGMRES, more
    ("coarse_solve_unequilibrated_rhs", "eq_solve((int)L->ndof, M->coarse_lu, M->coarse_d, M->coarse_piv, t);",
     "lu_solve((int)L->ndof, M->coarse_lu, M->coarse_piv, t);", 0, "test_standalone_gmg_reduces_residual"),
    ("fgmres_restart_residual_sign", "for (long i = 0; i < n; ++i) V[i] = w[i] / beta;",
     "for (long i = 0; i < n; ++i) V[i] = -w[i] / beta;", 0, "test_fgmres_reaches_direct_solution[2]"),
    ("fgmres_update_uses_v", "for (long t = 0; t < n; ++t) x[t] = x[t] + y[i] * Z[(long)i * n + t];",
     "for (long t = 0; t < n; ++t) x[t] = x[t] + y[i] * V[(long)i * n + t];", 0,
     "test_fgmres_reaches_direct_solution[2]"),
    # Galerkin coarse operator (R L_f P)
    ("galerkin_weight", "return d == 0 ? 1.0 : ((d == 1 || d == -1) ? 0.5 : 0.0);",
     "return d == 0 ? 1.0 : ((d == 1 || d == -1) ? 0.25 : 0.0);", 0,
     "test_galerkin_equals_rediscretisation_without_obstacles[2]"),
    ("galerkin_coarse_identity_lost", "Cc->val[q] = (Cc->fixed[row] && Cc->col[q] == row) ? 1.0 : 0.0;",
     "Cc->val[q] = 0.0;", 0, "test_galerkin_equals_rediscretisation_without_obstacles[2]"),
    ("galerkin_column_weight_shifted", "wj = wj * q1_weight(ja[k] - 2 * Ja[k]);",
     "wj = wj * q1_weight(ja[k] - 2 * Ja[k] + 1);", 0, "test_galerkin_pressure_block_closed_form[2]"),
]


def _mutate(src, old, new, occ):
    idx = -1
    for _ in range(occ + 1):
        idx = src.index(old, idx + 1)
    return src[:idx] + new + src[idx + len(old):]


def _run_pins(text, pins, workdir):
    """Compile `text` as the oracle and run the given pins against it; returns
    (pytest return code, names of the failed pins)."""
    c = os.path.join(workdir, "fc_oracle_variant.c")
    so = os.path.join(workdir, "libfc_oracle_variant.so")
    with open(c, "w") as f:
        f.write(text)
    O.compile_source(c, so)
    env = dict(os.environ, FC_ORACLE_LIB=so, OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", "-rf"] + [PINS + p for p in pins]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, re.findall(r"FAILED \S+::(\S+)", r.stdout)


@pytest.fixture(scope="module")
def outcomes():
    """Every mutant (and the unaltered control) through its pin, in parallel."""
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


def test_mutant_texts_are_unique_in_the_oracle():
    """Each original text occurs at least occ+1 times, so every mutant alters
    the place it names."""
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
