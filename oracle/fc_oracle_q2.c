/*
 * fc_oracle_q2.c -- plain, slow FP64 CPU oracle for the restricted additive
 * smoother with the Q2-Q1 (Taylor-Hood) element pair and a lower-corner
 * ownership rule.
 *
 * TEST INFRASTRUCTURE ONLY, like fc_oracle.c (which it includes for the
 * level set, the body force, the boundary quadrature rule and the dense
 * equilibrated LU: the same readings as the Q1-Q1 oracle).  Nothing in the
 * product library links, includes or calls it.
 *
 * The paper's method (Sec. 2-3) uses equal-order Q1-Q1 with the local L2
 * pressure projection; its restricted prolongation R~_i writes p_i and the
 * velocity DoFs "at the same node".  With Q2 velocities most velocity nodes
 * (edge midpoints, face and cell centres) are not at a pressure node, so
 * this variant fixes an owner for each: the Q2 node with fine index
 * (2a + s) (s in {0,1}^d) belongs to the pressure vertex a at the lower
 * corner of its cell, edge or face.  Every other part follows the paper:
 *   - weak form of eq. stokes_weak_fcm with the alpha-scaled volume terms and
 *     the symmetric Nitsche terms on Gamma_D (lambda = beta eta / h_min);
 *   - Q2 velocity per component and Q1 pressure, inf-sup stable, so no
 *     pressure stabilisation (c = 0);
 *   - cut-cell volume rule: the same recursive box split as the Q1 oracle,
 *     leaves with the tensor 3-point Gauss rule (exact for the Q2 products
 *     on uncut boxes); boundary points: the Q1 oracle's rule;
 *   - strong Dirichlet data per preset on the box faces at every Q2 node on
 *     them, eliminated symmetrically;
 *   - patch S_i of pressure vertex a: the pressures of the 3^d vertices
 *     around a and the velocities of every Q2 node in the cells touching
 *     them (fine indices 2a-4 .. 2a+4 per direction), constrained DoFs
 *     excluded; exact local solves (Sec. 3.1.2) by LU with partial pivoting
 *     of D L_i D, D = (row max |L_i|)^{-1/2} (the pressure block is zero, so
 *     the diagonal cannot scale it);
 *   - hierarchy by uniform halving; velocity transfer = Q2 interpolation
 *     (nested spaces), pressure transfer = Q1 interpolation, R = P^T;
 *     direct coarse solve; V-cycle; FGMRES(m) with MGS; standalone GMG.
 *
 * DoF layout: velocity first, Q2 node (I, J, K) (I fastest, 0 .. 2 n_k) with
 * its d components, then the pressure at vertex (i, j, k) (i fastest).
 */
#include "fc_oracle.c"

#define Q2PMAX 2214 /* 9^3 * 3 + 27 */
#define Q2OMAX 25   /* 2^3 * 3 + 1 */

typedef struct {
  or_level* g;          /* geometry, boundary points, parameters */
  int dim, nf[3], nv1[3];
  long nvnode, nv, np, ndof, ncell;
  long* rowptr;
  long* col;
  double* val;
  double* rhs;
  unsigned char* fixed;
  double* wfix;
  /* cache_inverse: per patch */
  int* pn;
  long* pdof;   /* [np][Q2PMAX] */
  int* pown;    /* [np][Q2OMAX] */
  double* pinv; /* [np][Q2OMAX][Q2PMAX] */
} q2_level;

typedef struct {
  double A[27][27];    /* velocity block per component */
  double B[3][27][8];  /* velocity node a comp c, pressure vertex b */
  double f[3][27];
  double fluid_volume, boundary_measure;
  int nvol, nbnd;
} q2_elem;

/* ------------------------------------------------------------------------ */
/* Q2 basis: tensor products of q0 = (1-t)(1-2t), q1 = 4t(1-t), q2 = t(2t-1) */
/* ------------------------------------------------------------------------ */

static void q2_1d(double t, double* v, double* d) {
  v[0] = (1.0 - t) * (1.0 - 2.0 * t);
  v[1] = 4.0 * t * (1.0 - t);
  v[2] = t * (2.0 * t - 1.0);
  d[0] = 4.0 * t - 3.0;
  d[1] = 4.0 - 8.0 * t;
  d[2] = 4.0 * t - 1.0;
}

/* values and gradients of the 3^d Q2 functions (local a = ax + 3 ay + 9 az)
 * and the 2^d Q1 functions (bit k = position in direction k) at x */
static void q2_basis(int dim, const double* x0, const double* h, const double* x, double* val, double (*grad)[3],
                     double* pval) {
  double v[3][3], d[3][3], t[3] = {0, 0, 0};
  for (int k = 0; k < 3; ++k) {
    t[k] = k < dim ? (x[k] - x0[k]) / h[k] : 0.0;
    q2_1d(t[k], v[k], d[k]);
  }
  const int na = dim == 3 ? 27 : 9;
  for (int a = 0; a < na; ++a) {
    const int ia[3] = {a % 3, (a / 3) % 3, a / 9};
    double f = 1.0;
    for (int k = 0; k < dim; ++k) f = f * v[k][ia[k]];
    val[a] = f;
    for (int k = 0; k < 3; ++k) grad[a][k] = 0.0;
    for (int k = 0; k < dim; ++k) {
      double g = d[k][ia[k]] / h[k];
      for (int m = 0; m < dim; ++m)
        if (m != k) g = g * v[m][ia[m]];
      grad[a][k] = g;
    }
  }
  for (int b = 0; b < (1 << dim); ++b) {
    double f = 1.0;
    for (int k = 0; k < dim; ++k) f = f * (((b >> k) & 1) ? t[k] : 1.0 - t[k]);
    pval[b] = f;
  }
}

/* ------------------------------------------------------------------------ */
/* Element data                                                              */
/* ------------------------------------------------------------------------ */

typedef struct {
  const or_level* L;
  double x0[3];
  q2_elem* e;
} q2_ctx;

static void q2_vol_point(q2_ctx* q, const double* x, double w) {
  const or_level* L = q->L;
  const int dim = L->dim, na = dim == 3 ? 27 : 9, nb = 1 << dim;
  double val[27], grad[27][3], pv[8], f[3];
  q2_basis(dim, q->x0, L->h, x, val, grad, pv);
  const double al = alpha_at(L, x);
  force_at(L, x, f);
  q2_elem* e = q->e;
  for (int a = 0; a < na; ++a)
    for (int b = a; b < na; ++b) {
      double g = 0.0;
      for (int k = 0; k < dim; ++k) g = g + grad[a][k] * grad[b][k];
      e->A[a][b] = e->A[a][b] + w * al * L->eta * g;
    }
  for (int c = 0; c < dim; ++c)
    for (int a = 0; a < na; ++a) {
      for (int b = 0; b < nb; ++b) e->B[c][a][b] = e->B[c][a][b] - w * al * grad[a][c] * pv[b];
      e->f[c][a] = e->f[c][a] + w * al * f[c] * val[a];
    }
  if (al == 1.0) e->fluid_volume = e->fluid_volume + w;
  e->nvol++;
}

static void q2_vol_box(q2_ctx* q, const double* lo, const double* hb, int level) {
  const or_level* L = q->L;
  const int dim = L->dim;
  int npos = 0, ns = 0;
  const int m3 = dim == 3 ? 3 : 1;
  for (int k = 0; k < m3; ++k)
    for (int j = 0; j < 3; ++j)
      for (int i = 0; i < 3; ++i) {
        double x[3] = {lo[0] + hb[0] * (0.5 * i), lo[1] + hb[1] * (0.5 * j), dim == 3 ? lo[2] + hb[2] * (0.5 * k) : 0.0};
        if (phi_all(L, x) > 0.0) npos++;
        ns++;
      }
  if (npos != 0 && npos != ns && level < L->qdepth) {
    double hc[3] = {hb[0] * 0.5, hb[1] * 0.5, hb[2] * 0.5};
    for (int ch = 0; ch < (1 << dim); ++ch) {
      double lc[3] = {lo[0], lo[1], lo[2]};
      for (int k = 0; k < dim; ++k)
        if ((ch >> k) & 1) lc[k] = lo[k] + hc[k];
      q2_vol_box(q, lc, hc, level + 1);
    }
    return;
  }
  /* tensor 3-point Gauss rule: nodes 1/2 - sqrt(3/5)/2, 1/2, 1/2 + sqrt(3/5)/2,
   * weights 5/18, 8/18, 5/18 of the box width */
  const double gp[3] = {0.5 - 0.5 * sqrt(0.6), 0.5, 0.5 + 0.5 * sqrt(0.6)};
  const double gw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  for (int k = 0; k < (dim == 3 ? 3 : 1); ++k)
    for (int j = 0; j < 3; ++j)
      for (int i = 0; i < 3; ++i) {
        double x[3] = {lo[0] + hb[0] * gp[i], lo[1] + hb[1] * gp[j], dim == 3 ? lo[2] + hb[2] * gp[k] : 0.0};
        double w = (hb[0] * gw[i]) * (hb[1] * gw[j]);
        if (dim == 3) w = w * (hb[2] * gw[k]);
        q2_vol_point(q, x, w);
      }
}

static void q2_compute_elem(const or_level* L, long cell, q2_elem* e) {
  memset(e, 0, sizeof(*e));
  const int dim = L->dim, na = dim == 3 ? 27 : 9, nb = 1 << dim;
  long idx[3];
  q2_ctx q;
  q.L = L;
  q.e = e;
  cell_x0(L, cell, q.x0, idx);
  q2_vol_box(&q, q.x0, L->h, 0);
  /* Nitsche terms on Gamma_D, the same as the Q1 element's with Q2 functions */
  for (long p = L->cell_bstart[cell]; p < L->cell_bstart[cell + 1]; ++p) {
    const or_bpoint* bp = &L->bp[p];
    double val[27], grad[27][3], pv[8], dn[27];
    q2_basis(dim, q.x0, L->h, bp->x, val, grad, pv);
    for (int a = 0; a < na; ++a) {
      double s = 0.0;
      for (int k = 0; k < dim; ++k) s = s + bp->n[k] * grad[a][k];
      dn[a] = s;
    }
    for (int a = 0; a < na; ++a)
      for (int b = a; b < na; ++b) {
        double t = -L->eta * val[a] * dn[b] - L->eta * dn[a] * val[b] + L->lambda * val[a] * val[b];
        e->A[a][b] = e->A[a][b] + bp->w * t;
      }
    for (int c = 0; c < dim; ++c)
      for (int a = 0; a < na; ++a)
        for (int b = 0; b < nb; ++b) e->B[c][a][b] = e->B[c][a][b] + bp->w * val[a] * bp->n[c] * pv[b];
    e->boundary_measure = e->boundary_measure + bp->w;
    e->nbnd++;
  }
  for (int a = 0; a < na; ++a)
    for (int b = 0; b < a; ++b) e->A[a][b] = e->A[b][a];
}

/* ------------------------------------------------------------------------ */
/* Level, DoFs, Dirichlet data                                               */
/* ------------------------------------------------------------------------ */

q2_level* q2_level_new(int dim, const int* n, const double* lo, const double* hi, int nshape, const double* shapes,
                       double alpha, int qdepth, double eta, double beta, double omega, int preset, int force_kind,
                       const double* force, double ubar) {
  q2_level* Q = (q2_level*)calloc(1, sizeof(q2_level));
  Q->g = or_level_new(dim, n, lo, hi, nshape, shapes, alpha, qdepth, eta, beta, omega, preset, force_kind, force, ubar);
  Q->dim = dim;
  Q->nvnode = 1;
  Q->np = 1;
  for (int k = 0; k < 3; ++k) {
    Q->nf[k] = k < dim ? 2 * n[k] + 1 : 1;
    Q->nv1[k] = k < dim ? n[k] + 1 : 1;
    Q->nvnode *= Q->nf[k];
    Q->np *= Q->nv1[k];
  }
  Q->nv = Q->nvnode * dim;
  Q->ndof = Q->nv + Q->np;
  Q->ncell = Q->g->ncell;
  return Q;
}

void q2_level_free(q2_level* Q) {
  if (!Q) return;
  or_level_free(Q->g);
  free(Q->rowptr); free(Q->col); free(Q->val); free(Q->rhs); free(Q->fixed); free(Q->wfix);
  free(Q->pn); free(Q->pdof); free(Q->pown); free(Q->pinv);
  free(Q);
}

long q2_ndof(const q2_level* Q) { return Q->ndof; }
long q2_nv(const q2_level* Q) { return Q->nv; }
long q2_np(const q2_level* Q) { return Q->np; }
long q2_nnz(const q2_level* Q) { return Q->rowptr ? Q->rowptr[Q->ndof] : 0; }

static long q2_vnode(const q2_level* Q, long I, long J, long K) { return I + Q->nf[0] * (J + (long)Q->nf[1] * K); }
static long q2_pnode(const q2_level* Q, long i, long j, long k) { return i + Q->nv1[0] * (j + (long)Q->nv1[1] * k); }

/* velocity component c at Q2 node (I, J, K): 1 if constrained, *w its value
 * (the presets of the Q1 oracle evaluated at the node's position) */
static int q2_dirichlet(const q2_level* Q, long I, long J, long K, int c, double* w) {
  const or_level* L = Q->g;
  const int dim = Q->dim;
  *w = 0.0;
  const int wall = (J == 0 || J == Q->nf[1] - 1) || (dim == 3 && (K == 0 || K == Q->nf[2] - 1));
  if (L->preset == 0) {
    const int inflow = I == 0;
    if (!wall && !inflow) return 0;
    if (!wall && inflow && c == 0) {
      const double y = L->lo[1] + 0.5 * (double)J * L->h[1];
      const double s = (y - L->lo[1]) / (L->hi[1] - L->lo[1]);
      double v = 4.0 * L->ubar * s * (1.0 - s);
      if (dim == 3) {
        const double z = L->lo[2] + 0.5 * (double)K * L->h[2];
        const double t = (z - L->lo[2]) / (L->hi[2] - L->lo[2]);
        v = v * 4.0 * t * (1.0 - t);
      }
      *w = v;
    }
    return 1;
  }
  if (L->preset == 1) return wall;
  return 0;
}

int q2_cell_element(const q2_level* Q, long cell, double* A, double* B, double* f, double* stats) {
  if (cell < 0 || cell >= Q->ncell) return -1;
  q2_elem e;
  q2_compute_elem(Q->g, cell, &e);
  const int na = Q->dim == 3 ? 27 : 9, nb = 1 << Q->dim;
  for (int a = 0; a < na; ++a)
    for (int b = 0; b < na; ++b) A[a * na + b] = e.A[a][b];
  for (int c = 0; c < Q->dim; ++c)
    for (int a = 0; a < na; ++a) {
      for (int b = 0; b < nb; ++b) B[(c * na + a) * nb + b] = e.B[c][a][b];
      f[c * na + a] = e.f[c][a];
    }
  stats[0] = e.fluid_volume;
  stats[1] = e.boundary_measure;
  stats[2] = e.nvol;
  stats[3] = e.nbnd;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Assembly: element triplets, stable sort by (row, col), sums in cell order */
/* ------------------------------------------------------------------------ */

typedef struct {
  long r, c;
  long seq;
  double v;
} q2_trip;

static int trip_cmp(const void* a, const void* b) {
  const q2_trip* x = (const q2_trip*)a;
  const q2_trip* y = (const q2_trip*)b;
  if (x->r != y->r) return x->r < y->r ? -1 : 1;
  if (x->c != y->c) return x->c < y->c ? -1 : 1;
  return x->seq < y->seq ? -1 : (x->seq > y->seq ? 1 : 0);
}

void q2_assemble(q2_level* Q) {
  if (Q->rowptr) return;
  const or_level* L = Q->g;
  const int dim = Q->dim, na = dim == 3 ? 27 : 9, nb = 1 << dim;
  const long per = (long)na * na * dim + 2L * dim * na * nb;
  q2_trip* T = (q2_trip*)malloc(sizeof(q2_trip) * (size_t)(per * Q->ncell));
  double* rhs = (double*)calloc((size_t)Q->ndof, sizeof(double));
  q2_elem* E = (q2_elem*)malloc(sizeof(q2_elem) * (size_t)Q->ncell);
#pragma omp parallel for schedule(dynamic, 8)
  for (long cell = 0; cell < Q->ncell; ++cell) q2_compute_elem(L, cell, &E[cell]);
  long nt = 0;
  for (long cell = 0; cell < Q->ncell; ++cell) {
    const q2_elem* e = &E[cell];
    long ci[3] = {cell % L->n[0], (cell / L->n[0]) % L->n[1], dim == 3 ? cell / ((long)L->n[0] * L->n[1]) : 0};
    long vd[27], pd[8];
    for (int a = 0; a < na; ++a)
      vd[a] = q2_vnode(Q, 2 * ci[0] + a % 3, 2 * ci[1] + (a / 3) % 3, dim == 3 ? 2 * ci[2] + a / 9 : 0);
    for (int b = 0; b < nb; ++b)
      pd[b] = Q->nv + q2_pnode(Q, ci[0] + (b & 1), ci[1] + ((b >> 1) & 1), dim == 3 ? ci[2] + ((b >> 2) & 1) : 0);
    for (int c = 0; c < dim; ++c) {
      for (int a = 0; a < na; ++a) {
        for (int b = 0; b < na; ++b) {
          T[nt] = (q2_trip){vd[a] * dim + c, vd[b] * dim + c, nt, e->A[a][b]};
          nt++;
        }
        for (int b = 0; b < nb; ++b) {
          T[nt] = (q2_trip){vd[a] * dim + c, pd[b], nt, e->B[c][a][b]};
          nt++;
          T[nt] = (q2_trip){pd[b], vd[a] * dim + c, nt, e->B[c][a][b]};
          nt++;
        }
        rhs[vd[a] * dim + c] = rhs[vd[a] * dim + c] + e->f[c][a];
      }
    }
  }
  free(E);
  qsort(T, (size_t)nt, sizeof(q2_trip), trip_cmp);
  /* merge */
  long* rowptr = (long*)calloc((size_t)Q->ndof + 1, sizeof(long));
  long* col = (long*)malloc(sizeof(long) * (size_t)nt);
  double* val = (double*)malloc(sizeof(double) * (size_t)nt);
  long nnz = 0;
  for (long t = 0; t < nt;) {
    long u = t;
    double s = 0.0;
    while (u < nt && T[u].r == T[t].r && T[u].c == T[t].c) s = s + T[u++].v;
    col[nnz] = T[t].c;
    val[nnz] = s;
    rowptr[T[t].r + 1]++;
    nnz++;
    t = u;
  }
  free(T);
  for (long r = 0; r < Q->ndof; ++r) rowptr[r + 1] += rowptr[r];
  /* Dirichlet data and symmetric elimination */
  unsigned char* fixed = (unsigned char*)calloc((size_t)Q->ndof, 1);
  double* wfix = (double*)calloc((size_t)Q->ndof, sizeof(double));
  for (long K = 0; K < Q->nf[2]; ++K)
    for (long J = 0; J < Q->nf[1]; ++J)
      for (long I = 0; I < Q->nf[0]; ++I)
        for (int c = 0; c < dim; ++c) {
          double w;
          if (q2_dirichlet(Q, I, J, K, c, &w)) {
            const long d = q2_vnode(Q, I, J, K) * dim + c;
            fixed[d] = 1;
            wfix[d] = w;
          }
        }
  for (long r = 0; r < Q->ndof; ++r) {
    if (fixed[r]) {
      for (long p = rowptr[r]; p < rowptr[r + 1]; ++p) val[p] = col[p] == r ? 1.0 : 0.0;
      rhs[r] = wfix[r];
      continue;
    }
    for (long p = rowptr[r]; p < rowptr[r + 1]; ++p)
      if (fixed[col[p]]) {
        rhs[r] = rhs[r] - val[p] * wfix[col[p]];
        val[p] = 0.0;
      }
  }
  Q->rowptr = rowptr;
  Q->col = col;
  Q->val = val;
  Q->rhs = rhs;
  Q->fixed = fixed;
  Q->wfix = wfix;
}

void q2_csr_copy(const q2_level* Q, long* rowptr, long* col, double* val, double* rhs, unsigned char* fixed) {
  memcpy(rowptr, Q->rowptr, sizeof(long) * (size_t)(Q->ndof + 1));
  memcpy(col, Q->col, sizeof(long) * (size_t)q2_nnz(Q));
  memcpy(val, Q->val, sizeof(double) * (size_t)q2_nnz(Q));
  memcpy(rhs, Q->rhs, sizeof(double) * (size_t)Q->ndof);
  memcpy(fixed, Q->fixed, (size_t)Q->ndof);
}

static void q2_spmv(const q2_level* Q, const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (long r = 0; r < Q->ndof; ++r) {
    double s = 0.0;
    for (long p = Q->rowptr[r]; p < Q->rowptr[r + 1]; ++p) s = s + Q->val[p] * x[Q->col[p]];
    y[r] = s;
  }
}

void q2_apply(const q2_level* Q, const double* x, double* y) { q2_spmv(Q, x, y); }

void q2_residual(const q2_level* Q, const double* b, const double* x, double* r) {
  q2_spmv(Q, x, r);
  for (long k = 0; k < Q->ndof; ++k) r[k] = b[k] - r[k];
}

/* ------------------------------------------------------------------------ */
/* Patches with the lower-corner ownership rule                              */
/* ------------------------------------------------------------------------ */

/* DoFs of the patch of pressure vertex `vert`: velocities (node-lex, then
 * component) of the Q2 nodes with fine index 2a-4 .. 2a+4, then the
 * pressures of the vertices a-1 .. a+1; constrained DoFs left out.  own[q]:
 * local index of the owned DoF q (velocity of the Q2 node 2a + s, s in
 * {0,1}^d with s_x fastest, component inner; the pressure p_a last) or -1. */
static int q2_patch_dofs_(const q2_level* Q, long vert, long* dofs, int* own) {
  const int dim = Q->dim;
  long a[3] = {vert % Q->nv1[0], (vert / Q->nv1[0]) % Q->nv1[1], dim == 3 ? vert / ((long)Q->nv1[0] * Q->nv1[1]) : 0};
  const int no = (1 << dim) * dim + 1;
  for (int q = 0; q < Q2OMAX; ++q) own[q] = -1;
  int n = 0;
  const int r3 = dim == 3 ? 9 : 1;
  for (int dz = 0; dz < r3; ++dz)
    for (int dy = 0; dy < 9; ++dy)
      for (int dx = 0; dx < 9; ++dx) {
        const long I = 2 * a[0] - 4 + dx, J = 2 * a[1] - 4 + dy, K = dim == 3 ? 2 * a[2] - 4 + dz : 0;
        if (I < 0 || I >= Q->nf[0] || J < 0 || J >= Q->nf[1] || K < 0 || K >= Q->nf[2]) continue;
        const long vn = q2_vnode(Q, I, J, K);
        const long s0 = I - 2 * a[0], s1 = J - 2 * a[1], s2 = dim == 3 ? K - 2 * a[2] : 0;
        const int owned = s0 >= 0 && s0 <= 1 && s1 >= 0 && s1 <= 1 && s2 >= 0 && s2 <= 1;
        for (int c = 0; c < dim; ++c) {
          const long d = vn * dim + c;
          if (Q->fixed[d]) continue;
          if (owned) own[(int)((s0 + 2 * s1 + 4 * s2) * dim + c)] = n;
          dofs[n++] = d;
        }
      }
  for (int dz = 0; dz < (dim == 3 ? 3 : 1); ++dz)
    for (int dy = 0; dy < 3; ++dy)
      for (int dx = 0; dx < 3; ++dx) {
        const long i = a[0] - 1 + dx, j = a[1] - 1 + dy, k = dim == 3 ? a[2] - 1 + dz : 0;
        if (i < 0 || i >= Q->nv1[0] || j < 0 || j >= Q->nv1[1] || k < 0 || k >= Q->nv1[2]) continue;
        const long d = Q->nv + q2_pnode(Q, i, j, k);
        if (i == a[0] && j == a[1] && k == a[2]) own[no - 1] = n;
        dofs[n++] = d;
      }
  return n;
}

int q2_patch_dofs(const q2_level* Q, long vert, long* dofs, int* own) { return q2_patch_dofs_(Q, vert, dofs, own); }

/* dense L_i = R_i L R_i^T from the assembled rows */
static void q2_patch_matrix_(const q2_level* Q, int n, const long* dofs, double* Li) {
  for (int p = 0; p < n; ++p) {
    for (int q = 0; q < n; ++q) Li[(long)p * n + q] = 0.0;
    const long r = dofs[p];
    for (long t = Q->rowptr[r]; t < Q->rowptr[r + 1]; ++t) {
      /* dofs are sorted: binary search for the column */
      long lo = 0, hi = n - 1, cidx = Q->col[t];
      while (lo <= hi) {
        long mid = (lo + hi) / 2;
        if (dofs[mid] == cidx) { Li[(long)p * n + mid] = Q->val[t]; break; }
        if (dofs[mid] < cidx) lo = mid + 1;
        else hi = mid - 1;
      }
    }
  }
}

int q2_patch_matrix(const q2_level* Q, long vert, double* Li, long* dofs, int* own) {
  int n = q2_patch_dofs_(Q, vert, dofs, own);
  q2_patch_matrix_(Q, n, dofs, Li);
  return n;
}

/* symmetric row-max equilibration D L D, LU with partial pivoting */
static void q2_eq_factor(int n, double* a, double* dsc, int* piv, int* st) {
  for (int r = 0; r < n; ++r) {
    double m = 0.0;
    for (int c = 0; c < n; ++c) {
      const double v = fabs(a[(long)r * n + c]);
      if (v > m) m = v;
    }
    dsc[r] = m > 0.0 ? 1.0 / sqrt(m) : 1.0;
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) a[(long)r * n + c] = dsc[r] * a[(long)r * n + c] * dsc[c];
  *st = lu_factor(n, a, piv);
}

static void q2_eq_solve(int n, const double* lu, const double* dsc, const int* piv, double* b) {
  for (int r = 0; r < n; ++r) b[r] = b[r] * dsc[r];
  lu_solve(n, lu, piv, b);
  for (int r = 0; r < n; ++r) b[r] = b[r] * dsc[r];
}

/* owned rows of L_i^{-1} (= solutions of L_i z = e_k, L_i symmetric) */
static int q2_inverse_rows_(const q2_level* Q, long vert, int* n_out, long* dofs, int* own, double* rows) {
  const int n = q2_patch_dofs_(Q, vert, dofs, own);
  double* Li = (double*)malloc(sizeof(double) * (size_t)n * n);
  int* piv = (int*)malloc(sizeof(int) * (size_t)n);
  double* dsc = (double*)malloc(sizeof(double) * (size_t)n);
  q2_patch_matrix_(Q, n, dofs, Li);
  int st;
  q2_eq_factor(n, Li, dsc, piv, &st);
  for (int k = 0; k < Q2OMAX; ++k) {
    double* z = rows + (long)k * Q2PMAX;
    for (int q = 0; q < Q2PMAX; ++q) z[q] = 0.0;
    if (own[k] < 0 || st != 0) continue;
    z[own[k]] = 1.0;
    q2_eq_solve(n, Li, dsc, piv, z);
  }
  free(Li);
  free(piv);
  free(dsc);
  *n_out = n;
  return st;
}

int q2_patch_inverse_rows(const q2_level* Q, long vert, long* dofs, int* own, double* rows) {
  int n;
  const int st = q2_inverse_rows_(Q, vert, &n, dofs, own, rows);
  return st == 0 ? n : -1;
}

int q2_build_inverse(q2_level* Q) {
  if (Q->pinv) return 0;
  const long np = Q->np;
  Q->pn = (int*)malloc(sizeof(int) * (size_t)np);
  Q->pdof = (long*)malloc(sizeof(long) * (size_t)np * Q2PMAX);
  Q->pown = (int*)malloc(sizeof(int) * (size_t)np * Q2OMAX);
  Q->pinv = (double*)malloc(sizeof(double) * (size_t)np * Q2OMAX * Q2PMAX);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 2) reduction(+ : bad)
  for (long v = 0; v < np; ++v) {
    int n;
    const int st = q2_inverse_rows_(Q, v, &n, Q->pdof + v * Q2PMAX, Q->pown + v * Q2OMAX, Q->pinv + v * Q2OMAX * Q2PMAX);
    Q->pn[v] = n;
    if (st != 0) bad++;
  }
  return bad;
}

/* one RA sweep (eq. iteration with eq. smoother): r = b - L x, then every
 * patch adds omega (L_i^{-1} r_i) to the DoFs it owns; constrained DoFs take
 * their Dirichlet value (identity rows).  order: optional permutation. */
int q2_sweep(q2_level* Q, const double* b, double* x, const long* order) {
  if (!Q->pinv) q2_build_inverse(Q);
  double* r = (double*)malloc(sizeof(double) * (size_t)Q->ndof);
  double* xn = (double*)malloc(sizeof(double) * (size_t)Q->ndof);
  q2_residual(Q, b, x, r);
  memcpy(xn, x, sizeof(double) * (size_t)Q->ndof);
  const double om = Q->g->omega;
#pragma omp parallel for schedule(dynamic, 16)
  for (long t = 0; t < Q->np; ++t) {
    const long v = order ? order[t] : t;
    const int n = Q->pn[v];
    const long* pd = Q->pdof + v * Q2PMAX;
    const double* rows = Q->pinv + v * Q2OMAX * Q2PMAX;
    for (int k = 0; k < Q2OMAX; ++k) {
      const int o = Q->pown[v * Q2OMAX + k];
      if (o < 0) continue;
      double s = 0.0;
      for (int q = 0; q < n; ++q) s = s + rows[(long)k * Q2PMAX + q] * r[pd[q]];
      xn[pd[o]] = x[pd[o]] + om * s;
    }
  }
  for (long k = 0; k < Q->ndof; ++k)
    if (Q->fixed[k]) xn[k] = x[k] + r[k];
  memcpy(x, xn, sizeof(double) * (size_t)Q->ndof);
  free(r);
  free(xn);
  return 0;
}

void q2_owner_count(const q2_level* Q, int* count) {
  long* dofs = (long*)malloc(sizeof(long) * Q2PMAX);
  int own[Q2OMAX];
  memset(count, 0, sizeof(int) * (size_t)Q->ndof);
  for (long v = 0; v < Q->np; ++v) {
    q2_patch_dofs_(Q, v, dofs, own);
    for (int k = 0; k < Q2OMAX; ++k)
      if (own[k] >= 0) count[dofs[own[k]]]++;
  }
  free(dofs);
}

/* ------------------------------------------------------------------------ */
/* Transfers: Q2 interpolation of velocities, Q1 of pressures, R = P^T       */
/* ------------------------------------------------------------------------ */

/* weights of the coarse Q2 nodes 2m, 2m+1, 2m+2 of the coarse cell m that
 * holds fine Q2 node F (fine spacing = coarse spacing / 2, so F / 4 is the
 * position in coarse cells) */
static void q2_fine_weights(long F, long nc, long* base, double* w) {
  long m = F / 4;
  if (m >= nc) m = nc - 1;
  const double t = (double)(F - 4 * m) / 4.0;
  double d[3];
  q2_1d(t, w, d);
  *base = 2 * m;
}

static void q1_fine_weights(long f, long* lo, long* hi, double* wl, double* wh) {
  *lo = f / 2;
  *hi = (f + 1) / 2;
  if (*lo == *hi) { *wl = 1.0; *wh = 0.0; }
  else { *wl = 0.5; *wh = 0.5; }
}

/* xf += P ec, constrained fine DoFs untouched */
void q2_prolong_add(const q2_level* F, const q2_level* C, const double* ec, double* xf) {
  const int dim = F->dim;
  for (long K = 0; K < F->nf[2]; ++K)
    for (long J = 0; J < F->nf[1]; ++J)
      for (long I = 0; I < F->nf[0]; ++I) {
        long b[3] = {0, 0, 0};
        double w[3][3] = {{1, 0, 0}, {1, 0, 0}, {1, 0, 0}};
        const long Fi[3] = {I, J, K};
        for (int k = 0; k < dim; ++k) q2_fine_weights(Fi[k], C->g->n[k], &b[k], w[k]);
        const long vn = q2_vnode(F, I, J, K);
        for (int c = 0; c < dim; ++c) {
          const long d = vn * dim + c;
          if (F->fixed[d]) continue;
          double s = 0.0;
          for (int tz = 0; tz < (dim == 3 ? 3 : 1); ++tz)
            for (int ty = 0; ty < 3; ++ty)
              for (int tx = 0; tx < 3; ++tx) {
                const double wt = w[0][tx] * w[1][ty] * (dim == 3 ? w[2][tz] : 1.0);
                if (wt == 0.0) continue;
                const long cn = q2_vnode(C, b[0] + tx, b[1] + ty, dim == 3 ? b[2] + tz : 0);
                s = s + wt * ec[cn * dim + c];
              }
          xf[d] = xf[d] + s;
        }
      }
  for (long k = 0; k < F->nv1[2]; ++k)
    for (long j = 0; j < F->nv1[1]; ++j)
      for (long i = 0; i < F->nv1[0]; ++i) {
        long lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        double wl[3] = {1, 1, 1}, wh[3] = {0, 0, 0};
        const long fi[3] = {i, j, k};
        for (int q = 0; q < dim; ++q) q1_fine_weights(fi[q], &lo[q], &hi[q], &wl[q], &wh[q]);
        double s = 0.0;
        for (int t = 0; t < (1 << dim); ++t) {
          double wt = 1.0;
          long ic[3] = {0, 0, 0};
          for (int q = 0; q < dim; ++q) {
            const int bit = (t >> q) & 1;
            wt = wt * (bit ? wh[q] : wl[q]);
            ic[q] = bit ? hi[q] : lo[q];
          }
          if (wt == 0.0) continue;
          s = s + wt * ec[C->nv + q2_pnode(C, ic[0], ic[1], ic[2])];
        }
        const long d = F->nv + q2_pnode(F, i, j, k);
        xf[d] = xf[d] + s;
      }
}

/* bc = P^T rf (every fine DoF), then constrained coarse DoFs set to zero */
void q2_restrict(const q2_level* F, const q2_level* C, const double* rf, double* bc) {
  const int dim = F->dim;
  memset(bc, 0, sizeof(double) * (size_t)C->ndof);
  for (long K = 0; K < F->nf[2]; ++K)
    for (long J = 0; J < F->nf[1]; ++J)
      for (long I = 0; I < F->nf[0]; ++I) {
        long b[3] = {0, 0, 0};
        double w[3][3] = {{1, 0, 0}, {1, 0, 0}, {1, 0, 0}};
        const long Fi[3] = {I, J, K};
        for (int k = 0; k < dim; ++k) q2_fine_weights(Fi[k], C->g->n[k], &b[k], w[k]);
        const long vn = q2_vnode(F, I, J, K);
        for (int tz = 0; tz < (dim == 3 ? 3 : 1); ++tz)
          for (int ty = 0; ty < 3; ++ty)
            for (int tx = 0; tx < 3; ++tx) {
              const double wt = w[0][tx] * w[1][ty] * (dim == 3 ? w[2][tz] : 1.0);
              if (wt == 0.0) continue;
              const long cn = q2_vnode(C, b[0] + tx, b[1] + ty, dim == 3 ? b[2] + tz : 0);
              for (int c = 0; c < dim; ++c) bc[cn * dim + c] = bc[cn * dim + c] + wt * rf[vn * dim + c];
            }
      }
  for (long k = 0; k < F->nv1[2]; ++k)
    for (long j = 0; j < F->nv1[1]; ++j)
      for (long i = 0; i < F->nv1[0]; ++i) {
        long lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        double wl[3] = {1, 1, 1}, wh[3] = {0, 0, 0};
        const long fi[3] = {i, j, k};
        for (int q = 0; q < dim; ++q) q1_fine_weights(fi[q], &lo[q], &hi[q], &wl[q], &wh[q]);
        const double rv = rf[F->nv + q2_pnode(F, i, j, k)];
        for (int t = 0; t < (1 << dim); ++t) {
          double wt = 1.0;
          long ic[3] = {0, 0, 0};
          for (int q = 0; q < dim; ++q) {
            const int bit = (t >> q) & 1;
            wt = wt * (bit ? wh[q] : wl[q]);
            ic[q] = bit ? hi[q] : lo[q];
          }
          if (wt == 0.0) continue;
          const long d = C->nv + q2_pnode(C, ic[0], ic[1], ic[2]);
          bc[d] = bc[d] + wt * rv;
        }
      }
  for (long k = 0; k < C->ndof; ++k)
    if (C->fixed[k]) bc[k] = 0.0;
}

/* ------------------------------------------------------------------------ */
/* Multigrid, FGMRES, standalone GMG                                         */
/* ------------------------------------------------------------------------ */

typedef struct {
  int nlev;
  q2_level** lev;
  double* coarse_lu;
  double* coarse_d;
  int* coarse_piv;
  int nu_pre, nu_post;
} q2_mg;

q2_mg* q2_mg_new(int nlev, q2_level** levels, int nu_pre, int nu_post) {
  q2_mg* M = (q2_mg*)calloc(1, sizeof(q2_mg));
  M->nlev = nlev;
  M->lev = (q2_level**)malloc(sizeof(q2_level*) * (size_t)nlev);
  for (int l = 0; l < nlev; ++l) {
    M->lev[l] = levels[l];
    q2_assemble(levels[l]);
    if (l > 0) q2_build_inverse(levels[l]);
  }
  M->nu_pre = nu_pre;
  M->nu_post = nu_post;
  q2_level* C = M->lev[0];
  const long n = C->ndof;
  M->coarse_lu = (double*)calloc((size_t)(n * n), sizeof(double));
  M->coarse_piv = (int*)malloc(sizeof(int) * (size_t)n);
  M->coarse_d = (double*)malloc(sizeof(double) * (size_t)n);
  for (long r = 0; r < n; ++r)
    for (long p = C->rowptr[r]; p < C->rowptr[r + 1]; ++p) M->coarse_lu[r * n + C->col[p]] = C->val[p];
  int st;
  q2_eq_factor((int)n, M->coarse_lu, M->coarse_d, M->coarse_piv, &st);
  return M;
}

void q2_mg_free(q2_mg* M) {
  if (!M) return;
  free(M->lev);
  free(M->coarse_lu);
  free(M->coarse_d);
  free(M->coarse_piv);
  free(M);
}

static void q2_vcycle_(q2_mg* M, int l, double* x, const double* b) {
  q2_level* L = M->lev[l];
  if (l == 0) {
    double* t = (double*)malloc(sizeof(double) * (size_t)L->ndof);
    memcpy(t, b, sizeof(double) * (size_t)L->ndof);
    q2_eq_solve((int)L->ndof, M->coarse_lu, M->coarse_d, M->coarse_piv, t);
    memcpy(x, t, sizeof(double) * (size_t)L->ndof);
    free(t);
    return;
  }
  q2_level* C = M->lev[l - 1];
  for (int s = 0; s < M->nu_pre; ++s) q2_sweep(L, b, x, NULL);
  double* r = (double*)malloc(sizeof(double) * (size_t)L->ndof);
  q2_residual(L, b, x, r);
  double* bc = (double*)malloc(sizeof(double) * (size_t)C->ndof);
  double* xc = (double*)calloc((size_t)C->ndof, sizeof(double));
  q2_restrict(L, C, r, bc);
  q2_vcycle_(M, l - 1, xc, bc);
  q2_prolong_add(L, C, xc, x);
  for (int s = 0; s < M->nu_post; ++s) q2_sweep(L, b, x, NULL);
  free(r);
  free(bc);
  free(xc);
}

void q2_vcycle(q2_mg* M, double* x, const double* b) { q2_vcycle_(M, M->nlev - 1, x, b); }

int q2_fgmres(q2_mg* M, const double* b, double* x, double rtol, int maxit, int m, double* relres) {
  q2_level* L = M->lev[M->nlev - 1];
  const long n = L->ndof;
  double* V = (double*)malloc(sizeof(double) * (size_t)n * (m + 1));
  double* Z = (double*)malloc(sizeof(double) * (size_t)n * m);
  double* H = (double*)calloc((size_t)(m + 1) * m, sizeof(double));
  double* cs = (double*)malloc(sizeof(double) * (size_t)m);
  double* sn = (double*)malloc(sizeof(double) * (size_t)m);
  double* g = (double*)malloc(sizeof(double) * (size_t)(m + 1));
  double* w = (double*)malloc(sizeof(double) * (size_t)n);
  const double bn = sqrt(dot(n, b, b));
  int its = 0;
  if (bn == 0.0) {
    memset(x, 0, sizeof(double) * (size_t)n);
    *relres = 0.0;
    goto done;
  }
  for (;;) {
    q2_residual(L, b, x, w);
    const double beta = sqrt(dot(n, w, w));
    if (beta <= rtol * bn || its >= maxit) { *relres = beta / bn; break; }
    for (long i = 0; i < n; ++i) V[i] = w[i] / beta;
    memset(g, 0, sizeof(double) * (size_t)(m + 1));
    g[0] = beta;
    int j, k = 0;
    for (j = 0; j < m && its < maxit; ++j) {
      double* zj = Z + (long)j * n;
      memset(zj, 0, sizeof(double) * (size_t)n);
      q2_vcycle_(M, M->nlev - 1, zj, V + (long)j * n);
      its++;
      q2_apply(L, zj, w);
      for (int i = 0; i <= j; ++i) {
        const double hij = dot(n, w, V + (long)i * n);
        H[i * m + j] = hij;
        for (long t = 0; t < n; ++t) w[t] = w[t] - hij * V[(long)i * n + t];
      }
      const double hn = sqrt(dot(n, w, w));
      H[(j + 1) * m + j] = hn;
      if (hn != 0.0)
        for (long t = 0; t < n; ++t) V[(long)(j + 1) * n + t] = w[t] / hn;
      for (int i = 0; i < j; ++i) {
        const double a = H[i * m + j], c = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * c;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      const double a = H[j * m + j], c = H[(j + 1) * m + j];
      const double den = sqrt(a * a + c * c);
      cs[j] = den == 0.0 ? 1.0 : a / den;
      sn[j] = den == 0.0 ? 0.0 : c / den;
      H[j * m + j] = den;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      k = j + 1;
      if (fabs(g[j + 1]) <= rtol * bn || hn == 0.0) break;
    }
    double y[512];
    for (int i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int t = i + 1; t < k; ++t) s = s - H[i * m + t] * y[t];
      y[i] = s / H[i * m + i];
    }
    for (int i = 0; i < k; ++i)
      for (long t = 0; t < n; ++t) x[t] = x[t] + y[i] * Z[(long)i * n + t];
  }
done:
  free(V); free(Z); free(H); free(cs); free(sn); free(g); free(w);
  return its;
}

int q2_gmg_solve(q2_mg* M, const double* b, double* x, double red, int maxit, double* relred) {
  q2_level* L = M->lev[M->nlev - 1];
  const long n = L->ndof;
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  q2_residual(L, b, x, r);
  const double r0 = sqrt(dot(n, r, r));
  double rn = r0;
  int it = 0;
  while (it < maxit && rn > red * r0) {
    q2_vcycle_(M, M->nlev - 1, x, b);
    q2_residual(L, b, x, r);
    rn = sqrt(dot(n, r, r));
    it++;
  }
  *relred = r0 > 0 ? rn / r0 : 0.0;
  free(r);
  return it;
}
