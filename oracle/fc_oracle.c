/*
 * fc_oracle.c -- plain, slow FP64 CPU oracle for the restricted additive (RA)
 * smoother of the finite cell Stokes multigrid method (Saberi & Vogel,
 * "A restricted additive smoother for finite cell flow problems").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this file; only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load it (through oracle/oracle.py).  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * What it computes, in the paper's order and notation:
 *   - Stokes strong form and boundary conditions (Sec. 2, eq. stokes_strong,
 *     eq. stokes_bc);
 *   - the finite cell weak form with symmetric Nitsche terms on the obstacle
 *     boundary Gamma_D and the alpha-scaled volume terms (Sec. 2,
 *     eq. stokes_weak_fcm, eq. stokes_disc_weak_fcm_2);
 *   - equal-order Q1-Q1 with the local L2 pressure-projection stabilisation
 *     c(q,p) = -(1/eta)(q - Pi0 q, p - Pi0 p) (Sec. 2, eq. stabilization_l2);
 *   - the saddle-point system L x = b (Sec. 3, eq. linear_system);
 *   - the RA smoother x <- x + S (b - L x), S = sum_i Rt_i^T w_i L_i^{-1} R_i,
 *     one patch per pressure node, exact local LU solves, restricted write
 *     to p_i and the velocity DoFs of the same node (Sec. 3.1, eq. iteration,
 *     eq. smoother; Sec. 3.1.2 for the LU and the 1+d stored rows);
 *   - geometric multigrid on a nested uniform hierarchy (Sec. 3, Algorithm 1
 *     on a uniform grid), transfers R and P = R^T (eq. restriction_op), a
 *     direct coarse solve, a V-cycle, and FGMRES with the V-cycle as right
 *     preconditioner (Sec. 4, remark on Krylov methods).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - cut-cell volume rule: recursive 2^d split of a cell up to depth k where
 *     the level set changes sign among the 3^d sample points of a box, tensor
 *     2-point Gauss on leaves, alpha evaluated pointwise;
 *   - obstacle boundary rule: composite 2-point Gauss in the curve parameter
 *     (circle, ellipse), composite 2-point Gauss in cos(theta) times a uniform
 *     rule in phi (sphere); points binned into the cell containing them;
 *   - Nitsche parameter lambda = beta*eta/h_min, beta = 100;
 *   - c(.,.) integrated over the whole cell without alpha;
 *   - pressure nodes "connected to p_i": the 3^d nodes sharing a cell with it;
 *     velocity DoFs of the patch: the 5^d nodes around node i (structural);
 *     constrained and out-of-grid DoFs are excluded;
 *   - box faces carry strong Dirichlet values per preset, eliminated
 *     symmetrically (identity rows, values lifted into b).
 *
 * Floating point: plain IEEE double, compiled with -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif


/* ------------------------------------------------------------------------ */
/* Problem description                                                       */
/* ------------------------------------------------------------------------ */

typedef struct {
  int type;      /* 0: circle (2D) / sphere (3D), 1: ellipse (2D) */
  double c[3];   /* centre */
  double r[3];   /* radius / semi-axes a, b */
  double rot[2]; /* (cos theta, sin theta) of the ellipse's a-axis */
} or_shape;

typedef struct {
  double A[8][8];    /* scalar velocity block a(.,.) per component */
  double B[3][8][8]; /* B[c][a][b]: velocity node a comp c, pressure node b */
  double C[8][8];    /* stabilisation block c(.,.) */
  double f[3][8];    /* load f(v) per component */
  double fluid_volume;
  double boundary_measure;
  int nvol, nbnd;
} or_elem;

typedef struct {
  double x[3], n[3], w;
  int shape;
  long cell;
} or_bpoint;

typedef struct or_level {
  int dim, n[3], nn[3], ndpn;
  double lo[3], hi[3], h[3], hmin;
  long ncell, nnodes, ndof;
  int nshape;
  or_shape* shape;
  double alpha, eta, beta, lambda, omega, ubar;
  int qdepth, preset, force_kind;
  double force[3];
  /* boundary quadrature, binned per cell (cell_bstart has ncell+1 entries) */
  long nbp;
  or_bpoint* bp;
  long* cell_bstart;
  /* element cache (optional) */
  or_elem* elem;
  /* assembled operator: CSR with identity rows for constrained DoFs */
  long* rowptr;
  long* col;
  double* val;
  double* rhs;
  unsigned char* fixed;
  double* wfix;
  /* patches for cache_inverse: per node, n_i dofs and (d+1) rows */
  int* pn;       /* n_i per patch */
  long* pdof;    /* [nnodes][402] */
  int* pown;     /* [nnodes][4] local index of owned dof or -1 */
  double* pinv;  /* [nnodes][4][402] owned rows of L_i^{-1} */
  /* adaptive grids (fc_oracle_amr.c): the prolongation from the next coarser
   * level as a node-to-node sparse matrix (rows: nodes of this level), used
   * by or_prolong_add / or_restrict in place of the uniform Q1 weights */
  long* tp_rowptr;
  long* tp_col;
  double* tp_val;
  /* adaptive grids: the stride of the cached patch arrays (pdof, pinv)
   * when their patches exceed PMAX DoFs; 0 means PMAX */
  int pstride;
} or_level;

#define PMAX 402
#define OMAX 4

/* ------------------------------------------------------------------------ */
/* Level set (Sec. 2: Omega = fluid, Omega_e \ Omega = fictitious)           */
/* ------------------------------------------------------------------------ */

static double phi_shape(const or_shape* s, int dim, const double* x) {
  double dx = x[0] - s->c[0], dy = x[1] - s->c[1];
  if (s->type == 0) {
    double q = dx * dx + dy * dy;
    if (dim == 3) {
      double dz = x[2] - s->c[2];
      q = q + dz * dz;
    }
    return s->r[0] - sqrt(q);
  }
  {
    double xp = s->rot[0] * dx + s->rot[1] * dy;
    double yp = -s->rot[1] * dx + s->rot[0] * dy;
    double u = xp / s->r[0], v = yp / s->r[1];
    return 1.0 - (u * u + v * v);
  }
}

/* phi > 0 inside some obstacle (fictitious part), phi <= 0 in the fluid. */
static double phi_all(const or_level* L, const double* x) {
  double p = -1.0;
  for (int s = 0; s < L->nshape; ++s) {
    double q = phi_shape(&L->shape[s], L->dim, x);
    if (s == 0 || q > p) p = q;
  }
  return p;
}

double or_phi(const or_level* L, const double* x) { return phi_all(L, x); }

/* alpha = 1 in Omega, alpha_f << 1 in the fictitious part (Sec. 2). */
static double alpha_at(const or_level* L, const double* x) {
  return phi_all(L, x) > 0.0 ? L->alpha : 1.0;
}

/* ------------------------------------------------------------------------ */
/* Body force                                                                */
/* ------------------------------------------------------------------------ */

static void force_at(const or_level* L, const double* x, double* f) {
  const double pi = 3.14159265358979323846;
  f[0] = f[1] = f[2] = 0.0;
  switch (L->force_kind) {
    case 0:
      f[0] = L->force[0]; f[1] = L->force[1]; f[2] = L->force[2];
      break;
    case 1:
      f[0] = L->force[0] * sin(pi * x[0]);
      f[1] = L->force[1] * cos(pi * x[1]);
      break;
    case 2:
      f[0] = L->force[0] * sin(pi * x[1]);
      if (L->dim == 3) f[0] = f[0] * sin(pi * x[2]);
      break;
    case 3:
      f[0] = -L->force[0] * (pi / 2.0) * sin(pi * x[0] / 2.0);
      break;
    default:
      break;
  }
}

/* ------------------------------------------------------------------------ */
/* Q1 basis on an axis-aligned cell                                          */
/* ------------------------------------------------------------------------ */

/* Values and gradients of the 2^d trilinear nodal functions at x in the cell
 * with lower corner x0 and sizes h.  Local node a has bit k = position in
 * direction k (x fastest). */
static void q1_basis(int dim, const double* x0, const double* h, const double* x,
                     double* val, double (*grad)[3]) {
  double xi[3] = {0, 0, 0};
  for (int k = 0; k < dim; ++k) xi[k] = (x[k] - x0[k]) / h[k];
  int nloc = 1 << dim;
  for (int a = 0; a < nloc; ++a) {
    double f1[3], d1[3];
    for (int k = 0; k < dim; ++k) {
      int bit = (a >> k) & 1;
      f1[k] = bit ? xi[k] : 1.0 - xi[k];
      d1[k] = (bit ? 1.0 : -1.0) / h[k];
    }
    double v = 1.0;
    for (int k = 0; k < dim; ++k) v = v * f1[k];
    val[a] = v;
    for (int k = 0; k < 3; ++k) grad[a][k] = 0.0;
    for (int k = 0; k < dim; ++k) {
      double g = d1[k];
      for (int m = 0; m < dim; ++m)
        if (m != k) g = g * f1[m];
      grad[a][k] = g;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Volume quadrature: recursive box split on a sign change of phi            */
/* ------------------------------------------------------------------------ */

typedef struct {
  const or_level* L;
  double x0[3]; /* cell lower corner */
  or_elem* e;
} vol_ctx;

static void vol_point(vol_ctx* q, const double* x, double w) {
  const or_level* L = q->L;
  int dim = L->dim, nloc = 1 << dim;
  double val[8], grad[8][3];
  q1_basis(dim, q->x0, L->h, x, val, grad);
  double al = alpha_at(L, x);
  double f[3];
  force_at(L, x, f);
  or_elem* e = q->e;
  /* a(v,u) volume part: (eta grad v, alpha grad u), per component */
  for (int a = 0; a < nloc; ++a)
    for (int b = a; b < nloc; ++b) {
      double g = 0.0;
      for (int k = 0; k < dim; ++k) g = g + grad[a][k] * grad[b][k];
      e->A[a][b] = e->A[a][b] + w * al * L->eta * g;
    }
  /* b(v,p) volume part: -(div v, alpha p) */
  for (int c = 0; c < dim; ++c)
    for (int a = 0; a < nloc; ++a)
      for (int b = 0; b < nloc; ++b)
        e->B[c][a][b] = e->B[c][a][b] - w * al * grad[a][c] * val[b];
  /* f(v) volume part: (v, alpha f) */
  for (int c = 0; c < dim; ++c)
    for (int a = 0; a < nloc; ++a) e->f[c][a] = e->f[c][a] + w * al * f[c] * val[a];
  if (al == 1.0) e->fluid_volume = e->fluid_volume + w;
  e->nvol++;
}

static void vol_box(vol_ctx* q, const double* lo, const double* hb, int level) {
  const or_level* L = q->L;
  int dim = L->dim;
  /* sign of phi at the 3^d sample points (corners, edge/face midpoints, centre) */
  int npos = 0, ns = 0;
  int m3 = dim == 3 ? 3 : 1;
  for (int k = 0; k < m3; ++k)
    for (int j = 0; j < 3; ++j)
      for (int i = 0; i < 3; ++i) {
        double x[3] = {lo[0] + hb[0] * (0.5 * i), lo[1] + hb[1] * (0.5 * j),
                       dim == 3 ? lo[2] + hb[2] * (0.5 * k) : 0.0};
        if (phi_all(L, x) > 0.0) npos++;
        ns++;
      }
  int cut = (npos != 0 && npos != ns);
  if (cut && level < L->qdepth) {
    int nch = 1 << dim;
    double hc[3] = {hb[0] * 0.5, hb[1] * 0.5, hb[2] * 0.5};
    for (int ch = 0; ch < nch; ++ch) {
      double lc[3] = {lo[0], lo[1], lo[2]};
      for (int k = 0; k < dim; ++k)
        if ((ch >> k) & 1) lc[k] = lo[k] + hc[k];
      vol_box(q, lc, hc, level + 1);
    }
    return;
  }
  /* tensor 2-point Gauss rule on this machine */
  const double g[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
  double w = 1.0;
  for (int k = 0; k < dim; ++k) w = w * (hb[k] * 0.5);
  for (int k = 0; k < (dim == 3 ? 2 : 1); ++k)
    for (int j = 0; j < 2; ++j)
      for (int i = 0; i < 2; ++i) {
        double x[3] = {lo[0] + hb[0] * g[i], lo[1] + hb[1] * g[j],
                       dim == 3 ? lo[2] + hb[2] * g[k] : 0.0};
        vol_point(q, x, w);
      }
}

/* ------------------------------------------------------------------------ */
/* Obstacle boundary quadrature Gamma_D                                      */
/* ------------------------------------------------------------------------ */

static long cell_of_point(const or_level* L, const double* x, int* ok) {
  long idx[3] = {0, 0, 0};
  *ok = 1;
  for (int k = 0; k < L->dim; ++k) {
    if (x[k] < L->lo[k] || x[k] > L->hi[k]) { *ok = 0; return -1; }
    long i = (long)floor((x[k] - L->lo[k]) / L->h[k]);
    if (i >= L->n[k]) i = L->n[k] - 1;
    if (i < 0) i = 0;
    idx[k] = i;
  }
  return idx[0] + (long)L->n[0] * (idx[1] + (long)L->n[1] * idx[2]);
}

static int point_in_other_shape(const or_level* L, int s, const double* x) {
  for (int t = 0; t < L->nshape; ++t)
    if (t != s && phi_shape(&L->shape[t], L->dim, x) > 0.0) return 1;
  return 0;
}

/* Generate the boundary rule of all shapes (in shape order, then parameter
 * order), drop points outside the box or inside another obstacle. */
static long gen_bpoints(const or_level* L, or_bpoint* out) {
  const double pi = 3.14159265358979323846;
  const double g[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
  long cnt = 0;
  int k2 = 1 << L->qdepth;
  for (int s = 0; s < L->nshape; ++s) {
    const or_shape* sh = &L->shape[s];
    if (L->dim == 2) {
      double rmax = sh->type == 0 ? sh->r[0] : (sh->r[0] > sh->r[1] ? sh->r[0] : sh->r[1]);
      long N = 8L * (long)ceil(2.0 * pi * rmax / L->hmin) * k2;
      if (N < 64) N = 64;
      double dt = 2.0 * pi / (double)N;
      for (long m = 0; m < N; ++m)
        for (int j = 0; j < 2; ++j) {
          double t = dt * ((double)m + g[j]);
          double ct = cos(t), st = sin(t);
          double x[3], n[3] = {0, 0, 0}, w;
          if (sh->type == 0) {
            x[0] = sh->c[0] + sh->r[0] * ct;
            x[1] = sh->c[1] + sh->r[0] * st;
            n[0] = -ct; n[1] = -st;
            w = 0.5 * dt * sh->r[0];
          } else {
            double a = sh->r[0], b = sh->r[1];
            double cr = sh->rot[0], sr = sh->rot[1];
            x[0] = sh->c[0] + (cr * (a * ct) - sr * (b * st));
            x[1] = sh->c[1] + (sr * (a * ct) + cr * (b * st));
            double nx = b * ct, ny = a * st;
            double nl = sqrt(nx * nx + ny * ny);
            n[0] = -(cr * nx - sr * ny) / nl;
            n[1] = -(sr * nx + cr * ny) / nl;
            double sp = sqrt((a * st) * (a * st) + (b * ct) * (b * ct));
            w = 0.5 * dt * sp;
          }
          x[2] = 0.0;
          int ok;
          long cell = cell_of_point(L, x, &ok);
          if (!ok || point_in_other_shape(L, s, x)) continue;
          if (out) {
            or_bpoint* p = &out[cnt];
            for (int k = 0; k < 3; ++k) { p->x[k] = x[k]; p->n[k] = n[k]; }
            p->w = w; p->shape = s; p->cell = cell;
          }
          cnt++;
        }
    } else {
      double r = sh->r[0];
      long Nm = (long)ceil(2.0 * r / L->hmin) * k2;
      if (Nm < 8) Nm = 8;
      long Nf = 2L * (long)ceil(2.0 * pi * r / L->hmin) * k2;
      if (Nf < 16) Nf = 16;
      double dm = 2.0 / (double)Nm, df = 2.0 * pi / (double)Nf;
      double w = r * r * (0.5 * dm) * df;
      for (long m = 0; m < Nm; ++m)
        for (int j = 0; j < 2; ++j) {
          double mu = -1.0 + dm * ((double)m + g[j]);
          double st = sqrt(1.0 - mu * mu);
          for (long q = 0; q < Nf; ++q) {
            double ph = df * ((double)q + 0.5);
            double cp = cos(ph), sp = sin(ph);
            double e[3] = {st * cp, st * sp, mu};
            double x[3] = {sh->c[0] + r * e[0], sh->c[1] + r * e[1], sh->c[2] + r * e[2]};
            int ok;
            long cell = cell_of_point(L, x, &ok);
            if (!ok || point_in_other_shape(L, s, x)) continue;
            if (out) {
              or_bpoint* p = &out[cnt];
              for (int k = 0; k < 3; ++k) { p->x[k] = x[k]; p->n[k] = -e[k]; }
              p->w = w; p->shape = s; p->cell = cell;
            }
            cnt++;
          }
        }
    }
  }
  return cnt;
}

static void build_bpoints(or_level* L) {
  long cnt = gen_bpoints(L, NULL);
  or_bpoint* pts = (or_bpoint*)malloc(sizeof(or_bpoint) * (cnt > 0 ? cnt : 1));
  gen_bpoints(L, pts);
  /* stable counting sort by cell: keeps generation order inside a cell */
  long* start = (long*)calloc((size_t)L->ncell + 1, sizeof(long));
  for (long i = 0; i < cnt; ++i) start[pts[i].cell + 1]++;
  for (long c = 0; c < L->ncell; ++c) start[c + 1] += start[c];
  long* fill = (long*)malloc(sizeof(long) * (size_t)(L->ncell + 1));
  memcpy(fill, start, sizeof(long) * (size_t)(L->ncell + 1));
  or_bpoint* sorted = (or_bpoint*)malloc(sizeof(or_bpoint) * (cnt > 0 ? cnt : 1));
  for (long i = 0; i < cnt; ++i) sorted[fill[pts[i].cell]++] = pts[i];
  free(fill);
  free(pts);
  L->nbp = cnt;
  L->bp = sorted;
  L->cell_bstart = start;
}

/* ------------------------------------------------------------------------ */
/* Element data of one cell                                                  */
/* ------------------------------------------------------------------------ */

static void cell_x0(const or_level* L, long cell, double* x0, long* idx) {
  long i = cell % L->n[0];
  long j = (cell / L->n[0]) % L->n[1];
  long k = L->dim == 3 ? cell / ((long)L->n[0] * L->n[1]) : 0;
  idx[0] = i; idx[1] = j; idx[2] = k;
  x0[0] = L->lo[0] + (double)i * L->h[0];
  x0[1] = L->lo[1] + (double)j * L->h[1];
  x0[2] = L->dim == 3 ? L->lo[2] + (double)k * L->h[2] : 0.0;
}

static void compute_elem(const or_level* L, long cell, or_elem* e) {
  memset(e, 0, sizeof(*e));
  int dim = L->dim, nloc = 1 << dim;
  long idx[3];
  vol_ctx q;
  q.L = L;
  q.e = e;
  cell_x0(L, cell, q.x0, idx);
  /* volume terms */
  vol_box(&q, q.x0, L->h, 0);
  /* Nitsche boundary terms on Gamma_D (obstacles, w = 0):
   *   a: -(v, n.eta grad u) - (n.eta grad v, u) + (v, lambda u)
   *   b: +(v, n p)  (and its transpose (n q, u)) */
  for (long p = L->cell_bstart[cell]; p < L->cell_bstart[cell + 1]; ++p) {
    const or_bpoint* bp = &L->bp[p];
    double val[8], grad[8][3];
    q1_basis(dim, q.x0, L->h, bp->x, val, grad);
    double dn[8];
    for (int a = 0; a < nloc; ++a) {
      double s = 0.0;
      for (int k = 0; k < dim; ++k) s = s + bp->n[k] * grad[a][k];
      dn[a] = s;
    }
    for (int a = 0; a < nloc; ++a)
      for (int b = a; b < nloc; ++b) {
        double t = -L->eta * val[a] * dn[b] - L->eta * dn[a] * val[b] + L->lambda * val[a] * val[b];
        e->A[a][b] = e->A[a][b] + bp->w * t;
      }
    for (int c = 0; c < dim; ++c)
      for (int a = 0; a < nloc; ++a)
        for (int b = 0; b < nloc; ++b) e->B[c][a][b] = e->B[c][a][b] + bp->w * val[a] * bp->n[c] * val[b];
    e->boundary_measure = e->boundary_measure + bp->w;
    e->nbnd++;
  }
  /* mirror the symmetric a block */
  for (int a = 0; a < nloc; ++a)
    for (int b = 0; b < a; ++b) e->A[a][b] = e->A[b][a];
  /* stabilisation c(q,p) = -(1/eta) (q - Pi0 q, p - Pi0 p)_K over the whole
   * cell, Pi0 = cell mean; (q - Pi0 q, p - Pi0 p)_K = M_ab - m_a m_b / |K|.
   * Integrated with the tensor 2-point Gauss rule, exact for Q1 x Q1. */
  {
    const double g[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
    double w = 1.0;
    for (int k = 0; k < dim; ++k) w = w * (L->h[k] * 0.5);
    double M[8][8], m[8], vol = 0.0;
    memset(M, 0, sizeof(M));
    memset(m, 0, sizeof(m));
    for (int k = 0; k < (dim == 3 ? 2 : 1); ++k)
      for (int j = 0; j < 2; ++j)
        for (int i = 0; i < 2; ++i) {
          double x[3] = {q.x0[0] + L->h[0] * g[i], q.x0[1] + L->h[1] * g[j],
                         dim == 3 ? q.x0[2] + L->h[2] * g[k] : 0.0};
          double val[8], grad[8][3];
          q1_basis(dim, q.x0, L->h, x, val, grad);
          for (int a = 0; a < nloc; ++a) {
            m[a] = m[a] + w * val[a];
            for (int b = 0; b < nloc; ++b) M[a][b] = M[a][b] + w * val[a] * val[b];
          }
          vol = vol + w;
        }
    for (int a = 0; a < nloc; ++a)
      for (int b = a; b < nloc; ++b) {
        double v = -(1.0 / L->eta) * (M[a][b] - m[a] * m[b] / vol);
        e->C[a][b] = v;
        e->C[b][a] = v;
      }
  }
}

static const or_elem* get_elem(const or_level* L, long cell, or_elem* tmp) {
  if (L->elem) return &L->elem[cell];
  compute_elem(L, cell, tmp);
  return tmp;
}

/* ------------------------------------------------------------------------ */
/* Strong Dirichlet data on the box faces                                    */
/* ------------------------------------------------------------------------ */

static void node_idx(const or_level* L, long node, long* idx) {
  idx[0] = node % L->nn[0];
  idx[1] = (node / L->nn[0]) % L->nn[1];
  idx[2] = L->dim == 3 ? node / ((long)L->nn[0] * L->nn[1]) : 0;
}

/* returns 1 if velocity component c of node is constrained; *w its value */
static int dirichlet(const or_level* L, long node, int c, double* w) {
  long idx[3];
  node_idx(L, node, idx);
  *w = 0.0;
  if (c >= L->dim) return 0; /* pressure is never constrained */
  int dim = L->dim;
  if (L->preset == 0) { /* channel: inflow x = lo, walls on y (and z) faces */
    int wall = (idx[1] == 0 || idx[1] == L->n[1]);
    if (dim == 3) wall = wall || idx[2] == 0 || idx[2] == L->n[2];
    int inflow = idx[0] == 0;
    if (!wall && !inflow) return 0;
    if (!wall && inflow && c == 0) {
      double y = L->lo[1] + (double)idx[1] * L->h[1];
      double H = L->hi[1] - L->lo[1];
      double s = (y - L->lo[1]) / H;
      double v = 4.0 * L->ubar * s * (1.0 - s);
      if (dim == 3) {
        double z = L->lo[2] + (double)idx[2] * L->h[2];
        double t = (z - L->lo[2]) / (L->hi[2] - L->lo[2]);
        v = v * 4.0 * t * (1.0 - t);
      }
      *w = v;
    }
    return 1;
  }
  if (L->preset == 1) { /* porous: no-slip on y (and z) faces */
    int wall = (idx[1] == 0 || idx[1] == L->n[1]);
    if (dim == 3) wall = wall || idx[2] == 0 || idx[2] == L->n[2];
    return wall;
  }
  return 0; /* preset 2: no strong Dirichlet data */
}

/* ------------------------------------------------------------------------ */
/* Level construction and global assembly (CSR)                              */
/* ------------------------------------------------------------------------ */

or_level* or_level_new(int dim, const int* n, const double* lo, const double* hi, int nshape,
                       const double* shapes /* [nshape][9]: type,c0..2,r0..2,cos,sin */,
                       double alpha, int qdepth, double eta, double beta, double omega,
                       int preset, int force_kind, const double* force, double ubar) {
  or_level* L = (or_level*)calloc(1, sizeof(or_level));
  L->dim = dim;
  L->ndpn = dim + 1;
  L->hmin = 1e300;
  L->ncell = 1;
  L->nnodes = 1;
  for (int k = 0; k < 3; ++k) {
    L->n[k] = k < dim ? n[k] : 1;
    L->nn[k] = k < dim ? n[k] + 1 : 1;
    L->lo[k] = k < dim ? lo[k] : 0.0;
    L->hi[k] = k < dim ? hi[k] : 1.0;
    L->h[k] = k < dim ? (hi[k] - lo[k]) / (double)n[k] : 1.0;
    if (k < dim) {
      if (L->h[k] < L->hmin) L->hmin = L->h[k];
      L->ncell *= L->n[k];
      L->nnodes *= L->nn[k];
    }
  }
  L->ndof = L->nnodes * L->ndpn;
  L->nshape = nshape;
  L->shape = (or_shape*)calloc((size_t)(nshape > 0 ? nshape : 1), sizeof(or_shape));
  for (int s = 0; s < nshape; ++s) {
    const double* d = shapes + 9 * s;
    L->shape[s].type = (int)d[0];
    for (int k = 0; k < 3; ++k) { L->shape[s].c[k] = d[1 + k]; L->shape[s].r[k] = d[4 + k]; }
    L->shape[s].rot[0] = d[7];
    L->shape[s].rot[1] = d[8];
  }
  L->alpha = alpha;
  L->qdepth = qdepth;
  L->eta = eta;
  L->beta = beta;
  L->lambda = beta * eta / L->hmin;
  L->omega = omega;
  L->preset = preset;
  L->force_kind = force_kind;
  for (int k = 0; k < 3; ++k) L->force[k] = force ? force[k] : 0.0;
  L->ubar = ubar;
  build_bpoints(L);
  return L;
}

void or_level_free(or_level* L) {
  if (!L) return;
  free(L->shape); free(L->bp); free(L->cell_bstart); free(L->elem);
  free(L->rowptr); free(L->col); free(L->val); free(L->rhs); free(L->fixed); free(L->wfix);
  free(L->pn); free(L->pdof); free(L->pown); free(L->pinv);
  free(L->tp_rowptr); free(L->tp_col); free(L->tp_val);
  free(L);
}

long or_ndof(const or_level* L) { return L->ndof; }
long or_nnodes(const or_level* L) { return L->nnodes; }
long or_ncell(const or_level* L) { return L->ncell; }
long or_nbpoints(const or_level* L) { return L->nbp; }

/* element data of one cell, exported for the tests */
int or_cell_element(const or_level* L, long cell, double* A, double* B, double* C, double* f,
                    double* stats) {
  if (cell < 0 || cell >= L->ncell) return -1;
  or_elem e;
  compute_elem(L, cell, &e);
  int nloc = 1 << L->dim;
  for (int a = 0; a < nloc; ++a)
    for (int b = 0; b < nloc; ++b) {
      A[a * nloc + b] = e.A[a][b];
      C[a * nloc + b] = e.C[a][b];
      for (int c = 0; c < L->dim; ++c) B[(c * nloc + a) * nloc + b] = e.B[c][a][b];
    }
  for (int c = 0; c < L->dim; ++c)
    for (int a = 0; a < nloc; ++a) f[c * nloc + a] = e.f[c][a];
  stats[0] = e.fluid_volume;
  stats[1] = e.boundary_measure;
  stats[2] = e.nvol;
  stats[3] = e.nbnd;
  return 0;
}

void or_precompute_cells(or_level* L) {
  if (L->elem) return;
  L->elem = (or_elem*)malloc(sizeof(or_elem) * (size_t)L->ncell);
#pragma omp parallel for schedule(dynamic, 16)
  for (long c = 0; c < L->ncell; ++c) compute_elem(L, c, &L->elem[c]);
}

static long node_of(const or_level* L, long i, long j, long k) {
  return i + (long)L->nn[0] * (j + (long)L->nn[1] * k);
}

/* Row (node a, comp ca) of the unconstrained operator: entries for all DoFs
 * of the 3^d neighbour nodes, accumulated over the 2^d cells around node a.
 * out[nb][cb] for nb in 0..3^d-1 (lexicographic offsets -1..1, x fastest). */
static void raw_row(const or_level* L, long node, int ca, double* out, double* fval) {
  int dim = L->dim, nd = L->ndpn, nloc = 1 << dim;
  int nnb = dim == 3 ? 27 : 9;
  long ia[3];
  node_idx(L, node, ia);
  for (int t = 0; t < nnb * nd; ++t) out[t] = 0.0;
  *fval = 0.0;
  or_elem tmp;
  for (int cc = 0; cc < nloc; ++cc) {
    long ic[3] = {0, 0, 0};
    int inside = 1;
    for (int k = 0; k < dim; ++k) {
      ic[k] = ia[k] - 1 + ((cc >> k) & 1);
      if (ic[k] < 0 || ic[k] >= L->n[k]) inside = 0;
    }
    if (!inside) continue;
    long cell = ic[0] + (long)L->n[0] * (ic[1] + (long)L->n[1] * ic[2]);
    const or_elem* e = get_elem(L, cell, &tmp);
    int la = 0;
    for (int k = 0; k < dim; ++k) la |= (int)(ia[k] - ic[k]) << k;
    if (ca < dim) *fval = *fval + e->f[ca][la];
    for (int lb = 0; lb < nloc; ++lb) {
      int nb = 0, mul = 1;
      for (int k = 0; k < dim; ++k) {
        long ib = ic[k] + ((lb >> k) & 1);
        nb += (int)(ib - ia[k] + 1) * mul;
        mul *= 3;
      }
      for (int cb = 0; cb < nd; ++cb) {
        double v;
        if (ca < dim && cb < dim) v = (ca == cb) ? e->A[la][lb] : 0.0;
        else if (ca < dim) v = e->B[ca][la][lb];
        else if (cb < dim) v = e->B[cb][lb][la];
        else v = e->C[la][lb];
        out[nb * nd + cb] = out[nb * nd + cb] + v;
      }
    }
  }
}

/* Row of the eliminated system L x = b: identity for a constrained DoF,
 * otherwise constrained columns moved to the right-hand side. Returns b. */
static double sys_row(const or_level* L, long node, int ca, double* out) {
  int dim = L->dim, nd = L->ndpn;
  int nnb = dim == 3 ? 27 : 9;
  double w;
  if (dirichlet(L, node, ca, &w)) {
    for (int t = 0; t < nnb * nd; ++t) out[t] = 0.0;
    out[(dim == 3 ? 13 : 4) * nd + ca] = 1.0;
    return w;
  }
  double fval;
  raw_row(L, node, ca, out, &fval);
  long ia[3];
  node_idx(L, node, ia);
  double rhs = fval;
  for (int nb = 0; nb < nnb; ++nb) {
    long ib[3] = {0, 0, 0};
    int t = nb, inside = 1;
    for (int k = 0; k < dim; ++k) {
      ib[k] = ia[k] + (t % 3) - 1;
      t /= 3;
      if (ib[k] < 0 || ib[k] > L->n[k]) inside = 0;
    }
    if (!inside) {
      for (int cb = 0; cb < nd; ++cb) out[nb * nd + cb] = 0.0;
      continue;
    }
    long nbn = node_of(L, ib[0], ib[1], ib[2]);
    for (int cb = 0; cb < dim; ++cb) {
      double wb;
      if (dirichlet(L, nbn, cb, &wb)) {
        rhs = rhs - out[nb * nd + cb] * wb;
        out[nb * nd + cb] = 0.0;
      }
    }
  }
  return rhs;
}

/* Rows of the eliminated system for a list of DoFs (dense over the 3^d
 * neighbour nodes, layout [row][3^d][d+1]) and their right-hand sides. */
void or_dof_rows(const or_level* L, long nrows, const long* dofs, double* rows, double* rhs) {
  int nd = L->ndpn, nnb = L->dim == 3 ? 27 : 9;
#pragma omp parallel for schedule(dynamic, 4)
  for (long r = 0; r < nrows; ++r)
    rhs[r] = sys_row(L, dofs[r] / nd, (int)(dofs[r] % nd), rows + r * nnb * nd);
}

/* Full CSR assembly with sorted columns. */
void or_assemble(or_level* L) {
  if (L->rowptr) return;
  int dim = L->dim, nd = L->ndpn, nnb = dim == 3 ? 27 : 9;
  long nr = L->ndof;
  L->rowptr = (long*)malloc(sizeof(long) * (size_t)(nr + 1));
  L->rhs = (double*)malloc(sizeof(double) * (size_t)nr);
  L->fixed = (unsigned char*)calloc((size_t)nr, 1);
  L->wfix = (double*)calloc((size_t)nr, sizeof(double));
  /* structural columns: all DoFs of in-grid neighbour nodes */
  L->rowptr[0] = 0;
  for (long node = 0; node < L->nnodes; ++node) {
    long ia[3];
    node_idx(L, node, ia);
    int cnt = 0;
    for (int nb = 0; nb < nnb; ++nb) {
      int t = nb, inside = 1;
      for (int k = 0; k < dim; ++k) {
        long ib = ia[k] + (t % 3) - 1;
        t /= 3;
        if (ib < 0 || ib > L->n[k]) inside = 0;
      }
      cnt += inside;
    }
    for (int c = 0; c < nd; ++c) L->rowptr[node * nd + c + 1] = L->rowptr[node * nd + c] + (long)cnt * nd;
  }
  long nnz = L->rowptr[nr];
  L->col = (long*)malloc(sizeof(long) * (size_t)nnz);
  L->val = (double*)malloc(sizeof(double) * (size_t)nnz);
#pragma omp parallel for schedule(dynamic, 64)
  for (long node = 0; node < L->nnodes; ++node) {
    long ia[3];
    node_idx(L, node, ia);
    double row[27 * 4];
    for (int c = 0; c < nd; ++c) {
      long dof = node * nd + c;
      double w;
      L->fixed[dof] = (unsigned char)dirichlet(L, node, c, &w);
      L->wfix[dof] = w;
      L->rhs[dof] = sys_row(L, node, c, row);
      long pos = L->rowptr[dof];
      /* neighbour offsets in lexicographic order give ascending node ids */
      for (int nb = 0; nb < nnb; ++nb) {
        long ib[3] = {0, 0, 0};
        int t = nb, inside = 1;
        for (int k = 0; k < dim; ++k) {
          ib[k] = ia[k] + (t % 3) - 1;
          t /= 3;
          if (ib[k] < 0 || ib[k] > L->n[k]) inside = 0;
        }
        if (!inside) continue;
        long nbn = node_of(L, ib[0], ib[1], ib[2]);
        for (int cb = 0; cb < nd; ++cb) {
          L->col[pos] = nbn * nd + cb;
          L->val[pos] = row[nb * nd + cb];
          pos++;
        }
      }
    }
  }
}

long or_nnz(const or_level* L) { return L->rowptr ? L->rowptr[L->ndof] : 0; }

void or_csr_copy(const or_level* L, long* rowptr, long* col, double* val, double* rhs,
                 unsigned char* fixed) {
  memcpy(rowptr, L->rowptr, sizeof(long) * (size_t)(L->ndof + 1));
  memcpy(col, L->col, sizeof(long) * (size_t)or_nnz(L));
  memcpy(val, L->val, sizeof(double) * (size_t)or_nnz(L));
  memcpy(rhs, L->rhs, sizeof(double) * (size_t)L->ndof);
  memcpy(fixed, L->fixed, (size_t)L->ndof);
}

/* y = L x (assembled operator) */
static void spmv(const or_level* L, const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (long r = 0; r < L->ndof; ++r) {
    double s = 0.0;
    for (long p = L->rowptr[r]; p < L->rowptr[r + 1]; ++p) s = s + L->val[p] * x[L->col[p]];
    y[r] = s;
  }
}

/* r = b - L x */
void or_residual(const or_level* L, const double* b, const double* x, double* r) {
  spmv(L, x, r);
  for (long i = 0; i < L->ndof; ++i) r[i] = b[i] - r[i];
}

void or_apply(const or_level* L, const double* x, double* y) { spmv(L, x, y); }

/* ------------------------------------------------------------------------ */
/* Patches S_i (Sec. 3.1, eq. smoother)                                      */
/* ------------------------------------------------------------------------ */

/* DoFs of the patch of pressure node i, in local order: velocity DoFs of the
 * 5^d nodes around i (node-lex, x fastest; component inner), then pressure
 * DoFs of the 3^d nodes around i. Constrained and out-of-grid DoFs are left
 * out. own[c] = local index of the DoF (i, c) written back by Rt_i, or -1. */
static int patch_dofs(const or_level* L, long node, long* dofs, int* own) {
  int dim = L->dim, nd = L->ndpn;
  long ia[3];
  node_idx(L, node, ia);
  int n = 0;
  for (int c = 0; c < OMAX; ++c) own[c] = -1;
  int r5 = dim == 3 ? 5 : 1;
  for (int dz = 0; dz < r5; ++dz)
    for (int dy = 0; dy < 5; ++dy)
      for (int dx = 0; dx < 5; ++dx) {
        long ib[3] = {ia[0] + dx - 2, ia[1] + dy - 2, dim == 3 ? ia[2] + dz - 2 : 0};
        int inside = 1;
        for (int k = 0; k < dim; ++k)
          if (ib[k] < 0 || ib[k] > L->n[k]) inside = 0;
        if (!inside) continue;
        long nb = node_of(L, ib[0], ib[1], ib[2]);
        for (int c = 0; c < dim; ++c) {
          double w;
          if (dirichlet(L, nb, c, &w)) continue;
          if (nb == node) own[c] = n;
          dofs[n++] = nb * nd + c;
        }
      }
  int r3 = dim == 3 ? 3 : 1;
  for (int dz = 0; dz < r3; ++dz)
    for (int dy = 0; dy < 3; ++dy)
      for (int dx = 0; dx < 3; ++dx) {
        long ib[3] = {ia[0] + dx - 1, ia[1] + dy - 1, dim == 3 ? ia[2] + dz - 1 : 0};
        int inside = 1;
        for (int k = 0; k < dim; ++k)
          if (ib[k] < 0 || ib[k] > L->n[k]) inside = 0;
        if (!inside) continue;
        long nb = node_of(L, ib[0], ib[1], ib[2]);
        if (nb == node) own[dim] = n;
        dofs[n++] = nb * nd + dim;
      }
  return n;
}

int or_patch_dofs(const or_level* L, long node, long* dofs, int* own) {
  return patch_dofs(L, node, dofs, own);
}

/* L_i = R_i L R_i^T read from the assembled CSR (columns sorted) */
static void patch_matrix_csr(const or_level* L, int n, const long* dofs, double* Li) {
  for (int p = 0; p < n; ++p) {
    long r = dofs[p];
    long b = L->rowptr[r], e = L->rowptr[r + 1];
    for (int q = 0; q < n; ++q) {
      long cdof = dofs[q], lo = b, hi = e - 1;
      double v = 0.0;
      while (lo <= hi) {
        long mid = (lo + hi) / 2;
        if (L->col[mid] == cdof) { v = L->val[mid]; break; }
        if (L->col[mid] < cdof) lo = mid + 1; else hi = mid - 1;
      }
      Li[(long)p * n + q] = v;
    }
  }
}

/* L_i from rows computed on the fly (no assembled operator needed) */
static void patch_matrix_rows(const or_level* L, int n, const long* dofs, double* Li) {
  int dim = L->dim, nd = L->ndpn, nnb = dim == 3 ? 27 : 9;
  double row[27 * 4];
  for (int p = 0; p < n; ++p) {
    long node = dofs[p] / nd;
    int c = (int)(dofs[p] % nd);
    sys_row(L, node, c, row);
    long ia[3];
    node_idx(L, node, ia);
    for (int q = 0; q < n; ++q) {
      long nb = dofs[q] / nd;
      int cb = (int)(dofs[q] % nd);
      long ib[3];
      node_idx(L, nb, ib);
      int off = 0, mul = 1, near = 1;
      for (int k = 0; k < dim; ++k) {
        long d = ib[k] - ia[k];
        if (d < -1 || d > 1) near = 0;
        off += (int)(d + 1) * mul;
        mul *= 3;
      }
      Li[(long)p * n + q] = near ? row[off * nd + cb] : 0.0;
    }
  }
  (void)nnb;
}

int or_patch_matrix(const or_level* L, long node, double* Li, long* dofs, int* own) {
  int n = patch_dofs(L, node, dofs, own);
  if (L->rowptr) patch_matrix_csr(L, n, dofs, Li);
  else patch_matrix_rows(L, n, dofs, Li);
  return n;
}

/* ------------------------------------------------------------------------ */
/* Dense LU with partial pivoting (max |a|, lowest row index on ties)        */
/* ------------------------------------------------------------------------ */

static int lu_factor(int n, double* a, int* piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(a[(long)k * n + k]);
    for (int r = k + 1; r < n; ++r) {
      double v = fabs(a[(long)r * n + k]);
      if (v > best) { best = v; p = r; }
    }
    piv[k] = p;
    if (best == 0.0) return -1;
    if (p != k)
      for (int c = 0; c < n; ++c) {
        double t = a[(long)k * n + c];
        a[(long)k * n + c] = a[(long)p * n + c];
        a[(long)p * n + c] = t;
      }
    double d = a[(long)k * n + k];
    for (int r = k + 1; r < n; ++r) {
      double l = a[(long)r * n + k] / d;
      a[(long)r * n + k] = l;
      if (l != 0.0)
        for (int c = k + 1; c < n; ++c) a[(long)r * n + c] = a[(long)r * n + c] - l * a[(long)k * n + c];
    }
  }
  return 0;
}

static void lu_solve(int n, const double* lu, const int* piv, double* b) {
  for (int k = 0; k < n; ++k) {
    int p = piv[k];
    if (p != k) { double t = b[k]; b[k] = b[p]; b[p] = t; }
  }
  for (int r = 0; r < n; ++r) {
    double s = b[r];
    for (int c = 0; c < r; ++c) s = s - lu[(long)r * n + c] * b[c];
    b[r] = s;
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int c = r + 1; c < n; ++c) s = s - lu[(long)r * n + c] * b[c];
    b[r] = s / lu[(long)r * n + r];
  }
}

/* Local solves "down to machine accuracy" (Sec. 3.1.2).  The finite cell
 * blocks mix alpha-scaled and unscaled rows (entries from 1e-11 to 1 for
 * alpha = 1e-8), and partial pivoting alone then loses up to six digits.  The
 * LU is therefore taken of the symmetrically equilibrated block
 * D L_i D, D = diag(|L_i,jj|^{-1/2}), and L_i^{-1} r = D (D L_i D)^{-1} D r. */
static void eq_factor(int n, double* a, double* dsc, int* piv, int* st) {
  for (int j = 0; j < n; ++j) {
    double v = fabs(a[(long)j * n + j]);
    dsc[j] = v > 0.0 ? 1.0 / sqrt(v) : 1.0;
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) a[(long)r * n + c] = dsc[r] * a[(long)r * n + c] * dsc[c];
  *st = lu_factor(n, a, piv);
}

static void eq_solve(int n, const double* lu, const double* dsc, const int* piv, double* b) {
  for (int j = 0; j < n; ++j) b[j] = dsc[j] * b[j];
  lu_solve(n, lu, piv, b);
  for (int j = 0; j < n; ++j) b[j] = dsc[j] * b[j];
}

/* Dense solve A x = b (A overwritten), exported for tests. */
int or_dense_solve(int n, double* a, double* b) {
  int* piv = (int*)malloc(sizeof(int) * (size_t)n);
  int st = lu_factor(n, a, piv);
  if (st == 0) lu_solve(n, a, piv, b);
  free(piv);
  return st;
}

/* Equilibrated dense solve, exported for tests. */
int or_dense_solve_eq(int n, double* a, double* b) {
  int* piv = (int*)malloc(sizeof(int) * (size_t)n);
  double* dsc = (double*)malloc(sizeof(double) * (size_t)n);
  int st;
  eq_factor(n, a, dsc, piv, &st);
  if (st == 0) eq_solve(n, a, dsc, piv, b);
  free(piv);
  free(dsc);
  return st;
}

/* ------------------------------------------------------------------------ */
/* cache_inverse: owned rows of L_i^{-1} (Sec. 3.1.2)                        */
/* ------------------------------------------------------------------------ */

/* Owned rows of L_i^{-1}.  L_i is exactly symmetric (the assembly mirrors
 * a and c and uses one number for each B / B^T pair), so row k of L_i^{-1}
 * is the solution of L_i z = e_k. */
static int patch_inverse_rows(const or_level* L, long node, int* n_out, long* dofs, int* own,
                              double* rows /* [OMAX][PMAX] */) {
  int n = patch_dofs(L, node, dofs, own);
  double* Li = (double*)malloc(sizeof(double) * (size_t)n * n);
  int* piv = (int*)malloc(sizeof(int) * (size_t)n);
  double* dsc = (double*)malloc(sizeof(double) * (size_t)n);
  if (L->rowptr) patch_matrix_csr(L, n, dofs, Li);
  else patch_matrix_rows(L, n, dofs, Li);
  int st;
  eq_factor(n, Li, dsc, piv, &st);
  for (int c = 0; c < OMAX; ++c) {
    double* z = rows + c * PMAX;
    for (int q = 0; q < PMAX; ++q) z[q] = 0.0;
    if (own[c] < 0 || st != 0) continue;
    z[own[c]] = 1.0;
    eq_solve(n, Li, dsc, piv, z);
  }
  free(Li);
  free(piv);
  free(dsc);
  *n_out = n;
  return st;
}

int or_patch_inverse_rows(const or_level* L, long node, long* dofs, int* own, double* rows) {
  int n;
  int st = patch_inverse_rows(L, node, &n, dofs, own, rows);
  return st == 0 ? n : -1;
}

int or_build_inverse(or_level* L) {
  if (L->pinv) return 0;
  long np = L->nnodes;
  L->pn = (int*)malloc(sizeof(int) * (size_t)np);
  L->pdof = (long*)malloc(sizeof(long) * (size_t)np * PMAX);
  L->pown = (int*)malloc(sizeof(int) * (size_t)np * OMAX);
  L->pinv = (double*)malloc(sizeof(double) * (size_t)np * OMAX * PMAX);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : bad)
  for (long i = 0; i < np; ++i) {
    int n;
    int st = patch_inverse_rows(L, i, &n, L->pdof + i * PMAX, L->pown + i * OMAX,
                                L->pinv + i * OMAX * PMAX);
    L->pn[i] = n;
    if (st != 0) bad++;
  }
  return bad;
}

/* ------------------------------------------------------------------------ */
/* One RA smoother sweep (eq. iteration with eq. smoother)                   */
/* ------------------------------------------------------------------------ */

/* mode 0: cached owned rows (cache_inverse); mode 1: gather L_i, factor and
 * solve on every application (cache_matrix / cache_none semantics).
 * order: optional permutation of the patches (NULL = natural). The patch
 * corrections all read the same residual r = b - L x, so the order of the
 * patches does not change the result. */
int or_sweep(or_level* L, const double* b, double* x, int mode, const long* order) {
  long nd = L->ndpn;
  double* r = (double*)malloc(sizeof(double) * (size_t)L->ndof);
  double* xn = (double*)malloc(sizeof(double) * (size_t)L->ndof);
  or_residual(L, b, x, r);
  memcpy(xn, x, sizeof(double) * (size_t)L->ndof);
  if (mode == 0 && !L->pinv) or_build_inverse(L);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : bad)
  for (long t = 0; t < L->nnodes; ++t) {
    long i = order ? order[t] : t;
    long dofs[PMAX];
    int own[OMAX];
    double y[OMAX] = {0, 0, 0, 0};
    if (mode == 0) {
      int n = L->pn[i];
      const long PS = L->pstride ? L->pstride : PMAX;
      const long* pd = L->pdof + i * PS;
      const double* rows = L->pinv + i * OMAX * PS;
      for (int c = 0; c < OMAX; ++c) {
        if (L->pown[i * OMAX + c] < 0) continue;
        double s = 0.0;
        for (int q = 0; q < n; ++q) s = s + rows[c * PS + q] * r[pd[q]];
        y[c] = s;
      }
      for (int c = 0; c < OMAX; ++c) own[c] = L->pown[i * OMAX + c];
    } else {
      int n = patch_dofs(L, i, dofs, own);
      double* Li = (double*)malloc(sizeof(double) * (size_t)n * n);
      int* piv = (int*)malloc(sizeof(int) * (size_t)n);
      double* ri = (double*)malloc(sizeof(double) * (size_t)n);
      double* dsc = (double*)malloc(sizeof(double) * (size_t)n);
      int st;
      patch_matrix_csr(L, n, dofs, Li);
      for (int q = 0; q < n; ++q) ri[q] = r[dofs[q]];
      eq_factor(n, Li, dsc, piv, &st);
      if (st != 0) bad++;
      else {
        eq_solve(n, Li, dsc, piv, ri);
        for (int c = 0; c < OMAX; ++c)
          if (own[c] >= 0) y[c] = ri[own[c]];
      }
      free(Li); free(piv); free(ri); free(dsc);
    }
    /* restricted prolongation: write only the DoFs of node i */
    for (int c = 0; c < OMAX && c < nd; ++c)
      if (own[c] >= 0) xn[i * nd + c] = x[i * nd + c] + L->omega * y[c];
  }
  /* constrained DoFs take their Dirichlet value (identity rows) */
  for (long k = 0; k < L->ndof; ++k)
    if (L->fixed[k]) xn[k] = x[k] + r[k];
  memcpy(x, xn, sizeof(double) * (size_t)L->ndof);
  free(r);
  free(xn);
  return bad;
}

/* Sweep restricted to a subset of patches against a frozen residual r:
 * x[owned] += omega * (L_i^{-1} r_i)[owned] for the listed patches only.
 * Used to check that the sweep splits exactly into independent groups. */
void or_apply_patches(or_level* L, const double* r, double* x, long np, const long* list) {
  long nd = L->ndpn;
  if (!L->pinv) or_build_inverse(L);
  for (long t = 0; t < np; ++t) {
    long i = list[t];
    int n = L->pn[i];
    const long PS = L->pstride ? L->pstride : PMAX;
    const long* pd = L->pdof + i * PS;
    const double* rows = L->pinv + i * OMAX * PS;
    for (int c = 0; c < OMAX; ++c) {
      int o = L->pown[i * OMAX + c];
      if (o < 0) continue;
      double s = 0.0;
      for (int q = 0; q < n; ++q) s = s + rows[c * PS + q] * r[pd[q]];
      x[i * nd + c] = x[i * nd + c] + L->omega * s;
    }
  }
}

/* owner count: how many patches write each DoF (must be 1 per free DoF) */
void or_owner_count(const or_level* L, int* count) {
  long dofs[PMAX];
  int own[OMAX];
  memset(count, 0, sizeof(int) * (size_t)L->ndof);
  for (long i = 0; i < L->nnodes; ++i) {
    int n = patch_dofs(L, i, dofs, own);
    (void)n;
    for (int c = 0; c < OMAX; ++c)
      if (own[c] >= 0) count[dofs[own[c]]]++;
  }
}

/* ------------------------------------------------------------------------ */
/* Grid transfers (eq. restriction_op; P = R^T), Q1 interpolation            */
/* ------------------------------------------------------------------------ */

/* x_f += P e_c on every component; constrained fine DoFs are left alone. */
void or_prolong_add(const or_level* F, const or_level* Cc, const double* ec, double* xf) {
  int dim = F->dim, nd = F->ndpn;
  if (F->tp_rowptr) { /* adaptive grids: the stored node-to-node weights */
    for (long node = 0; node < F->nnodes; ++node)
      for (int c = 0; c < nd; ++c) {
        long dof = node * nd + c;
        if (F->fixed[dof]) continue;
        double s = 0.0;
        for (long q = F->tp_rowptr[node]; q < F->tp_rowptr[node + 1]; ++q) s = s + F->tp_val[q] * ec[F->tp_col[q] * nd + c];
        xf[dof] = xf[dof] + s;
      }
    return;
  }
  for (long node = 0; node < F->nnodes; ++node) {
    long ia[3];
    node_idx(F, node, ia);
    long lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) {
      lo[k] = ia[k] / 2;
      hi[k] = (ia[k] + 1) / 2;
    }
    for (int c = 0; c < nd; ++c) {
      long dof = node * nd + c;
      if (F->fixed[dof]) continue;
      double s = 0.0;
      for (int t = 0; t < (1 << dim); ++t) {
        long ic[3] = {0, 0, 0};
        double wgt = 1.0;
        int dup = 0;
        for (int k = 0; k < dim; ++k) {
          int bit = (t >> k) & 1;
          if (lo[k] == hi[k] && bit) dup = 1;
          ic[k] = bit ? hi[k] : lo[k];
          wgt = wgt * (lo[k] == hi[k] ? 1.0 : 0.5);
        }
        if (dup) continue;
        long cn = ic[0] + (long)Cc->nn[0] * (ic[1] + (long)Cc->nn[1] * ic[2]);
        s = s + wgt * ec[cn * nd + c];
      }
      xf[dof] = xf[dof] + s;
    }
  }
}

/* b_c = P^T r_f, then constrained coarse DoFs set to zero. */
void or_restrict(const or_level* F, const or_level* Cc, const double* rf, double* bc) {
  int dim = F->dim, nd = F->ndpn;
  memset(bc, 0, sizeof(double) * (size_t)Cc->ndof);
  if (F->tp_rowptr) { /* adaptive grids: the transpose of the stored weights */
    for (long node = 0; node < F->nnodes; ++node)
      for (long q = F->tp_rowptr[node]; q < F->tp_rowptr[node + 1]; ++q)
        for (int c = 0; c < nd; ++c) bc[F->tp_col[q] * nd + c] = bc[F->tp_col[q] * nd + c] + F->tp_val[q] * rf[node * nd + c];
    for (long k = 0; k < Cc->ndof; ++k)
      if (Cc->fixed[k]) bc[k] = 0.0;
    return;
  }
  for (long node = 0; node < F->nnodes; ++node) {
    long ia[3];
    node_idx(F, node, ia);
    long lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) {
      lo[k] = ia[k] / 2;
      hi[k] = (ia[k] + 1) / 2;
    }
    for (int t = 0; t < (1 << dim); ++t) {
      long ic[3] = {0, 0, 0};
      double wgt = 1.0;
      int dup = 0;
      for (int k = 0; k < dim; ++k) {
        int bit = (t >> k) & 1;
        if (lo[k] == hi[k] && bit) dup = 1;
        ic[k] = bit ? hi[k] : lo[k];
        wgt = wgt * (lo[k] == hi[k] ? 1.0 : 0.5);
      }
      if (dup) continue;
      long cn = ic[0] + (long)Cc->nn[0] * (ic[1] + (long)Cc->nn[1] * ic[2]);
      for (int c = 0; c < nd; ++c) bc[cn * nd + c] = bc[cn * nd + c] + wgt * rf[node * nd + c];
    }
  }
  for (long k = 0; k < Cc->ndof; ++k)
    if (Cc->fixed[k]) bc[k] = 0.0;
}

/* Galerkin coarse operator, the alternative to rediscretising the coarser
 * grids of the hierarchy (Sec. 3): L_c = R L_f P with the transfers above.
 * For free coarse DoFs (I,c) and (J,e):
 *   L_c[(I,c),(J,e)] = sum over free fine DoFs (i,c), (j,e) of
 *                      P[(i,c),(I,c)] L_f[(i,c),(j,e)] P[(j,e),(J,e)],
 * P[(i,c),(I,c)] = prod_k w(i_k - 2 I_k), w(0) = 1, w(+-1) = 1/2, else 0
 * (the Q1 interpolation of or_prolong_add; constrained fine DoFs have zero
 * rows of P).  Constrained coarse DoFs keep identity rows and zero columns,
 * as in the rediscretised operator.  Both levels must be assembled; the
 * values of C's operator are replaced (same structure), its right-hand side
 * is left alone (only the finest one is used). */
static double q1_weight(long d) { return d == 0 ? 1.0 : ((d == 1 || d == -1) ? 0.5 : 0.0); }

void or_galerkin(or_level* Cc, const or_level* F) {
  int dim = F->dim, nd = F->ndpn;
#pragma omp parallel for schedule(dynamic, 16)
  for (long row = 0; row < Cc->ndof; ++row) {
    long I = row / nd;
    int c = (int)(row % nd);
    long b = Cc->rowptr[row], e = Cc->rowptr[row + 1];
    for (long q = b; q < e; ++q) Cc->val[q] = (Cc->fixed[row] && Cc->col[q] == row) ? 1.0 : 0.0;
    if (Cc->fixed[row]) continue;
    long ia[3] = {0, 0, 0};
    node_idx(Cc, I, ia);
    /* fine nodes 2I + s, s in {-1, 0, 1}^d */
    for (int t = 0; t < (dim == 3 ? 27 : 9); ++t) {
      long fi[3] = {0, 0, 0};
      int tt = t, inside = 1;
      double wi = 1.0;
      for (int k = 0; k < dim; ++k) {
        long s = (tt % 3) - 1;
        tt /= 3;
        fi[k] = 2 * ia[k] + s;
        if (fi[k] < 0 || fi[k] > F->n[k]) inside = 0;
        wi = wi * q1_weight(s);
      }
      if (!inside) continue;
      long frow = node_of(F, fi[0], fi[1], fi[2]) * nd + c;
      if (F->fixed[frow]) continue;
      for (long p = F->rowptr[frow]; p < F->rowptr[frow + 1]; ++p) {
        long fcol = F->col[p];
        if (F->fixed[fcol]) continue;
        long j = fcol / nd;
        int ec = (int)(fcol % nd);
        long ja[3] = {0, 0, 0};
        node_idx(F, j, ja);
        /* coarse nodes J that fine node j interpolates from */
        for (long q = b; q < e; ++q) {
          long ccol = Cc->col[q];
          if ((int)(ccol % nd) != ec || Cc->fixed[ccol]) continue;
          long Ja[3] = {0, 0, 0};
          node_idx(Cc, ccol / nd, Ja);
          double wj = 1.0;
          for (int k = 0; k < dim; ++k) wj = wj * q1_weight(ja[k] - 2 * Ja[k]);
          if (wj != 0.0) Cc->val[q] = Cc->val[q] + wi * F->val[p] * wj;
        }
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Multigrid hierarchy, V-cycle and FGMRES                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
  int nlev;          /* levels 0 (coarsest) .. nlev-1 (finest) */
  or_level** lev;
  double* coarse_lu; /* dense LU of the equilibrated coarsest operator */
  double* coarse_d;
  int* coarse_piv;
  int nu_pre, nu_post, mode;
} or_mg;

or_mg* or_mg_new(int nlev, or_level** levels, int nu_pre, int nu_post, int mode) {
  or_mg* M = (or_mg*)calloc(1, sizeof(or_mg));
  M->nlev = nlev;
  M->lev = (or_level**)malloc(sizeof(or_level*) * (size_t)nlev);
  for (int l = 0; l < nlev; ++l) {
    M->lev[l] = levels[l];
    or_assemble(levels[l]);
    if (mode == 0 && l > 0) or_build_inverse(levels[l]);
  }
  M->nu_pre = nu_pre;
  M->nu_post = nu_post;
  M->mode = mode;
  or_level* C = M->lev[0];
  long n = C->ndof;
  M->coarse_lu = (double*)calloc((size_t)(n * n), sizeof(double));
  M->coarse_piv = (int*)malloc(sizeof(int) * (size_t)n);
  for (long r = 0; r < n; ++r)
    for (long p = C->rowptr[r]; p < C->rowptr[r + 1]; ++p) M->coarse_lu[r * n + C->col[p]] = C->val[p];
  M->coarse_d = (double*)malloc(sizeof(double) * (size_t)n);
  int st;
  eq_factor((int)n, M->coarse_lu, M->coarse_d, M->coarse_piv, &st);
  return M;
}

void or_mg_free(or_mg* M) {
  if (!M) return;
  free(M->lev);
  free(M->coarse_lu);
  free(M->coarse_d);
  free(M->coarse_piv);
  free(M);
}

static void vcycle(or_mg* M, int l, double* x, const double* b) {
  or_level* L = M->lev[l];
  if (l == 0) {
    double* t = (double*)malloc(sizeof(double) * (size_t)L->ndof);
    memcpy(t, b, sizeof(double) * (size_t)L->ndof);
    eq_solve((int)L->ndof, M->coarse_lu, M->coarse_d, M->coarse_piv, t);
    memcpy(x, t, sizeof(double) * (size_t)L->ndof);
    free(t);
    return;
  }
  or_level* C = M->lev[l - 1];
  for (int s = 0; s < M->nu_pre; ++s) or_sweep(L, b, x, M->mode, NULL);
  double* r = (double*)malloc(sizeof(double) * (size_t)L->ndof);
  or_residual(L, b, x, r);
  double* bc = (double*)malloc(sizeof(double) * (size_t)C->ndof);
  double* xc = (double*)calloc((size_t)C->ndof, sizeof(double));
  or_restrict(L, C, r, bc);
  vcycle(M, l - 1, xc, bc);
  or_prolong_add(L, C, xc, x);
  for (int s = 0; s < M->nu_post; ++s) or_sweep(L, b, x, M->mode, NULL);
  free(r); free(bc); free(xc);
}

void or_vcycle(or_mg* M, double* x, const double* b) { vcycle(M, M->nlev - 1, x, b); }

static double dot(long n, const double* a, const double* b) {
  double s = 0.0;
  for (long i = 0; i < n; ++i) s = s + a[i] * b[i];
  return s;
}

/* FGMRES(m), right preconditioned by one V-cycle from a zero initial guess,
 * modified Gram-Schmidt.  Stops when ||b - L x|| <= rtol ||b||; returns the
 * number of preconditioner applications, the true relative residual, and
 * (optionally) the history of estimated relative residuals. */
int or_fgmres(or_mg* M, const double* b, double* x, double rtol, int maxit, int m,
              double* relres, double* hist) {
  or_level* L = M->lev[M->nlev - 1];
  long n = L->ndof;
  double* V = (double*)malloc(sizeof(double) * (size_t)n * (m + 1));
  double* Z = (double*)malloc(sizeof(double) * (size_t)n * m);
  double* H = (double*)calloc((size_t)(m + 1) * m, sizeof(double));
  double* cs = (double*)malloc(sizeof(double) * (size_t)m);
  double* sn = (double*)malloc(sizeof(double) * (size_t)m);
  double* g = (double*)malloc(sizeof(double) * (size_t)(m + 1));
  double* w = (double*)malloc(sizeof(double) * (size_t)n);
  double bn = sqrt(dot(n, b, b));
  int its = 0;
  if (bn == 0.0) {
    memset(x, 0, sizeof(double) * (size_t)n);
    *relres = 0.0;
    goto done;
  }
  for (;;) {
    or_residual(L, b, x, w);
    double beta = sqrt(dot(n, w, w));
    if (beta <= rtol * bn || its >= maxit) { *relres = beta / bn; break; }
    for (long i = 0; i < n; ++i) V[i] = w[i] / beta;
    memset(g, 0, sizeof(double) * (size_t)(m + 1));
    g[0] = beta;
    int j, k = 0;
    for (j = 0; j < m && its < maxit; ++j) {
      double* zj = Z + (long)j * n;
      memset(zj, 0, sizeof(double) * (size_t)n);
      vcycle(M, M->nlev - 1, zj, V + (long)j * n);
      its++;
      or_apply(L, zj, w);
      for (int i = 0; i <= j; ++i) {
        double hij = dot(n, w, V + (long)i * n);
        H[i * m + j] = hij;
        for (long t = 0; t < n; ++t) w[t] = w[t] - hij * V[(long)i * n + t];
      }
      double hn = sqrt(dot(n, w, w));
      H[(j + 1) * m + j] = hn;
      if (hn != 0.0)
        for (long t = 0; t < n; ++t) V[(long)(j + 1) * n + t] = w[t] / hn;
      for (int i = 0; i < j; ++i) {
        double a = H[i * m + j], c = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * c;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      double a = H[j * m + j], c = H[(j + 1) * m + j];
      double den = sqrt(a * a + c * c);
      cs[j] = den == 0.0 ? 1.0 : a / den;
      sn[j] = den == 0.0 ? 0.0 : c / den;
      H[j * m + j] = den;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      if (hist) hist[its - 1] = fabs(g[j + 1]) / bn;
      k = j + 1;
      if (fabs(g[j + 1]) <= rtol * bn || hn == 0.0) break;
    }
    /* y = H^{-1} g, x += Z y */
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

/* Standalone GMG: V-cycles until ||r|| <= red * ||r0|| (Sec. 4 experiment). */
int or_gmg_solve(or_mg* M, const double* b, double* x, double red, int maxit, double* relred) {
  or_level* L = M->lev[M->nlev - 1];
  long n = L->ndof;
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  or_residual(L, b, x, r);
  double r0 = sqrt(dot(n, r, r)), rn = r0;
  int it = 0;
  while (it < maxit && rn > red * r0) {
    vcycle(M, M->nlev - 1, x, b);
    or_residual(L, b, x, r);
    rn = sqrt(dot(n, r, r));
    it++;
  }
  *relred = r0 > 0 ? rn / r0 : 0.0;
  free(r);
  return it;
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* boundary points (for the quadrature pins): x, n, w, shape */
void or_bpoints_copy(const or_level* L, double* xyz, double* nrm, double* w, long* cell) {
  for (long i = 0; i < L->nbp; ++i) {
    for (int k = 0; k < 3; ++k) { xyz[3 * i + k] = L->bp[i].x[k]; nrm[3 * i + k] = L->bp[i].n[k]; }
    w[i] = L->bp[i].w;
    cell[i] = L->bp[i].cell;
  }
}
