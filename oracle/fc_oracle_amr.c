/*
 * fc_oracle_amr.c -- plain, slow FP64 CPU oracle for the restricted additive
 * smoother on adaptive quadtree grids (2D): 2:1 balanced refinement towards
 * the obstacle boundaries, hanging nodes removed as constraints, and the
 * grid hierarchy of Algorithm 1.
 *
 * TEST INFRASTRUCTURE ONLY, like fc_oracle.c, which it includes: the element
 * integrals of a leaf cell are those of the uniform grid of the leaf's level
 * (fc_oracle.c's compute_elem on that grid), and the V-cycle, FGMRES,
 * standalone GMG and the RA sweep with cached owned rows are fc_oracle.c's,
 * run on levels whose operator, patches and prolongation are built here.
 * Nothing in the product library links, includes or calls it.
 *
 * What it computes (Sec. 3):
 *   - space tree: a root grid of nroot cells; every cell refined uniformly
 *     to level U; a leaf whose level set changes sign among its 3^d sample
 *     points (the cut-cell test of the volume rule) refined until level R;
 *     then the 2:1 balance: neighbouring leaves, across faces and corners,
 *     at most one level apart;
 *   - hanging nodes: a leaf corner in the middle of an edge of a coarser
 *     neighbour is constrained to the mean of that edge's end points (with
 *     corner balance those are never hanging) and carries no DoF; the
 *     operator and the load are assembled from the element data with every
 *     hanging corner expanded into its two parents (L = C^T L_raw C);
 *   - strong Dirichlet data of the box faces on the free nodes, eliminated
 *     symmetrically as in fc_oracle.c;
 *   - patch S_i of free pressure node i (Sec. 3.1): the pressures of the
 *     nodes connected to i, and the velocity DoFs of the nodes connected to
 *     any of them, where two free nodes are connected when a leaf cell has
 *     corners whose expansions contain them; constrained DoFs left out; the
 *     owned DoFs are p_i and the velocity of node i;
 *   - hierarchy (Algorithm 1): the next coarser grid replaces every leaf of
 *     the highest level with its parent (all siblings together) and is then
 *     balanced; repeated down to the root grid;
 *   - prolongation: a fine free node takes the coarse finite element
 *     function at its position (bilinear on the coarse leaf containing it,
 *     hanging coarse corners expanded); restriction its transpose, as in
 *     fc_oracle.c's transfers.
 * All levels share one lattice: the cells of the finest level R, so a leaf
 * of level r covers 2^(R - r) lattice cells per direction.
 */
#include "fc_oracle.c"

typedef struct {
  int R;           /* lattice level: lattice cells are the cells of level R */
  int nroot[2];
  int NX, NY;      /* lattice cells per direction: nroot << R */
  unsigned char* lev; /* [NY][NX]: level of the leaf covering the lattice cell */
} amr_tree;

static int amr_size(const amr_tree* T, int level) { return 1 << (T->R - level); }

/* refine the leaf covering lattice cell (X, Y) */
static void amr_refine_leaf(amr_tree* T, int X, int Y) {
  const int l = T->lev[(long)Y * T->NX + X], s = amr_size(T, l);
  const int X0 = X / s * s, Y0 = Y / s * s;
  for (int y = Y0; y < Y0 + s; ++y)
    for (int x = X0; x < X0 + s; ++x) T->lev[(long)y * T->NX + x] = (unsigned char)(l + 1);
}

/* 2:1 balance across faces and corners: refine coarse leaves next to
 * leaves more than one level finer, until none is left */
static void amr_balance(amr_tree* T) {
  int changed = 1;
  while (changed) {
    changed = 0;
    for (int Y = 0; Y < T->NY; ++Y)
      for (int X = 0; X < T->NX; ++X) {
        const int l = T->lev[(long)Y * T->NX + X];
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            const int x = X + dx, y = Y + dy;
            if (x < 0 || y < 0 || x >= T->NX || y >= T->NY) continue;
            if (T->lev[(long)y * T->NX + x] < l - 1) {
              amr_refine_leaf(T, x, y);
              changed = 1;
            }
          }
      }
  }
}

/* the level set changes sign among the 3^d sample points of the box */
static int amr_cut(const or_level* G, const double* lo, const double* hb) {
  int npos = 0;
  for (int j = 0; j < 3; ++j)
    for (int i = 0; i < 3; ++i) {
      double x[3] = {lo[0] + hb[0] * (0.5 * i), lo[1] + hb[1] * (0.5 * j), 0.0};
      if (phi_all(G, x) > 0.0) npos++;
    }
  return npos != 0 && npos != 9;
}

/* the finest grid: uniform to level U, cut leaves refined to level R, balanced.
 * G is any level of the problem (shapes, box). */
amr_tree* amr_tree_fine(const or_level* G, const int* nroot, int U, int R) {
  amr_tree* T = (amr_tree*)calloc(1, sizeof(amr_tree));
  T->R = R;
  T->nroot[0] = nroot[0];
  T->nroot[1] = nroot[1];
  T->NX = nroot[0] << R;
  T->NY = nroot[1] << R;
  T->lev = (unsigned char*)malloc((size_t)T->NX * T->NY);
  memset(T->lev, U, (size_t)T->NX * T->NY);
  const double hx = (G->hi[0] - G->lo[0]) / T->NX, hy = (G->hi[1] - G->lo[1]) / T->NY;
  for (int l = U; l < R; ++l) {
    const int s = amr_size(T, l);
    for (int Y = 0; Y < T->NY; Y += s)
      for (int X = 0; X < T->NX; X += s) {
        if (T->lev[(long)Y * T->NX + X] != l) continue;
        double lo[2] = {G->lo[0] + X * hx, G->lo[1] + Y * hy}, hb[2] = {s * hx, s * hy};
        if (amr_cut(G, lo, hb)) amr_refine_leaf(T, X, Y);
      }
  }
  amr_balance(T);
  return T;
}

/* Algorithm 1: every leaf of the highest level replaced with its parent,
 * then balanced */
amr_tree* amr_tree_coarsen(const amr_tree* F) {
  amr_tree* T = (amr_tree*)calloc(1, sizeof(amr_tree));
  *T = *F;
  T->lev = (unsigned char*)malloc((size_t)T->NX * T->NY);
  memcpy(T->lev, F->lev, (size_t)T->NX * T->NY);
  int rmax = 0;
  for (long c = 0; c < (long)T->NX * T->NY; ++c)
    if (T->lev[c] > rmax) rmax = T->lev[c];
  for (long c = 0; c < (long)T->NX * T->NY; ++c)
    if (T->lev[c] == rmax && rmax > 0) T->lev[c] = (unsigned char)(rmax - 1);
  amr_balance(T);
  return T;
}

void amr_tree_free(amr_tree* T) {
  if (!T) return;
  free(T->lev);
  free(T);
}

int amr_tree_level(const amr_tree* T, int X, int Y) { return T->lev[(long)Y * T->NX + X]; }

/* ------------------------------------------------------------------------ */
/* Nodes, hanging constraints and the level's operator                       */
/* ------------------------------------------------------------------------ */

typedef struct {
  const amr_tree* T;
  long nv;        /* lattice vertices (NX + 1)(NY + 1) */
  long* fid;      /* free node index of a vertex, -1 if none */
  long* hp;       /* [nv][2]: parent vertices of a hanging vertex, -1 otherwise */
  long nfree;
  long* fvert;    /* lattice vertex of each free node */
} amr_nodes;

static long amr_vid(const amr_tree* T, int X, int Y) { return (long)Y * (T->NX + 1) + X; }

static void amr_nodes_build(const amr_tree* T, amr_nodes* N) {
  N->T = T;
  N->nv = (long)(T->NX + 1) * (T->NY + 1);
  unsigned char* corner = (unsigned char*)calloc((size_t)N->nv, 1);
  N->hp = (long*)malloc(sizeof(long) * (size_t)N->nv * 2);
  for (long v = 0; v < 2 * N->nv; ++v) N->hp[v] = -1;
  for (int Y = 0; Y < T->NY; ++Y)
    for (int X = 0; X < T->NX; ++X) {
      const int s = amr_size(T, T->lev[(long)Y * T->NX + X]);
      if (X % s || Y % s) continue;
      corner[amr_vid(T, X, Y)] = corner[amr_vid(T, X + s, Y)] = 1;
      corner[amr_vid(T, X, Y + s)] = corner[amr_vid(T, X + s, Y + s)] = 1;
    }
  /* a corner in the middle of an edge of a leaf is hanging */
  for (int Y = 0; Y < T->NY; ++Y)
    for (int X = 0; X < T->NX; ++X) {
      const int s = amr_size(T, T->lev[(long)Y * T->NX + X]);
      if (X % s || Y % s || s < 2) continue;
      const int h = s / 2;
      const int mid[4][2] = {{X + h, Y}, {X + h, Y + s}, {X, Y + h}, {X + s, Y + h}};
      const int a[4][2] = {{X, Y}, {X, Y + s}, {X, Y}, {X + s, Y}};
      const int b[4][2] = {{X + s, Y}, {X + s, Y + s}, {X, Y + s}, {X + s, Y + s}};
      for (int e = 0; e < 4; ++e) {
        const long m = amr_vid(T, mid[e][0], mid[e][1]);
        if (!corner[m]) continue;
        N->hp[2 * m] = amr_vid(T, a[e][0], a[e][1]);
        N->hp[2 * m + 1] = amr_vid(T, b[e][0], b[e][1]);
      }
    }
  N->fid = (long*)malloc(sizeof(long) * (size_t)N->nv);
  N->nfree = 0;
  for (long v = 0; v < N->nv; ++v) N->fid[v] = (corner[v] && N->hp[2 * v] < 0) ? N->nfree++ : -1;
  N->fvert = (long*)malloc(sizeof(long) * (size_t)N->nfree);
  for (long v = 0; v < N->nv; ++v)
    if (N->fid[v] >= 0) N->fvert[N->fid[v]] = v;
  free(corner);
}

static void amr_nodes_free(amr_nodes* N) {
  free(N->fid);
  free(N->hp);
  free(N->fvert);
}

/* expansion of a lattice vertex into free nodes: (node, weight), 1 or 2 terms */
static int amr_expand(const amr_nodes* N, long v, long* node, double* w) {
  if (N->fid[v] >= 0) {
    node[0] = N->fid[v];
    w[0] = 1.0;
    return 1;
  }
  node[0] = N->fid[N->hp[2 * v]];
  node[1] = N->fid[N->hp[2 * v + 1]];
  w[0] = w[1] = 0.5;
  return 2;
}

/* sorted insertion into a small set */
static void set_add(long* a, int* n, long v) {
  int k = *n;
  for (int t = 0; t < k; ++t)
    if (a[t] == v) return;
  while (k > 0 && a[k - 1] > v) {
    a[k] = a[k - 1];
    --k;
  }
  a[k] = v;
  (*n)++;
}

#define AMR_ADJ 64 /* free nodes connected to one free node, at most */

/* the leaves of the tree: anchor (X, Y) and level, lattice order */
static long amr_leaves(const amr_tree* T, int* out /* [][3] or NULL */) {
  long n = 0;
  for (int Y = 0; Y < T->NY; ++Y)
    for (int X = 0; X < T->NX; ++X) {
      const int l = T->lev[(long)Y * T->NX + X], s = amr_size(T, l);
      if (X % s || Y % s) continue;
      if (out) {
        out[3 * n] = X;
        out[3 * n + 1] = Y;
        out[3 * n + 2] = l;
      }
      n++;
    }
  return n;
}

/* free-node adjacency: nodes sharing a leaf after expansion (incl. itself) */
static void amr_adjacency(const amr_nodes* N, long* adj /* [nfree][AMR_ADJ] */, int* nadj, int* err) {
  const amr_tree* T = N->T;
  for (long f = 0; f < N->nfree; ++f) nadj[f] = 0;
  long nl = amr_leaves(T, NULL);
  int* lv = (int*)malloc(sizeof(int) * 3 * (size_t)nl);
  amr_leaves(T, lv);
  for (long q = 0; q < nl; ++q) {
    const int X = lv[3 * q], Y = lv[3 * q + 1], s = amr_size(T, lv[3 * q + 2]);
    long nodes[8];
    int nn = 0;
    for (int c = 0; c < 4; ++c) {
      long nd2[2];
      double w2[2];
      const int k = amr_expand(N, amr_vid(T, X + (c & 1) * s, Y + (c >> 1) * s), nd2, w2);
      for (int t = 0; t < k; ++t) nodes[nn++] = nd2[t];
    }
    for (int a = 0; a < nn; ++a)
      for (int b = 0; b < nn; ++b) {
        if (nadj[nodes[a]] >= AMR_ADJ - 1) { *err = 1; continue; }
        set_add(adj + nodes[a] * AMR_ADJ, &nadj[nodes[a]], nodes[b]);
      }
  }
  free(lv);
}

/* Build the or_level of tree T.  ul[r] (r = 0..T->R): the uniform grids of
 * the problem at every level (element data of the leaves of that level);
 * C: the level's coarser neighbour in the hierarchy (its tree Tc) or NULL.
 * Returns NULL on a patch or adjacency overflow. */
or_level* amr_level_new(const amr_tree* T, or_level** ul, const amr_tree* Tc) {
  const or_level* G = ul[T->R];
  or_level* L = (or_level*)calloc(1, sizeof(or_level));
  L->dim = 2;
  L->ndpn = 3;
  for (int k = 0; k < 3; ++k) {
    L->n[k] = k < 2 ? (k == 0 ? T->NX : T->NY) : 1;
    L->nn[k] = L->n[k] + (k < 2 ? 1 : 0);
    L->lo[k] = G->lo[k];
    L->hi[k] = G->hi[k];
    L->h[k] = G->h[k];
  }
  L->hmin = G->hmin;
  L->alpha = G->alpha; L->eta = G->eta; L->beta = G->beta; L->lambda = G->lambda;
  L->omega = G->omega; L->ubar = G->ubar; L->qdepth = G->qdepth; L->preset = G->preset;
  amr_nodes N;
  amr_nodes_build(T, &N);
  const long nf = N.nfree, nd = 3;
  L->nnodes = nf;
  L->ndof = nf * nd;
  /* adjacency and CSR structure: rows (node, comp), columns of every
   * connected node, all components, ascending */
  long* adj = (long*)malloc(sizeof(long) * (size_t)nf * AMR_ADJ);
  int* nadj = (int*)malloc(sizeof(int) * (size_t)nf);
  int err = 0;
  amr_adjacency(&N, adj, nadj, &err);
  L->rowptr = (long*)malloc(sizeof(long) * (size_t)(L->ndof + 1));
  L->rowptr[0] = 0;
  for (long f = 0; f < nf; ++f)
    for (int c = 0; c < 3; ++c) L->rowptr[f * nd + c + 1] = L->rowptr[f * nd + c] + (long)nadj[f] * nd;
  const long nnz = L->rowptr[L->ndof];
  L->col = (long*)malloc(sizeof(long) * (size_t)nnz);
  L->val = (double*)calloc((size_t)nnz, sizeof(double));
  L->rhs = (double*)calloc((size_t)L->ndof, sizeof(double));
  L->fixed = (unsigned char*)calloc((size_t)L->ndof, 1);
  L->wfix = (double*)calloc((size_t)L->ndof, sizeof(double));
  for (long f = 0; f < nf; ++f)
    for (int c = 0; c < 3; ++c) {
      long p = L->rowptr[f * nd + c];
      for (int t = 0; t < nadj[f]; ++t)
        for (int e = 0; e < 3; ++e) L->col[p++] = adj[f * AMR_ADJ + t] * nd + e;
    }
  /* element contributions, hanging corners expanded */
  long nl = amr_leaves(T, NULL);
  int* lv = (int*)malloc(sizeof(int) * 3 * (size_t)nl);
  amr_leaves(T, lv);
  for (long q = 0; q < nl; ++q) {
    const int X = lv[3 * q], Y = lv[3 * q + 1], l = lv[3 * q + 2], s = amr_size(T, l);
    const or_level* U = ul[l];
    const long cell = (long)(X / s) + (long)U->n[0] * (Y / s);
    or_elem tmp;
    const or_elem* e = get_elem(U, cell, &tmp);
    long en[4][2];
    double ew[4][2];
    int ek[4];
    for (int a = 0; a < 4; ++a) ek[a] = amr_expand(&N, amr_vid(T, X + (a & 1) * s, Y + (a >> 1) * s), en[a], ew[a]);
    for (int a = 0; a < 4; ++a)
      for (int ta = 0; ta < ek[a]; ++ta) {
        const long fa = en[a][ta];
        const double wa = ew[a][ta];
        for (int c = 0; c < 2; ++c) L->rhs[fa * nd + c] = L->rhs[fa * nd + c] + wa * e->f[c][a];
        for (int b = 0; b < 4; ++b)
          for (int tb = 0; tb < ek[b]; ++tb) {
            const long fb = en[b][tb];
            const double w = wa * ew[b][tb];
            for (int r = 0; r < 3; ++r) {
              const long row = fa * nd + r;
              for (int cc = 0; cc < 3; ++cc) {
                double v;
                if (r < 2 && cc < 2) v = r == cc ? e->A[a][b] : 0.0;
                else if (r < 2) v = e->B[r][a][b];
                else if (cc < 2) v = e->B[cc][b][a];
                else v = e->C[a][b];
                if (v == 0.0 && !(r < 2 && cc < 2 && r == cc)) continue;
                const long colj = fb * nd + cc;
                long lo2 = L->rowptr[row], hi2 = L->rowptr[row + 1] - 1;
                while (lo2 <= hi2) {
                  const long mid = (lo2 + hi2) / 2;
                  if (L->col[mid] == colj) { L->val[mid] = L->val[mid] + w * v; break; }
                  if (L->col[mid] < colj) lo2 = mid + 1; else hi2 = mid - 1;
                }
              }
            }
          }
      }
  }
  free(lv);
  /* strong Dirichlet data on the free nodes of the box faces (presets of
   * fc_oracle.c) and their symmetric elimination */
  for (long f = 0; f < nf; ++f) {
    const long v = N.fvert[f];
    const int X = (int)(v % (T->NX + 1)), Y = (int)(v / (T->NX + 1));
    int fixed = 0;
    double w0 = 0.0;
    const int wall = Y == 0 || Y == T->NY;
    if (L->preset == 0) {
      fixed = wall || X == 0;
      if (!wall && X == 0) {
        const double y = L->lo[1] + (double)Y * L->h[1];
        const double sy = (y - L->lo[1]) / (L->hi[1] - L->lo[1]);
        w0 = 4.0 * L->ubar * sy * (1.0 - sy);
      }
    } else if (L->preset == 1) {
      fixed = wall;
    }
    if (fixed)
      for (int c = 0; c < 2; ++c) {
        L->fixed[f * nd + c] = 1;
        L->wfix[f * nd + c] = c == 0 ? w0 : 0.0;
      }
  }
  for (long r = 0; r < L->ndof; ++r) {
    if (L->fixed[r]) {
      for (long p = L->rowptr[r]; p < L->rowptr[r + 1]; ++p) L->val[p] = L->col[p] == r ? 1.0 : 0.0;
      L->rhs[r] = L->wfix[r];
      continue;
    }
    for (long p = L->rowptr[r]; p < L->rowptr[r + 1]; ++p)
      if (L->fixed[L->col[p]]) {
        L->rhs[r] = L->rhs[r] - L->val[p] * L->wfix[L->col[p]];
        L->val[p] = 0.0;
      }
  }
  /* patches and their owned rows */
  L->pn = (int*)malloc(sizeof(int) * (size_t)nf);
  L->pdof = (long*)malloc(sizeof(long) * (size_t)nf * PMAX);
  L->pown = (int*)malloc(sizeof(int) * (size_t)nf * OMAX);
  L->pinv = (double*)malloc(sizeof(double) * (size_t)nf * OMAX * PMAX);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : bad)
  for (long i = 0; i < nf; ++i) {
    long vel[AMR_ADJ * AMR_ADJ];
    int nv = 0;
    for (int t = 0; t < nadj[i]; ++t) {
      const long j = adj[i * AMR_ADJ + t];
      for (int u = 0; u < nadj[j]; ++u) {
        const long k = adj[j * AMR_ADJ + u];
        int seen = 0;
        for (int z = 0; z < nv; ++z)
          if (vel[z] == k) { seen = 1; break; }
        if (!seen) vel[nv++] = k;
      }
    }
    /* ascending node order */
    for (int a = 1; a < nv; ++a) {
      const long key = vel[a];
      int b = a - 1;
      while (b >= 0 && vel[b] > key) { vel[b + 1] = vel[b]; --b; }
      vel[b + 1] = key;
    }
    long* dofs = L->pdof + i * PMAX;
    int* own = L->pown + i * OMAX;
    for (int c = 0; c < OMAX; ++c) own[c] = -1;
    int n = 0;
    for (int z = 0; z < nv && n < PMAX; ++z)
      for (int c = 0; c < 2; ++c) {
        const long d = vel[z] * nd + c;
        if (L->fixed[d] || n >= PMAX) continue;
        if (vel[z] == i) own[c] = n;
        dofs[n++] = d;
      }
    for (int t = 0; t < nadj[i] && n < PMAX; ++t) {
      const long j = adj[i * AMR_ADJ + t];
      if (j == i) own[2] = n;
      dofs[n++] = j * nd + 2;
    }
    L->pn[i] = n;
    if (n >= PMAX) { bad++; continue; }
    double* Li = (double*)malloc(sizeof(double) * (size_t)n * n);
    int* piv = (int*)malloc(sizeof(int) * (size_t)n);
    double* dsc = (double*)malloc(sizeof(double) * (size_t)n);
    patch_matrix_csr(L, n, dofs, Li);
    int st;
    eq_factor(n, Li, dsc, piv, &st);
    double* rows = L->pinv + i * OMAX * PMAX;
    for (int c = 0; c < OMAX; ++c) {
      double* z = rows + c * PMAX;
      for (int t = 0; t < PMAX; ++t) z[t] = 0.0;
      if (own[c] < 0 || st != 0) continue;
      z[own[c]] = 1.0;
      eq_solve(n, Li, dsc, piv, z);
    }
    if (st != 0) bad++;
    free(Li); free(piv); free(dsc);
  }
  /* prolongation from the coarser tree: the coarse finite element function
   * at each fine free node */
  if (Tc) {
    amr_nodes Nc;
    amr_nodes_build(Tc, &Nc);
    L->tp_rowptr = (long*)malloc(sizeof(long) * (size_t)(nf + 1));
    long cap = nf * 8 + 16;
    L->tp_col = (long*)malloc(sizeof(long) * (size_t)cap);
    L->tp_val = (double*)malloc(sizeof(double) * (size_t)cap);
    L->tp_rowptr[0] = 0;
    for (long f = 0; f < nf; ++f) {
      const long v = N.fvert[f];
      const int X = (int)(v % (T->NX + 1)), Y = (int)(v / (T->NX + 1));
      const int cx = X < Tc->NX ? X : Tc->NX - 1, cy = Y < Tc->NY ? Y : Tc->NY - 1;
      const int s = amr_size(Tc, Tc->lev[(long)cy * Tc->NX + cx]);
      const int X0 = cx / s * s, Y0 = cy / s * s;
      const double tx = (double)(X - X0) / s, ty = (double)(Y - Y0) / s;
      long node[16];
      double wt[16];
      int nn = 0;
      for (int a = 0; a < 4; ++a) {
        const double wa = ((a & 1) ? tx : 1.0 - tx) * ((a >> 1) ? ty : 1.0 - ty);
        if (wa == 0.0) continue;
        long n2[2];
        double w2[2];
        const int k = amr_expand(&Nc, amr_vid(Tc, X0 + (a & 1) * s, Y0 + (a >> 1) * s), n2, w2);
        for (int t = 0; t < k; ++t) {
          int z = 0;
          while (z < nn && node[z] != n2[t]) ++z;
          if (z == nn) { node[nn] = n2[t]; wt[nn] = 0.0; nn++; }
          wt[z] = wt[z] + wa * w2[t];
        }
      }
      /* ascending coarse node order */
      for (int a = 1; a < nn; ++a) {
        const long kn = node[a];
        const double kw = wt[a];
        int b = a - 1;
        while (b >= 0 && node[b] > kn) { node[b + 1] = node[b]; wt[b + 1] = wt[b]; --b; }
        node[b + 1] = kn;
        wt[b + 1] = kw;
      }
      const long p0 = L->tp_rowptr[f];
      for (int z = 0; z < nn; ++z) {
        L->tp_col[p0 + z] = node[z];
        L->tp_val[p0 + z] = wt[z];
      }
      L->tp_rowptr[f + 1] = p0 + nn;
    }
    amr_nodes_free(&Nc);
  }
  free(adj);
  free(nadj);
  amr_nodes_free(&N);
  if (err || bad) {
    or_level_free(L);
    return NULL;
  }
  return L;
}

/* lattice vertex of free node f (for the tests) */
long amr_free_nodes(const amr_tree* T, long* fvert /* may be NULL */) {
  amr_nodes N;
  amr_nodes_build(T, &N);
  const long n = N.nfree;
  if (fvert)
    for (long f = 0; f < n; ++f) fvert[f] = N.fvert[f];
  amr_nodes_free(&N);
  return n;
}

/* hanging vertices and their parents (for the tests); returns their count */
long amr_hanging(const amr_tree* T, long* vert, long* par /* [][2] */) {
  amr_nodes N;
  amr_nodes_build(T, &N);
  long n = 0;
  for (long v = 0; v < N.nv; ++v)
    if (N.hp[2 * v] >= 0) {
      if (vert) vert[n] = v;
      if (par) { par[2 * n] = N.hp[2 * v]; par[2 * n + 1] = N.hp[2 * v + 1]; }
      n++;
    }
  amr_nodes_free(&N);
  return n;
}

/* cached patch data of free node i: dofs, owned local indices, owned rows */
int amr_patch_rows(const or_level* L, long i, long* dofs, int* own, double* rows) {
  const int n = L->pn[i];
  for (int t = 0; t < n; ++t) dofs[t] = L->pdof[i * PMAX + t];
  for (int c = 0; c < OMAX; ++c) own[c] = L->pown[i * OMAX + c];
  for (int c = 0; c < OMAX; ++c)
    for (int t = 0; t < PMAX; ++t) rows[c * PMAX + t] = L->pinv[(i * OMAX + c) * PMAX + t];
  return n;
}

/* the prolongation rows (for the tests) */
long amr_prolongation(const or_level* L, long* rowptr, long* col, double* val) {
  if (!L->tp_rowptr) return -1;
  const long nnz = L->tp_rowptr[L->nnodes];
  if (rowptr) memcpy(rowptr, L->tp_rowptr, sizeof(long) * (size_t)(L->nnodes + 1));
  if (col) memcpy(col, L->tp_col, sizeof(long) * (size_t)nnz);
  if (val) memcpy(val, L->tp_val, sizeof(double) * (size_t)nnz);
  return nnz;
}
