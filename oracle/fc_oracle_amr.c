/*
 * fc_oracle_amr.c -- plain, slow FP64 CPU oracle for the restricted additive
 * smoother on adaptive space-tree grids (quadtrees in 2D, octrees in 3D):
 * 2:1 balanced refinement towards the obstacle boundaries, hanging nodes
 * removed as constraints, and the grid hierarchy of Algorithm 1.
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
 *     then the 2:1 balance: neighbouring leaves, across faces, edges and
 *     corners, at most one level apart;
 *   - hanging nodes: a leaf corner in the middle of an edge of a coarser
 *     neighbour is constrained to the mean of that edge's end points; in 3D
 *     a corner in the middle of a face of a coarser neighbour to the mean of
 *     that face's four corners (with corner balance those are never
 *     hanging); hanging nodes carry no DoF; the operator and the load are
 *     assembled from the element data with every hanging corner expanded
 *     into its parents (L = C^T L_raw C);
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
 *     function at its position (multilinear on the coarse leaf containing
 *     it, hanging coarse corners expanded); restriction its transpose, as
 *     in fc_oracle.c's transfers.
 * All levels share one lattice: the cells of the finest level R, so a leaf
 * of level r covers 2^(R - r) lattice cells per direction.
 */
#include "fc_oracle.c"

typedef struct {
  int dim;
  int R;           /* lattice level: lattice cells are the cells of level R */
  int nroot[3];
  int NX, NY, NZ;  /* lattice cells per direction: nroot << R (NZ = 1 in 2D) */
  unsigned char* lev; /* [NZ][NY][NX]: level of the leaf covering the lattice cell */
} amr_tree;

static int amr_size(const amr_tree* T, int level) { return 1 << (T->R - level); }
static long amr_cell(const amr_tree* T, int X, int Y, int Z) { return ((long)Z * T->NY + Y) * T->NX + X; }

/* refine the leaf covering lattice cell (X, Y, Z) */
static void amr_refine_leaf(amr_tree* T, int X, int Y, int Z) {
  const int l = T->lev[amr_cell(T, X, Y, Z)], s = amr_size(T, l);
  const int X0 = X / s * s, Y0 = Y / s * s, Z0 = T->dim == 3 ? Z / s * s : 0, sz = T->dim == 3 ? s : 1;
  for (int z = Z0; z < Z0 + sz; ++z)
    for (int y = Y0; y < Y0 + s; ++y)
      for (int x = X0; x < X0 + s; ++x) T->lev[amr_cell(T, x, y, z)] = (unsigned char)(l + 1);
}

/* 2:1 balance across faces, edges and corners: refine coarse leaves next to
 * leaves more than one level finer, until none is left */
static void amr_balance(amr_tree* T) {
  const int rz = T->dim == 3 ? 1 : 0;
  int changed = 1;
  while (changed) {
    changed = 0;
    for (int Z = 0; Z < T->NZ; ++Z)
      for (int Y = 0; Y < T->NY; ++Y)
        for (int X = 0; X < T->NX; ++X) {
          const int l = T->lev[amr_cell(T, X, Y, Z)];
          for (int dz = -rz; dz <= rz; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
              for (int dx = -1; dx <= 1; ++dx) {
                const int x = X + dx, y = Y + dy, z = Z + dz;
                if (x < 0 || y < 0 || z < 0 || x >= T->NX || y >= T->NY || z >= T->NZ) continue;
                if (T->lev[amr_cell(T, x, y, z)] < l - 1) {
                  amr_refine_leaf(T, x, y, z);
                  changed = 1;
                }
              }
        }
  }
}

/* the level set changes sign among the 3^d sample points of the box */
static int amr_cut(const or_level* G, const double* lo, const double* hb) {
  const int dim = G->dim, m3 = dim == 3 ? 3 : 1;
  int npos = 0, ns = 0;
  for (int k = 0; k < m3; ++k)
    for (int j = 0; j < 3; ++j)
      for (int i = 0; i < 3; ++i) {
        double x[3] = {lo[0] + hb[0] * (0.5 * i), lo[1] + hb[1] * (0.5 * j), dim == 3 ? lo[2] + hb[2] * (0.5 * k) : 0.0};
        if (phi_all(G, x) > 0.0) npos++;
        ns++;
      }
  return npos != 0 && npos != ns;
}

/* the finest grid: uniform to level U, cut leaves refined to level R, balanced.
 * G is any level of the problem (shapes, box, dimension). */
amr_tree* amr_tree_fine(const or_level* G, const int* nroot, int U, int R) {
  amr_tree* T = (amr_tree*)calloc(1, sizeof(amr_tree));
  T->dim = G->dim;
  T->R = R;
  for (int k = 0; k < 3; ++k) T->nroot[k] = k < T->dim ? nroot[k] : 1;
  T->NX = T->nroot[0] << R;
  T->NY = T->nroot[1] << R;
  T->NZ = T->dim == 3 ? T->nroot[2] << R : 1;
  const long nc = (long)T->NX * T->NY * T->NZ;
  T->lev = (unsigned char*)malloc((size_t)nc);
  memset(T->lev, U, (size_t)nc);
  const double h[3] = {(G->hi[0] - G->lo[0]) / T->NX, (G->hi[1] - G->lo[1]) / T->NY,
                       T->dim == 3 ? (G->hi[2] - G->lo[2]) / T->NZ : 0.0};
  for (int l = U; l < R; ++l) {
    const int s = amr_size(T, l), sz = T->dim == 3 ? s : 1;
    for (int Z = 0; Z < T->NZ; Z += sz)
      for (int Y = 0; Y < T->NY; Y += s)
        for (int X = 0; X < T->NX; X += s) {
          if (T->lev[amr_cell(T, X, Y, Z)] != l) continue;
          double lo[3] = {G->lo[0] + X * h[0], G->lo[1] + Y * h[1], T->dim == 3 ? G->lo[2] + Z * h[2] : 0.0};
          double hb[3] = {s * h[0], s * h[1], s * h[2]};
          if (amr_cut(G, lo, hb)) amr_refine_leaf(T, X, Y, Z);
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
  const long nc = (long)T->NX * T->NY * T->NZ;
  T->lev = (unsigned char*)malloc((size_t)nc);
  memcpy(T->lev, F->lev, (size_t)nc);
  int rmax = 0;
  for (long c = 0; c < nc; ++c)
    if (T->lev[c] > rmax) rmax = T->lev[c];
  for (long c = 0; c < nc; ++c)
    if (T->lev[c] == rmax && rmax > 0) T->lev[c] = (unsigned char)(rmax - 1);
  amr_balance(T);
  return T;
}

void amr_tree_free(amr_tree* T) {
  if (!T) return;
  free(T->lev);
  free(T);
}

int amr_tree_level(const amr_tree* T, int X, int Y, int Z) { return T->lev[amr_cell(T, X, Y, Z)]; }

/* ------------------------------------------------------------------------ */
/* Nodes, hanging constraints and the level's operator                       */
/* ------------------------------------------------------------------------ */

typedef struct {
  const amr_tree* T;
  long nv;        /* lattice vertices */
  long* fid;      /* free node index of a vertex, -1 if none */
  long* hp;       /* [nv][4]: parent vertices of a hanging vertex */
  int* hn;        /* parents of a hanging vertex (2 edge, 4 face), 0 otherwise */
  long nfree;
  long* fvert;    /* lattice vertex of each free node */
} amr_nodes;

static long amr_vid(const amr_tree* T, int X, int Y, int Z) {
  return ((long)Z * (T->NY + 1) + Y) * (T->NX + 1) + X;
}

static void amr_vxyz(const amr_tree* T, long v, int* X, int* Y, int* Z) {
  *X = (int)(v % (T->NX + 1));
  *Y = (int)((v / (T->NX + 1)) % (T->NY + 1));
  *Z = (int)(v / ((long)(T->NX + 1) * (T->NY + 1)));
}

/* the leaves of the tree: anchor (X, Y, Z) and level, lattice order */
static long amr_leaves(const amr_tree* T, int* out /* [][4] or NULL */) {
  long n = 0;
  for (int Z = 0; Z < T->NZ; ++Z)
    for (int Y = 0; Y < T->NY; ++Y)
      for (int X = 0; X < T->NX; ++X) {
        const int l = T->lev[amr_cell(T, X, Y, Z)], s = amr_size(T, l);
        if (X % s || Y % s || (T->dim == 3 && Z % s)) continue;
        if (out) {
          out[4 * n] = X;
          out[4 * n + 1] = Y;
          out[4 * n + 2] = Z;
          out[4 * n + 3] = l;
        }
        n++;
      }
  return n;
}

/* corner a (bit k: +s in direction k) of the leaf at (X, Y, Z) */
static long amr_corner(const amr_tree* T, int X, int Y, int Z, int s, int a) {
  return amr_vid(T, X + (a & 1) * s, Y + ((a >> 1) & 1) * s, T->dim == 3 ? Z + ((a >> 2) & 1) * s : 0);
}

static void amr_nodes_build(const amr_tree* T, amr_nodes* N) {
  const int dim = T->dim, nc = 1 << dim;
  N->T = T;
  N->nv = (long)(T->NX + 1) * (T->NY + 1) * (dim == 3 ? T->NZ + 1 : 1);
  unsigned char* corner = (unsigned char*)calloc((size_t)N->nv, 1);
  N->hp = (long*)malloc(sizeof(long) * (size_t)N->nv * 4);
  N->hn = (int*)calloc((size_t)N->nv, sizeof(int));
  const long nl = amr_leaves(T, NULL);
  int* lv = (int*)malloc(sizeof(int) * 4 * (size_t)nl);
  amr_leaves(T, lv);
  for (long q = 0; q < nl; ++q) {
    const int s = amr_size(T, lv[4 * q + 3]);
    for (int a = 0; a < nc; ++a) corner[amr_corner(T, lv[4 * q], lv[4 * q + 1], lv[4 * q + 2], s, a)] = 1;
  }
  /* an edge midpoint (2 parents) or, in 3D, a face centre (4 parents) of a
   * leaf that is a corner of another leaf is hanging */
  for (long q = 0; q < nl; ++q) {
    const int X = lv[4 * q], Y = lv[4 * q + 1], Z = lv[4 * q + 2], s = amr_size(T, lv[4 * q + 3]);
    if (s < 2) continue;
    const int h = s / 2;
    /* edges: direction k, the other coordinates at 0 or s */
    for (int k = 0; k < dim; ++k)
      for (int e = 0; e < (dim == 3 ? 4 : 2); ++e) {
        int o[3] = {0, 0, 0}, t = 0;
        for (int m = 0; m < dim; ++m) {
          if (m == k) continue;
          o[m] = ((e >> t) & 1) * s;
          t++;
        }
        int a[3] = {X + o[0], Y + o[1], Z + o[2]}, b[3] = {a[0], a[1], a[2]}, mm[3] = {a[0], a[1], a[2]};
        b[k] += s;
        mm[k] += h;
        const long m = amr_vid(T, mm[0], mm[1], dim == 3 ? mm[2] : 0);
        if (!corner[m]) continue;
        N->hn[m] = 2;
        N->hp[4 * m] = amr_vid(T, a[0], a[1], dim == 3 ? a[2] : 0);
        N->hp[4 * m + 1] = amr_vid(T, b[0], b[1], dim == 3 ? b[2] : 0);
      }
    if (dim == 3)
      /* faces: normal direction k, at 0 or s */
      for (int k = 0; k < 3; ++k)
        for (int side = 0; side < 2; ++side) {
          const int u = k == 0 ? 1 : 0, w = k == 2 ? 1 : 2;  /* the in-face directions */
          int c0[3] = {X, Y, Z};
          c0[k] += side * s;
          int mm[3] = {c0[0], c0[1], c0[2]};
          mm[u] += h;
          mm[w] += h;
          const long m = amr_vid(T, mm[0], mm[1], mm[2]);
          if (!corner[m]) continue;
          N->hn[m] = 4;
          for (int t = 0; t < 4; ++t) {
            int c[3] = {c0[0], c0[1], c0[2]};
            c[u] += (t & 1) * s;
            c[w] += (t >> 1) * s;
            N->hp[4 * m + t] = amr_vid(T, c[0], c[1], c[2]);
          }
        }
  }
  N->fid = (long*)malloc(sizeof(long) * (size_t)N->nv);
  N->nfree = 0;
  for (long v = 0; v < N->nv; ++v) N->fid[v] = (corner[v] && N->hn[v] == 0) ? N->nfree++ : -1;
  N->fvert = (long*)malloc(sizeof(long) * (size_t)N->nfree);
  for (long v = 0; v < N->nv; ++v)
    if (N->fid[v] >= 0) N->fvert[N->fid[v]] = v;
  free(corner);
  free(lv);
}

static void amr_nodes_free(amr_nodes* N) {
  free(N->fid);
  free(N->hp);
  free(N->hn);
  free(N->fvert);
}

/* expansion of a lattice vertex into free nodes: (node, weight), 1, 2 or 4 terms */
static int amr_expand(const amr_nodes* N, long v, long* node, double* w) {
  if (N->fid[v] >= 0) {
    node[0] = N->fid[v];
    w[0] = 1.0;
    return 1;
  }
  const int k = N->hn[v];
  for (int t = 0; t < k; ++t) {
    node[t] = N->fid[N->hp[4 * v + t]];
    w[t] = 1.0 / k;
  }
  return k;
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

#define AMR_ADJ 192 /* free nodes connected to one free node, at most */

/* free-node adjacency: nodes sharing a leaf after expansion (incl. itself) */
static void amr_adjacency(const amr_nodes* N, long* adj /* [nfree][AMR_ADJ] */, int* nadj, int* err) {
  const amr_tree* T = N->T;
  const int nc = 1 << T->dim;
  for (long f = 0; f < N->nfree; ++f) nadj[f] = 0;
  long nl = amr_leaves(T, NULL);
  int* lv = (int*)malloc(sizeof(int) * 4 * (size_t)nl);
  amr_leaves(T, lv);
  for (long q = 0; q < nl; ++q) {
    const int s = amr_size(T, lv[4 * q + 3]);
    long nodes[32];
    int nn = 0;
    for (int c = 0; c < nc; ++c) {
      long n4[4];
      double w4[4];
      const int k = amr_expand(N, amr_corner(T, lv[4 * q], lv[4 * q + 1], lv[4 * q + 2], s, c), n4, w4);
      for (int t = 0; t < k; ++t) nodes[nn++] = n4[t];
    }
    for (int a = 0; a < nn; ++a)
      for (int b = 0; b < nn; ++b) {
        if (nadj[nodes[a]] >= AMR_ADJ - 1) { *err = 1; continue; }
        set_add(adj + nodes[a] * AMR_ADJ, &nadj[nodes[a]], nodes[b]);
      }
  }
  free(lv);
}

/* patch DoFs of free node i (velocity of the nodes connected to a pressure
 * node connected to i, ascending, then those pressures); own[c]: local
 * index of DoF c of node i or -1; returns the count (stops at cap) */
static int amr_patch_list(const or_level* L, const long* adj, const int* nadj, long i, long* dofs, int* own, int cap) {
  const int nd = L->ndpn, dim = L->dim;
  long* vel = (long*)malloc(sizeof(long) * (size_t)AMR_ADJ * AMR_ADJ);
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
  for (int c = 0; c < OMAX; ++c) own[c] = -1;
  int n = 0;
  for (int z = 0; z < nv; ++z)
    for (int c = 0; c < dim; ++c) {
      const long d = vel[z] * nd + c;
      if (L->fixed[d]) continue;
      if (n < cap) {
        if (vel[z] == i) own[c] = n;
        dofs[n] = d;
      }
      n++;
    }
  for (int t = 0; t < nadj[i]; ++t) {
    const long j = adj[i * AMR_ADJ + t];
    if (n < cap) {
      if (j == i) own[dim] = n;
      dofs[n] = j * nd + dim;
    }
    n++;
  }
  free(vel);
  return n;
}

/* Build the or_level of tree T.  ul[r] (r = 0..T->R): the uniform grids of
 * the problem at every level (element data of the leaves of that level);
 * Tc: the level's coarser neighbour in the hierarchy or NULL.  Returns NULL
 * on an adjacency overflow or a singular patch. */
or_level* amr_level_new(const amr_tree* T, or_level** ul, const amr_tree* Tc) {
  const or_level* G = ul[T->R];
  const int dim = T->dim, nd = dim + 1, nc = 1 << dim;
  or_level* L = (or_level*)calloc(1, sizeof(or_level));
  L->dim = dim;
  L->ndpn = nd;
  const int NL[3] = {T->NX, T->NY, T->NZ};
  for (int k = 0; k < 3; ++k) {
    L->n[k] = k < dim ? NL[k] : 1;
    L->nn[k] = L->n[k] + (k < dim ? 1 : 0);
    L->lo[k] = G->lo[k];
    L->hi[k] = G->hi[k];
    L->h[k] = G->h[k];
  }
  L->hmin = G->hmin;
  L->alpha = G->alpha; L->eta = G->eta; L->beta = G->beta; L->lambda = G->lambda;
  L->omega = G->omega; L->ubar = G->ubar; L->qdepth = G->qdepth; L->preset = G->preset;
  amr_nodes N;
  amr_nodes_build(T, &N);
  const long nf = N.nfree;
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
    for (int c = 0; c < nd; ++c) L->rowptr[f * nd + c + 1] = L->rowptr[f * nd + c] + (long)nadj[f] * nd;
  const long nnz = L->rowptr[L->ndof];
  L->col = (long*)malloc(sizeof(long) * (size_t)nnz);
  L->val = (double*)calloc((size_t)nnz, sizeof(double));
  L->rhs = (double*)calloc((size_t)L->ndof, sizeof(double));
  L->fixed = (unsigned char*)calloc((size_t)L->ndof, 1);
  L->wfix = (double*)calloc((size_t)L->ndof, sizeof(double));
  for (long f = 0; f < nf; ++f)
    for (int c = 0; c < nd; ++c) {
      long p = L->rowptr[f * nd + c];
      for (int t = 0; t < nadj[f]; ++t)
        for (int e = 0; e < nd; ++e) L->col[p++] = adj[f * AMR_ADJ + t] * nd + e;
    }
  /* element contributions, hanging corners expanded */
  long nl = amr_leaves(T, NULL);
  int* lv = (int*)malloc(sizeof(int) * 4 * (size_t)nl);
  amr_leaves(T, lv);
  for (long q = 0; q < nl; ++q) {
    const int X = lv[4 * q], Y = lv[4 * q + 1], Z = lv[4 * q + 2], l = lv[4 * q + 3], s = amr_size(T, l);
    const or_level* U = ul[l];
    const long cell = (long)(X / s) + (long)U->n[0] * ((Y / s) + (long)U->n[1] * (dim == 3 ? Z / s : 0));
    or_elem tmp;
    const or_elem* e = get_elem(U, cell, &tmp);
    long en[8][4];
    double ew[8][4];
    int ek[8];
    for (int a = 0; a < nc; ++a) ek[a] = amr_expand(&N, amr_corner(T, X, Y, Z, s, a), en[a], ew[a]);
    for (int a = 0; a < nc; ++a)
      for (int ta = 0; ta < ek[a]; ++ta) {
        const long fa = en[a][ta];
        const double wa = ew[a][ta];
        for (int c = 0; c < dim; ++c) L->rhs[fa * nd + c] = L->rhs[fa * nd + c] + wa * e->f[c][a];
        for (int b = 0; b < nc; ++b)
          for (int tb = 0; tb < ek[b]; ++tb) {
            const long fb = en[b][tb];
            const double w = wa * ew[b][tb];
            for (int r = 0; r < nd; ++r) {
              const long row = fa * nd + r;
              for (int cc = 0; cc < nd; ++cc) {
                double v;
                if (r < dim && cc < dim) v = r == cc ? e->A[a][b] : 0.0;
                else if (r < dim) v = e->B[r][a][b];
                else if (cc < dim) v = e->B[cc][b][a];
                else v = e->C[a][b];
                if (v == 0.0 && !(r < dim && cc < dim && r == cc)) continue;
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
    int X, Y, Z;
    amr_vxyz(T, N.fvert[f], &X, &Y, &Z);
    int fixed = 0;
    double w0 = 0.0;
    int wall = Y == 0 || Y == T->NY;
    if (dim == 3) wall = wall || Z == 0 || Z == T->NZ;
    if (L->preset == 0) {
      fixed = wall || X == 0;
      if (!wall && X == 0) {
        const double y = L->lo[1] + (double)Y * L->h[1];
        const double sy = (y - L->lo[1]) / (L->hi[1] - L->lo[1]);
        w0 = 4.0 * L->ubar * sy * (1.0 - sy);
        if (dim == 3) {
          const double z = L->lo[2] + (double)Z * L->h[2];
          const double sz = (z - L->lo[2]) / (L->hi[2] - L->lo[2]);
          w0 = w0 * 4.0 * sz * (1.0 - sz);
        }
      }
    } else if (L->preset == 1) {
      fixed = wall;
    }
    if (fixed)
      for (int c = 0; c < dim; ++c) {
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
  /* patches and their owned rows (stride: the largest patch) */
  int ps = 1;
  {
    long dummy[1];
    int own[OMAX];
    for (long i = 0; i < nf; ++i) {
      const int n = amr_patch_list(L, adj, nadj, i, dummy, own, 0);
      if (n > ps) ps = n;
    }
  }
  L->pstride = ps;
  L->pn = (int*)malloc(sizeof(int) * (size_t)nf);
  L->pdof = (long*)malloc(sizeof(long) * (size_t)nf * ps);
  L->pown = (int*)malloc(sizeof(int) * (size_t)nf * OMAX);
  L->pinv = (double*)malloc(sizeof(double) * (size_t)nf * OMAX * ps);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : bad)
  for (long i = 0; i < nf; ++i) {
    long* dofs = L->pdof + i * ps;
    int* own = L->pown + i * OMAX;
    const int n = amr_patch_list(L, adj, nadj, i, dofs, own, ps);
    L->pn[i] = n;
    double* Li = (double*)malloc(sizeof(double) * (size_t)n * n);
    int* piv = (int*)malloc(sizeof(int) * (size_t)n);
    double* dsc = (double*)malloc(sizeof(double) * (size_t)n);
    patch_matrix_csr(L, n, dofs, Li);
    int st;
    eq_factor(n, Li, dsc, piv, &st);
    double* rows = L->pinv + i * OMAX * ps;
    for (int c = 0; c < OMAX; ++c) {
      double* z = rows + (long)c * ps;
      for (int t = 0; t < ps; ++t) z[t] = 0.0;
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
    long cap = nf * 32 + 16;
    L->tp_col = (long*)malloc(sizeof(long) * (size_t)cap);
    L->tp_val = (double*)malloc(sizeof(double) * (size_t)cap);
    L->tp_rowptr[0] = 0;
    for (long f = 0; f < nf; ++f) {
      int X, Y, Z;
      amr_vxyz(T, N.fvert[f], &X, &Y, &Z);
      const int cx = X < Tc->NX ? X : Tc->NX - 1, cy = Y < Tc->NY ? Y : Tc->NY - 1;
      const int cz = dim == 3 ? (Z < Tc->NZ ? Z : Tc->NZ - 1) : 0;
      const int s = amr_size(Tc, Tc->lev[amr_cell(Tc, cx, cy, cz)]);
      const int X0 = cx / s * s, Y0 = cy / s * s, Z0 = dim == 3 ? cz / s * s : 0;
      const double t[3] = {(double)(X - X0) / s, (double)(Y - Y0) / s, dim == 3 ? (double)(Z - Z0) / s : 0.0};
      long node[64];
      double wt[64];
      int nn = 0;
      for (int a = 0; a < nc; ++a) {
        double wa = 1.0;
        for (int k = 0; k < dim; ++k) wa = wa * (((a >> k) & 1) ? t[k] : 1.0 - t[k]);
        if (wa == 0.0) continue;
        long n4[4];
        double w4[4];
        const int k = amr_expand(&Nc, amr_corner(Tc, X0, Y0, Z0, s, a), n4, w4);
        for (int u = 0; u < k; ++u) {
          int z = 0;
          while (z < nn && node[z] != n4[u]) ++z;
          if (z == nn) { node[nn] = n4[u]; wt[nn] = 0.0; nn++; }
          wt[z] = wt[z] + wa * w4[u];
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

/* lattice vertex of each free node (for the tests); returns their count */
long amr_free_nodes(const amr_tree* T, long* fvert /* may be NULL */) {
  amr_nodes N;
  amr_nodes_build(T, &N);
  const long n = N.nfree;
  if (fvert)
    for (long f = 0; f < n; ++f) fvert[f] = N.fvert[f];
  amr_nodes_free(&N);
  return n;
}

/* hanging vertices, their parent counts and parents (for the tests) */
long amr_hanging(const amr_tree* T, long* vert, int* npar, long* par /* [][4] */) {
  amr_nodes N;
  amr_nodes_build(T, &N);
  long n = 0;
  for (long v = 0; v < N.nv; ++v)
    if (N.hn[v] > 0) {
      if (vert) vert[n] = v;
      if (npar) npar[n] = N.hn[v];
      if (par)
        for (int t = 0; t < 4; ++t) par[4 * n + t] = t < N.hn[v] ? N.hp[4 * v + t] : -1;
      n++;
    }
  amr_nodes_free(&N);
  return n;
}

/* cached patch data of free node i: dofs, owned local indices, owned rows
 * (rows[c][0 .. n-1]) */
int amr_patch_rows(const or_level* L, long i, long* dofs, int* own, double* rows, int cap) {
  const int n = L->pn[i], ps = L->pstride;
  if (n > cap) return -1;
  for (int t = 0; t < n; ++t) dofs[t] = L->pdof[i * ps + t];
  for (int c = 0; c < OMAX; ++c) own[c] = L->pown[i * OMAX + c];
  for (int c = 0; c < OMAX; ++c)
    for (int t = 0; t < n; ++t) rows[(long)c * cap + t] = L->pinv[(i * OMAX + c) * ps + t];
  return n;
}

int amr_patch_stride(const or_level* L) { return L->pstride; }

/* the prolongation rows (for the tests) */
long amr_prolongation(const or_level* L, long* rowptr, long* col, double* val) {
  if (!L->tp_rowptr) return -1;
  const long nnz = L->tp_rowptr[L->nnodes];
  if (rowptr) memcpy(rowptr, L->tp_rowptr, sizeof(long) * (size_t)(L->nnodes + 1));
  if (col) memcpy(col, L->tp_col, sizeof(long) * (size_t)nnz);
  if (val) memcpy(val, L->tp_val, sizeof(double) * (size_t)nnz);
  return nnz;
}
