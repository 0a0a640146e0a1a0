// fc_amr.cu -- adaptive space-tree grids (quadtrees in 2D, octrees in 3D)
// for the finite cell Stokes multigrid (Sec. 3): the tree refined towards
// the obstacle boundaries with 2:1 balance, its hierarchy (Algorithm 1),
// hanging nodes removed as constraints, the operator assembled from the GPU
// element data, the patches of the RA smoother and the transfers; and the
// GPU kernels of the adaptive levels: node-block residual, patch apply with
// the restricted write, prolongation and restriction, dense coarsest
// operator.
//
// The grid: a lattice of the finest cells (fc_grid.n); a leaf of level r
// covers 2^(R - r) lattice cells per direction, R = depth - 1; the root grid
// is fc_grid.n / 2^R.  Every cell is refined uniformly to level U
// (fc_options.amr_uniform), a leaf whose level set changes sign among its
// 3^d sample points (the cut-cell test of the volume rule) is refined to
// level R, and the tree is then 2:1 balanced across faces, edges and
// corners.  A leaf corner in the middle of an edge of a coarser leaf is
// hanging with the edge's two end points as parents; in 3D a corner in the
// middle of a face of a coarser leaf hangs on the face's four corners.
// Under corner balance the parents are never hanging themselves; a hanging
// vertex takes the mean of its parents and carries no DoF.  The next coarser
// grid of the hierarchy replaces every leaf of the highest level with its
// parent (Algorithm 1), then balances.  DoFs: the free (non-hanging) lattice
// vertices in lattice order (x fastest, then y, then z), the velocity
// components and then p per node.
//
// Operator: element data of a leaf of level r from the element kernel on
// the uniform grid of level r (same quadrature rules as the uniform path);
// the pressure stabilisation in closed form per leaf; every hanging corner
// expanded into its parents (L = C^T L_raw C); strong Dirichlet data of the
// box faces eliminated symmetrically (identity rows, zero columns, values
// lifted into b).  Patch S_i (Sec. 3.1): the pressures of the nodes
// connected to free node i and the velocity DoFs of the nodes connected to
// any of them (two free nodes are connected when a leaf has corners whose
// expansions contain them), constrained DoFs left out; owned: p_i and the
// velocity of node i.  Prolongation: a fine free node takes the coarse
// finite element function at its position; restriction its transpose,
// constrained coarse DoFs zeroed.
#include <math.h>
#include <stdlib.h>

#include <algorithm>
#include <vector>

#include "fc_internal.cuh"

namespace fc {

namespace {

// ---------------------------------------------------------------- tree
double host_phi(const std::vector<Shape>& sh, int dim, const double* x) {
  double p = -1.0;
  for (size_t t = 0; t < sh.size(); ++t) {
    const Shape& s = sh[t];
    const double dx = x[0] - s.c[0], dy = x[1] - s.c[1];
    double q;
    if (s.type == 0) {
      double d2 = dx * dx + dy * dy;
      if (dim == 3) {
        const double dz = x[2] - s.c[2];
        d2 = d2 + dz * dz;
      }
      q = s.r[0] - sqrt(d2);
    } else {
      const double xp = s.rot[0] * dx + s.rot[1] * dy;
      const double yp = -s.rot[1] * dx + s.rot[0] * dy;
      const double u = xp / s.r[0], v = yp / s.r[1];
      const double uu = u * u, vv = v * v;
      q = 1.0 - (uu + vv);
    }
    if (t == 0 || q > p) p = q;
  }
  return p;
}

int tsize(const AmrTree& T, int level) { return 1 << (T.R - level); }
size_t tcell(const AmrTree& T, int X, int Y, int Z) { return ((size_t)Z * T.NY + Y) * T.NX + X; }

void refine_leaf(AmrTree& T, int X, int Y, int Z) {
  const int l = T.lev[tcell(T, X, Y, Z)], s = tsize(T, l);
  const int X0 = X / s * s, Y0 = Y / s * s, Z0 = T.dim == 3 ? Z / s * s : 0, sz = T.dim == 3 ? s : 1;
  for (int z = Z0; z < Z0 + sz; ++z)
    for (int y = Y0; y < Y0 + s; ++y)
      for (int x = X0; x < X0 + s; ++x) T.lev[tcell(T, x, y, z)] = (unsigned char)(l + 1);
}

// refine leaves next to (face, edge or corner) leaves more than one level
// finer, until there are none
void balance(AmrTree& T) {
  const int rz = T.dim == 3 ? 1 : 0;
  bool changed = true;
  while (changed) {
    changed = false;
    for (int Z = 0; Z < T.NZ; ++Z)
      for (int Y = 0; Y < T.NY; ++Y)
        for (int X = 0; X < T.NX; ++X) {
          const int l = T.lev[tcell(T, X, Y, Z)];
          for (int dz = -rz; dz <= rz; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
              for (int dx = -1; dx <= 1; ++dx) {
                const int x = X + dx, y = Y + dy, z = Z + dz;
                if (x < 0 || y < 0 || z < 0 || x >= T.NX || y >= T.NY || z >= T.NZ) continue;
                if (T.lev[tcell(T, x, y, z)] < l - 1) {
                  refine_leaf(T, x, y, z);
                  changed = true;
                }
              }
        }
  }
}

long long vid(const AmrTree& T, int X, int Y, int Z) {
  return ((long long)Z * (T.NY + 1) + Y) * (T.NX + 1) + X;
}

void vxyz(const AmrTree& T, long long v, int* X, int* Y, int* Z) {
  *X = (int)(v % (T.NX + 1));
  *Y = (int)((v / (T.NX + 1)) % (T.NY + 1));
  *Z = (int)(v / ((long long)(T.NX + 1) * (T.NY + 1)));
}

// corner a of the leaf at (X, Y, Z) of size s: bit k of a = +s along axis k
long long corner_vid(const AmrTree& T, int X, int Y, int Z, int s, int a) {
  return vid(T, X + (a & 1) * s, Y + ((a >> 1) & 1) * s, T.dim == 3 ? Z + ((a >> 2) & 1) * s : 0);
}

// leaves in lattice order: (X, Y, Z, level)
std::vector<int> leaves(const AmrTree& T) {
  std::vector<int> out;
  for (int Z = 0; Z < T.NZ; ++Z)
    for (int Y = 0; Y < T.NY; ++Y)
      for (int X = 0; X < T.NX; ++X) {
        const int l = T.lev[tcell(T, X, Y, Z)], s = tsize(T, l);
        if (X % s || Y % s || (T.dim == 3 && Z % s)) continue;
        out.push_back(X);
        out.push_back(Y);
        out.push_back(Z);
        out.push_back(l);
      }
  return out;
}

// free nodes, hanging vertices and their parents; false if a parent is
// itself hanging (a tree that is not corner-balanced)
bool build_nodes(const AmrTree& T, const std::vector<int>& lf, AmrHost& H) {
  const int dim = T.dim, nc = 1 << dim;
  const long long nv = (long long)(T.NX + 1) * (T.NY + 1) * (dim == 3 ? T.NZ + 1 : 1);
  std::vector<unsigned char> corner((size_t)nv, 0);
  H.hp.assign((size_t)nv * 4, -1);
  H.hn.assign((size_t)nv, 0);
  const size_t nl = lf.size() / 4;
  for (size_t q = 0; q < nl; ++q) {
    const int s = tsize(T, lf[4 * q + 3]);
    for (int a = 0; a < nc; ++a) corner[corner_vid(T, lf[4 * q], lf[4 * q + 1], lf[4 * q + 2], s, a)] = 1;
  }
  for (size_t q = 0; q < nl; ++q) {
    const int P[3] = {lf[4 * q], lf[4 * q + 1], lf[4 * q + 2]}, s = tsize(T, lf[4 * q + 3]);
    if (s < 2) continue;
    const int h = s / 2;
    // edges along axis k: the other axes at 0 or s
    for (int k = 0; k < dim; ++k)
      for (int e = 0; e < (1 << (dim - 1)); ++e) {
        int a[3] = {P[0], P[1], P[2]}, bit = 0;
        for (int m = 0; m < dim; ++m)
          if (m != k) a[m] += ((e >> bit++) & 1) * s;
        int b[3] = {a[0], a[1], a[2]}, mid[3] = {a[0], a[1], a[2]};
        b[k] += s;
        mid[k] += h;
        const long long m = vid(T, mid[0], mid[1], mid[2]);
        if (!corner[m]) continue;
        H.hn[m] = 2;
        H.hp[4 * m] = vid(T, a[0], a[1], a[2]);
        H.hp[4 * m + 1] = vid(T, b[0], b[1], b[2]);
      }
    if (dim == 3)
      // faces normal to axis k at 0 or s; u, w the in-face axes
      for (int k = 0; k < 3; ++k)
        for (int side = 0; side < 2; ++side) {
          const int u = k == 0 ? 1 : 0, w = k == 2 ? 1 : 2;
          int c0[3] = {P[0], P[1], P[2]};
          c0[k] += side * s;
          int mid[3] = {c0[0], c0[1], c0[2]};
          mid[u] += h;
          mid[w] += h;
          const long long m = vid(T, mid[0], mid[1], mid[2]);
          if (!corner[m]) continue;
          H.hn[m] = 4;
          for (int t = 0; t < 4; ++t) {
            int c[3] = {c0[0], c0[1], c0[2]};
            c[u] += (t & 1) * s;
            c[w] += (t >> 1) * s;
            H.hp[4 * m + t] = vid(T, c[0], c[1], c[2]);
          }
        }
  }
  H.fid.assign((size_t)nv, -1);
  H.nfree = 0;
  for (long long v = 0; v < nv; ++v)
    if (corner[v] && H.hn[v] == 0) H.fid[v] = H.nfree++;
  H.fvert.resize((size_t)H.nfree);
  for (long long v = 0; v < nv; ++v)
    if (H.fid[v] >= 0) H.fvert[H.fid[v]] = v;
  for (long long v = 0; v < nv; ++v)
    for (int t = 0; t < H.hn[v]; ++t)
      if (H.fid[H.hp[4 * v + t]] < 0) return false;
  return true;
}

// a lattice vertex as free nodes with weights: 1, 2 or 4 terms
int expand(const AmrHost& H, long long v, long long* node, double* w) {
  if (H.fid[v] >= 0) {
    node[0] = H.fid[v];
    w[0] = 1.0;
    return 1;
  }
  const int k = H.hn[v];
  for (int t = 0; t < k; ++t) {
    node[t] = H.fid[H.hp[4 * v + t]];
    w[t] = 1.0 / k;
  }
  return k;
}

}  // namespace

AmrTree amr_tree_fine(const std::vector<Shape>& sh, int dim, const double* lo, const double* hi, const int* nroot,
                      int U, int R) {
  AmrTree T;
  T.dim = dim;
  T.R = R;
  for (int k = 0; k < 3; ++k) T.nroot[k] = k < dim ? nroot[k] : 1;
  T.NX = T.nroot[0] << R;
  T.NY = T.nroot[1] << R;
  T.NZ = dim == 3 ? T.nroot[2] << R : 1;
  T.lev.assign((size_t)T.NX * T.NY * T.NZ, (unsigned char)U);
  const double h[3] = {(hi[0] - lo[0]) / T.NX, (hi[1] - lo[1]) / T.NY, dim == 3 ? (hi[2] - lo[2]) / T.NZ : 0.0};
  const int m3 = dim == 3 ? 3 : 1, nsmp = dim == 3 ? 27 : 9;
  for (int l = U; l < R; ++l) {
    const int s = tsize(T, l), sz = dim == 3 ? s : 1;
    for (int Z = 0; Z < T.NZ; Z += sz)
      for (int Y = 0; Y < T.NY; Y += s)
        for (int X = 0; X < T.NX; X += s) {
          if (T.lev[tcell(T, X, Y, Z)] != l) continue;
          const double x0[3] = {lo[0] + X * h[0], lo[1] + Y * h[1], dim == 3 ? lo[2] + Z * h[2] : 0.0};
          int npos = 0;
          for (int k = 0; k < m3; ++k)
            for (int j = 0; j < 3; ++j)
              for (int i = 0; i < 3; ++i) {
                const double x[3] = {x0[0] + s * h[0] * (0.5 * i), x0[1] + s * h[1] * (0.5 * j),
                                     dim == 3 ? x0[2] + s * h[2] * (0.5 * k) : 0.0};
                if (host_phi(sh, dim, x) > 0.0) npos++;
              }
          if (npos != 0 && npos != nsmp) refine_leaf(T, X, Y, Z);
        }
  }
  balance(T);
  return T;
}

AmrTree amr_tree_coarsen(const AmrTree& F) {
  AmrTree T = F;
  int rmax = 0;
  for (unsigned char l : T.lev) rmax = std::max(rmax, (int)l);
  if (rmax > 0)
    for (auto& l : T.lev)
      if (l == rmax) l = (unsigned char)(rmax - 1);
  balance(T);
  return T;
}

// Host half of an adaptive level: nodes, leaves, adjacency, and (after the
// caller supplies the element data) operator, patches and transfers.
bool amr_structure(const AmrTree& T, AmrHost& H, std::vector<std::vector<long long>>& adj) {
  H.dim = T.dim;
  H.leaf = leaves(T);
  if (!build_nodes(T, H.leaf, H)) return false;
  const int nc = 1 << T.dim;
  adj.assign((size_t)H.nfree, {});
  const size_t nl = H.leaf.size() / 4;
  for (size_t q = 0; q < nl; ++q) {
    const int s = tsize(T, H.leaf[4 * q + 3]);
    long long nodes[32];
    int nn = 0;
    for (int c = 0; c < nc; ++c) {
      long long n4[4];
      double w4[4];
      const int k = expand(H, corner_vid(T, H.leaf[4 * q], H.leaf[4 * q + 1], H.leaf[4 * q + 2], s, c), n4, w4);
      for (int t = 0; t < k; ++t) nodes[nn++] = n4[t];
    }
    for (int a = 0; a < nn; ++a)
      for (int b = 0; b < nn; ++b) {
        auto& v = adj[nodes[a]];
        if (std::find(v.begin(), v.end(), nodes[b]) == v.end()) v.push_back(nodes[b]);
      }
  }
  for (auto& v : adj) std::sort(v.begin(), v.end());
  return true;
}

// Assembly from the element data of the leaves (per leaf, leaf order: eA
// NC x NC, eB d x NC x NC, eF d x NC with NC = 2^d corners), Dirichlet data,
// patches, node blocks.  g: the lattice geometry (box, parameters, preset).
// Returns the largest patch.
int amr_assemble(const AmrTree& T, const LevelGeom& g, const std::vector<double>& eA, const std::vector<double>& eB,
                 const std::vector<double>& eF, const std::vector<std::vector<long long>>& adj, AmrHost& H) {
  const int dim = T.dim, NC = 1 << dim, nd = dim + 1;
  const long long nf = H.nfree, ndof = nf * nd;
  H.rowptr.assign((size_t)ndof + 1, 0);
  for (long long f = 0; f < nf; ++f)
    for (int c = 0; c < nd; ++c) H.rowptr[f * nd + c + 1] = H.rowptr[f * nd + c] + (int)adj[f].size() * nd;
  H.col.resize((size_t)H.rowptr[ndof]);
  H.val.assign((size_t)H.rowptr[ndof], 0.0);
  H.rhs.assign((size_t)ndof, 0.0);
  H.fixed.assign((size_t)ndof, 0);
  H.wfix.assign((size_t)ndof, 0.0);
  for (long long f = 0; f < nf; ++f)
    for (int c = 0; c < nd; ++c) {
      int p = H.rowptr[f * nd + c];
      for (long long j : adj[f])
        for (int e = 0; e < nd; ++e) H.col[p++] = (int)(j * nd + e);
    }
  // every row of node f has the columns of adj[f] x (the d + 1 components),
  // so entry (f, c; g, e) sits at rowptr[f nd + c] + nd pos(g in adj[f]) + e
  auto slot_of = [&](long long f, long long g) {
    const auto& v = adj[f];
    return (int)(std::lower_bound(v.begin(), v.end(), g) - v.begin()) * nd;
  };
  const size_t nl = H.leaf.size() / 4;
  for (size_t q = 0; q < nl; ++q) {
    const int X = H.leaf[4 * q], Y = H.leaf[4 * q + 1], Z = H.leaf[4 * q + 2], l = H.leaf[4 * q + 3];
    const int s = tsize(T, l);
    const double* A = &eA[q * NC * NC];
    const double* B = &eB[q * dim * NC * NC];
    const double* F = &eF[q * dim * NC];
    // pressure stabilisation in closed form on the leaf (eq. stabilization_l2)
    double vol = 1.0;
    for (int k = 0; k < dim; ++k) vol = vol * (g.h[k] * s);
    double C[8][8];
    for (int a = 0; a < NC; ++a)
      for (int b = 0; b < NC; ++b) {
        double m = 1.0;
        for (int k = 0; k < dim; ++k) m = m * (((a >> k) & 1) == ((b >> k) & 1) ? 1.0 / 3.0 : 1.0 / 6.0);
        C[a][b] = -(1.0 / g.eta) * (vol * m - vol / (double)(NC * NC));
      }
    long long en[8][4];
    double ew[8][4];
    int ek[8];
    for (int a = 0; a < NC; ++a) ek[a] = expand(H, corner_vid(T, X, Y, Z, s, a), en[a], ew[a]);
    for (int a = 0; a < NC; ++a)
      for (int ta = 0; ta < ek[a]; ++ta) {
        const long long fa = en[a][ta];
        const double wa = ew[a][ta];
        for (int c = 0; c < dim; ++c) H.rhs[fa * nd + c] = H.rhs[fa * nd + c] + wa * F[c * NC + a];
        double* rows[4];
        for (int c = 0; c < nd; ++c) rows[c] = &H.val[H.rowptr[fa * nd + c]];
        for (int b = 0; b < NC; ++b)
          for (int tb = 0; tb < ek[b]; ++tb) {
            const long long fb = en[b][tb];
            const double w = wa * ew[b][tb];
            const int sb = slot_of(fa, fb);
            for (int c = 0; c < dim; ++c) {
              rows[c][sb + c] = rows[c][sb + c] + w * A[a * NC + b];
              rows[c][sb + dim] = rows[c][sb + dim] + w * B[(c * NC + a) * NC + b];
              rows[dim][sb + c] = rows[dim][sb + c] + w * B[(c * NC + b) * NC + a];
            }
            rows[dim][sb + dim] = rows[dim][sb + dim] + w * C[a][b];
          }
      }
  }
  // strong Dirichlet data (the presets of the uniform grids)
  for (long long f = 0; f < nf; ++f) {
    int X, Y, Z;
    vxyz(T, H.fvert[f], &X, &Y, &Z);
    bool wall = Y == 0 || Y == T.NY;
    if (dim == 3) wall = wall || Z == 0 || Z == T.NZ;
    bool fixed = false;
    double w0 = 0.0;
    if (g.preset == 0) {
      fixed = wall || X == 0;
      if (!wall && X == 0) {
        const double y = g.lo[1] + (double)Y * g.h[1];
        const double sy = (y - g.lo[1]) / (g.hi[1] - g.lo[1]);
        w0 = 4.0 * g.ubar * sy * (1.0 - sy);
        if (dim == 3) {
          const double z = g.lo[2] + (double)Z * g.h[2];
          const double sz = (z - g.lo[2]) / (g.hi[2] - g.lo[2]);
          w0 = w0 * 4.0 * sz * (1.0 - sz);
        }
      }
    } else if (g.preset == 1) {
      fixed = wall;
    }
    if (fixed)
      for (int c = 0; c < dim; ++c) {
        H.fixed[f * nd + c] = 1;
        H.wfix[f * nd + c] = c == 0 ? w0 : 0.0;
      }
  }
  for (long long r = 0; r < ndof; ++r) {
    if (H.fixed[r]) {
      for (int p = H.rowptr[r]; p < H.rowptr[r + 1]; ++p) H.val[p] = H.col[p] == r ? 1.0 : 0.0;
      H.rhs[r] = H.wfix[r];
      continue;
    }
    for (int p = H.rowptr[r]; p < H.rowptr[r + 1]; ++p)
      if (H.fixed[H.col[p]]) {
        H.rhs[r] = H.rhs[r] - H.val[p] * H.wfix[H.col[p]];
        H.val[p] = 0.0;
      }
  }
  // patches
  H.pstart.assign((size_t)nf + 1, 0);
  H.pdof.clear();
  H.pown.assign((size_t)nf * nd, -1);
  int maxn = 0;
  std::vector<long long> vel;
  std::vector<long long> seen((size_t)nf, -1);  // last patch that listed the node
  for (long long i = 0; i < nf; ++i) {
    vel.clear();
    for (long long j : adj[i])
      for (long long k : adj[j])
        if (seen[k] != i) {
          seen[k] = i;
          vel.push_back(k);
        }
    std::sort(vel.begin(), vel.end());
    int n = 0;
    for (long long k : vel)
      for (int c = 0; c < dim; ++c) {
        const long long d = k * nd + c;
        if (H.fixed[d]) continue;
        if (k == i) H.pown[i * nd + c] = n;
        H.pdof.push_back((int)d);
        n++;
      }
    for (long long j : adj[i]) {
      if (j == i) H.pown[i * nd + dim] = n;
      H.pdof.push_back((int)(j * nd + dim));
      n++;
    }
    H.pstart[i + 1] = H.pstart[i] + n;
    maxn = std::max(maxn, n);
  }
  // node blocks of the operator: the velocity rows couple the same component
  // only, with one scalar A for every component (identity rows on
  // constrained nodes, whose components are constrained together)
  H.nbp.assign((size_t)nf + 1, 0);
  H.nbc.clear();
  H.nbv.clear();
  for (long long f = 0; f < nf; ++f) {
    for (size_t t = 0; t < adj[f].size(); ++t) {
      const int sb = (int)t * nd;
      auto at = [&](int c, int e) { return H.val[H.rowptr[f * nd + c] + sb + e]; };
      H.nbc.push_back((int)adj[f][t]);
      H.nbv.push_back(at(0, 0));
      for (int c = 0; c < dim; ++c) H.nbv.push_back(at(c, dim));
      for (int c = 0; c < dim; ++c) H.nbv.push_back(at(dim, c));
      H.nbv.push_back(at(dim, dim));
    }
    H.nbp[f + 1] = (int)H.nbc.size();
  }
  return maxn;
}

// prolongation from the coarser tree Tc (nodes Hc) to the fine level H, and
// its transpose
void amr_transfers(const AmrTree& T, AmrHost& H, const AmrTree& Tc, const AmrHost& Hc) {
  const int dim = T.dim, NC = 1 << dim;
  const long long nf = H.nfree;
  H.prp.assign((size_t)nf + 1, 0);
  H.pcl.clear();
  H.pvl.clear();
  for (long long f = 0; f < nf; ++f) {
    int X, Y, Z;
    vxyz(T, H.fvert[f], &X, &Y, &Z);
    const int cx = std::min(X, Tc.NX - 1), cy = std::min(Y, Tc.NY - 1), cz = dim == 3 ? std::min(Z, Tc.NZ - 1) : 0;
    const int s = tsize(Tc, Tc.lev[tcell(Tc, cx, cy, cz)]);
    const int X0 = cx / s * s, Y0 = cy / s * s, Z0 = dim == 3 ? cz / s * s : 0;
    const double t[3] = {(double)(X - X0) / s, (double)(Y - Y0) / s, dim == 3 ? (double)(Z - Z0) / s : 0.0};
    long long node[64];
    double wt[64];
    int nn = 0;
    for (int a = 0; a < NC; ++a) {
      double wa = 1.0;
      for (int k = 0; k < dim; ++k) wa = wa * (((a >> k) & 1) ? t[k] : 1.0 - t[k]);
      if (wa == 0.0) continue;
      long long n4[4];
      double w4[4];
      const int k = expand(Hc, corner_vid(Tc, X0, Y0, Z0, s, a), n4, w4);
      for (int u = 0; u < k; ++u) {
        int z = 0;
        while (z < nn && node[z] != n4[u]) ++z;
        if (z == nn) { node[nn] = n4[u]; wt[nn] = 0.0; nn++; }
        wt[z] = wt[z] + wa * w4[u];
      }
    }
    std::vector<int> ord(nn);
    for (int z = 0; z < nn; ++z) ord[z] = z;
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return node[a] < node[b]; });
    for (int z : ord) {
      H.pcl.push_back((int)node[z]);
      H.pvl.push_back(wt[z]);
    }
    H.prp[f + 1] = (int)H.pcl.size();
  }
  // transpose: per coarse node, the fine nodes (ascending) and weights
  const long long nc = Hc.nfree;
  H.rrp.assign((size_t)nc + 1, 0);
  for (int c : H.pcl) H.rrp[c + 1]++;
  for (long long c = 0; c < nc; ++c) H.rrp[c + 1] += H.rrp[c];
  H.rcl.assign(H.pcl.size(), 0);
  H.rvl.assign(H.pcl.size(), 0.0);
  std::vector<int> pos(H.rrp.begin(), H.rrp.end() - 1);
  for (long long f = 0; f < nf; ++f)
    for (int p = H.prp[f]; p < H.prp[f + 1]; ++p) {
      const int c = H.pcl[p];
      H.rcl[pos[c]] = (int)f;
      H.rvl[pos[c]] = H.pvl[p];
      pos[c]++;
    }
}

std::vector<long long> amr_leaf_cells(const AmrTree& T, const AmrHost& H, int level, std::vector<long long>* slots) {
  std::vector<long long> cells;
  const size_t nl = H.leaf.size() / 4;
  const int s = tsize(T, level);
  const long long nxr = (long long)T.nroot[0] << level, nyr = (long long)T.nroot[1] << level;
  for (size_t q = 0; q < nl; ++q) {
    if (H.leaf[4 * q + 3] != level) continue;
    cells.push_back(H.leaf[4 * q] / s + nxr * (H.leaf[4 * q + 1] / s + nyr * (H.leaf[4 * q + 2] / s)));
    if (slots) slots->push_back((long long)q);
  }
  return cells;
}

// ------------------------------------------------------------- kernels
namespace {

// r = b - L x (L x when b is null) on node blocks: LPN lanes per free node,
// each over every LPN-th neighbour (index, then the record A, B_0 .. B_{d-1},
// T_0 .. T_{d-1}, C as 16-byte loads, then the neighbour's DoFs), a shuffle
// sum of the d + 1 row sums
template <int DIM, int LPN>
__global__ void __launch_bounds__(256)
    amr_residual_kernel(long long nf, const int* __restrict__ nbp, const int* __restrict__ nbc,
                        const double* __restrict__ nbv, const double* __restrict__ x,
                        const double* __restrict__ b, double* __restrict__ r) {
  constexpr int ND = DIM + 1, NBV = 2 * DIM + 2;
  const int lane = threadIdx.x % LPN;
  const long long gf = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / LPN;
  const long long f = gf < nf ? gf : nf - 1;
  double acc[ND];
#pragma unroll
  for (int c = 0; c < ND; ++c) acc[c] = 0.0;
  for (int p = nbp[f] + lane; p < nbp[f + 1]; p += LPN) {
    const long long g = nbc[p];
    const double2* v2 = reinterpret_cast<const double2*>(nbv + NBV * (long long)p);
    double m[NBV];
#pragma unroll
    for (int t = 0; t < NBV / 2; ++t) {
      const double2 q = v2[t];
      m[2 * t] = q.x;
      m[2 * t + 1] = q.y;
    }
    double xs[ND];
#pragma unroll
    for (int c = 0; c < ND; ++c) xs[c] = x[ND * g + c];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      acc[c] = fma(m[0], xs[c], acc[c]);
      acc[c] = fma(m[1 + c], xs[DIM], acc[c]);
      acc[DIM] = fma(m[1 + DIM + c], xs[c], acc[DIM]);
    }
    acc[DIM] = fma(m[NBV - 1], xs[DIM], acc[DIM]);
  }
  // the row sums (2D: a zero fourth) reduce-scattered over the LPN lanes
  const double a4[4] = {acc[0], acc[1], acc[2], ND == 4 ? acc[ND - 1] : 0.0};
  int c = 0;
  const double s = reduce_scatter4<LPN>(a4, lane, &c);
  if (gf >= nf || lane % (LPN / 4) != 0 || c >= ND) return;
  const long long row = f * ND + c;
  r[row] = b ? b[row] - s : s;
}

// patch apply: TPP lanes per patch over the patch's slot records (the DoF
// index in the bits of a double, then the d + 1 owned-row coefficients;
// 2D: two 16-byte loads per 32-byte record; 3D: five 8-byte loads per
// 40-byte record); y_k = sum_j rows[k][j] r[dof_j]; restricted write
// x[owned] += omega y (constrained velocity DoFs: identity rows, x += r)
template <int DIM, int TPP>
__global__ void __launch_bounds__(256)
    amr_apply_kernel(long long np, const long long* __restrict__ pstart, const int* __restrict__ pown,
                     const double* __restrict__ rows, const unsigned char* __restrict__ fixed,
                     const double* __restrict__ r, double omega, double* __restrict__ x) {
  constexpr int ND = DIM + 1, REC = ND + 1;
  const int lane = threadIdx.x % TPP;
  const long long gi = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / TPP;
  const bool valid = gi < np;
  const long long i = valid ? gi : np - 1;
  const long long s0 = pstart[i];
  const int n = (int)(pstart[i + 1] - s0);
  double y[ND];
#pragma unroll
  for (int k = 0; k < ND; ++k) y[k] = 0.0;
  if constexpr (DIM == 2) {
    const double2* rec = reinterpret_cast<const double2*>(rows + REC * s0);
#pragma unroll 4
    for (int j = lane; j < n; j += TPP) {
      const double2 a = __ldcs(rec + 2 * j), c = __ldcs(rec + 2 * j + 1);
      const double rv = r[__double_as_longlong(a.x)];
      y[0] = fma(a.y, rv, y[0]);
      y[1] = fma(c.x, rv, y[1]);
      y[2] = fma(c.y, rv, y[2]);
    }
  } else {
    const double* rec = rows + REC * s0;
#pragma unroll 4
    for (int j = lane; j < n; j += TPP) {
      const double* q = rec + REC * j;
      const double rv = r[__double_as_longlong(__ldcs(q))];
#pragma unroll
      for (int k = 0; k < ND; ++k) y[k] = fma(__ldcs(q + 1 + k), rv, y[k]);
    }
  }
  // the four row sums (2D: the fourth is zero) reduce-scattered over the
  // TPP lanes: the lanes with lane % (TPP / 4) == 0 write row `row`
  constexpr int Q = TPP / 4;
  const double y4[4] = {y[0], y[1], y[2], ND == 4 ? y[ND - 1] : 0.0};
  int row = 0;
  const double yk = reduce_scatter4<TPP>(y4, lane, &row);
  if (!valid || lane % Q != 0 || row >= ND) return;
  const long long d = i * ND + row;
  if (fixed[d]) x[d] += r[d];
  else if (pown[i * ND + row] >= 0) x[d] += omega * yk;
}

// x_f += P e_c per component, constrained fine DoFs left alone
template <int ND>
__global__ void amr_prolong_kernel(long long nf, const int* __restrict__ prp, const int* __restrict__ pcl,
                                   const double* __restrict__ pvl, const unsigned char* __restrict__ fixed,
                                   const double* __restrict__ ec, double* __restrict__ xf) {
  const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  double s[ND];
  for (int c = 0; c < ND; ++c) s[c] = 0.0;
  for (int p = prp[f]; p < prp[f + 1]; ++p)
    for (int c = 0; c < ND; ++c) s[c] = fma(pvl[p], ec[(long long)pcl[p] * ND + c], s[c]);
  for (int c = 0; c < ND; ++c)
    if (!fixed[f * ND + c]) xf[f * ND + c] += s[c];
}

// b_c = P^T r_f (gather over the fine nodes of each coarse node), then
// constrained coarse DoFs zeroed
template <int ND>
__global__ void amr_restrict_kernel(long long nc, const int* __restrict__ rrp, const int* __restrict__ rcl,
                                    const double* __restrict__ rvl, const unsigned char* __restrict__ cfixed,
                                    const double* __restrict__ rf, double* __restrict__ bc) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  double s[ND];
  for (int k = 0; k < ND; ++k) s[k] = 0.0;
  for (int p = rrp[c]; p < rrp[c + 1]; ++p)
    for (int k = 0; k < ND; ++k) s[k] = fma(rvl[p], rf[(long long)rcl[p] * ND + k], s[k]);
  for (int k = 0; k < ND; ++k) bc[c * ND + k] = cfixed[c * ND + k] ? 0.0 : s[k];
}

// dense row-major copy of a CSR matrix
__global__ void amr_dense_kernel(long long n, const int* __restrict__ rp, const int* __restrict__ col,
                                 const double* __restrict__ val, double* __restrict__ M) {
  const long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  for (long long c = 0; c < n; ++c) M[row * n + c] = 0.0;
  for (int p = rp[row]; p < rp[row + 1]; ++p) M[row * n + col[p]] = val[p];
}

unsigned nblocks(long long threads) { return (unsigned)((threads + 255) / 256); }

}  // namespace

static int amr_apply_lanes(long long npatch);

template <int DIM, int LPN>
static void residual_as(const AmrLevel& A, const double* x, const double* b, double* r, cudaStream_t s) {
  amr_residual_kernel<DIM, LPN><<<nblocks(A.nfree * LPN), 256, 0, s>>>(A.nfree, A.nbp, A.nbc, A.nbv, x, b, r);
}

cudaError_t launch_amr_residual(const AmrLevel& A, const double* x, const double* b, double* r, cudaStream_t s) {
  if (A.nfree == 0) return cudaSuccess;
  const int t = amr_apply_lanes(A.nfree);  // the apply's rule: two waves of resident threads
  if (A.dim == 2) {
    if (t == 4) residual_as<2, 4>(A, x, b, r, s);
    else if (t == 8) residual_as<2, 8>(A, x, b, r, s);
    else residual_as<2, 16>(A, x, b, r, s);
  } else {
    if (t == 4) residual_as<3, 4>(A, x, b, r, s);
    else if (t == 8) residual_as<3, 8>(A, x, b, r, s);
    else residual_as<3, 16>(A, x, b, r, s);
  }
  note_launches(1);
  return cudaGetLastError();
}

// lanes per patch (and per node in the residual): the fewest of 4, 8, 16
// that give the launch two waves of resident threads (2048 per SM), so that
// small levels still fill the GPU;
// FC_AMR_LANES = 4, 8 or 16 in the environment fixes it (tests, tuning)
static int amr_apply_lanes(long long npatch) {
  if (const char* e = getenv("FC_AMR_LANES")) {
    const int t = atoi(e);
    if (t == 4 || t == 8 || t == 16) return t;
  }
  int per_sm = 0, nsm = 0;  // the current device's SM count (cached per device, thread-safe)
  if (persistent_ctas((const void*)amr_apply_kernel<2, 4>, 256, 0, &per_sm, &nsm) != cudaSuccess || nsm <= 0)
    nsm = 1;
  const long long want = 2LL * nsm * 2048;
  for (int t = 4; t < 16; t *= 2)
    if (npatch * t >= want) return t;
  return 16;
}

template <int DIM, int TPP>
static void apply_as(const AmrLevel& A, const double* r, double omega, double* x, cudaStream_t s) {
  amr_apply_kernel<DIM, TPP><<<nblocks(A.nfree * TPP), 256, 0, s>>>(A.nfree, A.pstart, A.pown, A.rows, A.fixed, r,
                                                                     omega, x);
}

cudaError_t launch_amr_apply(const AmrLevel& A, const double* r, double omega, double* x, cudaStream_t s) {
  if (A.nfree == 0) return cudaSuccess;
  const int t = amr_apply_lanes(A.nfree);
  if (A.dim == 2) {
    if (t == 4) apply_as<2, 4>(A, r, omega, x, s);
    else if (t == 8) apply_as<2, 8>(A, r, omega, x, s);
    else apply_as<2, 16>(A, r, omega, x, s);
  } else {
    if (t == 4) apply_as<3, 4>(A, r, omega, x, s);
    else if (t == 8) apply_as<3, 8>(A, r, omega, x, s);
    else apply_as<3, 16>(A, r, omega, x, s);
  }
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_amr_prolong_add(const AmrLevel& F, const double* ec, double* xf, cudaStream_t s) {
  if (F.nfree == 0) return cudaSuccess;
  if (F.dim == 2)
    amr_prolong_kernel<3><<<nblocks(F.nfree), 256, 0, s>>>(F.nfree, F.prp, F.pcl, F.pvl, F.fixed, ec, xf);
  else
    amr_prolong_kernel<4><<<nblocks(F.nfree), 256, 0, s>>>(F.nfree, F.prp, F.pcl, F.pvl, F.fixed, ec, xf);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_amr_restrict(const AmrLevel& F, const AmrLevel& C, const double* rf, double* bc, cudaStream_t s) {
  if (C.nfree == 0) return cudaSuccess;
  if (F.dim == 2)
    amr_restrict_kernel<3><<<nblocks(C.nfree), 256, 0, s>>>(C.nfree, F.rrp, F.rcl, F.rvl, C.fixed, rf, bc);
  else
    amr_restrict_kernel<4><<<nblocks(C.nfree), 256, 0, s>>>(C.nfree, F.rrp, F.rcl, F.rvl, C.fixed, rf, bc);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_amr_dense(const AmrLevel& A, double* M, cudaStream_t s) {
  const long long n = A.nfree * (A.dim + 1);
  amr_dense_kernel<<<nblocks(n), 256, 0, s>>>(n, A.rowptr, A.col, A.val, M);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace fc
