// fc_amr.cu -- adaptive quadtree grids (2D) for the finite cell Stokes
// multigrid (Sec. 3): the space tree refined towards the obstacle
// boundaries with 2:1 balance, its hierarchy (Algorithm 1), hanging nodes
// removed as constraints, the operator assembled from the GPU element data,
// the patches of the RA smoother and the transfers; and the GPU kernels of
// the adaptive levels: CSR residual, patch apply with the restricted write,
// prolongation and restriction, dense coarsest operator.
//
// The grid: a lattice of the finest cells (fc_grid.n); a leaf of level r
// covers 2^(R - r) lattice cells per direction, R = depth - 1; the root grid
// is fc_grid.n / 2^R.  Every cell is refined uniformly to level U
// (fc_options.amr_uniform), a leaf whose level set changes sign among its
// 3 x 3 sample points (the cut-cell test of the volume rule) is refined to
// level R, and the tree is then 2:1 balanced across faces and corners.  A
// leaf corner in the middle of an edge of a coarser leaf is hanging: its
// value is the mean of that edge's end points (never hanging themselves
// under corner balance), and it carries no DoF.  The next coarser grid of
// the hierarchy replaces every leaf of the highest level with its parent
// (Algorithm 1), then balances.  DoFs: the free (non-hanging) lattice
// vertices in lattice order (y-major, x fastest), (u, v, p) per node.
//
// Operator: element data of a leaf of level r from the element kernel on
// the uniform grid of level r (same quadrature rules as the uniform path);
// the pressure stabilisation in closed form per leaf; every hanging corner
// expanded into its parents with weight 1/2 (L = C^T L_raw C); strong
// Dirichlet data of the box faces eliminated symmetrically (identity rows,
// zero columns, values lifted into b).  Patch S_i (Sec. 3.1): the pressures
// of the nodes connected to free node i and the velocity DoFs of the nodes
// connected to any of them (two free nodes are connected when a leaf has
// corners whose expansions contain them), constrained DoFs left out; owned:
// p_i and the velocity of node i.  Prolongation: a fine free node takes the
// coarse finite element function at its position; restriction its
// transpose, constrained coarse DoFs zeroed.
#include <math.h>

#include <algorithm>
#include <vector>

#include "fc_internal.cuh"

namespace fc {

namespace {

// ---------------------------------------------------------------- tree
double host_phi(const std::vector<Shape>& sh, double x, double y) {
  double p = -1.0;
  for (size_t t = 0; t < sh.size(); ++t) {
    const Shape& s = sh[t];
    const double dx = x - s.c[0], dy = y - s.c[1];
    double q;
    if (s.type == 0) {
      const double d2 = dx * dx + dy * dy;
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

void refine_leaf(AmrTree& T, int X, int Y) {
  const int l = T.lev[(size_t)Y * T.NX + X], s = tsize(T, l);
  const int X0 = X / s * s, Y0 = Y / s * s;
  for (int y = Y0; y < Y0 + s; ++y)
    for (int x = X0; x < X0 + s; ++x) T.lev[(size_t)y * T.NX + x] = (unsigned char)(l + 1);
}

void balance(AmrTree& T) {
  bool changed = true;
  while (changed) {
    changed = false;
    for (int Y = 0; Y < T.NY; ++Y)
      for (int X = 0; X < T.NX; ++X) {
        const int l = T.lev[(size_t)Y * T.NX + X];
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            const int x = X + dx, y = Y + dy;
            if (x < 0 || y < 0 || x >= T.NX || y >= T.NY) continue;
            if (T.lev[(size_t)y * T.NX + x] < l - 1) {
              refine_leaf(T, x, y);
              changed = true;
            }
          }
      }
  }
}

long long vid(const AmrTree& T, int X, int Y) { return (long long)Y * (T.NX + 1) + X; }

// free nodes, hanging vertices and their parents
struct Nodes {
  std::vector<long long> fid;   // per lattice vertex: free index or -1
  std::vector<long long> hp;    // per lattice vertex: two parents or -1
  std::vector<long long> fvert; // per free node: lattice vertex
  long long nfree = 0;
};

void build_nodes(const AmrTree& T, Nodes& N) {
  const long long nv = (long long)(T.NX + 1) * (T.NY + 1);
  std::vector<unsigned char> corner((size_t)nv, 0);
  N.hp.assign((size_t)nv * 2, -1);
  for (int Y = 0; Y < T.NY; ++Y)
    for (int X = 0; X < T.NX; ++X) {
      const int s = tsize(T, T.lev[(size_t)Y * T.NX + X]);
      if (X % s || Y % s) continue;
      corner[vid(T, X, Y)] = corner[vid(T, X + s, Y)] = 1;
      corner[vid(T, X, Y + s)] = corner[vid(T, X + s, Y + s)] = 1;
    }
  for (int Y = 0; Y < T.NY; ++Y)
    for (int X = 0; X < T.NX; ++X) {
      const int s = tsize(T, T.lev[(size_t)Y * T.NX + X]);
      if (X % s || Y % s || s < 2) continue;
      const int h = s / 2;
      // edges: bottom, top, left, right (midpoint, end points)
      const int e[4][6] = {{X + h, Y, X, Y, X + s, Y},
                           {X + h, Y + s, X, Y + s, X + s, Y + s},
                           {X, Y + h, X, Y, X, Y + s},
                           {X + s, Y + h, X + s, Y, X + s, Y + s}};
      for (int k = 0; k < 4; ++k) {
        const long long m = vid(T, e[k][0], e[k][1]);
        if (!corner[m]) continue;
        N.hp[2 * m] = vid(T, e[k][2], e[k][3]);
        N.hp[2 * m + 1] = vid(T, e[k][4], e[k][5]);
      }
    }
  N.fid.assign((size_t)nv, -1);
  N.nfree = 0;
  for (long long v = 0; v < nv; ++v)
    if (corner[v] && N.hp[2 * v] < 0) N.fid[v] = N.nfree++;
  N.fvert.resize((size_t)N.nfree);
  for (long long v = 0; v < nv; ++v)
    if (N.fid[v] >= 0) N.fvert[N.fid[v]] = v;
}

int expand(const Nodes& N, long long v, long long* node, double* w) {
  if (N.fid[v] >= 0) {
    node[0] = N.fid[v];
    w[0] = 1.0;
    return 1;
  }
  node[0] = N.fid[N.hp[2 * v]];
  node[1] = N.fid[N.hp[2 * v + 1]];
  w[0] = w[1] = 0.5;
  return 2;
}

// leaves in lattice order: (X, Y, level)
std::vector<int> leaves(const AmrTree& T) {
  std::vector<int> out;
  for (int Y = 0; Y < T.NY; ++Y)
    for (int X = 0; X < T.NX; ++X) {
      const int l = T.lev[(size_t)Y * T.NX + X], s = tsize(T, l);
      if (X % s || Y % s) continue;
      out.push_back(X);
      out.push_back(Y);
      out.push_back(l);
    }
  return out;
}

}  // namespace

AmrTree amr_tree_fine(const std::vector<Shape>& sh, const double* lo, const double* hi, const int* nroot, int U,
                      int R) {
  AmrTree T;
  T.R = R;
  T.nroot[0] = nroot[0];
  T.nroot[1] = nroot[1];
  T.NX = nroot[0] << R;
  T.NY = nroot[1] << R;
  T.lev.assign((size_t)T.NX * T.NY, (unsigned char)U);
  const double hx = (hi[0] - lo[0]) / T.NX, hy = (hi[1] - lo[1]) / T.NY;
  for (int l = U; l < R; ++l) {
    const int s = tsize(T, l);
    for (int Y = 0; Y < T.NY; Y += s)
      for (int X = 0; X < T.NX; X += s) {
        if (T.lev[(size_t)Y * T.NX + X] != l) continue;
        const double x0 = lo[0] + X * hx, y0 = lo[1] + Y * hy, bx = s * hx, by = s * hy;
        int npos = 0;
        for (int j = 0; j < 3; ++j)
          for (int i = 0; i < 3; ++i)
            if (host_phi(sh, x0 + bx * (0.5 * i), y0 + by * (0.5 * j)) > 0.0) npos++;
        if (npos != 0 && npos != 9) refine_leaf(T, X, Y);
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
  Nodes N;
  build_nodes(T, N);
  H.nfree = N.nfree;
  H.fvert = N.fvert;
  H.fid = N.fid;
  H.hp = N.hp;
  H.leaf = leaves(T);
  adj.assign((size_t)N.nfree, {});
  const size_t nl = H.leaf.size() / 3;
  for (size_t q = 0; q < nl; ++q) {
    const int X = H.leaf[3 * q], Y = H.leaf[3 * q + 1], s = tsize(T, H.leaf[3 * q + 2]);
    long long nodes[8];
    int nn = 0;
    for (int c = 0; c < 4; ++c) {
      long long n2[2];
      double w2[2];
      const int k = expand(N, vid(T, X + (c & 1) * s, Y + (c >> 1) * s), n2, w2);
      for (int t = 0; t < k; ++t) nodes[nn++] = n2[t];
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

// Assembly from the element data of the leaves (eA 4 x 4, eB 2 x 4 x 4,
// eF 2 x 4 per leaf, leaf order), Dirichlet data, patches.  g: the lattice
// geometry (box, parameters, preset).  Returns the largest patch.
int amr_assemble(const AmrTree& T, const LevelGeom& g, const std::vector<double>& eA, const std::vector<double>& eB,
                 const std::vector<double>& eF, const std::vector<std::vector<long long>>& adj, AmrHost& H) {
  Nodes N;
  N.fid = H.fid;
  N.hp = H.hp;
  N.fvert = H.fvert;
  N.nfree = H.nfree;
  const long long nf = H.nfree, nd = 3, ndof = nf * nd;
  H.rowptr.assign((size_t)ndof + 1, 0);
  for (long long f = 0; f < nf; ++f)
    for (int c = 0; c < 3; ++c) H.rowptr[f * nd + c + 1] = H.rowptr[f * nd + c] + (int)adj[f].size() * 3;
  H.col.resize((size_t)H.rowptr[ndof]);
  H.val.assign((size_t)H.rowptr[ndof], 0.0);
  H.rhs.assign((size_t)ndof, 0.0);
  H.fixed.assign((size_t)ndof, 0);
  H.wfix.assign((size_t)ndof, 0.0);
  for (long long f = 0; f < nf; ++f)
    for (int c = 0; c < 3; ++c) {
      int p = H.rowptr[f * nd + c];
      for (long long j : adj[f])
        for (int e = 0; e < 3; ++e) H.col[p++] = (int)(j * nd + e);
    }
  auto add = [&](long long row, long long colj, double v) {
    int lo = H.rowptr[row], hi = H.rowptr[row + 1] - 1;
    while (lo <= hi) {
      const int mid = (lo + hi) / 2;
      if (H.col[mid] == colj) { H.val[mid] = H.val[mid] + v; return; }
      if (H.col[mid] < colj) lo = mid + 1; else hi = mid - 1;
    }
  };
  const size_t nl = H.leaf.size() / 3;
  for (size_t q = 0; q < nl; ++q) {
    const int X = H.leaf[3 * q], Y = H.leaf[3 * q + 1], l = H.leaf[3 * q + 2], s = tsize(T, l);
    const double* A = &eA[q * 16];
    const double* B = &eB[q * 32];
    const double* F = &eF[q * 8];
    // pressure stabilisation in closed form on the leaf (eq. stabilization_l2)
    const double vol = (g.h[0] * s) * (g.h[1] * s);
    double C[4][4];
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        double m = 1.0;
        for (int k = 0; k < 2; ++k) m = m * (((a >> k) & 1) == ((b >> k) & 1) ? 1.0 / 3.0 : 1.0 / 6.0);
        C[a][b] = -(1.0 / g.eta) * (vol * m - vol * 0.0625);
      }
    long long en[4][2];
    double ew[4][2];
    int ek[4];
    for (int a = 0; a < 4; ++a) ek[a] = expand(N, vid(T, X + (a & 1) * s, Y + (a >> 1) * s), en[a], ew[a]);
    for (int a = 0; a < 4; ++a)
      for (int ta = 0; ta < ek[a]; ++ta) {
        const long long fa = en[a][ta];
        const double wa = ew[a][ta];
        for (int c = 0; c < 2; ++c) H.rhs[fa * nd + c] = H.rhs[fa * nd + c] + wa * F[c * 4 + a];
        for (int b = 0; b < 4; ++b)
          for (int tb = 0; tb < ek[b]; ++tb) {
            const long long fb = en[b][tb];
            const double w = wa * ew[b][tb];
            for (int c = 0; c < 2; ++c) {
              add(fa * nd + c, fb * nd + c, w * A[a * 4 + b]);
              add(fa * nd + c, fb * nd + 2, w * B[(c * 4 + a) * 4 + b]);
              add(fa * nd + 2, fb * nd + c, w * B[(c * 4 + b) * 4 + a]);
            }
            add(fa * nd + 2, fb * nd + 2, w * C[a][b]);
          }
      }
  }
  // strong Dirichlet data (the presets of the uniform grids)
  for (long long f = 0; f < nf; ++f) {
    const long long v = H.fvert[f];
    const int X = (int)(v % (T.NX + 1)), Y = (int)(v / (T.NX + 1));
    const bool wall = Y == 0 || Y == T.NY;
    bool fixed = false;
    double w0 = 0.0;
    if (g.preset == 0) {
      fixed = wall || X == 0;
      if (!wall && X == 0) {
        const double y = g.lo[1] + (double)Y * g.h[1];
        const double sy = (y - g.lo[1]) / (g.hi[1] - g.lo[1]);
        w0 = 4.0 * g.ubar * sy * (1.0 - sy);
      }
    } else if (g.preset == 1) {
      fixed = wall;
    }
    if (fixed)
      for (int c = 0; c < 2; ++c) {
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
  H.pown.assign((size_t)nf * 3, -1);
  int maxn = 0;
  std::vector<long long> vel;
  for (long long i = 0; i < nf; ++i) {
    vel.clear();
    for (long long j : adj[i])
      for (long long k : adj[j]) vel.push_back(k);
    std::sort(vel.begin(), vel.end());
    vel.erase(std::unique(vel.begin(), vel.end()), vel.end());
    int n = 0;
    for (long long k : vel)
      for (int c = 0; c < 2; ++c) {
        const long long d = k * nd + c;
        if (H.fixed[d]) continue;
        if (k == i) H.pown[i * 3 + c] = n;
        H.pdof.push_back((int)d);
        n++;
      }
    for (long long j : adj[i]) {
      if (j == i) H.pown[i * 3 + 2] = n;
      H.pdof.push_back((int)(j * nd + 2));
      n++;
    }
    H.pstart[i + 1] = H.pstart[i] + n;
    maxn = std::max(maxn, n);
  }
  // node blocks of the operator: the velocity rows couple the same component
  // only, with one scalar A for both (identity rows on constrained nodes)
  H.nbp.assign((size_t)nf + 1, 0);
  H.nbc.clear();
  H.nbv.clear();
  auto at = [&](long long row, long long colj) {
    int lo = H.rowptr[row], hi = H.rowptr[row + 1] - 1;
    while (lo <= hi) {
      const int mid = (lo + hi) / 2;
      if (H.col[mid] == colj) return H.val[mid];
      if (H.col[mid] < colj) lo = mid + 1; else hi = mid - 1;
    }
    return 0.0;
  };
  for (long long f = 0; f < nf; ++f) {
    for (long long g2 : adj[f]) {
      H.nbc.push_back((int)g2);
      H.nbv.push_back(at(f * nd + 0, g2 * nd + 0));
      H.nbv.push_back(at(f * nd + 0, g2 * nd + 2));
      H.nbv.push_back(at(f * nd + 1, g2 * nd + 2));
      H.nbv.push_back(at(f * nd + 2, g2 * nd + 0));
      H.nbv.push_back(at(f * nd + 2, g2 * nd + 1));
      H.nbv.push_back(at(f * nd + 2, g2 * nd + 2));
    }
    H.nbp[f + 1] = (int)H.nbc.size();
  }
  return maxn;
}

// prolongation from the coarser tree Tc (nodes Hc) to the fine level H, and
// its transpose
void amr_transfers(const AmrTree& T, AmrHost& H, const AmrTree& Tc, const AmrHost& Hc) {
  Nodes Nc;
  Nc.fid = Hc.fid;
  Nc.hp = Hc.hp;
  Nc.fvert = Hc.fvert;
  Nc.nfree = Hc.nfree;
  const long long nf = H.nfree;
  H.prp.assign((size_t)nf + 1, 0);
  H.pcl.clear();
  H.pvl.clear();
  for (long long f = 0; f < nf; ++f) {
    const long long v = H.fvert[f];
    const int X = (int)(v % (T.NX + 1)), Y = (int)(v / (T.NX + 1));
    const int cx = std::min(X, Tc.NX - 1), cy = std::min(Y, Tc.NY - 1);
    const int s = tsize(Tc, Tc.lev[(size_t)cy * Tc.NX + cx]);
    const int X0 = cx / s * s, Y0 = cy / s * s;
    const double tx = (double)(X - X0) / s, ty = (double)(Y - Y0) / s;
    long long node[16];
    double wt[16];
    int nn = 0;
    for (int a = 0; a < 4; ++a) {
      const double wa = ((a & 1) ? tx : 1.0 - tx) * ((a >> 1) ? ty : 1.0 - ty);
      if (wa == 0.0) continue;
      long long n2[2];
      double w2[2];
      const int k = expand(Nc, vid(Tc, X0 + (a & 1) * s, Y0 + (a >> 1) * s), n2, w2);
      for (int t = 0; t < k; ++t) {
        int z = 0;
        while (z < nn && node[z] != n2[t]) ++z;
        if (z == nn) { node[nn] = n2[t]; wt[nn] = 0.0; nn++; }
        wt[z] = wt[z] + wa * w2[t];
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
  const size_t nl = H.leaf.size() / 3;
  for (size_t q = 0; q < nl; ++q) {
    if (H.leaf[3 * q + 2] != level) continue;
    const int s = tsize(T, level);
    const long long nxr = (long long)T.nroot[0] << level;
    cells.push_back(H.leaf[3 * q] / s + nxr * (H.leaf[3 * q + 1] / s));
    if (slots) slots->push_back((long long)q);
  }
  return cells;
}

// ------------------------------------------------------------- kernels
namespace {

// r = b - L x (L x when b is null) on node blocks: 4 lanes per free node,
// each over every 4th neighbour (index, then the record A, B_0, B_1, T_0,
// T_1, C as three 16-byte loads, then the neighbour's u, v, p), a shuffle
// sum of the three row sums
__global__ void __launch_bounds__(256)
    amr_residual_kernel(long long nf, const int* __restrict__ nbp, const int* __restrict__ nbc,
                        const double* __restrict__ nbv, const double* __restrict__ x,
                        const double* __restrict__ b, double* __restrict__ r) {
  constexpr int LPN = 4;
  const int lane = threadIdx.x % LPN;
  const long long gf = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / LPN;
  const long long f = gf < nf ? gf : nf - 1;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (int p = nbp[f] + lane; p < nbp[f + 1]; p += LPN) {
    const long long g = nbc[p];
    const double2* v = reinterpret_cast<const double2*>(nbv + 6 * (long long)p);
    const double2 m0 = v[0], m1 = v[1], m2 = v[2];  // (A, B0), (B1, T0), (T1, C)
    const double xu = x[3 * g], xv = x[3 * g + 1], xp = x[3 * g + 2];
    a0 += m0.x * xu + m0.y * xp;
    a1 += m0.x * xv + m1.x * xp;
    a2 += m1.y * xu + m2.x * xv + m2.y * xp;
  }
#pragma unroll
  for (int o = LPN / 2; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
  }
  if (gf >= nf || lane >= 3) return;
  const double s = lane == 0 ? a0 : (lane == 1 ? a1 : a2);
  const long long row = f * 3 + lane;
  r[row] = b ? b[row] - s : s;
}

// patch apply: 4 lanes per patch over the patch's slot records (dof index
// in the bits of a double, then the 3 owned-row coefficients: two 16-byte
// loads per slot); y_k = sum_j rows[k][j] r[dof_j]; restricted write
// x[owned] += omega y (constrained velocity DoFs: identity rows, x += r)
__global__ void __launch_bounds__(256)
    amr_apply_kernel(long long np, const long long* __restrict__ pstart, const int* __restrict__ pown,
                     const double* __restrict__ rows, const unsigned char* __restrict__ fixed,
                     const double* __restrict__ r, double omega, double* __restrict__ x) {
  constexpr int TPP = 4;
  const int lane = threadIdx.x % TPP;
  const long long gi = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / TPP;
  const bool valid = gi < np;
  const long long i = valid ? gi : np - 1;
  const long long s0 = pstart[i];
  const int n = (int)(pstart[i + 1] - s0);
  const double2* rec = reinterpret_cast<const double2*>(rows + 4 * s0);
  double y[3] = {0.0, 0.0, 0.0};
#pragma unroll 4
  for (int j = lane; j < n; j += TPP) {
    const double2 a = __ldcs(rec + 2 * j), c = __ldcs(rec + 2 * j + 1);
    const double rv = r[__double_as_longlong(a.x)];
    y[0] += a.y * rv;
    y[1] += c.x * rv;
    y[2] += c.y * rv;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int o = TPP / 2; o > 0; o >>= 1) y[k] += __shfl_xor_sync(0xffffffffu, y[k], o);
  if (!valid || lane >= 3) return;
  const long long d = i * 3 + lane;
  const double yk = lane == 0 ? y[0] : (lane == 1 ? y[1] : y[2]);
  if (fixed[d]) x[d] += r[d];
  else if (pown[i * 3 + lane] >= 0) x[d] += omega * yk;
}

// x_f += P e_c per component, constrained fine DoFs left alone
__global__ void amr_prolong_kernel(long long nf, const int* __restrict__ prp, const int* __restrict__ pcl,
                                   const double* __restrict__ pvl, const unsigned char* __restrict__ fixed,
                                   const double* __restrict__ ec, double* __restrict__ xf) {
  const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  double s[3] = {0.0, 0.0, 0.0};
  for (int p = prp[f]; p < prp[f + 1]; ++p)
    for (int c = 0; c < 3; ++c) s[c] = s[c] + pvl[p] * ec[(long long)pcl[p] * 3 + c];
  for (int c = 0; c < 3; ++c)
    if (!fixed[f * 3 + c]) xf[f * 3 + c] += s[c];
}

// b_c = P^T r_f (gather over the fine nodes of each coarse node), then
// constrained coarse DoFs zeroed
__global__ void amr_restrict_kernel(long long nc, const int* __restrict__ rrp, const int* __restrict__ rcl,
                                    const double* __restrict__ rvl, const unsigned char* __restrict__ cfixed,
                                    const double* __restrict__ rf, double* __restrict__ bc) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  double s[3] = {0.0, 0.0, 0.0};
  for (int p = rrp[c]; p < rrp[c + 1]; ++p)
    for (int k = 0; k < 3; ++k) s[k] = s[k] + rvl[p] * rf[(long long)rcl[p] * 3 + k];
  for (int k = 0; k < 3; ++k) bc[c * 3 + k] = cfixed[c * 3 + k] ? 0.0 : s[k];
}

// dense row-major copy of a CSR matrix
__global__ void amr_dense_kernel(long long n, const int* __restrict__ rp, const int* __restrict__ col,
                                 const double* __restrict__ val, double* __restrict__ M) {
  const long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  for (long long c = 0; c < n; ++c) M[row * n + c] = 0.0;
  for (int p = rp[row]; p < rp[row + 1]; ++p) M[row * n + col[p]] = val[p];
}

unsigned nblocks(long long n) { return (unsigned)((n + 255) / 256); }

}  // namespace

cudaError_t launch_amr_residual(const AmrLevel& A, const double* x, const double* b, double* r, cudaStream_t s) {
  amr_residual_kernel<<<nblocks(A.nfree * 4), 256, 0, s>>>(A.nfree, A.nbp, A.nbc, A.nbv, x, b, r);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_amr_apply(const AmrLevel& A, const double* r, double omega, double* x, cudaStream_t s) {
  amr_apply_kernel<<<nblocks(A.nfree * 4), 256, 0, s>>>(A.nfree, A.pstart, A.pown, A.rows, A.fixed, r, omega, x);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_amr_prolong_add(const AmrLevel& F, const double* ec, double* xf, cudaStream_t s) {
  amr_prolong_kernel<<<nblocks(F.nfree), 256, 0, s>>>(F.nfree, F.prp, F.pcl, F.pvl, F.fixed, ec, xf);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_amr_restrict(const AmrLevel& F, const AmrLevel& C, const double* rf, double* bc, cudaStream_t s) {
  amr_restrict_kernel<<<nblocks(C.nfree), 256, 0, s>>>(C.nfree, F.rrp, F.rcl, F.rvl, C.fixed, rf, bc);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_amr_dense(const AmrLevel& A, double* M, cudaStream_t s) {
  const long long n = A.nfree * 3;
  amr_dense_kernel<<<nblocks(n), 256, 0, s>>>(n, A.rowptr, A.col, A.val, M);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace fc
