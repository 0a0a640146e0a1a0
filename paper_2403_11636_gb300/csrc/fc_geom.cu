// fc_geom.cu -- finite cell element data on the GPU (paper Sec. 2).
//
// One warp per background cell computes
//   a(v,u) = (eta grad v, alpha grad u) - (v, n.eta grad u)_G - (n.eta grad v, u)_G + (v, lambda u)_G
//   b(v,p) = -(div v, alpha p) + (v, n p)_G
//   f(v)   = (v, alpha f)
// for the nodal functions of the cell (eq. stokes_disc_weak_fcm_2): the 2^d
// Q1 functions for velocity and pressure (the paper's pair), or the 3^d Q2
// velocity functions with the Q1 pressure functions (Taylor-Hood variant),
// with Gamma_D the obstacle boundary (no-slip, w = 0).  The volume rule is
// the recursive box split: a box is split into 2^d children when the level
// set changes sign among its 3^d sample points, down to the quadrature depth;
// leaves take the tensor 2-point (Q1) or 3-point (Q2) Gauss rule with alpha
// evaluated at each point.  The boundary rule is composite 2-point Gauss in the curve
// parameter (circle / ellipse) or in cos(theta) times a uniform rule in the
// azimuth (sphere); every rule point is owned by the cell that contains it.
//
// The warp walks the split tree in depth-first order (children in
// lexicographic order) and adds point contributions in rule order, so every
// entry is a sum over the same points in the same order as the definition;
// the points themselves (level set, basis, force) are evaluated one per lane
// and broadcast.  This translation unit is compiled with --fmad=false.
#include <math.h>

#include "fc_internal.cuh"

namespace fc {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kStack = 48;

__device__ __forceinline__ double phi_shape(const Shape& s, int dim, const double* x) {
  double dx = x[0] - s.c[0], dy = x[1] - s.c[1];
  if (s.type == 0) {
    double q = dx * dx + dy * dy;
    if (dim == 3) {
      double dz = x[2] - s.c[2];
      q = q + dz * dz;
    }
    return s.r[0] - sqrt(q);
  }
  double xp = s.rot[0] * dx + s.rot[1] * dy;
  double yp = -s.rot[1] * dx + s.rot[0] * dy;
  double u = xp / s.r[0], v = yp / s.r[1];
  return 1.0 - (u * u + v * v);
}

// Sign of the level set: only shapes whose bounding box meets the cell can
// be positive at a point of the cell, so the candidate list decides it.
__device__ __forceinline__ bool inside_obstacle(const Shape* sh, const int* cand, int nc, int dim,
                                                const double* x) {
  double p = -1.0;
  for (int t = 0; t < nc; ++t) {
    double q = phi_shape(sh[cand[t]], dim, x);
    if (t == 0 || q > p) p = q;
  }
  return p > 0.0;
}

__device__ __forceinline__ void q1_basis(int dim, const double* x0, const double* h,
                                         const double* x, double* val, double (*grad)[3]) {
  double xi[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < dim; ++k) xi[k] = (x[k] - x0[k]) / h[k];
  const int nloc = 1 << dim;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    if (a >= nloc) break;
    double f1[3], d1[3];
    for (int k = 0; k < dim; ++k) {
      int bit = (a >> k) & 1;
      f1[k] = bit ? xi[k] : 1.0 - xi[k];
      d1[k] = (bit ? 1.0 : -1.0) / h[k];
    }
    double v = 1.0;
    for (int k = 0; k < dim; ++k) v = v * f1[k];
    val[a] = v;
    grad[a][0] = grad[a][1] = grad[a][2] = 0.0;
    for (int k = 0; k < dim; ++k) {
      double gk = d1[k];
      for (int m = 0; m < dim; ++m)
        if (m != k) gk = gk * f1[m];
      grad[a][k] = gk;
    }
  }
}

__device__ __forceinline__ void force_at(const LevelGeom& g, const double* x, double* f) {
  f[0] = f[1] = f[2] = 0.0;
  switch (g.force_kind) {
    case 0:
      f[0] = g.force[0]; f[1] = g.force[1]; f[2] = g.force[2];
      break;
    case 1:
      f[0] = g.force[0] * sin(kPi * x[0]);
      f[1] = g.force[1] * cos(kPi * x[1]);
      break;
    case 2:
      f[0] = g.force[0] * sin(kPi * x[1]);
      if (g.dim == 3) f[0] = f[0] * sin(kPi * x[2]);
      break;
    case 3:
      f[0] = -g.force[0] * (kPi / 2.0) * sin(kPi * x[0] / 2.0);
      break;
    default:
      break;
  }
}

// Entries handled by one lane: e = lane + 32 t.  Entry index space:
// [A upper triangle (a <= b, a-major)] [B (c, a, b)] [F (c, a)], with NV
// velocity and NP pressure functions per cell (Q1: 2^d and 2^d; Q2: 3^d
// and 2^d).
template <int DIM, int Q = 1>
struct Entries {
  static constexpr int NV = Q == 2 ? (DIM == 3 ? 27 : 9) : (1 << DIM);
  static constexpr int NP = 1 << DIM;
  static constexpr int NA = NV * (NV + 1) / 2;
  static constexpr int NB = DIM * NV * NP;
  static constexpr int NF = DIM * NV;
  static constexpr int NE = NA + NB + NF;
  static constexpr int PER = (NE + 31) / 32;
  static constexpr int NG1 = Q + 1;  // Gauss points per direction on a leaf
  static constexpr int NG = DIM == 3 ? NG1 * NG1 * NG1 : NG1 * NG1;
  // warps per CTA: the per-warp point queue grows with the basis and static
  // shared memory is limited to 48 KB per CTA
  static constexpr int WARPS = Q == 2 ? (DIM == 3 ? 1 : 3) : 4;
  // CTAs per SM the 3D Q1 kernel is compiled for (at most 128 registers:
  // the FP64 quadrature is latency-bound, more resident warps hide it)
  static constexpr int MINB = DIM == 3 && Q == 1 ? 4 : 1;
};

struct EntryId {
  int kind, c, a, b;  // kind 0 A, 1 B, 2 F, -1 none
};

template <int DIM, int Q = 1>
__device__ EntryId entry_of(int e) {
  using E = Entries<DIM, Q>;
  EntryId id{-1, 0, 0, 0};
  if (e < E::NA) {
    int a = 0, rem = e;
    while (rem >= E::NV - a) { rem -= E::NV - a; ++a; }
    id.kind = 0; id.a = a; id.b = a + rem;
  } else if (e < E::NA + E::NB) {
    int t = e - E::NA;
    id.kind = 1; id.c = t / (E::NV * E::NP); id.a = (t / E::NP) % E::NV; id.b = t % E::NP;
  } else if (e < E::NE) {
    int t = e - E::NA - E::NB;
    id.kind = 2; id.c = t / E::NV; id.a = t % E::NV;
  }
  return id;
}

// Q2 functions on [0, 1]: q0 = (1-t)(1-2t), q1 = 4t(1-t), q2 = t(2t-1)
__device__ __forceinline__ void q2_1d(double t, double* v, double* d) {
  v[0] = (1.0 - t) * (1.0 - 2.0 * t);
  v[1] = 4.0 * t * (1.0 - t);
  v[2] = t * (2.0 * t - 1.0);
  d[0] = 4.0 * t - 3.0;
  d[1] = 4.0 - 8.0 * t;
  d[2] = 4.0 * t - 1.0;
}

// velocity values / gradients (NV) and pressure values (NP) at x
template <int DIM, int Q>
__device__ __forceinline__ void elem_basis(const double* x0, const double* h, const double* x, double* val,
                                           double (*grad)[3], double* pval) {
  if (Q == 1) {
    q1_basis(DIM, x0, h, x, val, grad);
    for (int a = 0; a < (1 << DIM); ++a) pval[a] = val[a];
    return;
  }
  double v[3][3], d[3][3], t[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < 3; ++k) {
    t[k] = k < DIM ? (x[k] - x0[k]) / h[k] : 0.0;
    q2_1d(t[k], v[k], d[k]);
  }
  constexpr int NV = DIM == 3 ? 27 : 9;
  for (int a = 0; a < NV; ++a) {
    const int ia[3] = {a % 3, (a / 3) % 3, a / 9};
    double f = 1.0;
    for (int k = 0; k < DIM; ++k) f = f * v[k][ia[k]];
    val[a] = f;
    grad[a][0] = grad[a][1] = grad[a][2] = 0.0;
    for (int k = 0; k < DIM; ++k) {
      double gk = d[k][ia[k]] / h[k];
      for (int m = 0; m < DIM; ++m)
        if (m != k) gk = gk * v[m][ia[m]];
      grad[a][k] = gk;
    }
  }
  for (int b = 0; b < (1 << DIM); ++b) {
    double f = 1.0;
    for (int k = 0; k < DIM; ++k) f = f * (((b >> k) & 1) ? t[k] : 1.0 - t[k]);
    pval[b] = f;
  }
}

template <int DIM, int Q>
struct WarpShared {
  static constexpr int NV = Entries<DIM, Q>::NV, NP = Entries<DIM, Q>::NP;
  int cand[kMaxShapesPerCell];
  double stk_lo[kStack][3];
  int stk_lev[kStack];
  // Gauss points of the volume rule waiting for evaluation, in rule order:
  // position and weight, then per point alpha, force, basis values and
  // gradients (filled one point per lane)
  double px[32][3];
  double pw[32];
  double pal[32];
  double pf[32][3];
  double pval[32][NV];
  double pgrad[32][NV][3];
  double ppv[32][Q == 2 ? NP : 1];  // Q1: the pressure functions are the velocity ones (pval)
};

// Angular index range [lo, hi] (before wrapping) of rule points t = step *
// (m + off) that can fall in the box [bx0, bx1] x [by0, by1], seen from the
// centre (cx, cy) after the map (dx, dy) -> ((R^T d)_x / a, (R^T d)_y / b).
// Returns false when the box contains the centre (all indices).
__device__ bool angular_range(double bx0, double bx1, double by0, double by1, double cx, double cy,
                              double ca, double sa, double a, double b, double step, double off,
                              long long* mlo, long long* mhi) {
  if (cx >= bx0 && cx <= bx1 && cy >= by0 && cy <= by1) return false;
  double mx = 0.5 * (bx0 + bx1) - cx, my = 0.5 * (by0 + by1) - cy;
  double ur = (ca * mx + sa * my) / a, vr = (-sa * mx + ca * my) / b;
  double tref = atan2(vr, ur);
  double dmin = 0.0, dmax = 0.0;
  for (int k = 0; k < 4; ++k) {
    double X = (k & 1) ? bx1 : bx0, Y = (k & 2) ? by1 : by0;
    double dx = X - cx, dy = Y - cy;
    double u = (ca * dx + sa * dy) / a, v = (-sa * dx + ca * dy) / b;
    // angle of (u, v) relative to the reference direction
    double cr = ur * v - vr * u, dt = ur * u + vr * v;
    double d = atan2(cr, dt);
    if (k == 0 || d < dmin) dmin = d;
    if (k == 0 || d > dmax) dmax = d;
  }
  double tlo = tref + dmin, thi = tref + dmax;
  *mlo = (long long)floor(tlo / step - off) - 1;
  *mhi = (long long)floor(thi / step - off) + 1;
  return true;
}

template <int DIM, int Q>
__global__ void __launch_bounds__(Entries<DIM, Q>::WARPS * 32, Entries<DIM, Q>::MINB)
    cell_elements_kernel(LevelGeom g, double* __restrict__ eA, double* __restrict__ eB,
                         double* __restrict__ eF, double* __restrict__ estat,
                         unsigned* __restrict__ d_err, const double* __restrict__ refA,
                         const double* __restrict__ refB, unsigned char* __restrict__ cclass,
                         const long long* __restrict__ cell_list, long long nlist) {
  using E = Entries<DIM, Q>;
  constexpr int NL = E::NV, NP = E::NP, WARPS = E::WARPS;
  __shared__ WarpShared<DIM, Q> wsh[WARPS];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  WarpShared<DIM, Q>& S = wsh[wib];
  // with a cell list (the leaves of one level of an adaptive grid), slot q
  // integrates cell cell_list[q] of g and writes its outputs at position q
  const long long slot = (long long)blockIdx.x * WARPS + wib;
  if (slot >= (cell_list ? nlist : g.ncell)) return;
  const long long cell = cell_list ? cell_list[slot] : slot;
  const unsigned FULL = 0xffffffffu;

  long long ci = cell % g.n[0];
  long long cj = (cell / g.n[0]) % g.n[1];
  long long ck = DIM == 3 ? cell / ((long long)g.n[0] * g.n[1]) : 0;
  double x0[3];
  x0[0] = g.lo[0] + (double)ci * g.h[0];
  x0[1] = g.lo[1] + (double)cj * g.h[1];
  x0[2] = DIM == 3 ? g.lo[2] + (double)ck * g.h[2] : 0.0;
  double x1[3] = {x0[0] + g.h[0], x0[1] + g.h[1], DIM == 3 ? x0[2] + g.h[2] : 0.0};

  // ---- candidate shapes (bounding boxes meeting the slightly enlarged cell)
  int nc = 0;
  for (int base = 0; base < g.nshape; base += 32) {
    int s = base + lane;
    bool hit = false;
    if (s < g.nshape) {
      const Shape& sh = g.shapes[s];
      hit = true;
      for (int k = 0; k < DIM; ++k) {
        double m = 1e-9 * g.h[k];
        if (sh.c[k] + sh.bbr < x0[k] - m || sh.c[k] - sh.bbr > x1[k] + m) hit = false;
      }
    }
    unsigned bal = __ballot_sync(FULL, hit);
    int pos = nc + __popc(bal & ((1u << lane) - 1u));
    if (hit && pos < kMaxShapesPerCell) S.cand[pos] = s;
    nc += __popc(bal);
  }
  if (nc > kMaxShapesPerCell) {
    if (lane == 0) atomicOr(d_err, kErrTooManyShapes);
    nc = kMaxShapesPerCell;
  }
  __syncwarp();

  double acc[E::PER];
#pragma unroll
  for (int t = 0; t < E::PER; ++t) acc[t] = 0.0;
  double fluid_volume = 0.0, bmeasure = 0.0;
  int nvol = 0, nbnd = 0;
  bool split = false, al_mixed = false;
  double al_first = -1.0;

  // ---- volume rule: depth-first over the split tree.  The Gauss points of
  // the leaves are queued in rule order and evaluated 32 at a time, one
  // point per lane (level set, alpha, basis, force); the lanes then add the
  // queued points to their entries in queue order, so every entry is still
  // the sum over the points in rule order.
  const double gq[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
  // 3-point Gauss (Q2 leaves): nodes 1/2 -+ sqrt(3/5)/2, 1/2, weights 5/18, 8/18, 5/18
  const double gq3[3] = {0.5 - 0.5 * sqrt(0.6), 0.5, 0.5 + 0.5 * sqrt(0.6)};
  const double gw3[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  constexpr int NG = E::NG;
  int npt = 0;
  auto flush = [&]() {
    if (lane < npt) {
      const double x[3] = {S.px[lane][0], S.px[lane][1], S.px[lane][2]};
      S.pal[lane] = inside_obstacle(g.shapes, S.cand, nc, DIM, x) ? g.alpha : 1.0;
      double val[NL], grad[NL][3], pv[NP];
      elem_basis<DIM, Q>(x0, g.h, x, val, grad, pv);
      for (int a = 0; a < NL; ++a) {
        S.pval[lane][a] = val[a];
        for (int k = 0; k < 3; ++k) S.pgrad[lane][a][k] = grad[a][k];
      }
      if (Q == 2)
        for (int b = 0; b < NP; ++b) S.ppv[lane][b] = pv[b];
      double f[3] = {0.0, 0.0, 0.0};
      force_at(g, x, f);
      for (int k = 0; k < 3; ++k) S.pf[lane][k] = f[k];
    }
    __syncwarp();
    for (int q = 0; q < npt; ++q) {
      const double w = S.pw[q], al = S.pal[q];
#pragma unroll
      for (int t = 0; t < E::PER; ++t) {
        EntryId id = entry_of<DIM, Q>(lane + 32 * t);
        if (id.kind == 0) {
          double gg = 0.0;
          for (int kk = 0; kk < DIM; ++kk) gg = gg + S.pgrad[q][id.a][kk] * S.pgrad[q][id.b][kk];
          acc[t] = acc[t] + w * al * g.eta * gg;
        } else if (id.kind == 1) {
          acc[t] = acc[t] - w * al * S.pgrad[q][id.a][id.c] * (Q == 2 ? S.ppv[q][id.b] : S.pval[q][id.b]);
        } else if (id.kind == 2) {
          acc[t] = acc[t] + w * al * S.pf[q][id.c] * S.pval[q][id.a];
        }
      }
      if (al == 1.0) fluid_volume = fluid_volume + w;
      if (al_first < 0.0) al_first = al;
      else if (al != al_first) al_mixed = true;
      nvol++;
    }
    __syncwarp();
    npt = 0;
  };
  int sp = 0;
  if (lane == 0) {
    S.stk_lo[0][0] = x0[0]; S.stk_lo[0][1] = x0[1]; S.stk_lo[0][2] = x0[2];
    S.stk_lev[0] = 0;
  }
  sp = 1;
  __syncwarp();
  while (sp > 0) {
    --sp;
    double lo[3] = {S.stk_lo[sp][0], S.stk_lo[sp][1], S.stk_lo[sp][2]};
    int level = S.stk_lev[sp];
    __syncwarp();
    double hb[3];
    for (int k = 0; k < 3; ++k) {
      double v = g.h[k];
      for (int l = 0; l < level; ++l) v = v * 0.5;
      hb[k] = v;
    }
    // sign at the 3^d sample points
    constexpr int NS = DIM == 3 ? 27 : 9;
    bool pos = false;
    if (lane < NS) {
      int i = lane % 3, j = (lane / 3) % 3, k = lane / 9;
      double x[3] = {lo[0] + hb[0] * (0.5 * i), lo[1] + hb[1] * (0.5 * j),
                     DIM == 3 ? lo[2] + hb[2] * (0.5 * k) : 0.0};
      pos = inside_obstacle(g.shapes, S.cand, nc, DIM, x);
    }
    unsigned bal = __ballot_sync(FULL, pos);
    int npos = __popc(bal);
    bool cut = (npos != 0 && npos != NS);
    if (cut && level < g.qdepth) {
      split = true;
      // push the 2^d children in reverse so that child 0 is processed first
      constexpr int NCH = 1 << DIM;
      if (lane == 0) {
        for (int ch = NCH - 1; ch >= 0; --ch) {
          double lc[3] = {lo[0], lo[1], lo[2]};
          for (int k = 0; k < DIM; ++k)
            if ((ch >> k) & 1) lc[k] = lo[k] + hb[k] * 0.5;
          if (sp + (NCH - 1 - ch) < kStack) {
            S.stk_lo[sp + (NCH - 1 - ch)][0] = lc[0];
            S.stk_lo[sp + (NCH - 1 - ch)][1] = lc[1];
            S.stk_lo[sp + (NCH - 1 - ch)][2] = lc[2];
            S.stk_lev[sp + (NCH - 1 - ch)] = level + 1;
          }
        }
      }
      sp += NCH;
      if (sp > kStack) {
        if (lane == 0) atomicOr(d_err, kErrBadIndex);
        sp = 0;
      }
      __syncwarp();
      continue;
    }
    // a leaf: queue its Gauss points
    if (npt + NG > 32) flush();
    if (Q == 1) {
      double w = 1.0;
      for (int k = 0; k < DIM; ++k) w = w * (hb[k] * 0.5);
      if (lane < NG) {
        const int i = lane & 1, j = (lane >> 1) & 1, k = lane >> 2;
        S.px[npt + lane][0] = lo[0] + hb[0] * gq[i];
        S.px[npt + lane][1] = lo[1] + hb[1] * gq[j];
        S.px[npt + lane][2] = DIM == 3 ? lo[2] + hb[2] * gq[k] : 0.0;
        S.pw[npt + lane] = w;
      }
    } else if (lane < NG) {
      const int i = lane % 3, j = (lane / 3) % 3, k = lane / 9;
      S.px[npt + lane][0] = lo[0] + hb[0] * gq3[i];
      S.px[npt + lane][1] = lo[1] + hb[1] * gq3[j];
      S.px[npt + lane][2] = DIM == 3 ? lo[2] + hb[2] * gq3[k] : 0.0;
      double w = (hb[0] * gw3[i]) * (hb[1] * gw3[j]);
      if (DIM == 3) w = w * (hb[2] * gw3[k]);
      S.pw[npt + lane] = w;
    }
    npt += NG;
    __syncwarp();
  }
  if (npt > 0) flush();

  // ---- boundary rule of every candidate shape, points owned by this cell
  const int k2 = 1 << g.qdepth;
  for (int t = 0; t < nc; ++t) {
    const int s = S.cand[t];
    const Shape sh = g.shapes[s];
    if (DIM == 2) {
      double rmax = sh.type == 0 ? sh.r[0] : (sh.r[0] > sh.r[1] ? sh.r[0] : sh.r[1]);
      long long N = 8LL * (long long)ceil(2.0 * kPi * rmax / g.hmin) * k2;
      if (N < 64) N = 64;
      double dt = 2.0 * kPi / (double)N;
      double a = sh.type == 0 ? sh.r[0] : sh.r[0], b = sh.type == 0 ? sh.r[0] : sh.r[1];
      double ca = sh.type == 0 ? 1.0 : sh.rot[0], sa = sh.type == 0 ? 0.0 : sh.rot[1];
      double mg = 1e-9 * g.h[0];
      long long mlo = 0, mhi = N - 1;
      if (angular_range(x0[0] - mg, x1[0] + mg, x0[1] - mg, x1[1] + mg, sh.c[0], sh.c[1], ca, sa,
                        a, b, dt, 0.5, &mlo, &mhi)) {
        if (mhi - mlo + 1 >= N) { mlo = 0; mhi = N - 1; }
      }
      long long cnt = mhi - mlo + 1;
      long long start = ((mlo % N) + N) % N;
      // ascending order of m: the wrapped head [0, e] precedes [start, N-1]
      long long e_wrap = start + cnt - 1 - N;  // last index of the wrapped part, < 0 if none
      long long seg_b[2], seg_e[2];
      int nseg = 0;
      if (e_wrap >= 0) { seg_b[nseg] = 0; seg_e[nseg] = e_wrap; nseg++; seg_b[nseg] = start; seg_e[nseg] = N - 1; nseg++; }
      else { seg_b[0] = start; seg_e[0] = start + cnt - 1; nseg = 1; }
      for (int sg = 0; sg < nseg; ++sg) {
        long long npts = 2 * (seg_e[sg] - seg_b[sg] + 1);
        for (long long base = 0; base < npts; base += 32) {
          long long pidx = base + lane;
          bool ok = false;
          double px = 0, py = 0, nx = 0, ny = 0, wgt = 0;
          if (pidx < npts) {
            long long m = seg_b[sg] + pidx / 2;
            int j = (int)(pidx & 1);
            double tt = dt * ((double)m + gq[j]);
            double ct = cos(tt), st = sin(tt);
            if (sh.type == 0) {
              px = sh.c[0] + sh.r[0] * ct;
              py = sh.c[1] + sh.r[0] * st;
              nx = -ct; ny = -st;
              wgt = 0.5 * dt * sh.r[0];
            } else {
              double cr = sh.rot[0], sr = sh.rot[1];
              px = sh.c[0] + (cr * (a * ct) - sr * (b * st));
              py = sh.c[1] + (sr * (a * ct) + cr * (b * st));
              double tx = b * ct, ty = a * st;
              double nl = sqrt(tx * tx + ty * ty);
              nx = -(cr * tx - sr * ty) / nl;
              ny = -(sr * tx + cr * ty) / nl;
              double spd = sqrt((a * st) * (a * st) + (b * ct) * (b * ct));
              wgt = 0.5 * dt * spd;
            }
            double xx[3] = {px, py, 0.0};
            ok = true;
            long long idx[2];
            for (int k = 0; k < 2; ++k) {
              if (xx[k] < g.lo[k] || xx[k] > g.hi[k]) { ok = false; break; }
              long long ii = (long long)floor((xx[k] - g.lo[k]) / g.h[k]);
              if (ii >= g.n[k]) ii = g.n[k] - 1;
              if (ii < 0) ii = 0;
              idx[k] = ii;
            }
            if (ok && (idx[0] != ci || idx[1] != cj)) ok = false;
            if (ok) {
              for (int u = 0; u < nc; ++u)
                if (S.cand[u] != s && phi_shape(g.shapes[S.cand[u]], 2, xx) > 0.0) { ok = false; break; }
            }
          }
          // each lane evaluates the basis at its own point; the points are
          // then added in rule order with their values broadcast by shuffle
          double lval[NL], ldn[NL], lpv[NP];
          {
            double bx[3] = {px, py, 0.0};
            double val[NL], grad[NL][3];
            elem_basis<DIM, Q>(x0, g.h, bx, val, grad, lpv);
            for (int q = 0; q < NL; ++q) {
              double sdn = 0.0;
              const double bnl[3] = {nx, ny, 0.0};
              for (int k = 0; k < DIM; ++k) sdn = sdn + bnl[k] * grad[q][k];
              lval[q] = val[q];
              ldn[q] = sdn;
            }
          }
          unsigned vb = __ballot_sync(FULL, ok);
          while (vb) {
            int src = __ffs(vb) - 1;
            vb &= vb - 1;
            double bn[3] = {__shfl_sync(FULL, nx, src), __shfl_sync(FULL, ny, src), 0.0};
            double bw = __shfl_sync(FULL, wgt, src);
            double val[NL], dn[NL], pv[NP];
#pragma unroll
            for (int q = 0; q < NL; ++q) {
              val[q] = __shfl_sync(FULL, lval[q], src);
              dn[q] = __shfl_sync(FULL, ldn[q], src);
            }
#pragma unroll
            for (int q = 0; q < NP; ++q) pv[q] = __shfl_sync(FULL, lpv[q], src);
#pragma unroll
            for (int u = 0; u < E::PER; ++u) {
              EntryId id = entry_of<DIM, Q>(lane + 32 * u);
              if (id.kind == 0) {
                double tv = -g.eta * val[id.a] * dn[id.b] - g.eta * dn[id.a] * val[id.b] +
                            g.lambda * val[id.a] * val[id.b];
                acc[u] = acc[u] + bw * tv;
              } else if (id.kind == 1) {
                acc[u] = acc[u] + bw * val[id.a] * bn[id.c] * pv[id.b];
              }
            }
            bmeasure = bmeasure + bw;
            nbnd++;
          }
        }
      }
    } else {
      const double r = sh.r[0];
      long long Nm = (long long)ceil(2.0 * r / g.hmin) * k2;
      if (Nm < 8) Nm = 8;
      long long Nf = 2LL * (long long)ceil(2.0 * kPi * r / g.hmin) * k2;
      if (Nf < 16) Nf = 16;
      double dm = 2.0 / (double)Nm, df = 2.0 * kPi / (double)Nf;
      double wgt = r * r * (0.5 * dm) * df;
      double mz = 1e-9 * g.h[2];
      long long m0 = (long long)floor((((x0[2] - mz) - sh.c[2]) / r + 1.0) / dm) - 1;
      long long m1 = (long long)floor((((x1[2] + mz) - sh.c[2]) / r + 1.0) / dm) + 1;
      if (m0 < 0) m0 = 0;
      if (m1 > Nm - 1) m1 = Nm - 1;
      double mgx = 1e-9 * g.h[0], mgy = 1e-9 * g.h[1];
      for (long long m = m0; m <= m1; ++m) {
        for (int j = 0; j < 2; ++j) {
          double mu = -1.0 + dm * ((double)m + gq[j]);
          double st = sqrt(1.0 - mu * mu);
          double rho = r * st;
          // ring bounding box against the cell's xy box
          if (sh.c[0] + rho < x0[0] - mgx || sh.c[0] - rho > x1[0] + mgx ||
              sh.c[1] + rho < x0[1] - mgy || sh.c[1] - rho > x1[1] + mgy)
            continue;
          long long qlo = 0, qhi = Nf - 1;
          if (angular_range(x0[0] - mgx, x1[0] + mgx, x0[1] - mgy, x1[1] + mgy, sh.c[0], sh.c[1],
                            1.0, 0.0, 1.0, 1.0, df, 0.5, &qlo, &qhi)) {
            if (qhi - qlo + 1 >= Nf) { qlo = 0; qhi = Nf - 1; }
          }
          long long cnt = qhi - qlo + 1;
          long long start = ((qlo % Nf) + Nf) % Nf;
          long long e_wrap = start + cnt - 1 - Nf;
          long long seg_b[2], seg_e[2];
          int nseg = 0;
          if (e_wrap >= 0) { seg_b[nseg] = 0; seg_e[nseg] = e_wrap; nseg++; seg_b[nseg] = start; seg_e[nseg] = Nf - 1; nseg++; }
          else { seg_b[0] = start; seg_e[0] = start + cnt - 1; nseg = 1; }
          for (int sg = 0; sg < nseg; ++sg) {
            long long npts = seg_e[sg] - seg_b[sg] + 1;
            for (long long base = 0; base < npts; base += 32) {
              long long pidx = base + lane;
              bool ok = false;
              double ex = 0, ey = 0;
              double xx[3] = {0, 0, 0};
              if (pidx < npts) {
                long long q = seg_b[sg] + pidx;
                double ph = df * ((double)q + 0.5);
                double cp = cos(ph), spv = sin(ph);
                ex = st * cp;
                ey = st * spv;
                xx[0] = sh.c[0] + r * ex;
                xx[1] = sh.c[1] + r * ey;
                xx[2] = sh.c[2] + r * mu;
                ok = true;
                long long idx[3];
                for (int k = 0; k < 3; ++k) {
                  if (xx[k] < g.lo[k] || xx[k] > g.hi[k]) { ok = false; break; }
                  long long ii = (long long)floor((xx[k] - g.lo[k]) / g.h[k]);
                  if (ii >= g.n[k]) ii = g.n[k] - 1;
                  if (ii < 0) ii = 0;
                  idx[k] = ii;
                }
                if (ok && (idx[0] != ci || idx[1] != cj || idx[2] != ck)) ok = false;
                if (ok) {
                  for (int u = 0; u < nc; ++u)
                    if (S.cand[u] != s && phi_shape(g.shapes[S.cand[u]], 3, xx) > 0.0) { ok = false; break; }
                }
              }
              double lval[NL], ldn[NL], lpv[NP];
              {
                double val[NL], grad[NL][3];
                elem_basis<DIM, Q>(x0, g.h, xx, val, grad, lpv);
                const double bnl[3] = {-ex, -ey, -mu};
                for (int qq = 0; qq < NL; ++qq) {
                  double sdn = 0.0;
                  for (int k = 0; k < DIM; ++k) sdn = sdn + bnl[k] * grad[qq][k];
                  lval[qq] = val[qq];
                  ldn[qq] = sdn;
                }
              }
              unsigned vb = __ballot_sync(FULL, ok);
              while (vb) {
                int src = __ffs(vb) - 1;
                vb &= vb - 1;
                double bn[3] = {-__shfl_sync(FULL, ex, src), -__shfl_sync(FULL, ey, src), -mu};
                double val[NL], dn[NL], pv[NP];
#pragma unroll
                for (int qq = 0; qq < NL; ++qq) {
                  val[qq] = __shfl_sync(FULL, lval[qq], src);
                  dn[qq] = __shfl_sync(FULL, ldn[qq], src);
                }
#pragma unroll
                for (int qq = 0; qq < NP; ++qq) pv[qq] = __shfl_sync(FULL, lpv[qq], src);
#pragma unroll
                for (int u = 0; u < E::PER; ++u) {
                  EntryId id = entry_of<DIM, Q>(lane + 32 * u);
                  if (id.kind == 0) {
                    double tv = -g.eta * val[id.a] * dn[id.b] - g.eta * dn[id.a] * val[id.b] +
                                g.lambda * val[id.a] * val[id.b];
                    acc[u] = acc[u] + wgt * tv;
                  } else if (id.kind == 1) {
                    acc[u] = acc[u] + wgt * val[id.a] * bn[id.c] * pv[id.b];
                  }
                }
                bmeasure = bmeasure + wgt;
                nbnd++;
              }
            }
          }
        }
      }
    }
  }

  // ---- write back (A mirrored).  A plain cell (not split, one alpha at all
  // its Gauss points, no boundary points) takes alpha times the reference
  // element matrices of the same rule on an uncut cell: the same values up
  // to rounding, but bit-identical across plain cells, which makes the
  // patch blocks of uncut regions bit-identical (patch classes).
  const bool plain = refA != nullptr && !split && nbnd == 0 && !al_mixed && al_first > 0.0;
  double* A = eA + slot * NL * NL;
  double* B = eB + slot * DIM * NL * NP;
  double* F = eF + slot * DIM * NL;
#pragma unroll
  for (int t = 0; t < E::PER; ++t) {
    EntryId id = entry_of<DIM, Q>(lane + 32 * t);
    if (id.kind == 0) {
      double v = plain ? al_first * refA[id.a * NL + id.b] : acc[t];
      A[id.a * NL + id.b] = v;
      A[id.b * NL + id.a] = v;
    } else if (id.kind == 1) {
      B[(id.c * NL + id.a) * NP + id.b] = plain ? al_first * refB[(id.c * NL + id.a) * NP + id.b] : acc[t];
    } else if (id.kind == 2) {
      F[id.c * NL + id.a] = acc[t];
    }
  }
  if (lane == 0 && cclass) cclass[slot] = plain ? (al_first == 1.0 ? 1 : 2) : 0;
  if (lane == 0 && estat) {
    estat[slot * 4 + 0] = fluid_volume;
    estat[slot * 4 + 1] = bmeasure;
    estat[slot * 4 + 2] = (double)nvol;
    estat[slot * 4 + 3] = (double)nbnd;
  }
}

template <int DIM, int Q>
void run_elements(const LevelGeom& g, double* eA, double* eB, double* eF, double* estat, unsigned* d_err,
                  const double* refA, const double* refB, unsigned char* cclass, cudaStream_t s,
                  const long long* cell_list = nullptr, long long nlist = 0) {
  constexpr int W = Entries<DIM, Q>::WARPS;
  const long long blocks = ((cell_list ? nlist : g.ncell) + W - 1) / W;
  if (blocks == 0) return;
  cell_elements_kernel<DIM, Q><<<(unsigned)blocks, W * 32, 0, s>>>(g, eA, eB, eF, estat, d_err, refA, refB, cclass,
                                                                   cell_list, nlist);
}

}  // namespace

cudaError_t launch_cell_elements(const LevelGeom& g, double* eA, double* eB, double* eF,
                                 double* estat, unsigned* d_err, const double* refA, const double* refB,
                                 unsigned char* cclass, cudaStream_t s) {
  if (g.dim == 2) run_elements<2, 1>(g, eA, eB, eF, estat, d_err, refA, refB, cclass, s);
  else run_elements<3, 1>(g, eA, eB, eF, estat, d_err, refA, refB, cclass, s);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_cell_elements_list(const LevelGeom& g, const long long* cells, long long ncells, double* eA,
                                      double* eB, double* eF, unsigned* d_err, cudaStream_t s) {
  if (g.dim == 2) run_elements<2, 1>(g, eA, eB, eF, nullptr, d_err, nullptr, nullptr, nullptr, s, cells, ncells);
  else run_elements<3, 1>(g, eA, eB, eF, nullptr, d_err, nullptr, nullptr, nullptr, s, cells, ncells);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_cell_elements_q2(const LevelGeom& g, double* eA, double* eB, double* eF, double* estat,
                                    unsigned* d_err, cudaStream_t s) {
  if (g.dim == 2) run_elements<2, 2>(g, eA, eB, eF, estat, d_err, nullptr, nullptr, nullptr, s);
  else run_elements<3, 2>(g, eA, eB, eF, estat, d_err, nullptr, nullptr, nullptr, s);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace fc
