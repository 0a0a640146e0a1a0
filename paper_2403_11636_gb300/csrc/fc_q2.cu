// fc_q2.cu -- the Q2-Q1 (Taylor-Hood) variant of the finite cell Stokes
// operator: Q2 velocities at the nodes of the half-spaced grid (2 n_k + 1
// per direction), Q1 pressures at the vertices, no pressure stabilisation
// (the pair is inf-sup stable).  The weak form is the paper's (Sec. 2,
// eq. stokes_weak_fcm with the symmetric Nitsche terms; element data from
// fc_geom.cu with the Q2 basis and 3-point Gauss leaves).
//
// Vector layout (ndof = (prod_k nf_k) d + prod_k (n_k + 1)): the velocity
// block, Q2 node (I, J, K) with I fastest and its d components inner, then
// the pressure at vertex (i, j, k), i fastest.
//
// Operator storage, structure of arrays (Q2 node or vertex index fastest):
//   A [5^d offsets][nq]        velocity-velocity, the same for every component
//                              (node I to node I + o, o in [-2, 2]^d);
//   B [3^d offsets][d][nq]     row (I, c) to the pressure at vertex
//                              floor(I / 2) - 1 + o, o in [0, 2]^d;
//   T [5^d offsets][d][np]     row of vertex v to velocity (2 v + o, c),
//                              o in [-2, 2]^d (the entries of B, transposed).
// Structurally absent couplings are stored as zero.  Constrained velocity
// DoFs (all components of a node on a Dirichlet face) have identity rows;
// their columns are skipped in the operator (their values live in b).
#include <math.h>

#include <algorithm>

#include "fc_internal.cuh"

namespace fc {

namespace {

template <int DIM>
struct Q2D {
  static constexpr int NV = DIM == 3 ? 27 : 9;    // Q2 functions per cell
  static constexpr int NP = 1 << DIM;             // Q1 functions per cell
  static constexpr int W5 = DIM == 3 ? 125 : 25;  // 5^d window
  static constexpr int W3 = DIM == 3 ? 27 : 9;    // 3^d window
};

__device__ __forceinline__ void q2_decode(const int* nf, int dim, long long i, int* I) {
  I[0] = (int)(i % nf[0]);
  I[1] = (int)((i / nf[0]) % nf[1]);
  I[2] = dim == 3 ? (int)(i / ((long long)nf[0] * nf[1])) : 0;
}

__device__ __forceinline__ long long q2_index(const int* nf, const int* I) {
  return I[0] + (long long)nf[0] * (I[1] + (long long)nf[1] * I[2]);
}

// ---- masks and Dirichlet values at the Q2 nodes (the presets of the Q1
// path evaluated at each node's position)
template <int DIM>
__global__ void q2_mask_kernel(LevelGeom g, Q2Grid q, unsigned char* __restrict__ mask, double* __restrict__ wfix) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= q.nq) return;
  int I[3];
  q2_decode(q.nf, DIM, i, I);
  const bool wall = I[1] == 0 || I[1] == q.nf[1] - 1 || (DIM == 3 && (I[2] == 0 || I[2] == q.nf[2] - 1));
  bool fixed = false;
  double w0 = 0.0;
  if (g.preset == 0) {
    const bool inflow = I[0] == 0;
    fixed = wall || inflow;
    if (!wall && inflow) {
      const double y = g.lo[1] + 0.5 * (double)I[1] * g.h[1];
      const double s = (y - g.lo[1]) / (g.hi[1] - g.lo[1]);
      double v = 4.0 * g.ubar * s * (1.0 - s);
      if (DIM == 3) {
        const double z = g.lo[2] + 0.5 * (double)I[2] * g.h[2];
        const double t = (z - g.lo[2]) / (g.hi[2] - g.lo[2]);
        v = v * 4.0 * t * (1.0 - t);
      }
      w0 = v;
    }
  } else if (g.preset == 1) {
    fixed = wall;
  }
  mask[i] = fixed ? (unsigned char)((1 << DIM) - 1) : 0;
  for (int c = 0; c < DIM; ++c) wfix[i * DIM + c] = c == 0 ? w0 : 0.0;
}

// ---- assembly: each stencil entry gathers its element contributions from
// the cells shared by its row and column node, in cell order
template <int DIM>
__global__ void q2_assemble_vel_kernel(LevelGeom g, Q2Grid q, const double* __restrict__ eA,
                                       const double* __restrict__ eB, double* __restrict__ A,
                                       double* __restrict__ B) {
  using D = Q2D<DIM>;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= q.nq) return;
  int I[3];
  q2_decode(q.nf, DIM, i, I);
  // cells containing node I: per direction the cells c with 2c <= I <= 2c + 2
  int clo[3] = {0, 0, 0}, chi[3] = {0, 0, 0};
  for (int k = 0; k < DIM; ++k) {
    clo[k] = max(0, (I[k] - 1) / 2);
    chi[k] = min(g.n[k] - 1, I[k] / 2);
  }
  for (int o = 0; o < D::W5; ++o) {
    const int off[3] = {o % 5 - 2, (o / 5) % 5 - 2, DIM == 3 ? o / 25 - 2 : 0};
    double s = 0.0;
    for (int cz = clo[2]; cz <= chi[2]; ++cz)
      for (int cy = clo[1]; cy <= chi[1]; ++cy)
        for (int cx = clo[0]; cx <= chi[0]; ++cx) {
          const int c[3] = {cx, cy, cz};
          int la[3], lb[3];
          bool ok = true;
          for (int k = 0; k < DIM; ++k) {
            la[k] = I[k] - 2 * c[k];
            lb[k] = la[k] + off[k];
            if (lb[k] < 0 || lb[k] > 2) ok = false;
          }
          if (!ok) continue;
          const long long cell = cx + (long long)g.n[0] * (cy + (long long)g.n[1] * cz);
          const int a = la[0] + 3 * la[1] + (DIM == 3 ? 9 * la[2] : 0);
          const int b = lb[0] + 3 * lb[1] + (DIM == 3 ? 9 * lb[2] : 0);
          s = s + eA[(cell * D::NV + a) * D::NV + b];
        }
    A[(long long)o * q.nq + i] = s;
  }
  // B: vertices floor(I/2) - 1 + o
  for (int o = 0; o < D::W3; ++o) {
    const int off[3] = {o % 3, (o / 3) % 3, DIM == 3 ? o / 9 : 0};
    int v[3] = {0, 0, 0};
    for (int k = 0; k < DIM; ++k) v[k] = I[k] / 2 - 1 + off[k];
    for (int cc = 0; cc < DIM; ++cc) {
      double s = 0.0;
      for (int cz = clo[2]; cz <= chi[2]; ++cz)
        for (int cy = clo[1]; cy <= chi[1]; ++cy)
          for (int cx = clo[0]; cx <= chi[0]; ++cx) {
            const int c[3] = {cx, cy, cz};
            int la[3], lb[3];
            bool ok = true;
            for (int k = 0; k < DIM; ++k) {
              la[k] = I[k] - 2 * c[k];
              lb[k] = v[k] - c[k];
              if (lb[k] < 0 || lb[k] > 1) ok = false;
            }
            if (!ok) continue;
            const long long cell = cx + (long long)g.n[0] * (cy + (long long)g.n[1] * cz);
            const int a = la[0] + 3 * la[1] + (DIM == 3 ? 9 * la[2] : 0);
            const int b = lb[0] + 2 * lb[1] + (DIM == 3 ? 4 * lb[2] : 0);
            s = s + eB[((cell * DIM + cc) * D::NV + a) * D::NP + b];
          }
      B[((long long)o * DIM + cc) * q.nq + i] = s;
    }
  }
}

// T: row of vertex v, column (2 v + o, c) = B of row (2 v + o, c), column v
template <int DIM>
__global__ void q2_assemble_pres_kernel(Q2Grid q, const double* __restrict__ B, double* __restrict__ T) {
  using D = Q2D<DIM>;
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= q.np) return;
  int V[3];
  q2_decode(q.nv1, DIM, v, V);
  for (int o = 0; o < D::W5; ++o) {
    const int off[3] = {o % 5 - 2, (o / 5) % 5 - 2, DIM == 3 ? o / 25 - 2 : 0};
    int I[3] = {0, 0, 0};
    bool in = true;
    for (int k = 0; k < DIM; ++k) {
      I[k] = 2 * V[k] + off[k];
      if (I[k] < 0 || I[k] >= q.nf[k]) in = false;
    }
    int ob = 0;  // offset of v in the B window of node I
    if (in) {
      int m = 1;
      for (int k = 0; k < DIM; ++k) {
        ob += (V[k] - (I[k] / 2 - 1)) * m;
        m *= 3;
      }
    }
    const long long ni = in ? q2_index(q.nf, I) : 0;
    for (int c = 0; c < DIM; ++c) T[((long long)o * DIM + c) * q.np + v] = in ? B[((long long)ob * DIM + c) * q.nq + ni] : 0.0;
  }
}

// b: the load of the free velocity rows minus the lifted Dirichlet values,
// w on constrained rows, 0 (no pressure load) minus the lifting on pressure
// rows
template <int DIM>
__global__ void q2_rhs_kernel(LevelGeom g, Q2Grid q, const double* __restrict__ eF, const double* __restrict__ A,
                              const double* __restrict__ T, const unsigned char* __restrict__ mask,
                              const double* __restrict__ wfix, double* __restrict__ b) {
  using D = Q2D<DIM>;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < q.nq) {
    const long long i = t;
    int I[3];
    q2_decode(q.nf, DIM, i, I);
    if (mask[i]) {
      for (int c = 0; c < DIM; ++c) b[i * DIM + c] = wfix[i * DIM + c];
      return;
    }
    int clo[3] = {0, 0, 0}, chi[3] = {0, 0, 0};
    for (int k = 0; k < DIM; ++k) {
      clo[k] = max(0, (I[k] - 1) / 2);
      chi[k] = min(g.n[k] - 1, I[k] / 2);
    }
    for (int c = 0; c < DIM; ++c) {
      double s = 0.0;
      for (int cz = clo[2]; cz <= chi[2]; ++cz)
        for (int cy = clo[1]; cy <= chi[1]; ++cy)
          for (int cx = clo[0]; cx <= chi[0]; ++cx) {
            const long long cell = cx + (long long)g.n[0] * (cy + (long long)g.n[1] * cz);
            const int la[3] = {I[0] - 2 * cx, I[1] - 2 * cy, DIM == 3 ? I[2] - 2 * cz : 0};
            const int a = la[0] + 3 * la[1] + (DIM == 3 ? 9 * la[2] : 0);
            s = s + eF[(cell * DIM + c) * D::NV + a];
          }
      // lifting: constrained velocity columns of the same component
      for (int o = 0; o < D::W5; ++o) {
        const int J[3] = {I[0] + o % 5 - 2, I[1] + (o / 5) % 5 - 2, DIM == 3 ? I[2] + o / 25 - 2 : 0};
        bool in = true;
        for (int k = 0; k < DIM; ++k)
          if (J[k] < 0 || J[k] >= q.nf[k]) in = false;
        if (!in) continue;
        const long long j = q2_index(q.nf, J);
        if (!mask[j]) continue;
        s = s - A[(long long)o * q.nq + i] * wfix[j * DIM + c];
      }
      b[i * DIM + c] = s;
    }
  } else if (t < q.nq + q.np) {
    const long long v = t - q.nq;
    int V[3];
    q2_decode(q.nv1, DIM, v, V);
    double s = 0.0;
    for (int o = 0; o < D::W5; ++o) {
      const int J[3] = {2 * V[0] + o % 5 - 2, 2 * V[1] + (o / 5) % 5 - 2, DIM == 3 ? 2 * V[2] + o / 25 - 2 : 0};
      bool in = true;
      for (int k = 0; k < DIM; ++k)
        if (J[k] < 0 || J[k] >= q.nf[k]) in = false;
      if (!in) continue;
      const long long j = q2_index(q.nf, J);
      if (!mask[j]) continue;
      for (int c = 0; c < DIM; ++c) s = s - T[((long long)o * DIM + c) * q.np + v] * wfix[j * DIM + c];
    }
    b[q.nq * DIM + v] = s;
  }
}

// ---- residual r = b - L x (or L x when b is null); optional unpadded
// output r and padded copies (velocity halo 4 nodes, pressure halo 1
// vertex, zero halos) for the patch gathers
template <int DIM>
__global__ void __launch_bounds__(256)
    q2_residual_kernel(Q2Grid q, const double* __restrict__ A, const double* __restrict__ B,
                       const double* __restrict__ T, const unsigned char* __restrict__ mask,
                       const double* __restrict__ x, const double* __restrict__ b, double* __restrict__ r,
                       double* __restrict__ rpv, double* __restrict__ rpp) {
  using D = Q2D<DIM>;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const double* xp = x + q.nq * DIM;
  if (t < q.nq) {
    const long long i = t;
    int I[3];
    q2_decode(q.nf, DIM, i, I);
    double acc[3] = {0.0, 0.0, 0.0};
    if (mask[i]) {
      for (int c = 0; c < DIM; ++c) acc[c] = x[i * DIM + c];
    } else {
      for (int o = 0; o < D::W5; ++o) {
        const int J[3] = {I[0] + o % 5 - 2, I[1] + (o / 5) % 5 - 2, DIM == 3 ? I[2] + o / 25 - 2 : 0};
        bool in = true;
        for (int k = 0; k < DIM; ++k)
          if (J[k] < 0 || J[k] >= q.nf[k]) in = false;
        if (!in) continue;
        const long long j = q2_index(q.nf, J);
        if (mask[j]) continue;
        const double a = A[(long long)o * q.nq + i];
        for (int c = 0; c < DIM; ++c) acc[c] = acc[c] + a * x[j * DIM + c];
      }
      for (int o = 0; o < D::W3; ++o) {
        int V[3] = {0, 0, 0};
        bool in = true;
        const int off[3] = {o % 3, (o / 3) % 3, DIM == 3 ? o / 9 : 0};
        for (int k = 0; k < DIM; ++k) {
          V[k] = I[k] / 2 - 1 + off[k];
          if (V[k] < 0 || V[k] >= q.nv1[k]) in = false;
        }
        if (!in) continue;
        const double pv = xp[q2_index(q.nv1, V)];
        for (int c = 0; c < DIM; ++c) acc[c] = acc[c] + B[((long long)o * DIM + c) * q.nq + i] * pv;
      }
    }
    long long pq = 0;
    if (rpv) {
      int P[3] = {I[0] + 4, I[1] + 4, DIM == 3 ? I[2] + 4 : 0};
      pq = P[0] + (long long)(q.nf[0] + 8) * (P[1] + (long long)(q.nf[1] + 8) * P[2]);
    }
    for (int c = 0; c < DIM; ++c) {
      const double v = b ? b[i * DIM + c] - acc[c] : acc[c];
      if (r) r[i * DIM + c] = v;
      if (rpv) rpv[pq * DIM + c] = v;
    }
  } else if (t < q.nq + q.np) {
    const long long v = t - q.nq;
    int V[3];
    q2_decode(q.nv1, DIM, v, V);
    double acc = 0.0;
    for (int o = 0; o < D::W5; ++o) {
      const int J[3] = {2 * V[0] + o % 5 - 2, 2 * V[1] + (o / 5) % 5 - 2, DIM == 3 ? 2 * V[2] + o / 25 - 2 : 0};
      bool in = true;
      for (int k = 0; k < DIM; ++k)
        if (J[k] < 0 || J[k] >= q.nf[k]) in = false;
      if (!in) continue;
      const long long j = q2_index(q.nf, J);
      if (mask[j]) continue;
      for (int c = 0; c < DIM; ++c) acc = acc + T[((long long)o * DIM + c) * q.np + v] * x[j * DIM + c];
    }
    const double val = b ? b[q.nq * DIM + v] - acc : acc;
    if (r) r[q.nq * DIM + v] = val;
    if (rpp) {
      const int P[3] = {V[0] + 1, V[1] + 1, DIM == 3 ? V[2] + 1 : 0};
      rpp[P[0] + (long long)(q.nv1[0] + 2) * (P[1] + (long long)(q.nv1[1] + 2) * P[2])] = val;
    }
  }
}

// ---- transfers: Q2 interpolation of velocities (nested spaces), Q1 of
// pressures; R = P^T, constrained coarse DoFs zeroed after restriction,
// constrained fine DoFs untouched by prolongation
__device__ __forceinline__ void q2_fine_w(int F, int nc, int* base, double* w) {
  int m = F / 4;
  if (m >= nc) m = nc - 1;
  const double t = (double)(F - 4 * m) / 4.0;
  w[0] = (1.0 - t) * (1.0 - 2.0 * t);
  w[1] = 4.0 * t * (1.0 - t);
  w[2] = t * (2.0 * t - 1.0);
  *base = 2 * m;
}

template <int DIM>
__global__ void q2_prolong_kernel(Q2Grid f, Q2Grid c, const unsigned char* __restrict__ fmask,
                                  const double* __restrict__ ec, double* __restrict__ xf) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < f.nq) {
    if (fmask[t]) return;
    int I[3];
    q2_decode(f.nf, DIM, t, I);
    int base[3] = {0, 0, 0};
    double w[3][3] = {{1, 0, 0}, {1, 0, 0}, {1, 0, 0}};
    for (int k = 0; k < DIM; ++k) q2_fine_w(I[k], c.nv1[k] - 1, &base[k], w[k]);
    double s[3] = {0.0, 0.0, 0.0};
    for (int tz = 0; tz < (DIM == 3 ? 3 : 1); ++tz)
      for (int ty = 0; ty < 3; ++ty)
        for (int tx = 0; tx < 3; ++tx) {
          const double wt = w[0][tx] * w[1][ty] * (DIM == 3 ? w[2][tz] : 1.0);
          if (wt == 0.0) continue;
          const int J[3] = {base[0] + tx, base[1] + ty, DIM == 3 ? base[2] + tz : 0};
          const long long j = q2_index(c.nf, J);
          for (int cc = 0; cc < DIM; ++cc) s[cc] = s[cc] + wt * ec[j * DIM + cc];
        }
    for (int cc = 0; cc < DIM; ++cc) xf[t * DIM + cc] = xf[t * DIM + cc] + s[cc];
  } else if (t < f.nq + f.np) {
    const long long v = t - f.nq;
    int V[3];
    q2_decode(f.nv1, DIM, v, V);
    double s = 0.0;
    for (int bits = 0; bits < (1 << DIM); ++bits) {
      double wt = 1.0;
      int U[3] = {0, 0, 0};
      bool dup = false;
      for (int k = 0; k < DIM; ++k) {
        const int lo = V[k] / 2, hi = (V[k] + 1) / 2, bit = (bits >> k) & 1;
        if (lo == hi && bit) dup = true;
        U[k] = bit ? hi : lo;
        wt = wt * (lo == hi ? 1.0 : 0.5);
      }
      if (dup) continue;
      s = s + wt * ec[c.nq * DIM + q2_index(c.nv1, U)];
    }
    xf[f.nq * DIM + v] = xf[f.nq * DIM + v] + s;
  }
}

// restriction as a gather over the fine DoFs that interpolate from each
// coarse DoF (the same weights as the prolongation, transposed)
template <int DIM>
__global__ void q2_restrict_kernel(Q2Grid f, Q2Grid c, const unsigned char* __restrict__ cmask,
                                   const double* __restrict__ rf, double* __restrict__ bc) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < c.nq) {
    int J[3];
    q2_decode(c.nf, DIM, t, J);
    double s[3] = {0.0, 0.0, 0.0};
    if (!cmask[t]) {
      // fine Q2 nodes F with F / 4 in the coarse cells touching J: F in [2J - 4, 2J + 4]
      int flo[3] = {0, 0, 0}, fhi[3] = {0, 0, 0};
      for (int k = 0; k < DIM; ++k) {
        flo[k] = max(0, 2 * J[k] - 4);
        fhi[k] = min(f.nf[k] - 1, 2 * J[k] + 4);
      }
      for (int Fz = flo[2]; Fz <= fhi[2]; ++Fz)
        for (int Fy = flo[1]; Fy <= fhi[1]; ++Fy)
          for (int Fx = flo[0]; Fx <= fhi[0]; ++Fx) {
            const int F[3] = {Fx, Fy, Fz};
            double wt = 1.0;
            for (int k = 0; k < DIM; ++k) {
              int base;
              double w[3];
              q2_fine_w(F[k], c.nv1[k] - 1, &base, w);
              const int l = J[k] - base;
              wt = (l >= 0 && l <= 2) ? wt * w[l] : 0.0;
            }
            if (wt == 0.0) continue;
            const long long fi = q2_index(f.nf, F);
            for (int cc = 0; cc < DIM; ++cc) s[cc] = s[cc] + wt * rf[fi * DIM + cc];
          }
    }
    for (int cc = 0; cc < DIM; ++cc) bc[t * DIM + cc] = s[cc];
  } else if (t < c.nq + c.np) {
    const long long u = t - c.nq;
    int U[3];
    q2_decode(c.nv1, DIM, u, U);
    double s = 0.0;
    int flo[3] = {0, 0, 0}, fhi[3] = {0, 0, 0};
    for (int k = 0; k < DIM; ++k) {
      flo[k] = max(0, 2 * U[k] - 1);
      fhi[k] = min(f.nv1[k] - 1, 2 * U[k] + 1);
    }
    for (int vz = flo[2]; vz <= fhi[2]; ++vz)
      for (int vy = flo[1]; vy <= fhi[1]; ++vy)
        for (int vx = flo[0]; vx <= fhi[0]; ++vx) {
          const int V[3] = {vx, vy, vz};
          double wt = 1.0;
          for (int k = 0; k < DIM; ++k) wt = wt * (V[k] == 2 * U[k] ? 1.0 : 0.5);
          s = s + wt * rf[f.nq * DIM + q2_index(f.nv1, V)];
        }
    bc[c.nq * DIM + u] = s;
  }
}

// dense coarsest operator, row-major (rows and columns in the vector layout)
template <int DIM>
__global__ void q2_dense_kernel(Q2Grid q, const double* __restrict__ A, const double* __restrict__ B,
                                const double* __restrict__ T, const unsigned char* __restrict__ mask,
                                double* __restrict__ M) {
  using D = Q2D<DIM>;
  const long long n = q.nq * DIM + q.np;
  const long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  for (long long c = 0; c < n; ++c) M[row * n + c] = 0.0;
  if (row < q.nq * DIM) {
    const long long i = row / DIM;
    const int c = (int)(row % DIM);
    if (mask[i]) { M[row * n + row] = 1.0; return; }
    int I[3];
    q2_decode(q.nf, DIM, i, I);
    for (int o = 0; o < D::W5; ++o) {
      const int J[3] = {I[0] + o % 5 - 2, I[1] + (o / 5) % 5 - 2, DIM == 3 ? I[2] + o / 25 - 2 : 0};
      bool in = true;
      for (int k = 0; k < DIM; ++k)
        if (J[k] < 0 || J[k] >= q.nf[k]) in = false;
      if (!in) continue;
      const long long j = q2_index(q.nf, J);
      if (mask[j]) continue;
      M[row * n + j * DIM + c] = A[(long long)o * q.nq + i];
    }
    for (int o = 0; o < D::W3; ++o) {
      int V[3] = {0, 0, 0};
      bool in = true;
      const int off[3] = {o % 3, (o / 3) % 3, DIM == 3 ? o / 9 : 0};
      for (int k = 0; k < DIM; ++k) {
        V[k] = I[k] / 2 - 1 + off[k];
        if (V[k] < 0 || V[k] >= q.nv1[k]) in = false;
      }
      if (!in) continue;
      M[row * n + q.nq * DIM + q2_index(q.nv1, V)] = B[((long long)o * DIM + c) * q.nq + i];
    }
  } else {
    const long long v = row - q.nq * DIM;
    int V[3];
    q2_decode(q.nv1, DIM, v, V);
    for (int o = 0; o < D::W5; ++o) {
      const int J[3] = {2 * V[0] + o % 5 - 2, 2 * V[1] + (o / 5) % 5 - 2, DIM == 3 ? 2 * V[2] + o / 25 - 2 : 0};
      bool in = true;
      for (int k = 0; k < DIM; ++k)
        if (J[k] < 0 || J[k] >= q.nf[k]) in = false;
      if (!in) continue;
      const long long j = q2_index(q.nf, J);
      if (mask[j]) continue;
      for (int c = 0; c < DIM; ++c) M[row * n + j * DIM + c] = T[((long long)o * DIM + c) * q.np + v];
    }
  }
}

unsigned blocks_for(long long n) { return (unsigned)((n + 255) / 256); }

}  // namespace

Q2Grid make_q2grid(const LevelGeom& g) {
  Q2Grid q;
  q.nq = 1;
  q.np = 1;
  for (int k = 0; k < 3; ++k) {
    q.nf[k] = k < g.dim ? 2 * g.n[k] + 1 : 1;
    q.nv1[k] = k < g.dim ? g.n[k] + 1 : 1;
    q.nq *= q.nf[k];
    q.np *= q.nv1[k];
  }
  return q;
}

cudaError_t launch_q2_masks(const LevelGeom& g, const Q2Grid& q, unsigned char* mask, double* wfix, cudaStream_t s) {
  if (g.dim == 2) q2_mask_kernel<2><<<blocks_for(q.nq), 256, 0, s>>>(g, q, mask, wfix);
  else q2_mask_kernel<3><<<blocks_for(q.nq), 256, 0, s>>>(g, q, mask, wfix);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_q2_assemble(const LevelGeom& g, const Q2Grid& q, const double* eA, const double* eB,
                               const double* eF, const unsigned char* mask, const double* wfix, double* A,
                               double* B, double* T, double* b, cudaStream_t s) {
  if (g.dim == 2) {
    q2_assemble_vel_kernel<2><<<blocks_for(q.nq), 256, 0, s>>>(g, q, eA, eB, A, B);
    q2_assemble_pres_kernel<2><<<blocks_for(q.np), 256, 0, s>>>(q, B, T);
    if (b) q2_rhs_kernel<2><<<blocks_for(q.nq + q.np), 256, 0, s>>>(g, q, eF, A, T, mask, wfix, b);
  } else {
    q2_assemble_vel_kernel<3><<<blocks_for(q.nq), 256, 0, s>>>(g, q, eA, eB, A, B);
    q2_assemble_pres_kernel<3><<<blocks_for(q.np), 256, 0, s>>>(q, B, T);
    if (b) q2_rhs_kernel<3><<<blocks_for(q.nq + q.np), 256, 0, s>>>(g, q, eF, A, T, mask, wfix, b);
  }
  note_launches(b ? 3 : 2);
  return cudaGetLastError();
}

cudaError_t launch_q2_residual(int dim, const Q2Grid& q, const double* A, const double* B, const double* T,
                               const unsigned char* mask, const double* x, const double* b, double* r, double* rpv,
                               double* rpp, cudaStream_t s) {
  if (dim == 2) q2_residual_kernel<2><<<blocks_for(q.nq + q.np), 256, 0, s>>>(q, A, B, T, mask, x, b, r, rpv, rpp);
  else q2_residual_kernel<3><<<blocks_for(q.nq + q.np), 256, 0, s>>>(q, A, B, T, mask, x, b, r, rpv, rpp);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_q2_prolong_add(int dim, const Q2Grid& f, const Q2Grid& c, const unsigned char* fmask,
                                  const double* ec, double* xf, cudaStream_t s) {
  if (dim == 2) q2_prolong_kernel<2><<<blocks_for(f.nq + f.np), 256, 0, s>>>(f, c, fmask, ec, xf);
  else q2_prolong_kernel<3><<<blocks_for(f.nq + f.np), 256, 0, s>>>(f, c, fmask, ec, xf);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_q2_restrict(int dim, const Q2Grid& f, const Q2Grid& c, const unsigned char* cmask,
                               const double* rf, double* bc, cudaStream_t s) {
  if (dim == 2) q2_restrict_kernel<2><<<blocks_for(c.nq + c.np), 256, 0, s>>>(f, c, cmask, rf, bc);
  else q2_restrict_kernel<3><<<blocks_for(c.nq + c.np), 256, 0, s>>>(f, c, cmask, rf, bc);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_q2_dense(int dim, const Q2Grid& q, const double* A, const double* B, const double* T,
                            const unsigned char* mask, double* M, cudaStream_t s) {
  const long long n = q.nq * dim + q.np;
  if (dim == 2) q2_dense_kernel<2><<<blocks_for(n), 256, 0, s>>>(q, A, B, T, mask, M);
  else q2_dense_kernel<3><<<blocks_for(n), 256, 0, s>>>(q, A, B, T, mask, M);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace fc
