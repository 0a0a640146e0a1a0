// fc_patch.cu -- the restricted additive patch smoother (paper Sec. 3.1).
//
// Patch S_i of pressure node i: velocity DoFs of the 5^d nodes around i and
// pressure DoFs of the 3^d nodes around i (the pressures sharing a cell with
// p_i and the velocities coupled to them through B^T, taken structurally),
// without constrained or out-of-grid DoFs.  L_i = R_i L R_i^T is
//   [ A_i  B_i ]      A_i = blockdiag(K, .., K): the velocity form acts on
//   [ B_i' C_i ]      each component alike (eq. stokes_disc_weak_fcm_2).
// The local solve is exact (Sec. 3.1.2).  It is taken on the symmetrically
// equilibrated block D L_i D (D = |diag L_i|^{-1/2}) so that it reaches
// machine accuracy although alpha-scaled and unscaled rows differ by many
// orders of magnitude, and through the block elimination
//   K~ = LU (partial pivoting), W~_c = K~^{-1} B~_c,
//   S~ = C~ - sum_c B~_c' W~_c  (LU, partial pivoting)
// instead of a dense LU of the whole (5^d d + 3^d)-square block: 4.4 instead
// of 43 MFLOP per 3D patch.
//
// One CTA per patch builds the block factors in shared memory and then
//   mode 0 (cache_inverse): writes the 1+d owned rows of L_i^{-1} (the rows
//          that R~_i^T keeps, Sec. 3.1.2);
//   mode 1 (cache_matrix):  writes the block factors for later solves;
//   mode 2 (cache_none):    solves with the gathered residual at once and
//          updates the owned DoFs (nothing stored).
#include <cuda_bf16.h>
#include <stdlib.h>
#include <math.h>

#include <algorithm>

#include "fc_internal.cuh"

namespace fc {

namespace {

template <int DIM>
struct PatchDims {
  static constexpr int NU = DIM == 3 ? 125 : 25;   // velocity nodes (5^d)
  static constexpr int NP = DIM == 3 ? 27 : 9;     // pressure nodes (3^d)
  static constexpr int ND = DIM + 1;
  static constexpr int SP = 2 * DIM + 2;
  static constexpr int NSLOT = NU * DIM + NP;
  static constexpr int NCOL = DIM * NP + 1 + DIM;  // B columns, e_centre, residual columns
  // factor record (doubles): K LU (column-major), W (col-major), S LU, du, dp
  static constexpr int REC = NU * NU + DIM * NP * NU + NP * NP + NU + NP;
  static constexpr int RECI = NU + NP;
};

template <int DIM>
__device__ __forceinline__ void vel_off(int v, int* o) {
  o[0] = v % 5 - 2;
  o[1] = (v / 5) % 5 - 2;
  o[2] = DIM == 3 ? v / 25 - 2 : 0;
}
template <int DIM>
__device__ __forceinline__ void prs_off(int p, int* o) {
  o[0] = p % 3 - 1;
  o[1] = (p / 3) % 3 - 1;
  o[2] = DIM == 3 ? p / 9 - 1 : 0;
}
template <int DIM>
__device__ __forceinline__ int nb_index(const int* d) {
  return (d[0] + 1) + 3 * (d[1] + 1) + (DIM == 3 ? 9 * (d[2] + 1) : 0);
}

// CTA-cooperative LU with partial pivoting (max |a|, lowest row on ties),
// row-major n x n with leading dimension ld.
__device__ void cta_lu(double* A, int n, int ld, int* piv, int* s_flag) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  for (int k = 0; k < n; ++k) {
    if (warp == 0) {
      double best = -1.0;
      int bi = k;
      for (int r = k + lane; r < n; r += 32) {
        double v = fabs(A[r * ld + k]);
        if (v > best) { best = v; bi = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_down_sync(0xffffffffu, best, o);
        int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if (lane == 0) {
        piv[k] = bi;
        if (best == 0.0) *s_flag = 1;
      }
    }
    __syncthreads();
    int p = piv[k];
    if (p != k)
      for (int c = tid; c < n; c += nt) {
        double t = A[k * ld + c];
        A[k * ld + c] = A[p * ld + c];
        A[p * ld + c] = t;
      }
    __syncthreads();
    double d = A[k * ld + k];
    for (int r = k + 1 + tid; r < n; r += nt) A[r * ld + k] = d != 0.0 ? A[r * ld + k] / d : 0.0;
    __syncthreads();
    int m = n - k - 1;
    for (int t = tid; t < m * m; t += nt) {
      int r = k + 1 + t / m, c = k + 1 + t % m;
      A[r * ld + c] = A[r * ld + c] - A[r * ld + k] * A[k * ld + c];
    }
    __syncthreads();
  }
}

// z <- A^{-1} z with the row-major LU and pivots (one thread)
__device__ void lu_solve_vec(const double* A, int n, int ld, const int* piv, double* z) {
  for (int k = 0; k < n; ++k) {
    int p = piv[k];
    if (p != k) { double t = z[k]; z[k] = z[p]; z[p] = t; }
  }
  for (int r = 0; r < n; ++r) {
    double s = z[r];
    for (int c = 0; c < r; ++c) s = s - A[r * ld + c] * z[c];
    z[r] = s;
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = z[r];
    for (int c = r + 1; c < n; ++c) s = s - A[r * ld + c] * z[c];
    z[r] = s / A[r * ld + r];
  }
}

// W <- A^{-1} W for ncol right-hand sides (column-major, length n) with the
// row-major LU and pivots of A, all threads of the CTA cooperating: the row
// swaps per column, then column-oriented forward and back substitution with
// one barrier per pivot step (each step updates every column at once).
__device__ void cta_lu_solve_multi(const double* A, int n, const int* piv, double* W, int ncol) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int col = tid; col < ncol; col += nt) {
    double* z = W + col * n;
    for (int k = 0; k < n; ++k) {
      int p = piv[k];
      if (p != k) { double t = z[k]; z[k] = z[p]; z[p] = t; }
    }
  }
  __syncthreads();
  for (int k = 0; k < n - 1; ++k) {
    const int m = n - 1 - k;
    for (int t = tid; t < m * ncol; t += nt) {
      const int col = t / m, r = k + 1 + t % m;
      W[col * n + r] = W[col * n + r] - A[r * n + k] * W[col * n + k];
    }
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {
    const double d = A[k * n + k];
    for (int col = tid; col < ncol; col += nt) W[col * n + k] = W[col * n + k] / d;
    __syncthreads();
    for (int t = tid; t < k * ncol; t += nt) {
      const int col = t / k, r = t % k;
      W[col * n + r] = W[col * n + r] - A[r * n + k] * W[col * n + k];
    }
    __syncthreads();
  }
}

template <int DIM, int MODE>
__global__ void __launch_bounds__(1024)
    patch_factor_kernel(LevelGeom g, const double* __restrict__ st, const unsigned char* __restrict__ mask,
                        double omega, double* __restrict__ coef, double* __restrict__ fac,
                        int* __restrict__ fpiv, const double* __restrict__ rpad, double* __restrict__ x,
                        unsigned* __restrict__ d_err, const int* __restrict__ work,
                        const int* __restrict__ outidx) {
  using P = PatchDims<DIM>;
  constexpr int NU = P::NU, NP = P::NP, ND = P::ND, SP = P::SP, NCOL = P::NCOL;
  extern __shared__ double smem[];
  double* K = smem;                 // NU x NU row-major
  double* W = K + NU * NU;          // NCOL columns of length NU
  double* S = W + NCOL * NU;        // NP x NP row-major
  double* du = S + NP * NP;         // NU
  double* dp = du + NU;             // NP
  double* rp = dp + NP;             // NP: scaled pressure residual (mode 2) / scratch
  double* zp = rp + NP;             // (DIM+1) x NP scratch
  double* yo = zp + (DIM + 1) * NP; // ND owned results
  int* pivK = (int*)(yo + ND);      // NU
  int* pivS = pivK + NU;            // NP
  long long* nodeU = (long long*)(((uintptr_t)(pivS + NP) + 7) & ~(uintptr_t)7);  // NU
  long long* nodeP = nodeU + NU;    // NP
  unsigned char* au = (unsigned char*)(nodeP + NP);  // NU
  unsigned char* ap = au + NU;      // NP
  __shared__ int s_flag;

  const int tid = threadIdx.x, nt = blockDim.x;
  // block blockIdx.x factors patch work[blockIdx.x] (all patches in order
  // without a work list) and stores into block blockIdx.x
  const long long widx = blockIdx.x;
  const long long i = work ? work[widx] : widx;
  const int ia[3] = {(int)(i % g.nn[0]), (int)((i / g.nn[0]) % g.nn[1]),
                     DIM == 3 ? (int)(i / ((long long)g.nn[0] * g.nn[1])) : 0};
  if (tid == 0) s_flag = 0;

  // ---- patch DoFs
  for (int v = tid; v < NU; v += nt) {
    int o[3];
    vel_off<DIM>(v, o);
    int b0 = ia[0] + o[0], b1 = ia[1] + o[1], b2 = ia[2] + o[2];
    bool in = b0 >= 0 && b0 <= g.n[0] && b1 >= 0 && b1 <= g.n[1] && (DIM == 2 || (b2 >= 0 && b2 <= g.n[2]));
    long long bn = in ? b0 + (long long)g.nn[0] * (b1 + (long long)g.nn[1] * b2) : -1;
    nodeU[v] = bn;
    au[v] = (unsigned char)(in && !(mask[bn] & 1));
  }
  for (int p = tid; p < NP; p += nt) {
    int o[3];
    prs_off<DIM>(p, o);
    int b0 = ia[0] + o[0], b1 = ia[1] + o[1], b2 = ia[2] + o[2];
    bool in = b0 >= 0 && b0 <= g.n[0] && b1 >= 0 && b1 <= g.n[1] && (DIM == 2 || (b2 >= 0 && b2 <= g.n[2]));
    nodeP[p] = in ? b0 + (long long)g.nn[0] * (b1 + (long long)g.nn[1] * b2) : -1;
    ap[p] = (unsigned char)in;
  }
  __syncthreads();

  // ---- gather K, B (into W columns), C (into S)
  for (int e = tid; e < NU * NU; e += nt) {
    int v = e / NU, w = e % NU;
    double val = 0.0;
    if (au[v] && au[w]) {
      int ov[3], ow[3], d[3];
      vel_off<DIM>(v, ov);
      vel_off<DIM>(w, ow);
      bool adj = true;
      for (int k = 0; k < 3; ++k) { d[k] = ow[k] - ov[k]; if (d[k] < -1 || d[k] > 1) adj = false; }
      if (adj) val = st[((long long)nb_index<DIM>(d) * SP) * g.nnodes + nodeU[v]];
    } else if (v == w) {
      val = 1.0;
    }
    K[e] = val;
  }
  for (int e = tid; e < DIM * NP * NU; e += nt) {
    int col = e / NU, v = e % NU, c = col / NP, p = col % NP;
    double val = 0.0;
    if (au[v] && ap[p]) {
      int ov[3], op[3], d[3];
      vel_off<DIM>(v, ov);
      prs_off<DIM>(p, op);
      bool adj = true;
      for (int k = 0; k < 3; ++k) { d[k] = op[k] - ov[k]; if (d[k] < -1 || d[k] > 1) adj = false; }
      if (adj) val = st[((long long)nb_index<DIM>(d) * SP + 1 + c) * g.nnodes + nodeU[v]];
    }
    W[e] = val;
  }
  for (int e = tid; e < NP * NP; e += nt) {
    int p = e / NP, q = e % NP;
    double val = 0.0;
    if (ap[p] && ap[q]) {
      int op[3], oq[3], d[3];
      prs_off<DIM>(p, op);
      prs_off<DIM>(q, oq);
      bool adj = true;
      for (int k = 0; k < 3; ++k) { d[k] = oq[k] - op[k]; if (d[k] < -1 || d[k] > 1) adj = false; }
      if (adj) val = st[((long long)nb_index<DIM>(d) * SP + 1 + 2 * DIM) * g.nnodes + nodeP[p]];
    } else if (p == q) {
      val = 1.0;
    }
    S[e] = val;
  }
  __syncthreads();
  for (int v = tid; v < NU; v += nt) {
    double a = fabs(K[v * NU + v]);
    du[v] = (au[v] && a > 0.0) ? 1.0 / sqrt(a) : 1.0;
  }
  for (int p = tid; p < NP; p += nt) {
    double a = fabs(S[p * NP + p]);
    dp[p] = (ap[p] && a > 0.0) ? 1.0 / sqrt(a) : 1.0;
  }
  __syncthreads();
  // ---- equilibrate; extra right-hand sides: e_centre and (mode 2) D r
  const int v0 = DIM == 3 ? 62 : 12, p0 = DIM == 3 ? 13 : 4;
  for (int e = tid; e < NU * NU; e += nt) K[e] = du[e / NU] * K[e] * du[e % NU];
  for (int e = tid; e < DIM * NP * NU; e += nt) W[e] = du[e % NU] * W[e] * dp[(e / NU) % NP];
  for (int e = tid; e < NP * NP; e += nt) S[e] = dp[e / NP] * S[e] * dp[e % NP];
  for (int v = tid; v < NU; v += nt) {
    W[(DIM * NP) * NU + v] = v == v0 ? 1.0 : 0.0;
    for (int c = 0; c < DIM; ++c) {
      double rv = 0.0;
      if (MODE == 2 && au[v]) {
        int o[3];
        vel_off<DIM>(v, o);
        long long pn = pad_node(g, ia[0] + o[0], ia[1] + o[1], ia[2] + o[2]);
        rv = du[v] * rpad[pn * ND + c];
      }
      W[(DIM * NP + 1 + c) * NU + v] = rv;
    }
  }
  for (int p = tid; p < NP; p += nt) {
    double rv = 0.0;
    if (MODE == 2 && ap[p]) {
      int o[3];
      prs_off<DIM>(p, o);
      long long pn = pad_node(g, ia[0] + o[0], ia[1] + o[1], ia[2] + o[2]);
      rv = dp[p] * rpad[pn * ND + DIM];
    }
    rp[p] = rv;
  }
  __syncthreads();

  // ---- K~ = LU
  cta_lu(K, NU, NU, pivK, &s_flag);
  // ---- W~ = K~^{-1} [B~ | e_centre | D r_u]
  const int ncol = MODE == 2 ? NCOL : DIM * NP + 1;
  cta_lu_solve_multi(K, NU, pivK, W, ncol);
  __syncthreads();
  // ---- S~ = C~ - sum_c B~_c^T W~_c, B~ re-read from the operator (27 / 9
  // velocity nodes are adjacent to a pressure node)
  for (int e = tid; e < NP * NP; e += nt) {
    int p = e / NP, q = e % NP;
    double s = S[e];
    if (ap[p]) {
      int op[3];
      prs_off<DIM>(p, op);
      for (int t = 0; t < (DIM == 3 ? 27 : 9); ++t) {
        int d[3] = {t % 3 - 1, (t / 3) % 3 - 1, DIM == 3 ? t / 9 - 1 : 0};
        int ov[3] = {op[0] + d[0], op[1] + d[1], op[2] + d[2]};
        int v = (ov[0] + 2) + 5 * (ov[1] + 2) + (DIM == 3 ? 25 * (ov[2] + 2) : 0);
        if (!au[v]) continue;
        int dvp[3] = {-d[0], -d[1], -d[2]};  // pressure node relative to velocity node
        long long base = (long long)nb_index<DIM>(dvp) * SP;
        for (int c = 0; c < DIM; ++c) {
          double bt = du[v] * st[(base + 1 + c) * g.nnodes + nodeU[v]] * dp[p];
          s = s - bt * W[(c * NP + q) * NU + v];
        }
      }
    }
    S[e] = s;
  }
  __syncthreads();
  cta_lu(S, NP, NP, pivS, &s_flag);
  if (s_flag) {
    if (tid == 0) atomicOr(d_err, kErrSingularPatch);
  }

  if (MODE == 0) {
    // ---- owned rows: row k of L_i^{-1} = d_k (L~^{-1} e_k)^T D
    // z_p for each owned k: velocity c -> -S~^{-1} (row v0 of W~_c); pressure -> S~^{-1} e_p0
    if (tid < ND) {
      double* z = zp + tid * NP;
      for (int q = 0; q < NP; ++q)
        z[q] = tid < DIM ? -W[(tid * NP + q) * NU + v0] : (q == p0 ? 1.0 : 0.0);
      lu_solve_vec(S, NP, NP, pivS, z);
    }
    __syncthreads();
    double* out = coef + (outidx ? (long long)outidx[widx] : widx) * P::NSLOT * ND;
    for (int j = tid; j < P::NSLOT; j += nt) {
      double vals[ND];
      if (j < NU * DIM) {
        int v = j / DIM, c2 = j % DIM;
        for (int k = 0; k < ND; ++k) {
          double z = 0.0;
          if (au[v]) {
            double s = (k == c2) ? W[(DIM * NP) * NU + v] : 0.0;
            for (int q = 0; q < NP; ++q) s = s - W[(c2 * NP + q) * NU + v] * zp[k * NP + q];
            z = s;
          }
          bool own_ok = k < DIM ? au[v0] != 0 : true;
          double dk = k < DIM ? du[v0] : dp[p0];
          vals[k] = (own_ok && au[v]) ? dk * z * du[v] : 0.0;
        }
      } else {
        int p = j - NU * DIM;
        for (int k = 0; k < ND; ++k) {
          bool own_ok = k < DIM ? au[v0] != 0 : true;
          double dk = k < DIM ? du[v0] : dp[p0];
          vals[k] = (own_ok && ap[p]) ? dk * zp[k * NP + p] * dp[p] : 0.0;
        }
      }
      for (int k = 0; k < ND; ++k) out[(long long)j * ND + k] = vals[k];
    }
  } else if (MODE == 1) {
    // ---- store the block factors: K~ LU column-major, W~ (B~ columns),
    // S~ LU row-major, du, dp; pivots
    double* rec = fac + widx * P::REC;
    for (int e = tid; e < NU * NU; e += nt) {
      int c = e / NU, r = e % NU;
      rec[e] = K[r * NU + c];
    }
    for (int e = tid; e < DIM * NP * NU; e += nt) rec[NU * NU + e] = W[e];
    for (int e = tid; e < NP * NP; e += nt) rec[NU * NU + DIM * NP * NU + e] = S[e];
    for (int v = tid; v < NU; v += nt) rec[NU * NU + DIM * NP * NU + NP * NP + v] = du[v];
    for (int p = tid; p < NP; p += nt) rec[NU * NU + DIM * NP * NU + NP * NP + NU + p] = dp[p];
    int* ip = fpiv + widx * P::RECI;
    for (int v = tid; v < NU; v += nt) ip[v] = pivK[v];
    for (int p = tid; p < NP; p += nt) ip[NU + p] = pivS[p];
  } else {
    // ---- solve with the gathered residual: t = r~_p - sum_c W~_c^T r~_c,
    // z_p = S~^{-1} t, owned u_c = (K~^{-1} r~_c)[v0] - W~_c[v0,:] z_p
    for (int q = tid; q < NP; q += nt) {
      double s = rp[q];
      for (int c = 0; c < DIM; ++c) {
        // W~_c^T r~_c = B~_c^T (K~^{-1} r~_c) because K~ is symmetric; the
        // residual columns were solved in place, B~ is re-read.
        int op[3];
        prs_off<DIM>(q, op);
        if (!ap[q]) continue;
        for (int t = 0; t < (DIM == 3 ? 27 : 9); ++t) {
          int d[3] = {t % 3 - 1, (t / 3) % 3 - 1, DIM == 3 ? t / 9 - 1 : 0};
          int ov[3] = {op[0] + d[0], op[1] + d[1], op[2] + d[2]};
          int v = (ov[0] + 2) + 5 * (ov[1] + 2) + (DIM == 3 ? 25 * (ov[2] + 2) : 0);
          if (!au[v]) continue;
          int dvp[3] = {-d[0], -d[1], -d[2]};
          double bt = du[v] * st[((long long)nb_index<DIM>(dvp) * SP + 1 + c) * g.nnodes + nodeU[v]] * dp[q];
          s = s - bt * W[(DIM * NP + 1 + c) * NU + v];
        }
      }
      zp[q] = s;
    }
    __syncthreads();
    if (tid == 0) {
      lu_solve_vec(S, NP, NP, pivS, zp);
      for (int c = 0; c < DIM; ++c) {
        double s = W[(DIM * NP + 1 + c) * NU + v0];
        for (int q = 0; q < NP; ++q) s = s - W[(c * NP + q) * NU + v0] * zp[q];
        yo[c] = du[v0] * s;
      }
      yo[DIM] = dp[p0] * zp[p0];
      unsigned char m = mask[i];
      long long pc = pad_node(g, ia[0], ia[1], ia[2]);
      for (int c = 0; c < DIM; ++c) {
        if ((m >> c) & 1) x[i * ND + c] = x[i * ND + c] + rpad[pc * ND + c];
        else x[i * ND + c] = x[i * ND + c] + omega * yo[c];
      }
      x[i * ND + DIM] = x[i * ND + DIM] + omega * yo[DIM];
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 owned rows of a 3D patch (cache_inverse) by a banded LDL^T of the
// velocity block.  In lattice order (x fastest) a velocity node of the 5^3
// box couples only to nodes at most 1 + 5 + 25 = 31 positions away, so the
// equilibrated K~ = D K D is a band matrix of half-bandwidth 31.  When K~ is
// positive definite (the velocity form is coercive on the patch) it factors
// as K~ = L diag(d) L^T without pivoting and L keeps the band.  Then, per
// velocity component c,
//   Y_c = L^{-1} B~_c        (27 columns, each from its first structural
//                             nonzero row),
//   Yh_c = diag(d)^{-1/2} Y_c,   S~ -= Yh_c' Yh_c,   w_c = Yh_c' sh,
// with sh = diag(d)^{-1/2} L^{-1} e_centre, which gives the Schur complement
// S~ = C~ - sum_c B~_c' K~^{-1} B~_c and the centre rows w_c of
// W~_c = K~^{-1} B~_c without forming W~.  The owned columns of L~^{-1}
// (rows, by symmetry) follow from z_p (S~ z_p = -w_k for the velocity rows,
// e_p0 for the pressure row) and the 12 banded solves
//   z_u(c') = K~^{-1} (delta_{k c'} e_centre - B~_c' z_p).
// About 0.55 M FMA per patch against 2.2 M for the dense elimination of
// patch_factor_kernel, with the same result up to rounding.  The band solves
// run one column per warp: lane l carries entry k + l of the column through
// step k, so a step is one FMA per lane and two shuffles, no block barrier.
// A pivot d_k <= dmin (1e-14: K~ not positive definite to working accuracy)
// puts the patch on a redo list for the pivoted dense LU (patch_factor_kernel
// mode 0 with an output index).  FC_LDL_MIN_PIVOT overrides dmin (a value
// above 1 sends every patch to the dense LU, which validation runs use to
// compare the two paths).
constexpr int kBand = 32;       // stored band per column: diagonal + 31 below
constexpr int kTri = 31 * 32 / 2;  // trailing-update pairs (l, m), 1 <= m <= l <= 31

// y <- L^{-1} y for the unit lower band factor (column-major band Lb[k *
// kBand + l] = L(k + l, k)), rows f .. n-1 (rows above f are zero), by one
// warp.
__device__ __forceinline__ void band_forward(const double* Lb, double* y, int n, int f, int lane) {
  double v = f + lane < n ? y[f + lane] : 0.0;
  for (int k = f; k < n; ++k) {
    const double yk = __shfl_sync(0xffffffffu, v, 0);
    if (lane == 0) y[k] = yk;
    v = fma(-Lb[k * kBand + lane], yk, v);  // lane 0's result is shifted out
    v = __shfl_down_sync(0xffffffffu, v, 1);
    if (lane == 31) v = k + 32 < n ? y[k + 32] : 0.0;
  }
}

// y <- L^{-T} y (unit upper band L^T), by one warp: lane l carries entry
// i - l through step i (i = n-1 .. 0).
__device__ __forceinline__ void band_backward(const double* Lb, double* y, int n, int lane) {
  double v = n - 1 - lane >= 0 ? y[n - 1 - lane] : 0.0;
  for (int i = n - 1; i >= 0; --i) {
    const double xi = __shfl_sync(0xffffffffu, v, 0);
    if (lane == 0) y[i] = xi;
    const int r = i - lane;
    const double lv = lane > 0 && r >= 0 ? Lb[r * kBand + lane] : 0.0;  // L(i, i - l)
    v = fma(-lv, xi, v);
    v = __shfl_down_sync(0xffffffffu, v, 1);
    if (lane == 31) v = i - 32 >= 0 ? y[i - 32] : 0.0;
  }
}

// Work items of the Schur products of the 3D band kernel: the 378 pairs
// p <= q of S~ (item e, row-major over the upper triangle) and the 27
// centre-row products (items 378 + q), ordered by the first row their dot
// product reads (max of the two columns' first structural nonzeros), so the
// lanes of a warp run loops of similar length.
struct SchurOrder {
  unsigned short e[27 * 28 / 2 + 27];
};
__host__ __device__ constexpr int first_row_of(int q) { return (q % 3) + 5 * ((q / 3) % 3) + 25 * (q / 9); }
constexpr SchurOrder make_schur_order() {
  SchurOrder o{};
  constexpr int NP = 27, NPAIR = NP * (NP + 1) / 2;
  int key[NPAIR + NP] = {};
  int e = 0;
  for (int p = 0; p < NP; ++p)
    for (int q = p; q < NP; ++q, ++e) key[e] = first_row_of(p) > first_row_of(q) ? first_row_of(p) : first_row_of(q);
  for (int q = 0; q < NP; ++q, ++e) key[e] = first_row_of(q) > 62 ? first_row_of(q) : 62;
  int n = 0;
  for (int k = 0; k < 125; ++k)
    for (int j = 0; j < NPAIR + NP; ++j)
      if (key[j] == k) o.e[n++] = (unsigned short)j;
  return o;
}
__constant__ SchurOrder kSchurOrder = make_schur_order();

double ldl_min_pivot_env() {
  if (const char* env = getenv("FC_LDL_MIN_PIVOT")) {
    char* end = nullptr;
    const double v = strtod(env, &end);
    if (end != env && v >= 0.0) return v;
  }
  return 1e-14;
}

template <int DIM>
size_t ldl_rows_smem() {
  using P = PatchDims<DIM>;
  constexpr int NU = P::NU, NP = P::NP;
  const size_t d = (size_t)NU * kBand + (size_t)(NP + 1) * NU + NP * NP + 4 * NU + NP + 32 + 4 * NP + DIM * NP;
  const size_t b = d * 8 + (size_t)(NU + 2 * NP) * 4 + kTri * 2 + NU + NP + 16;
  return (b + 15) & ~(size_t)15;
}

// Record of the banded block factors of a 3D patch (cache_matrix), doubles:
// the band of L with 1/d_k on the diagonal (NU x kBand, column-major), the
// LU of S~ (row-major), the centre rows w_c of W~_c = K~^{-1} B~_c, du, dp;
// ints: the pivots of S~ and a dense-record index (-1: banded record).
constexpr int kBandRec = 125 * kBand + 27 * 27 + 3 * 27 + 125 + 27;
constexpr int kBandRecI = 27 + 1;

// MODE 0: owned rows (cache_inverse) into coef; MODE 1: the band factor
// record (cache_matrix) into coef / fpiv; MODE 2 (cache_none): solve with
// the gathered residual rpad and update the owned DoFs of x at once (x null:
// only factor K~ and list the patches whose block is not positive definite,
// which a sweep then leaves to the dense on-the-fly kernel).
template <int MODE>
__global__ void __launch_bounds__(256, 3)
    patch_rows_ldl_kernel(LevelGeom g, const double* __restrict__ st, const unsigned char* __restrict__ mask,
                          double* __restrict__ coef, int* __restrict__ fpiv, unsigned* __restrict__ d_err,
                          const int* __restrict__ work, int* __restrict__ redo_node, int* __restrict__ redo_out,
                          int* __restrict__ nredo, double dmin, const double* __restrict__ rpad,
                          double* __restrict__ x, double omega) {
  constexpr int DIM = 3;
  using P = PatchDims<DIM>;
  constexpr int NU = P::NU, NP = P::NP, ND = P::ND, SP = P::SP, NSLOT = P::NSLOT;
  constexpr int v0 = 62, p0 = 13;
  extern __shared__ double lsm[];
  double* Lb = lsm;                    // NU x kBand band of K~, then L and d
  double* Y = Lb + NU * kBand;         // (NP + 1) columns of length NU; later the 12 solves
  double* S = Y + (NP + 1) * NU;       // NP x NP
  double* sh = S + NP * NP;            // NU
  double* rd = sh + NU;                // 1 / d_k
  double* rsd = rd + NU;               // d_k^{-1/2}
  double* du = rsd + NU;               // NU
  double* colU = du + NU;              // 32: column k of the step, before scaling
  double* dp = colU + 32;              // NP
  double* zp = dp + NP;                // ND x NP
  double* w = zp + ND * NP;            // DIM x NP: centre rows of W~_c
  int* nodeU = (int*)(w + DIM * NP);   // NU
  int* nodeP = nodeU + NU;             // NP
  int* pivS = nodeP + NP;              // NP
  unsigned short* tri = (unsigned short*)(pivS + NP);  // kTri
  unsigned char* au = (unsigned char*)(tri + kTri);    // NU
  unsigned char* ap = au + NU;                         // NP
  __shared__ int s_flag, s_fail;

  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
  const long long widx = blockIdx.x;
  const long long i = work ? work[widx] : widx;
  const unsigned nx = (unsigned)g.nn[0], ny = (unsigned)g.nn[1];
  const int ia[3] = {(int)((unsigned)i % nx), (int)(((unsigned)i / nx) % ny), (int)((unsigned)i / (nx * ny))};
  const long long nn = g.nnodes;
  if (tid == 0) {
    s_flag = 0;
    s_fail = 0;
  }
  for (int e = tid; e < kTri; e += nt) {
    int l = 1;
    while (l * (l + 1) / 2 <= e) ++l;
    tri[e] = (unsigned short)((l << 8) | (e - l * (l - 1) / 2 + 1));
  }
  for (int v = tid; v < NU; v += nt) {
    int o[3];
    vel_off<DIM>(v, o);
    const int b0 = ia[0] + o[0], b1 = ia[1] + o[1], b2 = ia[2] + o[2];
    const bool in = b0 >= 0 && b0 <= g.n[0] && b1 >= 0 && b1 <= g.n[1] && b2 >= 0 && b2 <= g.n[2];
    const int bn = in ? b0 + g.nn[0] * (b1 + g.nn[1] * b2) : -1;
    nodeU[v] = bn;
    au[v] = (unsigned char)(in && !(mask[bn] & 1));
  }
  for (int p = tid; p < NP; p += nt) {
    int o[3];
    prs_off<DIM>(p, o);
    const int b0 = ia[0] + o[0], b1 = ia[1] + o[1], b2 = ia[2] + o[2];
    const bool in = b0 >= 0 && b0 <= g.n[0] && b1 >= 0 && b1 <= g.n[1] && b2 >= 0 && b2 <= g.n[2];
    nodeP[p] = in ? b0 + g.nn[0] * (b1 + g.nn[1] * b2) : -1;
    ap[p] = (unsigned char)in;
  }
  __syncthreads();

  // ---- gather the lower band of K (entry (k + l, k) from row k of the
  // operator), C into S; identity rows for absent DoFs
  for (int e = tid; e < NU * kBand; e += nt) {
    const int k = e >> 5, l = e & 31, r = k + l;
    double val = 0.0;
    if (r < NU) {
      if (au[k] && au[r]) {
        int ok[3], orr[3], d[3];
        vel_off<DIM>(k, ok);
        vel_off<DIM>(r, orr);
        bool adj = true;
        for (int t = 0; t < 3; ++t) { d[t] = orr[t] - ok[t]; if (d[t] < -1 || d[t] > 1) adj = false; }
        if (adj) val = st[((long long)nb_index<DIM>(d) * SP) * nn + nodeU[k]];
      } else if (l == 0) {
        val = 1.0;
      }
    }
    Lb[e] = val;
  }
  for (int e = tid; e < NP * NP; e += nt) {
    const int p = e / NP, q = e % NP;
    double val = 0.0;
    if (ap[p] && ap[q]) {
      int op[3], oq[3], d[3];
      prs_off<DIM>(p, op);
      prs_off<DIM>(q, oq);
      bool adj = true;
      for (int t = 0; t < 3; ++t) { d[t] = oq[t] - op[t]; if (d[t] < -1 || d[t] > 1) adj = false; }
      if (adj) val = st[((long long)nb_index<DIM>(d) * SP + 1 + 2 * DIM) * nn + nodeP[p]];
    } else if (p == q) {
      val = 1.0;
    }
    S[e] = val;
  }
  __syncthreads();
  for (int v = tid; v < NU; v += nt) {
    const double a = fabs(Lb[v * kBand]);
    du[v] = (au[v] && a > 0.0) ? 1.0 / sqrt(a) : 1.0;
  }
  for (int p = tid; p < NP; p += nt) {
    const double a = fabs(S[p * NP + p]);
    dp[p] = (ap[p] && a > 0.0) ? 1.0 / sqrt(a) : 1.0;
  }
  __syncthreads();
  for (int e = tid; e < NU * kBand; e += nt) {
    const int k = e >> 5, r = k + (e & 31);
    if (r < NU) Lb[e] = du[k] * Lb[e] * du[r];
  }
  for (int e = tid; e < NP * NP; e += nt) S[e] = dp[e / NP] * S[e] * dp[e % NP];
  __syncthreads();

  // ---- K~ = L diag(d) L^T, right-looking over the band
  for (int k = 0; k < NU; ++k) {
    if (warp == 0) {
      const double dk = Lb[k * kBand];
      const double u = Lb[k * kBand + lane];
      const double r = __drcp_rn(dk);  // 1 / d_k, correctly rounded
      if (lane == 0) {
        rd[k] = r;
        if (!(dk > dmin)) s_fail = 1;
      }
      colU[lane] = u;
      if (lane > 0) Lb[k * kBand + lane] = u * r;
    }
    __syncthreads();
    for (int e = tid; e < kTri; e += nt) {
      const int lm = tri[e], l = lm >> 8, m = lm & 255;
      if (k + l < NU) Lb[(k + m) * kBand + (l - m)] -= Lb[k * kBand + l] * colU[m];
    }
    __syncthreads();
  }
  if (s_fail) {  // not positive definite: the pivoted dense LU takes the patch
    if (tid == 0 && nredo) {
      const int slot = atomicAdd(nredo, 1);
      redo_node[slot] = (int)i;
      redo_out[slot] = (int)widx;
      if (MODE == 1) fpiv[widx * kBandRecI + NP] = -2;  // dense record pending
    }
    return;
  }
  if (MODE == 2 && !x) return;  // setup check only
  for (int k = tid; k < NU; k += nt) rsd[k] = sqrt(rd[k]);
  __syncthreads();

  // ---- per component: Y_c = L^{-1} B~_c, S~ -= Yh_c' Yh_c, w_c = Yh_c' sh
  for (int c = 0; c < DIM; ++c) {
    const int ncol = c == 0 ? NP + 1 : NP;  // column NP of component 0: L^{-1} e_centre
    for (int e = tid; e < ncol * NU; e += nt) {
      const int q = e / NU, v = e - q * NU;
      double val = 0.0;
      if (q == NP) {
        val = v == v0 ? 1.0 : 0.0;
      } else if (au[v] && ap[q]) {
        int ov[3], oq[3], d[3];
        vel_off<DIM>(v, ov);
        prs_off<DIM>(q, oq);
        bool adj = true;
        for (int t = 0; t < 3; ++t) { d[t] = oq[t] - ov[t]; if (d[t] < -1 || d[t] > 1) adj = false; }
        if (adj) val = du[v] * st[((long long)nb_index<DIM>(d) * SP + 1 + c) * nn + nodeU[v]] * dp[q];
      }
      Y[e] = val;
    }
    __syncthreads();
    for (int q = warp; q < ncol; q += nwarp) {
      int f = v0;
      if (q < NP) {
        int oq[3];
        prs_off<DIM>(q, oq);
        f = (oq[0] + 1) + 5 * (oq[1] + 1) + 25 * (oq[2] + 1);  // first velocity node next to q
      }
      double* y = Y + q * NU;
      band_forward(Lb, y, NU, f, lane);
      __syncwarp();
      for (int t = f + lane; t < NU; t += 32) y[t] *= rsd[t];
      if (q == NP)
        for (int t = lane; t < NU; t += 32) sh[t] = t >= f ? y[t] : 0.0;
      __syncwarp();
    }
    __syncthreads();
    constexpr int NPAIR = NP * (NP + 1) / 2;
    for (int it = tid; it < NPAIR + NP; it += nt) {
      const int e = kSchurOrder.e[it];
      if (e < NPAIR) {
        int p = 0, r = e;
        while (r >= NP - p) { r -= NP - p; ++p; }
        const int q = p + r;
        const double* yp = Y + p * NU;
        const double* yq = Y + q * NU;
        double acc = 0.0;
        for (int t = max(first_row_of(p), first_row_of(q)); t < NU; ++t) acc = fma(yp[t], yq[t], acc);
        S[p * NP + q] -= acc;
        if (p != q) S[q * NP + p] -= acc;
      } else {
        const int q = e - NPAIR;
        const double* yq = Y + q * NU;
        double acc = 0.0;
        for (int t = max(first_row_of(q), v0); t < NU; ++t) acc = fma(sh[t], yq[t], acc);
        w[c * NP + q] = acc;
      }
    }
    __syncthreads();
  }

  // ---- S~ = LU; z_p of the owned columns
  cta_lu(S, NP, NP, pivS, &s_flag);
  if (s_flag) {
    if (tid == 0) atomicOr(d_err, kErrSingularPatch);
  }
  if (MODE == 2) {
    // z_c = K~^{-1} (D r)_c, h = D r_p - sum_c B~_c' z_c, z_p = S~^{-1} h,
    // u_c(centre) = z_c(centre) - w_c . z_p; x[owned] += omega D (u, p)
    double* zc = Y;   // 3 columns of NU (Y is free after the Schur products)
    double* hq = zp;  // NP
    const long long pc = pad_node(g, ia[0], ia[1], ia[2]);
    const long long px = g.nn[0] + 4, py = g.nn[1] + 4;
    for (int e = tid; e < DIM * NU; e += nt) {
      const int c = e / NU, v = e - c * NU;
      int o[3];
      vel_off<DIM>(v, o);
      zc[e] = au[v] ? du[v] * rpad[(pc + o[0] + px * (o[1] + py * o[2])) * ND + c] : 0.0;
    }
    __syncthreads();
    if (warp < DIM) {
      double* y = zc + warp * NU;
      band_forward(Lb, y, NU, 0, lane);
      __syncwarp();
      for (int t = lane; t < NU; t += 32) y[t] *= rd[t];
      __syncwarp();
      band_backward(Lb, y, NU, lane);
    }
    __syncthreads();
    if (tid < NP) {
      const int q = tid;
      double hv = 0.0;
      if (ap[q]) {
        int oq[3];
        prs_off<DIM>(q, oq);
        double acc = rpad[(pc + oq[0] + px * (oq[1] + py * oq[2])) * ND + DIM];
        for (int t = 0; t < 27; ++t) {
          const int d[3] = {t % 3 - 1, (t / 3) % 3 - 1, t / 9 - 1};
          const int v = (oq[0] + d[0] + 2) + 5 * (oq[1] + d[1] + 2) + 25 * (oq[2] + d[2] + 2);
          if (!au[v]) continue;
          const int dvp[3] = {-d[0], -d[1], -d[2]};  // q relative to v
          const long long base = (long long)nb_index<DIM>(dvp) * SP;
          for (int c = 0; c < DIM; ++c) acc = fma(-st[(base + 1 + c) * nn + nodeU[v]] * du[v], zc[c * NU + v], acc);
        }
        hv = dp[q] * acc;
      }
      hq[q] = hv;
    }
    __syncthreads();
    if (tid == 0) {
      lu_solve_vec(S, NP, NP, pivS, hq);
      double y[ND];
      for (int c = 0; c < DIM; ++c) {
        double sv = zc[c * NU + v0];
        for (int q = 0; q < NP; ++q) sv = fma(-w[c * NP + q], hq[q], sv);
        y[c] = du[v0] * sv;
      }
      y[DIM] = dp[p0] * hq[p0];
      const unsigned char m = mask[i];
      for (int c = 0; c < DIM; ++c)
        x[i * ND + c] = x[i * ND + c] + (((m >> c) & 1) ? rpad[pc * ND + c] : omega * y[c]);
      x[i * ND + DIM] = x[i * ND + DIM] + omega * y[DIM];
    }
    return;
  }
  if (MODE == 1) {  // cache_matrix: store the band factors, S~ LU, w_c, du, dp
    double* rec = coef + widx * kBandRec;
    for (int e = tid; e < NU * kBand; e += nt) rec[e] = (e & (kBand - 1)) == 0 ? rd[e >> 5] : Lb[e];
    // S~ LU with the reciprocals of U's diagonal (the apply divides by none)
    for (int e = tid; e < NP * NP; e += nt) rec[NU * kBand + e] = e / NP == e % NP ? 1.0 / S[e] : S[e];
    for (int e = tid; e < DIM * NP; e += nt) rec[NU * kBand + NP * NP + e] = w[e];
    for (int v = tid; v < NU; v += nt) rec[NU * kBand + NP * NP + DIM * NP + v] = du[v];
    for (int p = tid; p < NP; p += nt) rec[NU * kBand + NP * NP + DIM * NP + NU + p] = dp[p];
    int* ip = fpiv + widx * kBandRecI;
    for (int p = tid; p < NP; p += nt) ip[p] = pivS[p];
    if (tid == 0) ip[NP] = -1;
    return;
  }
  if (tid < ND) {
    double* z = zp + tid * NP;
    for (int q = 0; q < NP; ++q) z[q] = tid < DIM ? -w[tid * NP + q] : (q == p0 ? 1.0 : 0.0);
    lu_solve_vec(S, NP, NP, pivS, z);
  }
  __syncthreads();

  // ---- right-hand sides delta_{k c'} e_centre - B~_c' z_p (12 columns of Y)
  for (int e = tid; e < DIM * NU; e += nt) {
    const int c2 = e / NU, v = e - c2 * NU;
    double g4[ND];
    for (int k = 0; k < ND; ++k) g4[k] = 0.0;
    if (au[v]) {
      int ov[3];
      vel_off<DIM>(v, ov);
      for (int qz = max(-1, ov[2] - 1); qz <= min(1, ov[2] + 1); ++qz)
        for (int qy = max(-1, ov[1] - 1); qy <= min(1, ov[1] + 1); ++qy)
          for (int qx = max(-1, ov[0] - 1); qx <= min(1, ov[0] + 1); ++qx) {
            const int q = (qx + 1) + 3 * (qy + 1) + 9 * (qz + 1);
            if (!ap[q]) continue;
            const int d[3] = {qx - ov[0], qy - ov[1], qz - ov[2]};
            const double b = du[v] * st[((long long)nb_index<DIM>(d) * SP + 1 + c2) * nn + nodeU[v]] * dp[q];
            for (int k = 0; k < ND; ++k) g4[k] = fma(-b, zp[k * NP + q], g4[k]);
          }
      if (v == v0) g4[c2] += 1.0;
    }
    for (int k = 0; k < ND; ++k) Y[(k * DIM + c2) * NU + v] = g4[k];
  }
  __syncthreads();
  for (int sidx = warp; sidx < ND * DIM; sidx += nwarp) {
    double* y = Y + sidx * NU;
    band_forward(Lb, y, NU, 0, lane);
    __syncwarp();
    for (int t = lane; t < NU; t += 32) y[t] *= rd[t];
    __syncwarp();
    band_backward(Lb, y, NU, lane);
    __syncwarp();
  }
  __syncthreads();

  // ---- owned rows of L_i^{-1} = d_k (L~^{-1} e_k)^T D, in the slot layout
  double* out = coef + widx * NSLOT * ND;
  for (int j = tid; j < NSLOT; j += nt) {
    double vals[ND];
    if (j < NU * DIM) {
      const int v = j / DIM, c2 = j - (j / DIM) * DIM;
      for (int k = 0; k < ND; ++k) {
        const bool own_ok = k < DIM ? au[v0] != 0 : true;
        const double dk = k < DIM ? du[v0] : dp[p0];
        vals[k] = (own_ok && au[v]) ? dk * Y[(k * DIM + c2) * NU + v] * du[v] : 0.0;
      }
    } else {
      const int p = j - NU * DIM;
      for (int k = 0; k < ND; ++k) {
        const bool own_ok = k < DIM ? au[v0] != 0 : true;
        const double dk = k < DIM ? du[v0] : dp[p0];
        vals[k] = (own_ok && ap[p]) ? dk * zp[k * NP + p] * dp[p] : 0.0;
      }
    }
    for (int k = 0; k < ND; ++k) out[(long long)j * ND + k] = vals[k];
  }
}

// cache_matrix apply with the banded factor records (3D): one 96-thread CTA
// per patch.  The record's band and S~ LU are staged in shared memory; warp
// c solves K~ z_c = (D r)_c (forward, 1/d, backward), then
//   h = D r_p - sum_c B~_c' z_c       (B~ re-read from the operator),
//   z_p = S~^{-1} h,   u_c(centre) = z_c(centre) - w_c . z_p,
// and the owned DoFs take omega D (u, p) (the restricted update).  Patches
// whose record is dense (index >= 0) are left to the dense apply over its
// node list.
__global__ void __launch_bounds__(96)
    band_factor_apply_kernel(LevelGeom g, const double* __restrict__ st, const double* __restrict__ fac,
                             const int* __restrict__ fpiv, const unsigned char* __restrict__ mask,
                             const double* __restrict__ rpad, double omega, double* __restrict__ x,
                             const int* __restrict__ prow) {
  constexpr int DIM = 3;
  using P = PatchDims<DIM>;
  constexpr int NU = P::NU, NP = P::NP, ND = P::ND, SP = P::SP;
  constexpr int v0 = 62, p0 = 13;
  __shared__ __align__(16) double sL[NU * kBand];
  __shared__ double sS[NP * NP];
  __shared__ double sz[DIM * NU], szd[DIM * NU];
  __shared__ double sh[NP];
  __shared__ int spiv[NP];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long i = blockIdx.x;
  const int pr = prow ? prow[i] : (int)i;
  const long long blk = pr < 0 ? -(long long)pr - 1 : pr;
  const int* ip = fpiv + blk * kBandRecI;
  if (ip[NP] >= 0) return;  // dense record: the dense apply takes this patch
  const double* rec = fac + blk * kBandRec;
  const double* wv = rec + NU * kBand + NP * NP;
  const double* du = wv + DIM * NP;
  const double* dp = du + NU;
  {
    const double2* src = reinterpret_cast<const double2*>(rec);
    double2* dst = reinterpret_cast<double2*>(sL);
    for (int e = tid; e < NU * kBand / 2; e += 96) dst[e] = __ldcs(src + e);
    for (int e = tid; e < NP * NP; e += 96) sS[e] = rec[NU * kBand + e];
    if (tid < NP) spiv[tid] = ip[tid];
  }
  const unsigned nx = (unsigned)g.nn[0], ny = (unsigned)g.nn[1];
  const int ia[3] = {(int)((unsigned)i % nx), (int)(((unsigned)i / nx) % ny), (int)((unsigned)i / (nx * ny))};
  const long long pbase = pad_node(g, ia[0], ia[1], ia[2]);
  const long long px = g.nn[0] + 4, py = g.nn[1] + 4;
  for (int e = tid; e < DIM * NU; e += 96) {
    const int c = e / NU, v = e - c * NU;
    int o[3];
    vel_off<DIM>(v, o);
    const int b0 = ia[0] + o[0], b1 = ia[1] + o[1], b2 = ia[2] + o[2];
    const bool in = b0 >= 0 && b0 <= g.n[0] && b1 >= 0 && b1 <= g.n[1] && b2 >= 0 && b2 <= g.n[2];
    const bool act = in && !(mask[b0 + (long long)g.nn[0] * (b1 + (long long)g.nn[1] * b2)] & 1);
    const long long pn = pbase + o[0] + px * (o[1] + py * o[2]);
    sz[e] = act ? du[v] * rpad[pn * ND + c] : 0.0;
  }
  __syncthreads();
  {  // z_c = K~^{-1} (D r)_c, one warp per component; szd = D z_c
    double* y = sz + warp * NU;
    band_forward(sL, y, NU, 0, lane);
    __syncwarp();
    for (int t = lane; t < NU; t += 32) y[t] *= sL[t * kBand];
    __syncwarp();
    band_backward(sL, y, NU, lane);
    __syncwarp();
    for (int t = lane; t < NU; t += 32) szd[warp * NU + t] = du[t] * y[t];
  }
  __syncthreads();
  if (warp == 0) {
    // h = D r_p - sum_c B~_c' z_c = dp (r_p - sum_c B_c' D z_c), lane q
    double hv = 0.0;
    if (lane < NP) {
      const int q = lane;
      int oq[3];
      prs_off<DIM>(q, oq);
      const int c0 = ia[0] + oq[0], c1 = ia[1] + oq[1], c2 = ia[2] + oq[2];
      const bool qin = c0 >= 0 && c0 <= g.n[0] && c1 >= 0 && c1 <= g.n[1] && c2 >= 0 && c2 <= g.n[2];
      if (qin) {
        const long long pq = pbase + oq[0] + px * (oq[1] + py * oq[2]);
        double acc = rpad[pq * ND + DIM];
        for (int t = 0; t < 27; ++t) {
          const int d[3] = {t % 3 - 1, (t / 3) % 3 - 1, t / 9 - 1};
          const int ov[3] = {oq[0] + d[0], oq[1] + d[1], oq[2] + d[2]};
          const int v = (ov[0] + 2) + 5 * (ov[1] + 2) + 25 * (ov[2] + 2);
          const int b0 = ia[0] + ov[0], b1 = ia[1] + ov[1], b2 = ia[2] + ov[2];
          if (b0 < 0 || b0 > g.n[0] || b1 < 0 || b1 > g.n[1] || b2 < 0 || b2 > g.n[2]) continue;
          const long long bn = b0 + (long long)g.nn[0] * (b1 + (long long)g.nn[1] * b2);
          if (mask[bn] & 1) continue;
          const int dvp[3] = {-d[0], -d[1], -d[2]};  // q relative to v
          const long long base = (long long)nb_index<DIM>(dvp) * SP;
          for (int c = 0; c < DIM; ++c) acc = fma(-st[(base + 1 + c) * g.nnodes + bn], szd[c * NU + v], acc);
        }
        hv = dp[q] * acc;
      }
      sh[q] = hv;
    }
    __syncwarp();
    // z_p = S~^{-1} h: row interchanges, then lane r carries z_p(r) through
    // the column steps of L (unit) and U (reciprocal diagonal stored)
    if (lane == 0)
      for (int k = 0; k < NP; ++k) {
        const int pk = spiv[k];
        if (pk != k) { const double t0 = sh[k]; sh[k] = sh[pk]; sh[pk] = t0; }
      }
    __syncwarp();
    double z = lane < NP ? sh[lane] : 0.0;
    for (int k = 0; k < NP - 1; ++k) {
      const double zk = __shfl_sync(0xffffffffu, z, k);
      if (lane > k && lane < NP) z = fma(-sS[lane * NP + k], zk, z);
    }
    for (int k = NP - 1; k >= 0; --k) {
      const double zk = __shfl_sync(0xffffffffu, z, k) * sS[k * NP + k];
      if (lane == k) z = zk;
      if (lane < k) z = fma(-sS[lane * NP + k], zk, z);
    }
    // owned update: u_c(centre) = z_c(centre) - w_c . z_p
    double y[ND];
    for (int c = 0; c < DIM; ++c) {
      double pc = lane < NP ? wv[c * NP + lane] * z : 0.0;
      for (int o = 16; o > 0; o >>= 1) pc += __shfl_xor_sync(0xffffffffu, pc, o);
      y[c] = du[v0] * (sz[c * NU + v0] - pc);
    }
    y[DIM] = dp[p0] * __shfl_sync(0xffffffffu, z, p0);
    if (lane == 0) {
      // restricted update of the node's own DoFs; a constrained velocity
      // component takes its residual (identity row)
      const unsigned char m = mask[i];
      for (int c = 0; c < DIM; ++c)
        x[i * ND + c] = x[i * ND + c] + (((m >> c) & 1) ? rpad[pbase * ND + c] : omega * y[c]);
      x[i * ND + DIM] = x[i * ND + DIM] + omega * y[DIM];
    }
  }
}

__global__ void mark_dense_records_kernel(const int* __restrict__ redo_out, int n, int* __restrict__ fpiv) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) fpiv[(long long)redo_out[j] * kBandRecI + 27] = j;
}

// nodes whose record (through prow) is dense, with that dense record's index
__global__ void dense_list_kernel(long long nnodes, const int* __restrict__ prow, const int* __restrict__ fpiv,
                                  int* __restrict__ lnode, int* __restrict__ lrec, int* __restrict__ nlist) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nnodes) return;
  const int pr = prow ? prow[i] : (int)i;
  const long long blk = pr < 0 ? -(long long)pr - 1 : pr;
  const int d = fpiv[blk * kBandRecI + 27];
  if (d >= 0) {
    const int k = atomicAdd(nlist, 1);
    lnode[k] = (int)i;
    lrec[k] = d;
  }
}

// ---------------------------------------------------------------------------
// cache_inverse apply: y = omega * Inv_i r_i, x[node i] += y.  One warp per
// patch; lane handles slots j = lane + 32 t, reads the ND coefficients of the
// slot with vector loads (streamed past L2: each row is read once per sweep)
// and the residual entry of the slot from the padded residual, whose zero
// halo covers the 5^d box so the gathers need no bounds checks.  The slot ->
// residual offset table is built once per block in shared memory, and the
// node index is decoded in 32-bit arithmetic (64-bit division would run on
// the FP64 pipe, 1/70 of the FP32 rate on this part).
// Row loads: rows shared by a class of patches stay in the caches; a
// patch's own rows are read once per sweep and streamed past L2.
template <typename V>
__device__ __forceinline__ V ldrow(const V* p, bool cached) {
  return cached ? __ldg(p) : __ldcs(p);
}

template <int DIM>
__device__ __forceinline__ void slot_table(const LevelGeom& g, int* soff) {
  constexpr int NU = PatchDims<DIM>::NU, ND = DIM + 1, NSLOT = PatchDims<DIM>::NSLOT;
  const int px = g.nn[0] + 4, py = g.nn[1] + 4;
  for (int j = threadIdx.x; j < NSLOT; j += blockDim.x) {
    int o[3], c;
    if (j < NU * DIM) {
      vel_off<DIM>(j / DIM, o);
      c = j % DIM;
    } else {
      prs_off<DIM>(j - NU * DIM, o);
      c = DIM;
    }
    soff[j] = (o[0] + px * (o[1] + py * o[2])) * ND + c;
  }
  __syncthreads();
}

template <int DIM>
__device__ __forceinline__ void decode_node(const LevelGeom& g, unsigned i, int* ia) {
  const unsigned nx = (unsigned)g.nn[0], ny = (unsigned)g.nn[1];
  unsigned t = i / nx;
  ia[0] = (int)(i - t * nx);
  if (DIM == 3) {
    unsigned u = t / ny;
    ia[1] = (int)(t - u * ny);
    ia[2] = (int)u;
  } else {
    ia[1] = (int)t;
    ia[2] = 0;
  }
}

template <int DIM>
__device__ __forceinline__ void finish_update(const LevelGeom& g, long long i, const int* ia,
                                              const unsigned char* mask, const double* rc,
                                              const double* y, double omega, double* x) {
  constexpr int ND = DIM + 1;
  unsigned char m = mask[i];
  for (int c = 0; c < DIM; ++c) {
    if ((m >> c) & 1) x[i * ND + c] = x[i * ND + c] + rc[c];
    else x[i * ND + c] = x[i * ND + c] + omega * y[c];
  }
  x[i * ND + DIM] = x[i * ND + DIM] + omega * y[DIM];
}

// Restricted prolongation R~_i^T for the apply kernels: lane c < d+1
// updates component c of node i from the warp-reduced y (all lanes hold the
// sums); constrained velocity components take the residual (identity row).
// x2, when given, receives the (hi, lo) float pair of the new value.
template <int ND>
__device__ __forceinline__ void owned_update(unsigned i, int lane, const unsigned char* mask, double rcv,
                                             double yv, double omega, double* x, float2* x2) {
  if (lane >= ND) return;
  const int c = lane;
  const size_t k = (size_t)i * ND + c;
  const bool fixed = c < ND - 1 && ((mask[i] >> c) & 1);
  const double nv = x[k] + (fixed ? rcv : omega * yv);
  x[k] = nv;
  if (x2) {
    float hi = (float)nv;
    x2[k] = make_float2(hi, (float)(nv - (double)hi));
  }
}

template <int N, typename T>
__device__ __forceinline__ T pick(const T* v, int c) {
  T r = v[0];
#pragma unroll
  for (int k = 1; k < N; ++k)
    if (c == k) r = v[k];
  return r;
}


template <int DIM, int TPP>
__global__ void __launch_bounds__(256)
    apply_fp64_kernel(LevelGeom g, const double* __restrict__ coef, const unsigned char* __restrict__ mask,
                      const double* __restrict__ rpad, double omega, double* __restrict__ x,
                      const int* __restrict__ prow) {
  using P = PatchDims<DIM>;
  constexpr int ND = P::ND, NSLOT = P::NSLOT;
  __shared__ int soff[NSLOT];
  slot_table<DIM>(g, soff);
  // a group of TPP lanes per patch; groups past the last patch still take
  // part in the shuffles of their warp
  const int lane = threadIdx.x % TPP;
  const unsigned gi = (unsigned)(((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) / TPP);
  const bool valid = gi < (unsigned)g.nnodes;
  const unsigned i = valid ? gi : (unsigned)g.nnodes - 1;
  int ia[3];
  decode_node<DIM>(g, i, ia);
  const long long pbase = pad_node(g, ia[0], ia[1], ia[2]);
  const double* rp = rpad + pbase * ND;
  const int pr = prow ? prow[i] : (int)i;
  const bool shared_rows = pr < 0;  // class rows: read through the cache
  const double* cf = coef + (size_t)(shared_rows ? -pr - 1 : pr) * NSLOT * ND;
  double y[4] = {0.0, 0.0, 0.0, 0.0};  // 2D: y[3] stays zero
  // Live velocity slots.  Slots of out-of-grid nodes and of wall layers
  // (every velocity component constrained) have zero coefficients; in 3D the
  // 5 x 5 x 5 velocity box is clipped per direction to its live layers
  // [x0, x1] x [y0, y1] x [z0, z1]: a patch walks rows of rx = 3 (x1 - x0 + 1)
  // contiguous slots (a y row of a z-plane holds 15), ny rows per z-plane,
  // nz planes, then its 3^d pressure slots.  Patches of a warp are
  // consecutive nodes of an x row and mostly share the clipping.
  int nv = P::NU * DIM, rx = nv, ny = 1, vbase = 0;  // unclipped: one run of all velocity slots
  if (DIM == 3 && g.dead_layer) {
    const unsigned char* dx = g.dead_layer;
    const unsigned char* dy = dx + g.nn[0];
    const unsigned char* dz = dy + g.nn[1];
    int x0 = -2, x1 = 2, y0 = -2, y1 = 2, z0 = -2, z1 = 2;
    while (x0 <= 2 && (ia[0] + x0 < 0 || ia[0] + x0 > g.n[0] || dx[ia[0] + x0])) ++x0;
    while (x1 >= x0 && (ia[0] + x1 < 0 || ia[0] + x1 > g.n[0] || dx[ia[0] + x1])) --x1;
    while (y0 <= 2 && (ia[1] + y0 < 0 || ia[1] + y0 > g.n[1] || dy[ia[1] + y0])) ++y0;
    while (y1 >= y0 && (ia[1] + y1 < 0 || ia[1] + y1 > g.n[1] || dy[ia[1] + y1])) --y1;
    while (z0 <= 2 && (ia[2] + z0 < 0 || ia[2] + z0 > g.n[2] || dz[ia[2] + z0])) ++z0;
    while (z1 >= z0 && (ia[2] + z1 < 0 || ia[2] + z1 > g.n[2] || dz[ia[2] + z1])) --z1;
    rx = 3 * (x1 - x0 + 1);
    ny = y1 - y0 + 1;
    nv = x1 >= x0 && y1 >= y0 && z1 >= z0 ? rx * ny * (z1 - z0 + 1) : 0;
    vbase = (z0 + 2) * 75 + (y0 + 2) * 15 + (x0 + 2) * 3;
  }
  // a patch whose node has every velocity component constrained owns only
  // its pressure: its velocity rows are zero and only row d is summed
  const bool wall = DIM == 3 && (mask[i] & 7) == 7;
  const int tot = nv + P::NP;
  int zi = 0, yi = 0, o = lane;  // loop index t = (zi ny + yi) rx + o while t < nv
  if (nv > 0)
    while (o >= rx) {
      o -= rx;
      if (++yi == ny) { yi = 0; ++zi; }
    }
  if (DIM == 3 && wall) {
    for (int t = lane; t < tot; t += TPP) {
      const int j = t < nv ? vbase + zi * 75 + yi * 15 + o : P::NU * DIM + (t - nv);
      if (nv > 0) {
        o += TPP;
        while (o >= rx) {
          o -= rx;
          if (++yi == ny) { yi = 0; ++zi; }
        }
      }
      y[ND - 1] += ldrow(cf + (size_t)j * ND + (ND - 1), shared_rows) * rp[soff[j]];
    }
  } else {
#pragma unroll 4
    for (int t = lane; t < tot; t += TPP) {
      const int j = t < nv ? vbase + zi * 75 + yi * 15 + o : P::NU * DIM + (t - nv);
      if (nv > 0) {
        o += TPP;
        while (o >= rx) {
          o -= rx;
          if (++yi == ny) { yi = 0; ++zi; }
        }
      }
      double rv = rp[soff[j]];
      if (ND == 4) {
        const double2* c2 = reinterpret_cast<const double2*>(cf + (size_t)j * 4);
        double2 a = ldrow(c2, shared_rows), b = ldrow(c2 + 1, shared_rows);
        y[0] += a.x * rv; y[1] += a.y * rv; y[2] += b.x * rv; y[3] += b.y * rv;
      } else {
#pragma unroll
        for (int k = 0; k < ND; ++k) y[k] += ldrow(cf + (size_t)j * ND + k, shared_rows) * rv;
      }
    }
  }
  if constexpr (TPP >= 4) {
    // the lane whose group-lane bits below TPP/4 are zero writes component c
    int c = 0;
    const double yc = reduce_scatter4<TPP>(y, lane, &c);
    if (valid && c < ND && (lane & (TPP / 4 - 1)) == 0) owned_update<ND>(i, c, mask, rp[c], yc, omega, x, nullptr);
  } else {
#pragma unroll
    for (int k = 0; k < ND; ++k)
#pragma unroll
      for (int o = TPP / 2; o > 0; o >>= 1) y[k] += __shfl_xor_sync(0xffffffffu, y[k], o);
    if (valid && lane < ND) owned_update<ND>(i, lane, mask, rp[lane], pick<ND>(y, lane), omega, x, nullptr);
  }
}

// float32 / bfloat16 rows with float32 residual and float32 accumulation
template <typename T>
__device__ __forceinline__ void load_row4(const T* p, float* v, bool cached);
template <>
__device__ __forceinline__ void load_row4<float>(const float* p, float* v, bool cached) {
  float4 a = ldrow(reinterpret_cast<const float4*>(p), cached);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
template <>
__device__ __forceinline__ void load_row4<__nv_bfloat16>(const __nv_bfloat16* p, float* v, bool cached) {
  uint2 a = ldrow(reinterpret_cast<const uint2*>(p), cached);
  v[0] = __uint_as_float(a.x << 16); v[1] = __uint_as_float(a.x & 0xffff0000u);
  v[2] = __uint_as_float(a.y << 16); v[3] = __uint_as_float(a.y & 0xffff0000u);
}

template <int DIM, typename T, int TPP>
__global__ void __launch_bounds__(256)
    apply_lowp_kernel(LevelGeom g, const T* __restrict__ coef, const unsigned char* __restrict__ mask,
                      const float* __restrict__ rpad, double omega, double* __restrict__ x,
                      const int* __restrict__ prow) {
  using P = PatchDims<DIM>;
  constexpr int ND = P::ND, NSLOT = P::NSLOT;
  __shared__ int soff[NSLOT];
  slot_table<DIM>(g, soff);
  const int lane = threadIdx.x % TPP;
  const unsigned gi = (unsigned)(((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) / TPP);
  const bool valid = gi < (unsigned)g.nnodes;
  const unsigned i = valid ? gi : (unsigned)g.nnodes - 1;
  int ia[3];
  decode_node<DIM>(g, i, ia);
  const long long pbase = pad_node(g, ia[0], ia[1], ia[2]);
  const float* rp = rpad + pbase * ND;
  const int pr = prow ? prow[i] : (int)i;
  const bool shared_rows = pr < 0;  // class rows: read through the cache
  const T* cf = coef + (size_t)(shared_rows ? -pr - 1 : pr) * NSLOT * ND;
  float y[ND];
#pragma unroll
  for (int k = 0; k < ND; ++k) y[k] = 0.0f;
#pragma unroll 2
  for (int j = lane; j < NSLOT; j += TPP) {
    float rv = rp[soff[j]];
    float cv[4];
    if (ND == 4) {
      load_row4<T>(cf + (size_t)j * 4, cv, shared_rows);
    } else {
#pragma unroll
      for (int k = 0; k < ND; ++k) cv[k] = (float)cf[(size_t)j * ND + k];  // 2D: scalar loads
    }
#pragma unroll
    for (int k = 0; k < ND; ++k) y[k] = fmaf(cv[k], rv, y[k]);
  }
#pragma unroll
  for (int k = 0; k < ND; ++k)
#pragma unroll
    for (int o = TPP / 2; o > 0; o >>= 1) y[k] += __shfl_xor_sync(0xffffffffu, y[k], o);
  if (valid && lane < ND)
    owned_update<ND>(i, lane, mask, (double)rp[lane], (double)pick<ND>(y, lane), omega, x, nullptr);
}

// Float-pair arithmetic (hi + lo of float32, about 48-bit significand) on the
// float32 pipes.  A product c r = (ch + cl)(rh + rl) is taken as the exact
// ch rh split by one FMA plus the cross terms in float32; it is added to the
// running sum with a two-sum on the high parts, the low parts accumulate
// plainly and are folded in once at the end (Dekker 1971; Knuth TAOCP 4.2.2).
struct df { float hi, lo; };
__device__ __forceinline__ df df_two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ df df_add(df a, df b) {
  df s = df_two_sum(a.hi, b.hi);
  df t = df_two_sum(a.lo, b.lo);
  s.lo += t.hi;
  float hi = s.hi + s.lo;
  float lo = s.lo - (hi - s.hi);
  lo += t.lo;
  float h2 = hi + lo;
  return {h2, lo - (h2 - hi)};
}
__device__ __forceinline__ df df_mul(df a, df b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  float hi = p + e;
  return {hi, e - (hi - p)};
}
// acc += c * r (c, r pairs); acc.lo collects every low-order term
__device__ __forceinline__ void df_fma_acc(df& acc, float ch, float cl, float rh, float rl) {
  float p = ch * rh;
  float pe = fmaf(ch, rh, -p);
  float cross = fmaf(ch, rl, cl * rh);
  float s = acc.hi + p;
  float bb = s - acc.hi;
  float e = (acc.hi - (s - bb)) + (p - bb);
  acc.hi = s;
  acc.lo += e + (pe + cross);
}

template <int DIM>
__global__ void __launch_bounds__(256)
    apply_df_kernel(LevelGeom g, const float2* __restrict__ coef, const unsigned char* __restrict__ mask,
                    const float2* __restrict__ rpad, double omega, double* __restrict__ x,
                    float2* __restrict__ xp2, float2 om2, const int* __restrict__ prow) {
  using P = PatchDims<DIM>;
  constexpr int ND = P::ND, NSLOT = P::NSLOT;
  __shared__ int soff[NSLOT];
  slot_table<DIM>(g, soff);
  const int lane = threadIdx.x & 31;
  const unsigned i = (unsigned)(((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (i >= (unsigned)g.nnodes) return;
  int ia[3];
  decode_node<DIM>(g, i, ia);
  const long long pbase = pad_node(g, ia[0], ia[1], ia[2]);
  const float2* rp = rpad + pbase * ND;
  const int pr = prow ? prow[i] : (int)i;
  const bool shared_rows = pr < 0;  // class rows: read through the cache
  const float2* cf = coef + (size_t)(shared_rows ? -pr - 1 : pr) * NSLOT * ND;
  df y[ND];
#pragma unroll
  for (int k = 0; k < ND; ++k) y[k] = {0.0f, 0.0f};
#pragma unroll 2
  for (int j = lane; j < NSLOT; j += 32) {
    float2 r2 = rp[soff[j]];
    float ch[4], cl[4];
    if (ND == 4) {
      const float4* c4 = reinterpret_cast<const float4*>(cf + (size_t)j * 4);
      float4 a = ldrow(c4, shared_rows), b = ldrow(c4 + 1, shared_rows);
      ch[0] = a.x; cl[0] = a.y; ch[1] = a.z; cl[1] = a.w;
      ch[2] = b.x; cl[2] = b.y; ch[3] = b.z; cl[3] = b.w;
    } else {
#pragma unroll
      for (int k = 0; k < ND; ++k) {
        float2 c2 = ldrow(cf + (size_t)j * ND + k, shared_rows);
        ch[k] = c2.x; cl[k] = c2.y;
      }
    }
#pragma unroll
    for (int k = 0; k < ND; ++k) df_fma_acc(y[k], ch[k], cl[k], r2.x, r2.y);
  }
#pragma unroll
  for (int k = 0; k < ND; ++k) {
    float h = y[k].hi + y[k].lo;
    y[k] = {h, y[k].lo - (h - y[k].hi)};
    for (int o = 16; o > 0; o >>= 1) {
      df other = {__shfl_xor_sync(0xffffffffu, y[k].hi, o), __shfl_xor_sync(0xffffffffu, y[k].lo, o)};
      y[k] = df_add(y[k], other);
    }
  }
  if (lane < ND) {
    float2 r2 = rp[lane];
    df yl = pick<ND>(y, lane);
    if (xp2) {
      // pair copy of x (padded like the residual), updated on the float32
      // pipes: x + omega y, or x + r on a constrained component
      const size_t k = (size_t)pbase * ND + lane;
      const float2 xv = xp2[k];
      const bool fixed = lane < DIM && ((mask[i] >> lane) & 1);
      const df add = fixed ? df{r2.x, r2.y} : df_mul({om2.x, om2.y}, yl);
      const df nv = df_add({xv.x, xv.y}, add);
      xp2[k] = make_float2(nv.hi, nv.lo);
    } else {
      owned_update<ND>(i, lane, mask, (double)r2.x + (double)r2.y, (double)yl.hi + (double)yl.lo, omega, x,
                       nullptr);
    }
  }
}

// ---------------------------------------------------------------------------
// cache_matrix apply: block solve with the stored factors, one warp per patch.
template <int DIM>
__global__ void __launch_bounds__(128)
    factor_apply_kernel(LevelGeom g, const double* __restrict__ fac, const int* __restrict__ fpiv,
                        const unsigned char* __restrict__ mask, const double* __restrict__ rpad,
                        double omega, double* __restrict__ x, const int* __restrict__ prow,
                        const int* __restrict__ lnode, const int* __restrict__ lrec, long long nlist) {
  using P = PatchDims<DIM>;
  constexpr int NU = P::NU, NP = P::NP, ND = P::ND;
  __shared__ double sz[4][DIM * NU + 2 * NP];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  // every node through prow, or (lnode) the listed nodes with their records
  const long long wi = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (wi >= (lnode ? nlist : g.nnodes)) return;
  const long long i = lnode ? (long long)lnode[wi] : wi;
  double* z = sz[wib];             // DIM vectors of NU (component-major)
  double* t = z + DIM * NU;        // NP
  double* zpv = t + NP;            // NP
  const int pr = lnode ? lrec[wi] : (prow ? prow[i] : (int)i);
  const long long blk = pr < 0 ? -(long long)pr - 1 : pr;
  const double* rec = fac + blk * (long long)P::REC;
  const double* LUc = rec;                        // column-major
  const double* Wm = rec + NU * NU;               // [c*NP+q][NU]
  const double* Sm = Wm + DIM * NP * NU;          // row-major NP x NP
  const double* du = Sm + NP * NP;
  const double* dp = du + NU;
  const int* piv = fpiv + blk * (long long)P::RECI;
  int ia[3] = {(int)(i % g.nn[0]), (int)((i / g.nn[0]) % g.nn[1]),
               DIM == 3 ? (int)(i / ((long long)g.nn[0] * g.nn[1])) : 0};
  long long pbase = pad_node(g, ia[0], ia[1], ia[2]);
  long long px = g.nn[0] + 4, py = g.nn[1] + 4;
  // scaled residual; inactive DoFs carry zero coefficients in du/B already
  // (du = 1 there but B rows are zero and K is identity), so zero them
  for (int v = lane; v < NU; v += 32) {
    int o[3];
    vel_off<DIM>(v, o);
    long long pn = pbase + o[0] + px * (o[1] + py * o[2]);
    int b0 = ia[0] + o[0], b1 = ia[1] + o[1], b2 = ia[2] + o[2];
    bool in = b0 >= 0 && b0 <= g.n[0] && b1 >= 0 && b1 <= g.n[1] && (DIM == 2 || (b2 >= 0 && b2 <= g.n[2]));
    bool act = in && !(mask[b0 + (long long)g.nn[0] * (b1 + (long long)g.nn[1] * b2)] & 1);
    for (int c = 0; c < DIM; ++c) z[c * NU + v] = act ? du[v] * rpad[pn * ND + c] : 0.0;
  }
  for (int p = lane; p < NP; p += 32) {
    int o[3];
    prs_off<DIM>(p, o);
    long long pn = pbase + o[0] + px * (o[1] + py * o[2]);
    t[p] = dp[p] * rpad[pn * ND + DIM];  // out-of-grid pressure: halo zero
  }
  __syncwarp();
  // t -= sum_c W~_c^T r~_c   (W~ = K~^{-1} B~ and K~ symmetric)
  for (int q = 0; q < NP; ++q) {
    double s = 0.0;
    for (int c = 0; c < DIM; ++c)
      for (int v = lane; v < NU; v += 32) s += Wm[(long long)(c * NP + q) * NU + v] * z[c * NU + v];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) t[q] -= s;
  }
  __syncwarp();
  // u* = K~^{-1} r~_c for every component (column-oriented sweeps)
  if (lane == 0)
    for (int k = 0; k < NU; ++k) {
      int p = piv[k];
      if (p != k)
        for (int c = 0; c < DIM; ++c) { double tmp = z[c * NU + k]; z[c * NU + k] = z[c * NU + p]; z[c * NU + p] = tmp; }
    }
  __syncwarp();
  for (int k = 0; k < NU; ++k) {
    double zk[DIM];
    for (int c = 0; c < DIM; ++c) zk[c] = z[c * NU + k];
    for (int r = k + 1 + lane; r < NU; r += 32) {
      double l = LUc[(long long)k * NU + r];
      for (int c = 0; c < DIM; ++c) z[c * NU + r] -= l * zk[c];
    }
    __syncwarp();
  }
  for (int k = NU - 1; k >= 0; --k) {
    double dkk = LUc[(long long)k * NU + k];
    double zk[DIM];
    for (int c = 0; c < DIM; ++c) zk[c] = z[c * NU + k] / dkk;
    __syncwarp();
    if (lane == 0)
      for (int c = 0; c < DIM; ++c) z[c * NU + k] = zk[c];
    for (int r = lane; r < k; r += 32) {
      double u = LUc[(long long)k * NU + r];
      for (int c = 0; c < DIM; ++c) z[c * NU + r] -= u * zk[c];
    }
    __syncwarp();
  }
  // z_p = S~^{-1} t
  if (lane == 0) {
    const int* pivS = piv + NU;
    for (int q = 0; q < NP; ++q) zpv[q] = t[q];
    for (int k = 0; k < NP; ++k) {
      int p = pivS[k];
      if (p != k) { double tmp = zpv[k]; zpv[k] = zpv[p]; zpv[p] = tmp; }
    }
    for (int r = 0; r < NP; ++r) {
      double s = zpv[r];
      for (int c = 0; c < r; ++c) s -= Sm[r * NP + c] * zpv[c];
      zpv[r] = s;
    }
    for (int r = NP - 1; r >= 0; --r) {
      double s = zpv[r];
      for (int c = r + 1; c < NP; ++c) s -= Sm[r * NP + c] * zpv[c];
      zpv[r] = s / Sm[r * NP + r];
    }
    const int v0 = DIM == 3 ? 62 : 12, p0 = DIM == 3 ? 13 : 4;
    double y[ND];
    for (int c = 0; c < DIM; ++c) {
      double s = z[c * NU + v0];
      for (int q = 0; q < NP; ++q) s -= Wm[(long long)(c * NP + q) * NU + v0] * zpv[q];
      y[c] = du[v0] * s;
    }
    y[DIM] = dp[p0] * zpv[p0];
    double rc[ND];
    for (int c = 0; c < ND; ++c) rc[c] = rpad[pbase * ND + c];
    finish_update<DIM>(g, i, ia, mask, rc, y, omega, x);
  }
}

// float64 rows -> storage precision
template <typename T>
__global__ void convert_kernel(long long n, const double* __restrict__ in, T* __restrict__ out) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    out[t] = (T)in[t];
}
template <>
__global__ void convert_kernel<__nv_bfloat16>(long long n, const double* __restrict__ in, __nv_bfloat16* __restrict__ out) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    out[t] = __double2bfloat16(in[t]);
}
template <>
__global__ void convert_kernel<float2>(long long n, const double* __restrict__ in, float2* __restrict__ out) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double v = in[t];
    float hi = (float)v;
    float lo = (float)(v - (double)hi);
    out[t] = make_float2(hi, lo);
  }
}

template <int DIM>
size_t factor_smem() {
  using P = PatchDims<DIM>;
  size_t d = (size_t)P::NU * P::NU + (size_t)P::NCOL * P::NU + P::NP * P::NP + P::NU + P::NP + P::NP +
             (DIM + 1) * P::NP + P::ND;
  size_t bytes = d * 8 + (P::NU + P::NP) * 4 + 8 + (P::NU + P::NP) * 8 + (P::NU + P::NP) + 16;
  return (bytes + 15) & ~(size_t)15;
}

template <int DIM, int MODE>
cudaError_t run_factor(const LevelGeom& g, const double* st, const unsigned char* mask, double omega,
                       double* coef, double* fac, int* fpiv, const double* rpad, double* x,
                       unsigned* d_err, const int* work, long long nwork, cudaStream_t s,
                       const int* outidx = nullptr) {
  size_t sm = factor_smem<DIM>();
  auto kern = patch_factor_kernel<DIM, MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const long long nb = work ? nwork : g.nnodes;
  if (nb <= 0) return cudaSuccess;
  // threads per CTA: the 3D block needs 220 KB of shared memory, so one CTA
  // fills an SM and its warps alone hide the shared-memory and barrier
  // latency; FC_FACTOR_THREADS overrides the choice for tuning runs
  int threads = DIM == 3 ? 1024 : 128;
  if (const char* env = getenv("FC_FACTOR_THREADS")) {
    int t = atoi(env);
    if (t >= 64 && t <= 1024 && t % 32 == 0) threads = t;
  }
  kern<<<(unsigned)nb, threads, sm, s>>>(g, st, mask, omega, coef, fac, fpiv, rpad, x, d_err, work, outidx);
  note_launches(1);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Persistent float-pair apply for the pair smoothing phase.  CTAs stay
// resident (one wave); each first copies the row blocks shared by the patch
// classes (at most two) into shared memory, then its warps stride over the
// patches.  A class patch reads its rows from shared memory, a unique patch
// streams its own rows from HBM; the residual gathers and the pair update of
// x are those of apply_df_kernel.
constexpr int kMaxClassBlocks = 2;

template <int DIM, bool SMEM, int TPP>
__device__ __forceinline__ void df_patch_dot(const float2* __restrict__ cf, const float2* __restrict__ rp,
                                             const int* soff, int lane, df* y) {
  using P = PatchDims<DIM>;
  constexpr int ND = P::ND, NSLOT = P::NSLOT;
#pragma unroll 2
  for (int j = lane; j < NSLOT; j += TPP) {
    float2 r2 = rp[soff[j]];
    float ch[4], cl[4];
    if (ND == 4) {
      const float4* c4 = reinterpret_cast<const float4*>(cf + (size_t)j * 4);
      float4 a, b;
      if (SMEM) { a = c4[0]; b = c4[1]; }
      else { a = __ldcs(c4); b = __ldcs(c4 + 1); }
      ch[0] = a.x; cl[0] = a.y; ch[1] = a.z; cl[1] = a.w;
      ch[2] = b.x; cl[2] = b.y; ch[3] = b.z; cl[3] = b.w;
    } else {
#pragma unroll
      for (int k = 0; k < ND; ++k) {
        float2 c2 = SMEM ? cf[(size_t)j * ND + k] : __ldcs(cf + (size_t)j * ND + k);
        ch[k] = c2.x; cl[k] = c2.y;
      }
    }
#pragma unroll
    for (int k = 0; k < ND; ++k) df_fma_acc(y[k], ch[k], cl[k], r2.x, r2.y);
  }
}

template <int DIM, int TPP>
__global__ void __launch_bounds__(256)
    apply_df_persistent_kernel(LevelGeom g, const float2* __restrict__ coef, const unsigned char* __restrict__ mask,
                               const float2* __restrict__ rpad, float2* __restrict__ xp2, float2 om2,
                               const int* __restrict__ prow, int2 cls_blk) {
  using P = PatchDims<DIM>;
  constexpr int ND = P::ND, NSLOT = P::NSLOT;
  __shared__ int soff[NSLOT];
  extern __shared__ float4 srow_raw[];
  float2* srows = reinterpret_cast<float2*>(srow_raw);
  const int nblk_sh = (cls_blk.x >= 0) + (cls_blk.y >= 0);
  const int blk_id[2] = {cls_blk.x, cls_blk.y};
  for (int b = 0; b < nblk_sh; ++b) {
    // element-wise float2 copy: 2D blocks (177 pairs) are only 8-byte aligned
    const float2* src = coef + (size_t)blk_id[b] * NSLOT * ND;
    float2* dst = srows + (size_t)b * NSLOT * ND;
    for (int t = threadIdx.x; t < NSLOT * ND; t += blockDim.x) dst[t] = __ldg(src + t);
  }
  slot_table<DIM>(g, soff);  // ends with __syncthreads()
  // groups of TPP lanes take one patch each (TPP = 32: a warp per patch);
  // every group of a warp runs the same number of passes so that the
  // shuffles below always see full warps
  const int lane = threadIdx.x % TPP;
  const unsigned gpb = blockDim.x / TPP;
  const unsigned ngroups = gridDim.x * gpb;
  const unsigned first = blockIdx.x * gpb + threadIdx.x / TPP;
  const unsigned warp_first = first - (threadIdx.x & 31) / TPP;
  for (unsigned i0 = warp_first; i0 < (unsigned)g.nnodes; i0 += ngroups) {
    const unsigned iv = i0 + (first - warp_first);
    const bool valid = iv < (unsigned)g.nnodes;
    const unsigned i = valid ? iv : (unsigned)g.nnodes - 1;
    int ia[3];
    decode_node<DIM>(g, i, ia);
    const long long pbase = pad_node(g, ia[0], ia[1], ia[2]);
    const float2* rp = rpad + pbase * ND;
    const int pr = prow ? prow[i] : (int)i;
    df y[ND];
#pragma unroll
    for (int k = 0; k < ND; ++k) y[k] = {0.0f, 0.0f};
    int sh = -1;
    if (pr < 0) {
      const int blk = -pr - 1;
      sh = blk == cls_blk.x ? 0 : (blk == cls_blk.y ? 1 : -1);
    }
    if (sh >= 0) {
      df_patch_dot<DIM, true, TPP>(srows + (size_t)sh * NSLOT * ND, rp, soff, lane, y);
    } else {
      const size_t blk = pr < 0 ? (size_t)(-pr - 1) : (size_t)pr;
      df_patch_dot<DIM, false, TPP>(coef + blk * NSLOT * ND, rp, soff, lane, y);
    }
#pragma unroll
    for (int k = 0; k < ND; ++k) {
      float h = y[k].hi + y[k].lo;
      y[k] = {h, y[k].lo - (h - y[k].hi)};
#pragma unroll
      for (int o = TPP / 2; o > 0; o >>= 1) {
        df other = {__shfl_xor_sync(0xffffffffu, y[k].hi, o), __shfl_xor_sync(0xffffffffu, y[k].lo, o)};
        y[k] = df_add(y[k], other);
      }
    }
    // lane t of the group updates component t (two per lane when TPP = 2)
#pragma unroll
    for (int t0 = 0; t0 < ND; t0 += TPP) {
      const int c = t0 + lane;
      if (!valid || c >= ND) break;
      const float2 r2 = rp[c];
      const df yl = pick<ND>(y, c);
      const size_t k = (size_t)pbase * ND + c;
      const float2 xv = xp2[k];
      const bool fixed = c < DIM && ((mask[i] >> c) & 1);
      const df add = fixed ? df{r2.x, r2.y} : df_mul({om2.x, om2.y}, yl);
      const df nv = df_add({xv.x, xv.y}, add);
      xp2[k] = make_float2(nv.hi, nv.lo);
    }
  }
}

// lanes per patch of the single-problem apply kernels: a warp per 3D patch
// (402 slots), 4 lanes per 2D patch (59 slots; a warp per 2D patch leaves
// the loads latency-bound).  FC_APPLY_TPP (2, 4, 8, 16, 32) overrides the
// choice of the float-pair apply for tuning runs.
int apply_tpp(int dim) {
  static const int env = [] {
    const char* e = getenv("FC_APPLY_TPP");
    const int t = e ? atoi(e) : 0;
    return (t == 2 || t == 4 || t == 8 || t == 16 || t == 32) ? t : 0;
  }();
  if (env) return env;
  return dim == 3 ? 32 : 4;
}

// lanes per patch of the FP64-row apply.  The kernel is bound by the FP64
// pipe (2 FMA per clock per SM on this part), so the group is kept small:
// each lane then accumulates more slots and the group's reduction adds
// little (8 lanes: 4 FP64 adds per lane, 2 % of a 3D patch's 1,608 FMA;
// 32 lanes: 6 per lane, 12 %).  4 lanes in 2D (59 slots).  FC_APPLY64_TPP
// (4, 8, 16, 32) overrides the 3D choice for tuning runs.
int apply64_tpp(int dim) {
  static const int env = [] {
    const char* e = getenv("FC_APPLY64_TPP");
    const int t = e ? atoi(e) : 0;
    return (t == 4 || t == 8 || t == 16 || t == 32) ? t : 0;
  }();
  if (dim == 2) return 4;
  return env ? env : 8;
}

template <int DIM, int TPP>
cudaError_t run_df_persistent_t(const LevelGeom& g, const float2* coef, const unsigned char* mask,
                                const float2* rpad, float2* xp2, float2 om2, const int* prow, int2 cls,
                                cudaStream_t s) {
  using P = PatchDims<DIM>;
  const size_t smem = (size_t)kMaxClassBlocks * P::NSLOT * P::ND * sizeof(float2);
  auto kern = apply_df_persistent_kernel<DIM, TPP>;
  int per_sm = 0, nsm = 0;
  cudaError_t e = persistent_ctas((const void*)kern, 256, smem, &per_sm, &nsm);
  if (e != cudaSuccess) return e;
  const long long need = (g.nnodes + 256 / TPP - 1) / (256 / TPP);
  const long long blocks = std::min<long long>((long long)per_sm * nsm, need);
  kern<<<(unsigned)std::max<long long>(blocks, 1), 256, smem, s>>>(g, coef, mask, rpad, xp2, om2, prow, cls);
  note_launches(1);
  return cudaGetLastError();
}

template <int DIM>
cudaError_t run_df_persistent(const LevelGeom& g, const float2* coef, const unsigned char* mask,
                              const float2* rpad, float2* xp2, float2 om2, const int* prow, int2 cls,
                              cudaStream_t s) {
  switch (apply_tpp(DIM)) {
    case 2: return run_df_persistent_t<DIM, 2>(g, coef, mask, rpad, xp2, om2, prow, cls, s);
    case 4: return run_df_persistent_t<DIM, 4>(g, coef, mask, rpad, xp2, om2, prow, cls, s);
    case 8: return run_df_persistent_t<DIM, 8>(g, coef, mask, rpad, xp2, om2, prow, cls, s);
    case 16: return run_df_persistent_t<DIM, 16>(g, coef, mask, rpad, xp2, om2, prow, cls, s);
    default: return run_df_persistent_t<DIM, 32>(g, coef, mask, rpad, xp2, om2, prow, cls, s);
  }
}
// ---------------------------------------------------------------------------
// Float-pair patch factorisation (rows for the reduced-precision modes).
// The same block elimination as patch_factor_kernel mode 0, with the gather
// and the equilibration in float64 and every elimination step -- the LU of
// K~, the multi-right-hand-side solves, the Schur complement S~ and its LU,
// the owned rows -- in float-pair arithmetic on the float32 pipes (about 48
// significant bits; the blocks are equilibrated, so the rows keep ~14
// digits).  FP64 runs at about 1/70 of FP32 on this part.
struct pr { float h, l; };
__device__ __forceinline__ pr pr_norm(float s, float e) {
  float h = s + e;
  return {h, e - (h - s)};
}
__device__ __forceinline__ pr pr_add(pr a, pr b) {
  float s = a.h + b.h;
  float bb = s - a.h;
  float e = (a.h - (s - bb)) + (b.h - bb);
  e += a.l + b.l;
  return pr_norm(s, e);
}
__device__ __forceinline__ pr pr_mul(pr a, pr b) {
  float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return pr_norm(p, e);
}
// c - a b: the product as p + e (exact FMA split plus the cross terms), a
// two-sum of the high parts, the low parts added, one renormalisation
__device__ __forceinline__ pr pr_fms(pr c, pr a, pr b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  const float s = c.h - p;
  const float bb = s - c.h;
  const float err = (c.h - (s - bb)) + (-p - bb);
  return pr_norm(s, (c.l - e) + err);
}
__device__ __forceinline__ pr pr_div(pr a, pr b) {
  float q1 = a.h / b.h;
  pr r = pr_fms(a, {q1, 0.0f}, b);
  float q2 = r.h / b.h;
  return pr_norm(q1, q2);
}
__device__ __forceinline__ pr pr_from(double v) {
  float h = (float)v;
  return {h, (float)(v - (double)h)};
}
__device__ __forceinline__ double pr_to(pr a) { return (double)a.h + (double)a.l; }

// Arithmetic of the CTA factorisations: float pairs (Ops = OpsPair) or
// plain float32 (Ops = OpsF32).
struct OpsPair {
  using T = pr;
  static __device__ __forceinline__ T zero() { return {0.0f, 0.0f}; }
  static __device__ __forceinline__ float mag(T a) { return fabsf(a.h); }
  static __device__ __forceinline__ bool nonzero(T a) { return a.h != 0.0f; }
  static __device__ __forceinline__ T fms(T c, T a, T b) { return pr_fms(c, a, b); }
  static __device__ __forceinline__ T div(T a, T b) { return pr_div(a, b); }
  static __device__ __forceinline__ T mul(T a, T b) { return pr_mul(a, b); }
  static __device__ __forceinline__ T shfl(T a, int src) {
    return {__shfl_sync(0xffffffffu, a.h, src), __shfl_sync(0xffffffffu, a.l, src)};
  }
};
struct OpsF32 {
  using T = float;
  static __device__ __forceinline__ T zero() { return 0.0f; }
  static __device__ __forceinline__ float mag(T a) { return fabsf(a); }
  static __device__ __forceinline__ bool nonzero(T a) { return a != 0.0f; }
  static __device__ __forceinline__ T fms(T c, T a, T b) { return fmaf(-a, b, c); }
  static __device__ __forceinline__ T div(T a, T b) { return a / b; }
  static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
  static __device__ __forceinline__ T shfl(T a, int src) { return __shfl_sync(0xffffffffu, a, src); }
};

// CTA LU with partial pivoting (max |a|, the high part for pairs; lowest
// row on ties) of the N x N matrix A (row-major).  Per pivot step: warp 0 finds the pivot, the
// rows are interchanged and the multipliers formed, then warp w updates the
// trailing rows w, w + nw, ... with its lanes on the columns and the pivot
// row held in registers (no index division in the inner loops).
template <int N, class Ops>
__device__ void cta_lu_rows(typename Ops::T* A, int* piv, int* s_flag, typename Ops::T* s_scal) {
  using T = typename Ops::T;
  constexpr int CJ = (N + 31) / 32;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int k = 0; k < N; ++k) {
    if (warp == 0) {
      float best = -1.0f;
      int bi = k;
      for (int r = k + lane; r < N; r += 32) {
        const float v = Ops::mag(A[r * N + k]);
        if (v > best) { best = v; bi = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if (lane == 0) {
        piv[k] = bi;
        s_scal[0] = A[bi * N + k];
        s_scal[1] = A[k * N + k];
        if (best == 0.0f) *s_flag = 1;
      }
    }
    __syncthreads();
    const int p = piv[k];
    const T pv = s_scal[0], akk = s_scal[1];
    // interchange rows k and p outside column k; column k gets the pivot and
    // the multipliers (row p's old entry is the old a_kk)
    if (p != k)
      for (int c = tid; c < N; c += nt)
        if (c != k) {
          const T t = A[k * N + c];
          A[k * N + c] = A[p * N + c];
          A[p * N + c] = t;
        }
    for (int r = k + tid; r < N; r += nt) {
      if (r == k) {
        A[k * N + k] = pv;
      } else {
        const T a = r == p ? akk : A[r * N + k];
        A[r * N + k] = Ops::nonzero(pv) ? Ops::div(a, pv) : Ops::zero();
      }
    }
    __syncthreads();
    T pk[CJ];
#pragma unroll
    for (int j = 0; j < CJ; ++j) {
      const int c = lane + 32 * j;
      pk[j] = (c > k && c < N) ? A[k * N + c] : Ops::zero();
    }
    int r = warp;
    if (r <= k) r += ((k + 1 - r + nw - 1) / nw) * nw;
    for (; r < N; r += nw) {
      const T m = A[r * N + k];
#pragma unroll
      for (int j = 0; j < CJ; ++j) {
        if (32 * j + 31 <= k) continue;  // whole 32-column chunk done (warp-uniform)
        const int c = lane + 32 * j;
        if (c > k && c < N) A[r * N + c] = Ops::fms(A[r * N + c], m, pk[j]);
      }
    }
    __syncthreads();
  }
}

// W <- A^{-1} W for ncol right-hand sides (column-major, length N) with the
// row-major LU of A and the row permutation perm (perm[r] = original
// row placed at r by the interchanges).  Warp w takes the columns w, w + nw,
// ... (CB of them at a time); lane l keeps rows l, l + 32, ... of those
// columns in registers, so an entry never leaves its lane and the
// substitutions need no block barrier: the entry of each pivot step is
// broadcast by shuffle.
template <int N, int CB, class Ops>
__device__ void cta_solve_cols(const typename Ops::T* A, const typename Ops::T* rdiag, const int* perm,
                               typename Ops::T* W, int ncol) {
  using T = typename Ops::T;
  constexpr int RI = (N + 31) / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int g0 = warp; g0 < ncol; g0 += nw * CB) {
    int nb = 0;  // columns of this group that exist (warp-uniform)
#pragma unroll
    for (int b = 0; b < CB; ++b)
      if (g0 + b * nw < ncol) nb = b + 1;
    T z[CB][RI];
#pragma unroll
    for (int b = 0; b < CB; ++b) {
      const int col = g0 + b * nw;
#pragma unroll
      for (int i = 0; i < RI; ++i) {
        const int r = lane + 32 * i;
        z[b][i] = (col < ncol && r < N) ? W[col * N + perm[r]] : Ops::zero();
      }
    }
    // forward substitution with the unit lower factor
#pragma unroll
    for (int kb = 0; kb < RI; ++kb) {
      for (int kl = 0; kl < 32; ++kl) {
        const int k = kb * 32 + kl;
        if (k >= N - 1) break;
        T wk[CB];
#pragma unroll
        for (int b = 0; b < CB; ++b) wk[b] = Ops::shfl(z[b][kb], kl);
#pragma unroll
        for (int i = 0; i < RI; ++i) {
          if (32 * i + 31 <= k) continue;  // rows of this chunk final (warp-uniform)
          const int r = lane + 32 * i;
          if (r > k && r < N) {
            const T l = A[r * N + k];
#pragma unroll
            for (int b = 0; b < CB; ++b)
              if (b < nb) z[b][i] = Ops::fms(z[b][i], l, wk[b]);
          }
        }
      }
    }
    // back substitution with the upper factor
#pragma unroll
    for (int kb = RI - 1; kb >= 0; --kb) {
      for (int kl = 31; kl >= 0; --kl) {
        const int k = kb * 32 + kl;
        if (k >= N) continue;
        const T rd = rdiag[k];
        T q[CB];
#pragma unroll
        for (int b = 0; b < CB; ++b) {
          if (b >= nb) continue;
          const T own = Ops::mul(z[b][kb], rd);  // meaningful in lane kl only
          q[b] = Ops::shfl(own, kl);
          if (lane == kl) z[b][kb] = q[b];
        }
#pragma unroll
        for (int i = 0; i < RI; ++i) {
          if (32 * i >= k) continue;  // no row of this chunk above k (warp-uniform)
          const int r = lane + 32 * i;
          if (r < k) {
            const T u = A[r * N + k];
#pragma unroll
            for (int b = 0; b < CB; ++b)
              if (b < nb) z[b][i] = Ops::fms(z[b][i], u, q[b]);
          }
        }
      }
    }
    __syncwarp();  // every lane's loads of the column precede the stores
#pragma unroll
    for (int b = 0; b < CB; ++b) {
      const int col = g0 + b * nw;
      if (col >= ncol) continue;
#pragma unroll
      for (int i = 0; i < RI; ++i) {
        const int r = lane + 32 * i;
        if (r < N) W[col * N + r] = z[b][i];
      }
    }
  }
}

// one thread: z <- A^{-1} z with the pair LU
__device__ void lu_solve_vec_pair(const pr* A, int n, const int* piv, pr* z) {
  for (int k = 0; k < n; ++k) {
    int p = piv[k];
    if (p != k) { pr t = z[k]; z[k] = z[p]; z[p] = t; }
  }
  for (int r = 0; r < n; ++r) {
    pr s = z[r];
    for (int c = 0; c < r; ++c) s = pr_fms(s, A[r * n + c], z[c]);
    z[r] = s;
  }
  for (int r = n - 1; r >= 0; --r) {
    pr s = z[r];
    for (int c = r + 1; c < n; ++c) s = pr_fms(s, A[r * n + c], z[c]);
    z[r] = pr_div(s, A[r * n + r]);
  }
}

template <int DIM>
__global__ void __launch_bounds__(1024)
    patch_factor_pair_kernel(LevelGeom g, const double* __restrict__ st, const unsigned char* __restrict__ mask,
                             double* __restrict__ coef, unsigned* __restrict__ d_err,
                             const int* __restrict__ work, const int* __restrict__ outidx) {
  using P = PatchDims<DIM>;
  constexpr int NU = P::NU, NP = P::NP, ND = P::ND, SP = P::SP;
  constexpr int NC = DIM * NP + 1;  // B columns and e_centre
  constexpr int C0 = DIM == 3 ? 13 : 4;  // neighbour index of the zero offset
  extern __shared__ double smem[];
  pr* K = reinterpret_cast<pr*>(smem);   // NU x NU
  pr* W = K + NU * NU;                   // NC x NU
  pr* S = W + NC * NU;                   // NP x NP
  pr* zp = S + NP * NP;                  // ND x NP
  double* du = reinterpret_cast<double*>(zp + ND * NP);  // NU
  double* dp = du + NU;                                 // NP
  int* pivK = reinterpret_cast<int*>(dp + NP);
  int* pivS = pivK + NU;
  long long* nodeU = reinterpret_cast<long long*>(((uintptr_t)(pivS + NP) + 7) & ~(uintptr_t)7);
  long long* nodeP = nodeU + NU;
  unsigned char* au = reinterpret_cast<unsigned char*>(nodeP + NP);
  unsigned char* ap = au + NU;
  int* perm = reinterpret_cast<int*>(((uintptr_t)(ap + NP) + 3) & ~(uintptr_t)3);  // NU
  pr* rdiag = reinterpret_cast<pr*>(((uintptr_t)(perm + NU) + 7) & ~(uintptr_t)7);  // NU
  __shared__ int s_flag;
  __shared__ pr s_scal[2];
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long widx = blockIdx.x;
  const long long i = work ? work[widx] : widx;
  const int ia[3] = {(int)(i % g.nn[0]), (int)((i / g.nn[0]) % g.nn[1]),
                     DIM == 3 ? (int)(i / ((long long)g.nn[0] * g.nn[1])) : 0};
  if (tid == 0) s_flag = 0;
  for (int v = tid; v < NU; v += nt) {
    int o[3];
    vel_off<DIM>(v, o);
    int b0 = ia[0] + o[0], b1 = ia[1] + o[1], b2 = ia[2] + o[2];
    bool in = b0 >= 0 && b0 <= g.n[0] && b1 >= 0 && b1 <= g.n[1] && (DIM == 2 || (b2 >= 0 && b2 <= g.n[2]));
    long long bn = in ? b0 + (long long)g.nn[0] * (b1 + (long long)g.nn[1] * b2) : -1;
    nodeU[v] = bn;
    au[v] = (unsigned char)(in && !(mask[bn] & 1));
  }
  for (int p = tid; p < NP; p += nt) {
    int o[3];
    prs_off<DIM>(p, o);
    int b0 = ia[0] + o[0], b1 = ia[1] + o[1], b2 = ia[2] + o[2];
    bool in = b0 >= 0 && b0 <= g.n[0] && b1 >= 0 && b1 <= g.n[1] && (DIM == 2 || (b2 >= 0 && b2 <= g.n[2]));
    nodeP[p] = in ? b0 + (long long)g.nn[0] * (b1 + (long long)g.nn[1] * b2) : -1;
    ap[p] = (unsigned char)in;
  }
  __syncthreads();
  // equilibration from the diagonal entries (float64)
  for (int v = tid; v < NU; v += nt) {
    double a = au[v] ? fabs(st[((long long)C0 * SP) * g.nnodes + nodeU[v]]) : 0.0;
    du[v] = (au[v] && a > 0.0) ? 1.0 / sqrt(a) : 1.0;
  }
  for (int p = tid; p < NP; p += nt) {
    double a = ap[p] ? fabs(st[((long long)C0 * SP + 1 + 2 * DIM) * g.nnodes + nodeP[p]]) : 0.0;
    dp[p] = (ap[p] && a > 0.0) ? 1.0 / sqrt(a) : 1.0;
  }
  __syncthreads();
  // gather, equilibrate (float64), store as pairs (structural zeros and the
  // identity rows of absent DoFs without float64 arithmetic)
  const int v0 = DIM == 3 ? 62 : 12, p0 = DIM == 3 ? 13 : 4;
  for (int e = tid; e < NU * NU; e += nt) {
    const int v = e / NU, w = e % NU;
    pr val = {v == w && !(au[v] && au[w]) ? 1.0f : 0.0f, 0.0f};
    if (au[v] && au[w]) {
      int ov[3], ow[3], d[3];
      vel_off<DIM>(v, ov);
      vel_off<DIM>(w, ow);
      bool adj = true;
      for (int k = 0; k < 3; ++k) { d[k] = ow[k] - ov[k]; if (d[k] < -1 || d[k] > 1) adj = false; }
      if (adj) val = pr_from(du[v] * st[((long long)nb_index<DIM>(d) * SP) * g.nnodes + nodeU[v]] * du[w]);
    }
    K[e] = val;
  }
  for (int e = tid; e < DIM * NP * NU; e += nt) {
    const int col = e / NU, v = e % NU, c = col / NP, p = col % NP;
    pr val = {0.0f, 0.0f};
    if (au[v] && ap[p]) {
      int ov[3], op[3], d[3];
      vel_off<DIM>(v, ov);
      prs_off<DIM>(p, op);
      bool adj = true;
      for (int k = 0; k < 3; ++k) { d[k] = op[k] - ov[k]; if (d[k] < -1 || d[k] > 1) adj = false; }
      if (adj) val = pr_from(du[v] * st[((long long)nb_index<DIM>(d) * SP + 1 + c) * g.nnodes + nodeU[v]] * dp[p]);
    }
    W[e] = val;
  }
  for (int v = tid; v < NU; v += nt) W[(DIM * NP) * NU + v] = pr{v == v0 ? 1.0f : 0.0f, 0.0f};
  for (int e = tid; e < NP * NP; e += nt) {
    const int p = e / NP, q = e % NP;
    pr val = {p == q && !(ap[p] && ap[q]) ? 1.0f : 0.0f, 0.0f};
    if (ap[p] && ap[q]) {
      int op[3], oq[3], d[3];
      prs_off<DIM>(p, op);
      prs_off<DIM>(q, oq);
      bool adj = true;
      for (int k = 0; k < 3; ++k) { d[k] = oq[k] - op[k]; if (d[k] < -1 || d[k] > 1) adj = false; }
      if (adj) val = pr_from(dp[p] * st[((long long)nb_index<DIM>(d) * SP + 1 + 2 * DIM) * g.nnodes + nodeP[p]] * dp[q]);
    }
    S[e] = val;
  }
  __syncthreads();
  cta_lu_rows<NU, OpsPair>(K, pivK, &s_flag, s_scal);
  // reciprocals of the pivots for the back substitution
  for (int k = tid; k < NU; k += nt) {
    const pr d = K[k * NU + k];
    rdiag[k] = d.h != 0.0f ? pr_div({1.0f, 0.0f}, d) : pr{0.0f, 0.0f};
  }
  if (tid == 0) {
    for (int r = 0; r < NU; ++r) perm[r] = r;
    for (int k = 0; k < NU; ++k) {
      const int pk = pivK[k];
      const int t = perm[k];
      perm[k] = perm[pk];
      perm[pk] = t;
    }
  }
  __syncthreads();
  cta_solve_cols<NU, 3, OpsPair>(K, rdiag, perm, W, NC);
  __syncthreads();
  // the LU of K~ is no longer needed: its space takes B~ in compact form,
  // Bc[(p * NT + t) * DIM + c] = B~_c of pressure p and its neighbour
  // velocity node t (3^d box around p)
  constexpr int NT = DIM == 3 ? 27 : 9;
  pr* Bc = K;
  for (int e = tid; e < NP * NT * DIM; e += nt) {
    const int p = e / (NT * DIM), rem = e - p * (NT * DIM), t = rem / DIM, c = rem - t * DIM;
    int op[3];
    prs_off<DIM>(p, op);
    const int d[3] = {t % 3 - 1, (t / 3) % 3 - 1, DIM == 3 ? t / 9 - 1 : 0};
    const int v = (op[0] + d[0] + 2) + 5 * (op[1] + d[1] + 2) + (DIM == 3 ? 25 * (op[2] + d[2] + 2) : 0);
    pr val = {0.0f, 0.0f};
    if (ap[p] && au[v]) {
      const int dvp[3] = {-d[0], -d[1], -d[2]};
      const long long base = (long long)nb_index<DIM>(dvp) * SP;
      val = pr_from(du[v] * st[(base + 1 + c) * g.nnodes + nodeU[v]] * dp[p]);
    }
    Bc[e] = val;
  }
  __syncthreads();
  // S~ = C~ - sum_c B~_c^T W~_c
  for (int e = tid; e < NP * NP; e += nt) {
    const int p = e / NP, q = e % NP;
    pr sv = S[e];
    if (ap[p]) {
      int op[3];
      prs_off<DIM>(p, op);
      for (int t = 0; t < NT; ++t) {
        const int d[3] = {t % 3 - 1, (t / 3) % 3 - 1, DIM == 3 ? t / 9 - 1 : 0};
        const int v = (op[0] + d[0] + 2) + 5 * (op[1] + d[1] + 2) + (DIM == 3 ? 25 * (op[2] + d[2] + 2) : 0);
        if (!au[v]) continue;
        for (int c = 0; c < DIM; ++c) sv = pr_fms(sv, Bc[(p * NT + t) * DIM + c], W[(c * NP + q) * NU + v]);
      }
    }
    S[e] = sv;
  }
  __syncthreads();
  cta_lu_rows<NP, OpsPair>(S, pivS, &s_flag, s_scal);
  if (s_flag && tid == 0) atomicOr(d_err, kErrSingularPatch);
  // owned rows: velocity c -> z_p = -S~^{-1} (row v0 of W~_c); pressure -> S~^{-1} e_p0
  if (tid < ND) {
    pr* z = zp + tid * NP;
    for (int q = 0; q < NP; ++q) {
      pr w = W[(tid * NP + q) * NU + v0];
      z[q] = tid < DIM ? pr{-w.h, -w.l} : pr{q == p0 ? 1.0f : 0.0f, 0.0f};
    }
    lu_solve_vec_pair(S, NP, pivS, z);
  }
  __syncthreads();
  double* out = coef + (outidx ? (long long)outidx[widx] : widx) * P::NSLOT * ND;
  for (int j = tid; j < P::NSLOT; j += nt) {
    double vals[ND];
    if (j < NU * DIM) {
      int v = j / DIM, c2 = j % DIM;
      for (int k = 0; k < ND; ++k) {
        double z = 0.0;
        if (au[v]) {
          pr s = (k == c2) ? W[(DIM * NP) * NU + v] : pr{0.0f, 0.0f};
          for (int q = 0; q < NP; ++q) s = pr_fms(s, W[(c2 * NP + q) * NU + v], zp[k * NP + q]);
          z = pr_to(s);
        }
        bool own_ok = k < DIM ? au[v0] != 0 : true;
        double dk = k < DIM ? du[v0] : dp[p0];
        vals[k] = (own_ok && au[v]) ? dk * z * du[v] : 0.0;
      }
    } else {
      int p = j - NU * DIM;
      for (int k = 0; k < ND; ++k) {
        bool own_ok = k < DIM ? au[v0] != 0 : true;
        double dk = k < DIM ? du[v0] : dp[p0];
        vals[k] = (own_ok && ap[p]) ? dk * pr_to(zp[k * NP + p]) * dp[p] : 0.0;
      }
    }
    for (int k = 0; k < ND; ++k) out[(long long)j * ND + k] = vals[k];
  }
}

// ---------------------------------------------------------------------------
// Float32 factorisation with iterative refinement, for rows stored in
// float32 or bfloat16.  The equilibrated block M~ = D L_i D (absent DoFs as
// identity rows) is gathered once in float64 and kept in float pairs in its
// sparse form (A~: 3^d velocity neighbours per velocity node; B~_c and C~ by
// pressure node and neighbour); its dense blocks are factored in float32
// (LU of A~, W = A~^{-1} B~, the Schur complement S~ = C~ - sum_c B~_c' W_c
// and its LU).  The owned columns z_k = M~^{-1} e_k (= the owned rows, M~
// being symmetric) are then solved with these factors through the block
// elimination and refined twice: r = e_k - M~ z_k in float pairs from the
// exact entries, z_k += M~^{-1} r.  Each step multiplies the error by about
// cond(M~) x 2^-24, so the rows reach float64-class accuracy before they are
// rounded to float32 / bfloat16, at a fraction of the cost of float-pair
// elimination.  Where cond(M~) x 2^-24 is not small the refinement does not
// converge; such patches are listed (redo_node / redo_out) for the
// float-pair elimination.
template <int DIM>
__global__ void __launch_bounds__(1024)
    patch_factor_ir_kernel(LevelGeom g, const double* __restrict__ st, const unsigned char* __restrict__ mask,
                           double* __restrict__ coef, unsigned* __restrict__ d_err,
                           const int* __restrict__ work, int* __restrict__ redo_node, int* __restrict__ redo_out,
                           int* __restrict__ nredo) {
  using P = PatchDims<DIM>;
  constexpr int NU = P::NU, NP = P::NP, ND = P::ND, SP = P::SP, NSLOT = P::NSLOT;
  constexpr int NT = DIM == 3 ? 27 : 9;   // 3^d neighbour offsets
  constexpr int NB = DIM * NP;            // columns of B~
  constexpr int NV = ND * DIM;            // velocity blocks of the ND owned vectors
  constexpr int C0 = DIM == 3 ? 13 : 4;   // offset index of the zero offset
  constexpr int NPASS = 3;                // first solve and two refinements
  const int v0 = DIM == 3 ? 62 : 12, p0 = DIM == 3 ? 13 : 4;
  extern __shared__ double smem[];
  pr* Asp = reinterpret_cast<pr*>(smem);  // [v][t]
  pr* Bsp = Asp + NU * NT;                // [(p * NT + t) * DIM + c]
  pr* Csp = Bsp + NP * NT * DIM;          // [p][t]
  pr* Zv = Csp + NP * NT;                 // [(k * DIM + c) * NU + v]
  pr* Zp = Zv + NV * NU;                  // [k * NP + p]
  double* du = reinterpret_cast<double*>(Zp + ND * NP);
  double* dp = du + NU;
  float* Af = reinterpret_cast<float*>(dp + NP);  // NU x NU
  float* Wf = Af + NU * NU;               // NB columns of NU
  float* Sf = Wf + NB * NU;               // NP x NP
  float* Rv = Sf + NP * NP;               // NV columns of NU
  float* Rp = Rv + NV * NU;               // ND x NP
  float* Hp = Rp + ND * NP;               // ND x NP
  float* rdiag = Hp + ND * NP;            // NU
  int* pivA = reinterpret_cast<int*>(rdiag + NU);
  int* permA = pivA + NU;
  int* pivS = permA + NU;
  long long* nodeU = reinterpret_cast<long long*>(((uintptr_t)(pivS + NP) + 7) & ~(uintptr_t)7);
  long long* nodeP = nodeU + NU;
  unsigned char* au = reinterpret_cast<unsigned char*>(nodeP + NP);
  unsigned char* ap = au + NU;
  __shared__ int s_flag;
  __shared__ float s_scal[2];
  __shared__ int s_rmax;  // largest |residual| of the last refinement (float bits)
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long widx = blockIdx.x;
  const long long i = work ? work[widx] : widx;
  const int ia[3] = {(int)(i % g.nn[0]), (int)((i / g.nn[0]) % g.nn[1]),
                     DIM == 3 ? (int)(i / ((long long)g.nn[0] * g.nn[1])) : 0};
  if (tid == 0) s_flag = 0;
  for (int v = tid; v < NU; v += nt) {
    int o[3];
    vel_off<DIM>(v, o);
    const int b0 = ia[0] + o[0], b1 = ia[1] + o[1], b2 = ia[2] + o[2];
    const bool in = b0 >= 0 && b0 <= g.n[0] && b1 >= 0 && b1 <= g.n[1] && (DIM == 2 || (b2 >= 0 && b2 <= g.n[2]));
    const long long bn = in ? b0 + (long long)g.nn[0] * (b1 + (long long)g.nn[1] * b2) : -1;
    nodeU[v] = bn;
    au[v] = (unsigned char)(in && !(mask[bn] & 1));
  }
  for (int p = tid; p < NP; p += nt) {
    int o[3];
    prs_off<DIM>(p, o);
    const int b0 = ia[0] + o[0], b1 = ia[1] + o[1], b2 = ia[2] + o[2];
    const bool in = b0 >= 0 && b0 <= g.n[0] && b1 >= 0 && b1 <= g.n[1] && (DIM == 2 || (b2 >= 0 && b2 <= g.n[2]));
    nodeP[p] = in ? b0 + (long long)g.nn[0] * (b1 + (long long)g.nn[1] * b2) : -1;
    ap[p] = (unsigned char)in;
  }
  __syncthreads();
  for (int v = tid; v < NU; v += nt) {
    const double a = au[v] ? fabs(st[((long long)C0 * SP) * g.nnodes + nodeU[v]]) : 0.0;
    du[v] = (au[v] && a > 0.0) ? 1.0 / sqrt(a) : 1.0;
  }
  for (int p = tid; p < NP; p += nt) {
    const double a = ap[p] ? fabs(st[((long long)C0 * SP + 1 + 2 * DIM) * g.nnodes + nodeP[p]]) : 0.0;
    dp[p] = (ap[p] && a > 0.0) ? 1.0 / sqrt(a) : 1.0;
  }
  // dense float32 blocks start from zero
  for (int e = tid; e < NU * NU; e += nt) Af[e] = 0.0f;
  for (int e = tid; e < NB * NU; e += nt) Wf[e] = 0.0f;
  for (int e = tid; e < NP * NP; e += nt) Sf[e] = 0.0f;
  __syncthreads();
  // the sparse equilibrated entries, float64 products kept as pairs
  for (int e = tid; e < NU * NT; e += nt) {
    const int v = e / NT, t = e - v * NT;
    const int d[3] = {t % 3 - 1, (t / 3) % 3 - 1, DIM == 3 ? t / 9 - 1 : 0};
    int ov[3];
    vel_off<DIM>(v, ov);
    const int ow[3] = {ov[0] + d[0], ov[1] + d[1], ov[2] + d[2]};
    const bool inbox = ow[0] >= -2 && ow[0] <= 2 && ow[1] >= -2 && ow[1] <= 2 && ow[2] >= -2 && ow[2] <= 2;
    pr val = {t == C0 && !au[v] ? 1.0f : 0.0f, 0.0f};
    if (inbox) {
      const int w = (ow[0] + 2) + 5 * (ow[1] + 2) + (DIM == 3 ? 25 * (ow[2] + 2) : 0);
      if (au[v] && au[w]) val = pr_from(du[v] * st[((long long)nb_index<DIM>(d) * SP) * g.nnodes + nodeU[v]] * du[w]);
      if (val.h != 0.0f) Af[v * NU + w] = val.h;
    }
    Asp[e] = val;
  }
  for (int e = tid; e < NP * NT * DIM; e += nt) {
    const int p = e / (NT * DIM), rem = e - p * (NT * DIM), t = rem / DIM, c = rem - t * DIM;
    int op[3];
    prs_off<DIM>(p, op);
    const int d[3] = {t % 3 - 1, (t / 3) % 3 - 1, DIM == 3 ? t / 9 - 1 : 0};
    const int v = (op[0] + d[0] + 2) + 5 * (op[1] + d[1] + 2) + (DIM == 3 ? 25 * (op[2] + d[2] + 2) : 0);
    pr val = {0.0f, 0.0f};
    if (ap[p] && au[v]) {
      const int dvp[3] = {-d[0], -d[1], -d[2]};
      val = pr_from(du[v] * st[((long long)nb_index<DIM>(dvp) * SP + 1 + c) * g.nnodes + nodeU[v]] * dp[p]);
      Wf[(c * NP + p) * NU + v] = val.h;
    }
    Bsp[e] = val;
  }
  for (int e = tid; e < NP * NT; e += nt) {
    const int p = e / NT, t = e - p * NT;
    const int d[3] = {t % 3 - 1, (t / 3) % 3 - 1, DIM == 3 ? t / 9 - 1 : 0};
    int op[3];
    prs_off<DIM>(p, op);
    const int oq[3] = {op[0] + d[0], op[1] + d[1], op[2] + d[2]};
    const bool inbox = oq[0] >= -1 && oq[0] <= 1 && oq[1] >= -1 && oq[1] <= 1 && oq[2] >= -1 && oq[2] <= 1;
    pr val = {t == C0 && !ap[p] ? 1.0f : 0.0f, 0.0f};
    if (inbox) {
      const int q = (oq[0] + 1) + 3 * (oq[1] + 1) + (DIM == 3 ? 9 * (oq[2] + 1) : 0);
      if (ap[p] && ap[q])
        val = pr_from(dp[p] * st[((long long)nb_index<DIM>(d) * SP + 1 + 2 * DIM) * g.nnodes + nodeP[p]] * dp[q]);
      if (val.h != 0.0f) Sf[p * NP + q] = val.h;
    }
    Csp[e] = val;
  }
  __syncthreads();
  // float32 LU of A~, W = A~^{-1} B~, S~ and its LU
  cta_lu_rows<NU, OpsF32>(Af, pivA, &s_flag, s_scal);
  for (int k = tid; k < NU; k += nt) {
    const float dk = Af[k * NU + k];
    rdiag[k] = dk != 0.0f ? 1.0f / dk : 0.0f;
  }
  if (tid == 0) {
    for (int r = 0; r < NU; ++r) permA[r] = r;
    for (int k = 0; k < NU; ++k) {
      const int pk = pivA[k];
      const int tmp = permA[k];
      permA[k] = permA[pk];
      permA[pk] = tmp;
    }
  }
  __syncthreads();
  cta_solve_cols<NU, 3, OpsF32>(Af, rdiag, permA, Wf, NB);
  __syncthreads();
  for (int e = tid; e < NP * NP; e += nt) {
    const int p = e / NP, q = e - p * NP;
    float sv = Sf[e];
    if (ap[p]) {
      int op[3];
      prs_off<DIM>(p, op);
      for (int t = 0; t < NT; ++t) {
        const int d[3] = {t % 3 - 1, (t / 3) % 3 - 1, DIM == 3 ? t / 9 - 1 : 0};
        const int v = (op[0] + d[0] + 2) + 5 * (op[1] + d[1] + 2) + (DIM == 3 ? 25 * (op[2] + d[2] + 2) : 0);
        if (!au[v]) continue;
        for (int c = 0; c < DIM; ++c) sv = fmaf(-Bsp[(p * NT + t) * DIM + c].h, Wf[(c * NP + q) * NU + v], sv);
      }
    }
    Sf[e] = sv;
  }
  __syncthreads();
  cta_lu_rows<NP, OpsF32>(Sf, pivS, &s_flag, s_scal);
  if (s_flag && tid == 0) atomicOr(d_err, kErrSingularPatch);
  // right-hand sides e_k (owned velocity components, then the owned
  // pressure) and zero solutions
  for (int e = tid; e < NV * NU; e += nt) {
    const int col = e / NU, v = e - col * NU, k = col / DIM, c = col - k * DIM;
    Rv[e] = (k < DIM && c == k && v == v0) ? 1.0f : 0.0f;
    Zv[e] = {0.0f, 0.0f};
  }
  for (int e = tid; e < ND * NP; e += nt) {
    const int k = e / NP, p = e - k * NP;
    Rp[e] = (k == DIM && p == p0) ? 1.0f : 0.0f;
    Zp[e] = {0.0f, 0.0f};
  }
  __syncthreads();
  for (int pass = 0; pass < NPASS; ++pass) {
    // block solve M~ (u, p) = (Rv, Rp) in float32, in place
    cta_solve_cols<NU, 3, OpsF32>(Af, rdiag, permA, Rv, NV);  // y_c = A~^{-1} f_c
    __syncthreads();
    for (int e = tid; e < ND * NP; e += nt) {  // h = g - sum_c B~_c' y_c
      const int k = e / NP, p = e - k * NP;
      float h = Rp[e];
      int op[3];
      prs_off<DIM>(p, op);
      for (int t = 0; t < NT; ++t) {
        const int d[3] = {t % 3 - 1, (t / 3) % 3 - 1, DIM == 3 ? t / 9 - 1 : 0};
        const int v = (op[0] + d[0] + 2) + 5 * (op[1] + d[1] + 2) + (DIM == 3 ? 25 * (op[2] + d[2] + 2) : 0);
        for (int c = 0; c < DIM; ++c) h = fmaf(-Bsp[(p * NT + t) * DIM + c].h, Rv[(k * DIM + c) * NU + v], h);
      }
      Hp[e] = h;
    }
    __syncthreads();
    if (tid < ND) {  // p = S~^{-1} h
      float* z = Hp + tid * NP;
      for (int k = 0; k < NP; ++k) {
        const int pk = pivS[k];
        if (pk != k) { const float tmp = z[k]; z[k] = z[pk]; z[pk] = tmp; }
      }
      for (int r = 0; r < NP; ++r) {
        float sv = z[r];
        for (int c = 0; c < r; ++c) sv = fmaf(-Sf[r * NP + c], z[c], sv);
        z[r] = sv;
      }
      for (int r = NP - 1; r >= 0; --r) {
        float sv = z[r];
        for (int c = r + 1; c < NP; ++c) sv = fmaf(-Sf[r * NP + c], z[c], sv);
        z[r] = sv / Sf[r * NP + r];
      }
    }
    __syncthreads();
    for (int e = tid; e < NV * NU; e += nt) {  // u_c = y_c - W_c p, then z += (u, p)
      const int col = e / NU, v = e - col * NU, k = col / DIM, c = col - k * DIM;
      float u = Rv[e];
      for (int q = 0; q < NP; ++q) u = fmaf(-Wf[(c * NP + q) * NU + v], Hp[k * NP + q], u);
      Zv[e] = pr_add(Zv[e], {u, 0.0f});
    }
    for (int e = tid; e < ND * NP; e += nt) Zp[e] = pr_add(Zp[e], {Hp[e], 0.0f});
    if (tid == 0) s_rmax = 0;
    __syncthreads();
    // residual e_k - M~ z in float pairs from the sparse entries (after the
    // last solve it only measures convergence)
    float rmax = 0.0f;
    for (int e = tid; e < NV * NU; e += nt) {
      const int col = e / NU, v = e - col * NU, k = col / DIM, c = col - k * DIM;
      pr sv = {(k < DIM && c == k && v == v0) ? 1.0f : 0.0f, 0.0f};
      int ov[3];
      vel_off<DIM>(v, ov);
      for (int t = 0; t < NT; ++t) {
        const int d[3] = {t % 3 - 1, (t / 3) % 3 - 1, DIM == 3 ? t / 9 - 1 : 0};
        const int ow[3] = {ov[0] + d[0], ov[1] + d[1], ov[2] + d[2]};
        if (ow[0] < -2 || ow[0] > 2 || ow[1] < -2 || ow[1] > 2 || ow[2] < -2 || ow[2] > 2) continue;
        const int w = (ow[0] + 2) + 5 * (ow[1] + 2) + (DIM == 3 ? 25 * (ow[2] + 2) : 0);
        sv = pr_fms(sv, Asp[v * NT + t], Zv[(k * DIM + c) * NU + w]);
        // pressure neighbour at the same offset (the 3^d box around the
        // patch centre), coupled through B~_c(v, q)
        const int oq[3] = {ov[0] + d[0], ov[1] + d[1], ov[2] + d[2]};
        if (oq[0] < -1 || oq[0] > 1 || oq[1] < -1 || oq[1] > 1 || oq[2] < -1 || oq[2] > 1) continue;
        const int q = (oq[0] + 1) + 3 * (oq[1] + 1) + (DIM == 3 ? 9 * (oq[2] + 1) : 0);
        // v relative to q is -d: offset index of -d
        const int tq = (-d[0] + 1) + 3 * (-d[1] + 1) + (DIM == 3 ? 9 * (-d[2] + 1) : 0);
        sv = pr_fms(sv, Bsp[(q * NT + tq) * DIM + c], Zp[k * NP + q]);
      }
      Rv[e] = sv.h + sv.l;
      rmax = fmaxf(rmax, fabsf(sv.h));
    }
    for (int e = tid; e < ND * NP; e += nt) {
      const int k = e / NP, p = e - k * NP;
      pr sv = {(k == DIM && p == p0) ? 1.0f : 0.0f, 0.0f};
      int op[3];
      prs_off<DIM>(p, op);
      for (int t = 0; t < NT; ++t) {
        const int d[3] = {t % 3 - 1, (t / 3) % 3 - 1, DIM == 3 ? t / 9 - 1 : 0};
        const int v = (op[0] + d[0] + 2) + 5 * (op[1] + d[1] + 2) + (DIM == 3 ? 25 * (op[2] + d[2] + 2) : 0);
        for (int c = 0; c < DIM; ++c) sv = pr_fms(sv, Bsp[(p * NT + t) * DIM + c], Zv[(k * DIM + c) * NU + v]);
        const int oq[3] = {op[0] + d[0], op[1] + d[1], op[2] + d[2]};
        if (oq[0] < -1 || oq[0] > 1 || oq[1] < -1 || oq[1] > 1 || oq[2] < -1 || oq[2] > 1) continue;
        const int q = (oq[0] + 1) + 3 * (oq[1] + 1) + (DIM == 3 ? 9 * (oq[2] + 1) : 0);
        sv = pr_fms(sv, Csp[p * NT + t], Zp[k * NP + q]);
      }
      Rp[e] = sv.h + sv.l;
      rmax = fmaxf(rmax, fabsf(sv.h));
    }
    // a NaN compares false everywhere: count it as no convergence
    if (rmax != rmax) rmax = 3.0e38f;
    atomicMax(&s_rmax, __float_as_int(rmax));
    __syncthreads();
  }
  // Refinement that did not bring the residual of the unit right-hand sides
  // below 1e-9 (an equilibrated block too ill-conditioned for float32
  // factors, typically a badly cut patch): the patch goes on the list that
  // the float-pair elimination rebuilds afterwards.
  if (tid == 0 && nredo && s_rmax > __float_as_int(1.0e-9f)) {
    const int slot = atomicAdd(nredo, 1);
    redo_node[slot] = (int)i;
    redo_out[slot] = (int)widx;
  }
  // owned rows of L_i^{-1} = D z_k D, in the slot layout
  double* out = coef + widx * NSLOT * ND;
  for (int j = tid; j < NSLOT; j += nt) {
    double vals[ND];
    if (j < NU * DIM) {
      const int v = j / DIM, c2 = j % DIM;
      for (int k = 0; k < ND; ++k) {
        const bool own_ok = k < DIM ? au[v0] != 0 : true;
        const double dk = k < DIM ? du[v0] : dp[p0];
        vals[k] = (own_ok && au[v]) ? dk * pr_to(Zv[(k * DIM + c2) * NU + v]) * du[v] : 0.0;
      }
    } else {
      const int p = j - NU * DIM;
      for (int k = 0; k < ND; ++k) {
        const bool own_ok = k < DIM ? au[v0] != 0 : true;
        const double dk = k < DIM ? du[v0] : dp[p0];
        vals[k] = (own_ok && ap[p]) ? dk * pr_to(Zp[k * NP + p]) * dp[p] : 0.0;
      }
    }
    for (int k = 0; k < ND; ++k) out[(long long)j * ND + k] = vals[k];
  }
}

template <int DIM>
size_t ir_factor_smem() {
  using P = PatchDims<DIM>;
  constexpr int NT = DIM == 3 ? 27 : 9, NB = DIM * P::NP, NV = P::ND * DIM;
  size_t b = (size_t)(P::NU * NT + P::NP * NT * DIM + P::NP * NT + NV * P::NU + P::ND * P::NP) * 8 +
             (size_t)(P::NU + P::NP) * 8 +
             (size_t)(P::NU * P::NU + NB * P::NU + P::NP * P::NP + NV * P::NU + 2 * P::ND * P::NP + P::NU) * 4 +
             (size_t)(2 * P::NU + P::NP) * 4 + 8 + (size_t)(P::NU + P::NP) * 8 + (P::NU + P::NP) + 16;
  return (b + 15) & ~(size_t)15;
}

template <int DIM>
cudaError_t run_ir_factor(const LevelGeom& g, const double* st, const unsigned char* mask, double* coef,
                          unsigned* d_err, const int* work, long long nwork, int* redo_node, int* redo_out,
                          int* nredo, cudaStream_t s) {
  const size_t sm = ir_factor_smem<DIM>();
  auto kern = patch_factor_ir_kernel<DIM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const long long nb = work ? nwork : g.nnodes;
  if (nb <= 0) return cudaSuccess;
  int threads = DIM == 3 ? 1024 : 128;
  if (const char* env = getenv("FC_FACTOR_THREADS")) {
    const int t = atoi(env);
    if (t >= 64 && t <= 1024 && t % 32 == 0) threads = t;
  }
  kern<<<(unsigned)nb, threads, sm, s>>>(g, st, mask, coef, d_err, work, redo_node, redo_out, nredo);
  note_launches(1);
  return cudaGetLastError();
}

template <int DIM>
size_t pair_factor_smem() {
  using P = PatchDims<DIM>;
  const int NC = DIM * P::NP + 1;
  size_t b = (size_t)(P::NU * P::NU + NC * P::NU + P::NP * P::NP + P::ND * P::NP) * 8 +
             (P::NU + P::NP) * 8 + (P::NU + P::NP) * 4 + 8 + (P::NU + P::NP) * 8 + (P::NU + P::NP) + 16 +
             P::NU * 4 + 4 + P::NU * 8 + 8;
  return (b + 15) & ~(size_t)15;
}

template <int DIM>
cudaError_t run_pair_factor(const LevelGeom& g, const double* st, const unsigned char* mask, double* coef,
                            unsigned* d_err, const int* work, long long nwork, const int* outidx,
                            cudaStream_t s) {
  size_t sm = pair_factor_smem<DIM>();
  auto kern = patch_factor_pair_kernel<DIM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const long long nb = work ? nwork : g.nnodes;
  if (nb <= 0) return cudaSuccess;
  int threads = DIM == 3 ? 1024 : 128;
  if (const char* env = getenv("FC_FACTOR_THREADS")) {
    int t = atoi(env);
    if (t >= 64 && t <= 1024 && t % 32 == 0) threads = t;
  }
  kern<<<(unsigned)nb, threads, sm, s>>>(g, st, mask, coef, d_err, work, outidx);
  note_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Q2-Q1 patches (2D).  Patch of vertex a: the Q2 nodes 2a - 4 .. 2a + 4 per
// direction (81 nodes, 2 components, node-major) and the pressures of the
// vertices a - 1 .. a + 1 (9): 171 slots; constrained and out-of-grid DoFs
// are absent (zero coefficients).  The vertex owns the Q2 nodes 2a + s,
// s in {0,1}^2, with both components (rows 2 (sx + 2 sy) + c) and its
// pressure (row 8).  The local solve is exact (Sec. 3.1.2) on the
// symmetrically scaled block D L_i D, D = (largest entry of the row)^{-1/2}
// taken per velocity node over both components, by block elimination:
// K~ = LU (partial pivoting), W~_c = K~^{-1} B~_c, S~ = -sum_c B~_c' W~_c
// (the pressure block of Q2-Q1 is zero), LU of S~.
struct Q2P {
  static constexpr int NV = 81, NP = 9, NSV = 162, NS = 171, NROWP = 10;  // 9 owned rows, padded
};

__device__ __forceinline__ bool q2_in(const Q2Grid& q, int I, int J) { return I >= 0 && I < q.nf[0] && J >= 0 && J < q.nf[1]; }

__global__ void __launch_bounds__(256)
    q2_patch_rows_kernel(Q2Grid q, const double* __restrict__ A, const double* __restrict__ B,
                         const unsigned char* __restrict__ mask, double* __restrict__ coef, unsigned* d_err) {
  constexpr int NV = Q2P::NV, NP = Q2P::NP;
  extern __shared__ double q2sm[];
  double* K = q2sm;                      // NV x NV row-major
  double* Bs = K + NV * NV;              // [c][NV][NP]
  double* W = Bs + 2 * NV * NP;          // [c*NP + q][NV] column-major
  double* S = W + 2 * NP * NV;           // NP x NP
  double* dv = S + NP * NP;              // NV
  double* dp = dv + NV;                  // NP
  double* Y = dp + NP;                   // [4][NV] owned velocity columns of K~^{-1}
  double* pv = Y + 4 * NV;               // [9][NP] pressure parts of the owned rows
  int* piv = reinterpret_cast<int*>(pv + 9 * NP);  // NV + NP
  int* act = piv + NV + NP;                        // NV + NP
  int* flag = act + NV + NP;
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long v = blockIdx.x;
  const int ax = (int)(v % q.nv1[0]), ay = (int)(v / q.nv1[0]);
  if (tid == 0) *flag = 0;
  for (int j = tid; j < NV + NP; j += nt) {
    if (j < NV) {
      const int I = 2 * ax - 4 + j % 9, J = 2 * ay - 4 + j / 9;
      act[j] = q2_in(q, I, J) && !mask[I + (long long)q.nf[0] * J];
    } else {
      const int t = j - NV, X = ax - 1 + t % 3, Y2 = ay - 1 + t / 3;
      act[j] = X >= 0 && X < q.nv1[0] && Y2 >= 0 && Y2 < q.nv1[1];
    }
  }
  __syncthreads();
  // gather K and B_c
  for (int t = tid; t < NV * NV; t += nt) {
    const int r = t / NV, c = t % NV;
    double val = 0.0;
    if (act[r] && act[c]) {
      const int ox = c % 9 - r % 9, oy = c / 9 - r / 9;
      if (ox >= -2 && ox <= 2 && oy >= -2 && oy <= 2) {
        const int I = 2 * ax - 4 + r % 9, J = 2 * ay - 4 + r / 9;
        const long long i = I + (long long)q.nf[0] * J;
        val = A[(long long)((ox + 2) + 5 * (oy + 2)) * q.nq + i];
      }
    } else if (r == c) {
      val = 1.0;
    }
    K[t] = val;
  }
  for (int t = tid; t < 2 * NV * NP; t += nt) {
    const int cc = t / (NV * NP), r = (t / NP) % NV, pq = t % NP;
    double val = 0.0;
    if (act[r] && act[NV + pq]) {
      const int I = 2 * ax - 4 + r % 9, J = 2 * ay - 4 + r / 9;
      const int X = ax - 1 + pq % 3, Y2 = ay - 1 + pq / 3;
      const int ox = X - (I / 2 - 1), oy = Y2 - (J / 2 - 1);
      if (ox >= 0 && ox <= 2 && oy >= 0 && oy <= 2) {
        const long long i = I + (long long)q.nf[0] * J;
        val = B[((long long)(ox + 3 * oy) * 2 + cc) * q.nq + i];
      }
    }
    Bs[t] = val;
  }
  __syncthreads();
  // scaling
  for (int j = tid; j < NV + NP; j += nt) {
    double m = 0.0;
    if (j < NV) {
      for (int c = 0; c < NV; ++c) m = fmax(m, fabs(K[j * NV + c]));
      for (int cc = 0; cc < 2; ++cc)
        for (int pq = 0; pq < NP; ++pq) m = fmax(m, fabs(Bs[(cc * NV + j) * NP + pq]));
      dv[j] = act[j] && m > 0.0 ? 1.0 / sqrt(m) : 1.0;
    } else {
      const int pq = j - NV;
      for (int cc = 0; cc < 2; ++cc)
        for (int r = 0; r < NV; ++r) m = fmax(m, fabs(Bs[(cc * NV + r) * NP + pq]));
      dp[pq] = act[j] && m > 0.0 ? 1.0 / sqrt(m) : 1.0;
    }
  }
  __syncthreads();
  for (int t = tid; t < NV * NV; t += nt) K[t] = dv[t / NV] * K[t] * dv[t % NV];
  for (int t = tid; t < 2 * NV * NP; t += nt) {
    const int r = (t / NP) % NV, pq = t % NP;
    Bs[t] = dv[r] * Bs[t] * dp[pq];
  }
  __syncthreads();
  cta_lu(K, NV, NV, piv, flag);
  // W~_c = K~^{-1} B~_c (columns c*NP + q)
  for (int t = tid; t < 2 * NP * NV; t += nt) {
    const int col = t / NV, r = t % NV, cc = col / NP, pq = col % NP;
    W[t] = Bs[(cc * NV + r) * NP + pq];
  }
  __syncthreads();
  cta_lu_solve_multi(K, NV, piv, W, 2 * NP);
  // S~ = -sum_c B~_c' W~_c (identity rows for absent pressures)
  for (int t = tid; t < NP * NP; t += nt) {
    const int r = t / NP, c = t % NP;
    double sum = 0.0;
    if (act[NV + r] && act[NV + c]) {
      for (int cc = 0; cc < 2; ++cc)
        for (int p = 0; p < NV; ++p) sum = sum - Bs[(cc * NV + p) * NP + r] * W[(cc * NP + c) * NV + p];
    } else if (r == c) {
      sum = 1.0;
    }
    S[t] = sum;
  }
  // the columns of K~^{-1} at the owned velocity nodes
  for (int t = tid; t < 4 * NV; t += nt) {
    const int s2 = t / NV, r = t % NV;
    const int own = (4 + (s2 & 1)) + 9 * (4 + (s2 >> 1));
    Y[t] = r == own ? 1.0 : 0.0;
  }
  __syncthreads();
  cta_lu(S, NP, NP, piv + NV, flag);
  cta_lu_solve_multi(K, NV, piv, Y, 4);
  // pressure parts: row (s2, c): S~^{-1} (-B~_c' y_s2); pressure row: S~^{-1} e_centre
  if (tid < 9) {
    double z[NP];
    const int k = tid;
    for (int pq = 0; pq < NP; ++pq) {
      if (k < 8) {
        const int s2 = k >> 1, cc = k & 1;
        double sum = 0.0;
        for (int p = 0; p < NV; ++p) sum = sum - Bs[(cc * NV + p) * NP + pq] * Y[s2 * NV + p];
        z[pq] = sum;
      } else {
        z[pq] = pq == 4 ? 1.0 : 0.0;
      }
    }
    lu_solve_vec(S, NP, NP, piv + NV, z);
    for (int pq = 0; pq < NP; ++pq) pv[k * NP + pq] = z[pq];
  }
  __syncthreads();
  // rows: velocity u_c' = delta_cc' y - W~_c' p, de-scaled; absent owned DoFs give zero rows
  double* out = coef + (size_t)v * Q2P::NS * Q2P::NROWP;
  for (int t = tid; t < Q2P::NS * Q2P::NROWP; t += nt) {
    const int slot = t / Q2P::NROWP, k = t % Q2P::NROWP;
    double val = 0.0;
    if (k < 9) {
      int orow;  // local index of the owned DoF of row k
      if (k < 8) {
        const int s2 = k >> 1;
        orow = (4 + (s2 & 1)) + 9 * (4 + (s2 >> 1));
      } else {
        orow = NV + 4;
      }
      if (act[orow]) {
        const double dk = k < 8 ? dv[orow] : dp[4];
        if (slot < Q2P::NSV) {
          const int p = slot / 2, c2 = slot % 2;
          if (act[p]) {
            double u = 0.0;
            if (k < 8 && c2 == (k & 1)) u = Y[(k >> 1) * NV + p];
            for (int pq = 0; pq < NP; ++pq) u = u - W[(c2 * NP + pq) * NV + p] * pv[k * NP + pq];
            val = dk * u * dv[p];
          }
        } else {
          const int pq = slot - Q2P::NSV;
          if (act[NV + pq]) val = dk * pv[k * NP + pq] * dp[pq];
        }
      }
    }
    out[t] = val;
  }
  if (tid == 0 && *flag) atomicOr(d_err, kErrSingularPatch);
}

// apply: 8 lanes per patch; y_k = sum_slots rows[slot][k] r[slot]; the
// restricted update writes the owned DoFs only (x += omega y, constrained
// velocity DoFs x += r)
__global__ void __launch_bounds__(256)
    q2_apply_kernel(Q2Grid q, const double* __restrict__ coef, const unsigned char* __restrict__ mask,
                    const double* __restrict__ rpv, const double* __restrict__ rpp, double omega,
                    double* __restrict__ x) {
  constexpr int TPP = 8;
  __shared__ int soff[Q2P::NS];
  const int PX = q.nf[0] + 8, PXP = q.nv1[0] + 2;
  for (int j = threadIdx.x; j < Q2P::NS; j += blockDim.x) {
    if (j < Q2P::NSV) {
      const int p = j / 2, c = j % 2;
      soff[j] = ((p % 9 - 4) + PX * (p / 9 - 4)) * 2 + c;
    } else {
      const int pq = j - Q2P::NSV;
      soff[j] = (pq % 3 - 1) + PXP * (pq / 3 - 1);
    }
  }
  __syncthreads();
  const int lane = threadIdx.x % TPP;
  const long long gi = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / TPP;
  const bool valid = gi < q.np;
  const long long v = valid ? gi : q.np - 1;
  const int ax = (int)(v % q.nv1[0]), ay = (int)(v / q.nv1[0]);
  const double* rv = rpv + ((long long)(2 * ay + 4) * PX + (2 * ax + 4)) * 2;
  const double* rp = rpp + (long long)(ay + 1) * PXP + (ax + 1);
  const double* cf = coef + (size_t)v * Q2P::NS * Q2P::NROWP;
  double y[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) y[k] = 0.0;
  for (int j = lane; j < Q2P::NS; j += TPP) {
    const double r = j < Q2P::NSV ? rv[soff[j]] : rp[soff[j]];
    const double2* c2 = reinterpret_cast<const double2*>(cf + (size_t)j * Q2P::NROWP);
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const double2 a = __ldcs(c2 + h);
      y[2 * h] += a.x * r;
      y[2 * h + 1] += a.y * r;
    }
    y[8] += __ldcs(cf + (size_t)j * Q2P::NROWP + 8) * r;
  }
  // reduce-scatter of rows 0-7 over the 8 lanes (halve the rows by lane
  // bits 2, 1, 0: lane l ends with the sum of row l) and a full sum of row 8
  const bool b2 = lane & 4, b1 = lane & 2, b0 = lane & 1;
  double k4[4], k2[2];
#pragma unroll
  for (int t = 0; t < 4; ++t)
    k4[t] = (b2 ? y[4 + t] : y[t]) + __shfl_xor_sync(0xffffffffu, b2 ? y[t] : y[4 + t], 4);
#pragma unroll
  for (int t = 0; t < 2; ++t)
    k2[t] = (b1 ? k4[2 + t] : k4[t]) + __shfl_xor_sync(0xffffffffu, b1 ? k4[t] : k4[2 + t], 2);
  const double yl = (b0 ? k2[1] : k2[0]) + __shfl_xor_sync(0xffffffffu, b0 ? k2[0] : k2[1], 1);
  double y8 = y[8];
#pragma unroll
  for (int o = TPP / 2; o > 0; o >>= 1) y8 += __shfl_xor_sync(0xffffffffu, y8, o);
  if (!valid) return;
  for (int k = lane; k < 9; k += TPP) {
    const double yk = k < 8 ? yl : y8;
    if (k < 8) {
      const int s2 = k >> 1, c = k & 1;
      const int I = 2 * ax + (s2 & 1), J = 2 * ay + (s2 >> 1);
      if (I >= q.nf[0] || J >= q.nf[1]) continue;
      const long long i = I + (long long)q.nf[0] * J;
      const double add = mask[i] ? rv[(((s2 & 1)) + PX * (s2 >> 1)) * 2 + c] : omega * yk;
      x[i * 2 + c] += add;
    } else {
      x[q.nq * 2 + v] += omega * yk;
    }
  }
}

// ---- Q2-Q1 patches in 3D: the Q2 nodes 2a-4 .. 2a+4 (9^3 = 729) with 3
// components, then the 27 pressures a-1 .. a+1; 25 owned rows (the 8 Q2
// nodes 2a + s, s in {0,1}^3 with s_x fastest, component inner; then p_a).
// Rows are stored [row][slot] with the slots padded to 2240.
struct Q2P3 {
  static constexpr int NV = 729, NP = 27, NSV = 2187, NS = 2214, NROW = 25, SP = 2240;
  // K couples Q2 nodes at most 2 apart per direction: in node-lexicographic
  // order (x fastest) that is a half bandwidth of 2 + 2*9 + 2*81
  static constexpr int KL = 182;
  // band row of the LU with row exchanges: KL below, 2 KL above (the fill a
  // row exchange can bring), the diagonal
  static constexpr int BW = 3 * KL + 1;
  static constexpr int NRHS = 3 * NP + 8;  // W~_c columns, then the 8 owned unit vectors
  static constexpr size_t WS = ((size_t)NV * BW + (size_t)NV * NRHS + (size_t)3 * NP * NV + 31) / 32 * 32;
};

__device__ __forceinline__ int q2p3_own(int s) { return (4 + (s & 1)) + 9 * (4 + ((s >> 1) & 1)) + 81 * (4 + (s >> 2)); }

// Owned rows of the equilibrated local inverse by block elimination, as in
// two dimensions, with K~ (729 x 729) factored by a banded LU with partial
// pivoting in global memory (one workspace per CTA, L2 resident):
//   K~ W~ = B~ (81 columns) and K~ Y = e_own (8 columns), solved together;
//   S~ = -sum_c B~_c' W~_c; pressure parts z = S~^{-1}(-B~_c' y) or
//   S~^{-1} e_centre; velocity parts delta y - W~ z; de-scaled.
// The RHS solves give each warp its own columns, so they need no CTA
// barrier; the LU takes three barriers per pivot step (four with a row
// exchange).  Persistent: CTA b takes vertices b, b + grid, ...
__global__ void __launch_bounds__(512)
    q2_patch_rows3_kernel(Q2Grid q, const double* __restrict__ A, const double* __restrict__ B,
                          const unsigned char* __restrict__ mask, double* __restrict__ coef,
                          double* __restrict__ work, unsigned* d_err) {
  using P = Q2P3;
  constexpr int NV = P::NV, NP = P::NP, KL = P::KL, BW = P::BW, NR = P::NRHS;
  __shared__ int act[NV + NP];
  __shared__ int rend[NV];    // last column of the nonzeros of row r (grows with fill)
  __shared__ int cstart[NV];  // first row with a nonzero of U in column k
  __shared__ int piv[NV];
  __shared__ double dv[NV], dp[NP];
  __shared__ double S[NP * NP];
  __shared__ int pivS[NP];
  __shared__ double pv[P::NROW * NP];
  __shared__ double lcol[KL];     // multipliers of the current pivot step
  __shared__ double urow[2 * KL];  // pivot row right of the diagonal
  __shared__ int s_cmax, flag;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
  double* Bd = work + (size_t)blockIdx.x * P::WS;  // [row][BW]: column c of row r at c - r + KL
  double* X = Bd + (size_t)NV * BW;                 // [rhs][NV]
  double* Bs = X + (size_t)NR * NV;                 // [c][pq][NV]
  for (long long v = blockIdx.x; v < q.np; v += gridDim.x) {
    const int ax = (int)(v % q.nv1[0]), ay = (int)((v / q.nv1[0]) % q.nv1[1]),
              az = (int)(v / ((long long)q.nv1[0] * q.nv1[1]));
    if (tid == 0) flag = 0;
    for (int j = tid; j < NV + NP; j += nt) {
      if (j < NV) {
        const int I = 2 * ax - 4 + j % 9, J = 2 * ay - 4 + (j / 9) % 9, K = 2 * az - 4 + j / 81;
        const bool in = I >= 0 && I < q.nf[0] && J >= 0 && J < q.nf[1] && K >= 0 && K < q.nf[2];
        act[j] = in && !mask[I + (long long)q.nf[0] * (J + (long long)q.nf[1] * K)];
        rend[j] = min(j + KL, NV - 1);
      } else {
        const int t = j - NV, X0 = ax - 1 + t % 3, Y0 = ay - 1 + (t / 3) % 3, Z0 = az - 1 + t / 9;
        act[j] = X0 >= 0 && X0 < q.nv1[0] && Y0 >= 0 && Y0 < q.nv1[1] && Z0 >= 0 && Z0 < q.nv1[2];
      }
    }
    __syncthreads();
    // gather the band of K (identity rows for absent nodes) and B_c
    for (int t = tid; t < NV * BW; t += nt) {
      const int r = t / BW, c = r - KL + t % BW;
      double val = 0.0;
      if (c >= 0 && c < NV) {
        if (act[r] && act[c]) {
          const int ox = c % 9 - r % 9, oy = (c / 9) % 9 - (r / 9) % 9, oz = c / 81 - r / 81;
          if (ox >= -2 && ox <= 2 && oy >= -2 && oy <= 2 && oz >= -2 && oz <= 2) {
            const int I = 2 * ax - 4 + r % 9, J = 2 * ay - 4 + (r / 9) % 9, K = 2 * az - 4 + r / 81;
            const long long i = I + (long long)q.nf[0] * (J + (long long)q.nf[1] * K);
            val = A[(long long)((ox + 2) + 5 * (oy + 2) + 25 * (oz + 2)) * q.nq + i];
          }
        } else if (r == c) {
          val = 1.0;
        }
      }
      Bd[t] = val;
    }
    for (int t = tid; t < 3 * NP * NV; t += nt) {
      const int cc = t / (NP * NV), pq = (t / NV) % NP, r = t % NV;
      double val = 0.0;
      if (act[r] && act[NV + pq]) {
        const int I = 2 * ax - 4 + r % 9, J = 2 * ay - 4 + (r / 9) % 9, K = 2 * az - 4 + r / 81;
        const int ox = ax - 1 + pq % 3 - (I / 2 - 1), oy = ay - 1 + (pq / 3) % 3 - (J / 2 - 1),
                  oz = az - 1 + pq / 9 - (K / 2 - 1);
        if (ox >= 0 && ox <= 2 && oy >= 0 && oy <= 2 && oz >= 0 && oz <= 2) {
          const long long i = I + (long long)q.nf[0] * (J + (long long)q.nf[1] * K);
          val = B[((long long)(ox + 3 * oy + 9 * oz) * 3 + cc) * q.nq + i];
        }
      }
      Bs[t] = val;
    }
    __syncthreads();
    // row-max equilibration: one scale per velocity node (K is shared by the
    // components), one per pressure
    for (int j = tid; j < NV + NP; j += nt) {
      double m = 0.0;
      if (j < NV) {
        for (int o = 0; o < BW; ++o) m = fmax(m, fabs(Bd[(size_t)j * BW + o]));
        for (int t = 0; t < 3 * NP; ++t) m = fmax(m, fabs(Bs[(size_t)t * NV + j]));
        dv[j] = act[j] && m > 0.0 ? 1.0 / sqrt(m) : 1.0;
      } else {
        const int pq = j - NV;
        for (int cc = 0; cc < 3; ++cc)
          for (int r = 0; r < NV; ++r) m = fmax(m, fabs(Bs[((size_t)cc * NP + pq) * NV + r]));
        dp[pq] = act[j] && m > 0.0 ? 1.0 / sqrt(m) : 1.0;
      }
    }
    __syncthreads();
    for (int t = tid; t < NV * BW; t += nt) {
      const int r = t / BW, c = r - KL + t % BW;
      if (c >= 0 && c < NV) Bd[t] = dv[r] * Bd[t] * dv[c];
    }
    for (int t = tid; t < NR * NV; t += nt) {
      const int m = t / NV, r = t % NV;
      if (m < 3 * NP) {
        const double s = dv[r] * Bs[t] * dp[m % NP];
        Bs[t] = s;
        X[t] = s;
      } else {
        X[t] = r == q2p3_own(m - 3 * NP) ? 1.0 : 0.0;
      }
    }
    __syncthreads();
    // banded LU with partial pivoting (max |a|, lowest row on ties)
    for (int k = 0; k < NV; ++k) {
      const int rlast = min(k + KL, NV - 1);
      if (warp == 0) {
        double best = -1.0;
        int bi = k;
        for (int r = k + lane; r <= rlast; r += 32) {
          const double a = fabs(Bd[(size_t)r * BW + (k - r + KL)]);
          if (a > best) { best = a; bi = r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
          const double ob = __shfl_down_sync(0xffffffffu, best, o);
          const int oi = __shfl_down_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) {
          piv[k] = bi;
          if (!(best > 0.0)) flag = 1;
          s_cmax = max(rend[k], rend[bi]);
          const int t = rend[k];
          rend[k] = rend[bi];
          rend[bi] = t;
        }
      }
      __syncthreads();
      const int p = piv[k];
      if (p != k) {
        const int cmax = s_cmax;
        for (int c = k + tid; c <= cmax; c += nt) {
          double* a = Bd + (size_t)k * BW + (c - k + KL);
          double* b = Bd + (size_t)p * BW + (c - p + KL);
          const double t = *a;
          *a = *b;
          *b = t;
        }
        __syncthreads();
      }
      const double d = Bd[(size_t)k * BW + KL];
      const int nr = rlast - k, ncol = rend[k] - k;
      for (int t = tid; t < nr + ncol; t += nt) {
        if (t < nr) {
          const int i = k + 1 + t;
          double* a = Bd + (size_t)i * BW + (k - i + KL);
          const double l = d != 0.0 ? *a / d : 0.0;
          *a = l;
          lcol[t] = l;
          if (l != 0.0) rend[i] = max(rend[i], rend[k]);
        } else {
          const int c = k + 1 + (t - nr);
          urow[t - nr] = Bd[(size_t)k * BW + (c - k + KL)];
        }
      }
      __syncthreads();
      for (int t = tid; t < nr * ncol; t += nt) {
        const int ii = t / ncol, cc = t % ncol;
        const double l = lcol[ii];
        if (l != 0.0) {
          const int i = k + 1 + ii, c = k + 1 + cc;
          double* a = Bd + (size_t)i * BW + (c - i + KL);
          *a = *a - l * urow[cc];
        }
      }
      __syncthreads();
    }
    if (tid == 0) {
      // first row with a nonzero of U in column k (non-decreasing in k)
      int i = 0;
      for (int k = 0; k < NV; ++k) {
        while (rend[i] < k) ++i;
        cstart[k] = i;
      }
    }
    __syncthreads();
    // solves: warp w takes the columns w, w + nwarp, ...; forward with the
    // row exchanges in pivot order, then backward with U
    for (int m = warp; m < NR; m += nwarp) {
      double* xm = X + (size_t)m * NV;
      for (int k = 0; k < NV; ++k) {
        const int p = piv[k];
        if (p != k && lane == 0) {
          const double t = xm[k];
          xm[k] = xm[p];
          xm[p] = t;
        }
        __syncwarp();
        const double xk = xm[k];
        const int rlast = min(k + KL, NV - 1);
        for (int i = k + 1 + lane; i <= rlast; i += 32) xm[i] = xm[i] - Bd[(size_t)i * BW + (k - i + KL)] * xk;
        __syncwarp();
      }
      for (int k = NV - 1; k >= 0; --k) {
        const double xk = xm[k] / Bd[(size_t)k * BW + KL];
        __syncwarp();
        if (lane == 0) xm[k] = xk;
        for (int i = cstart[k] + lane; i < k; i += 32) xm[i] = xm[i] - Bd[(size_t)i * BW + (k - i + KL)] * xk;
        __syncwarp();
      }
    }
    __syncthreads();
    // S~ = -sum_c B~_c' W~_c (identity rows and columns for absent pressures)
    for (int t = tid; t < NP * NP; t += nt) {
      const int r = t / NP, c = t % NP;
      double sum = 0.0;
      if (act[NV + r] && act[NV + c]) {
        for (int cc = 0; cc < 3; ++cc) {
          const double* bp = Bs + ((size_t)cc * NP + r) * NV;
          const double* wp = X + ((size_t)cc * NP + c) * NV;
          for (int j = 0; j < NV; ++j) sum = sum - bp[j] * wp[j];
        }
      } else if (r == c) {
        sum = 1.0;
      }
      S[t] = sum;
    }
    // right-hand sides of the pressure parts: -B~_c' y_s (row 3 s + c), e_centre
    for (int t = tid; t < P::NROW * NP; t += nt) {
      const int k = t / NP, pq = t % NP;
      double sum = 0.0;
      if (k < 24) {
        const double* bp = Bs + ((size_t)(k % 3) * NP + pq) * NV;
        const double* yp = X + ((size_t)3 * NP + k / 3) * NV;
        for (int j = 0; j < NV; ++j) sum = sum - bp[j] * yp[j];
      } else {
        sum = pq == 13 ? 1.0 : 0.0;
      }
      pv[t] = sum;
    }
    __syncthreads();
    cta_lu(S, NP, NP, pivS, &flag);
    if (tid < P::NROW) lu_solve_vec(S, NP, NP, pivS, pv + tid * NP);
    __syncthreads();
    // rows: velocity u_c' = delta_cc' y - W~_c' z, pressure z; de-scaled;
    // absent owned DoFs give zero rows
    double* out = coef + (size_t)v * P::NROW * P::SP;
    for (int t = tid; t < P::NROW * P::SP; t += nt) {
      const int k = t / P::SP, slot = t % P::SP;
      double val = 0.0;
      const int orow = k < 24 ? q2p3_own(k / 3) : NV + 13;
      if (slot < P::NS && act[orow]) {
        const double dk = k < 24 ? dv[orow] : dp[13];
        if (slot < P::NSV) {
          const int pn = slot / 3, c2 = slot % 3;
          if (act[pn]) {
            double u = (k < 24 && c2 == k % 3) ? X[((size_t)3 * NP + k / 3) * NV + pn] : 0.0;
            for (int pq = 0; pq < NP; ++pq) u = u - X[((size_t)c2 * NP + pq) * NV + pn] * pv[k * NP + pq];
            val = dk * u * dv[pn];
          }
        } else {
          const int pq = slot - P::NSV;
          if (act[NV + pq]) val = dk * pv[k * NP + pq] * dp[pq];
        }
      }
      out[t] = val;
    }
    if (tid == 0 && flag) atomicOr(d_err, kErrSingularPatch);
    __syncthreads();
  }
}

// ---- adaptive grids: owned rows of the patches (variable size).  L_i
// gathered from the CSR rows of the patch DoFs (binary search in each
// sorted row), symmetrically equilibrated D L_i D with D = |diag L_i|^-1/2,
// LU with partial pivoting, and the owned columns of (D L_i D)^-1 (= its
// owned rows, L_i symmetric) by a CTA-cooperative solve with the d + 1 unit
// vectors, de-scaled; rows of absent owned DoFs are zero.  The dense block
// lives in dynamic shared memory, one CTA per patch (the patches whose
// block fits; larger ones take the block elimination below).  Stored per
// slot as a record of d + 2 doubles: the DoF index in the bits of a double,
// then the d + 1 owned-row coefficients.
template <int DIM>
__global__ void __launch_bounds__(512)
    amr_patch_rows_kernel(long long np, const long long* __restrict__ pstart, const int* __restrict__ pdof,
                          const int* __restrict__ pown, const int* __restrict__ rp, const int* __restrict__ col,
                          const double* __restrict__ val, double* __restrict__ rows, unsigned* d_err) {
  constexpr int ND = DIM + 1, REC = ND + 1;
  extern __shared__ double am[];
  __shared__ int s_piv[kAmrMaxPatch];
  __shared__ int s_flag;
  double* base = am;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (long long p = blockIdx.x; p < np; p += gridDim.x) {
    const long long s0 = pstart[p];
    const int n = (int)(pstart[p + 1] - s0);
    double* K = base;               // n x n row-major
    double* dsc = K + (size_t)n * n;
    double* W = dsc + n;            // n x (d + 1), column-major
    if (tid == 0) s_flag = 0;
    for (int t = tid; t < n * n; t += nt) {
      const int a = t / n, b = t % n;
      const int ra = pdof[s0 + a], cb = pdof[s0 + b];
      double v = 0.0;
      int lo = rp[ra], hi = rp[ra + 1] - 1;
      while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int c = col[mid];
        if (c == cb) { v = val[mid]; break; }
        if (c < cb) lo = mid + 1; else hi = mid - 1;
      }
      K[t] = v;
    }
    __syncthreads();
    for (int a = tid; a < n; a += nt) {
      const double d = fabs(K[(size_t)a * n + a]);
      dsc[a] = d > 0.0 ? 1.0 / sqrt(d) : 1.0;
    }
    __syncthreads();
    for (int t = tid; t < n * n; t += nt) K[t] = dsc[t / n] * K[t] * dsc[t % n];
    __syncthreads();
    cta_lu(K, n, n, s_piv, &s_flag);
    for (int t = tid; t < ND * n; t += nt) {
      const int k = t / n, j = t % n, o = pown[p * ND + k];
      W[t] = (o >= 0 && j == o) ? 1.0 : 0.0;
    }
    __syncthreads();
    cta_lu_solve_multi(K, n, s_piv, W, ND);
    double* out = rows + REC * s0;
    for (int t = tid; t < REC * n; t += nt) {
      const int j = t / REC, f = t % REC;
      if (f == 0) {
        out[t] = __longlong_as_double((long long)pdof[s0 + j]);
      } else {
        const int k = f - 1, o = pown[p * ND + k];
        out[t] = o >= 0 ? dsc[o] * W[(size_t)k * n + j] * dsc[j] : 0.0;
      }
    }
    if (tid == 0 && s_flag) atomicOr(d_err, kErrSingularPatch);
    __syncthreads();  // the next patch reuses the block
  }
}

// ---- adaptive grids, larger patches: the owned rows by block elimination.
// The patch's velocity DoFs come node by node with all d components (the
// constrained ones leave with their node), and the velocity block is
// I_d (x) A_s with one scalar block A_s over the patch's velocity nodes, so
// with B_c the pressure-velocity block of component c and C the pressure
// block (all equilibrated as in the dense kernel, D = |diag L_i|^-1/2):
//   W_c = A_s^-1 B_c^T,   S = C - sum_c B_c W_c,
// and the rows of L_i^-1 (L_i symmetric) of the owned DoFs are
//   pressure q0:         p part z,       velocity part (a, c) -(W_c z)_a,
//                        z = S^-1 e_q0;
//   velocity (j0, c0):   p part -y,      velocity part d_{c c0} (A_s^-1 e_j0)_a
//                        + (W_c y)_a,    y = S^-1 (row j0 of W_c0).
// LU with partial pivoting of A_s (n_v^3 / 3 FMA against (d n_v + n_p)^3 / 3
// for the whole block), d n_p right-hand sides for W, LU of S.  Each CTA
// works on its own slice of a global workspace (persistent CTAs).
template <int DIM>
__global__ void __launch_bounds__(512)
    amr_patch_rows_schur_kernel(long long npatch, const long long* __restrict__ pstart, const int* __restrict__ pdof,
                                const int* __restrict__ pown, const int* __restrict__ rp,
                                const int* __restrict__ col, const double* __restrict__ val,
                                double* __restrict__ rows, double* work, long long wstride, int maxnv, int maxnp,
                                unsigned* d_err) {
  constexpr int ND = DIM + 1, REC = ND + 1;
  __shared__ int s_piv[kAmrMaxPatch];
  __shared__ int s_flag, s_bad, s_nvd;
  double* Ah = work + (long long)blockIdx.x * wstride;  // n_v x n_v row-major
  double* Bt = Ah + (size_t)maxnv * maxnv;              // B_c^T: column c n_p + q of length n_v
  double* W = Bt + (size_t)DIM * maxnp * maxnv;         // A_s^-1 B_c^T, same layout
  double* S = W + (size_t)DIM * maxnp * maxnv;          // n_p x n_p row-major
  double* Dg = S + (size_t)maxnp * maxnp;               // scaling per patch DoF
  double* Z = Dg + (size_t)DIM * maxnv + maxnp;         // d + 1 solves with S, column-major
  double* U0 = Z + (size_t)ND * maxnp;                  // A_s^-1 e_j0
  const int tid = threadIdx.x, nt = blockDim.x;
  auto entry = [&](int row, int cj) {
    int lo = rp[row], hi = rp[row + 1] - 1;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1;
      const int c = col[mid];
      if (c == cj) return val[mid];
      if (c < cj) lo = mid + 1; else hi = mid - 1;
    }
    return 0.0;
  };
  for (long long p = blockIdx.x; p < npatch; p += gridDim.x) {
    const long long s0 = pstart[p];
    const int n = (int)(pstart[p + 1] - s0);
    const int* dof = pdof + s0;
    if (tid == 0) { s_flag = 0; s_bad = 0; s_nvd = n; }
    __syncthreads();
    for (int j = tid; j < n; j += nt)
      if (dof[j] % ND == DIM) atomicMin(&s_nvd, j);
    __syncthreads();
    const int nvd = s_nvd, npp = n - nvd, nv = nvd / DIM;
    for (int j = tid; j < n; j += nt) {
      const int c = j % DIM;
      const bool ok = j >= nvd ? dof[j] % ND == DIM : (dof[j] % ND == c && dof[j] - c == dof[j - c]);
      if (!ok) s_bad = 1;
    }
    if (tid == 0 && (nvd % DIM != 0 || nv > maxnv || npp > maxnp)) s_bad = 1;
    __syncthreads();
    if (s_bad) {
      if (tid == 0) atomicOr(d_err, kErrBadIndex);
      continue;  // uniform: every thread read s_bad after the barrier
    }
    for (int t = tid; t < nv * nv; t += nt) Ah[t] = entry(dof[(t / nv) * DIM], dof[(t % nv) * DIM]);
    for (int t = tid; t < DIM * npp * nv; t += nt) {
      const int a = t % nv, cq = t / nv, c = cq / npp, q = cq % npp;
      Bt[t] = entry(dof[a * DIM + c], dof[nvd + q]);
    }
    for (int t = tid; t < npp * npp; t += nt) S[t] = entry(dof[nvd + t / npp], dof[nvd + t % npp]);
    __syncthreads();
    for (int j = tid; j < n; j += nt) {
      const double d = j < nvd ? fabs(Ah[(size_t)(j / DIM) * nv + j / DIM]) : fabs(S[(size_t)(j - nvd) * npp + j - nvd]);
      Dg[j] = d > 0.0 ? 1.0 / sqrt(d) : 1.0;
    }
    __syncthreads();
    for (int t = tid; t < nv * nv; t += nt) Ah[t] = Dg[(t / nv) * DIM] * Ah[t] * Dg[(t % nv) * DIM];
    for (int t = tid; t < DIM * npp * nv; t += nt) {
      const int a = t % nv, cq = t / nv, c = cq / npp, q = cq % npp;
      const double v = Dg[a * DIM + c] * Bt[t] * Dg[nvd + q];
      Bt[t] = v;
      W[t] = v;
    }
    for (int t = tid; t < npp * npp; t += nt) S[t] = Dg[nvd + t / npp] * S[t] * Dg[nvd + t % npp];
    __syncthreads();
    cta_lu(Ah, nv, nv, s_piv, &s_flag);
    cta_lu_solve_multi(Ah, nv, s_piv, W, DIM * npp);
    for (int t = tid; t < npp * npp; t += nt) {
      const int q = t / npp, r = t % npp;
      double acc = S[t];
      for (int c = 0; c < DIM; ++c) {
        const double* bq = Bt + (size_t)(c * npp + q) * nv;
        const double* wr = W + (size_t)(c * npp + r) * nv;
        for (int a = 0; a < nv; ++a) acc = fma(-bq[a], wr[a], acc);
      }
      S[t] = acc;
    }
    __syncthreads();
    cta_lu(S, npp, npp, s_piv + nv, &s_flag);
    // right-hand sides with S: row j0 of W_k for an owned velocity
    // component k, e_q0 for the owned pressure; A_s^-1 e_j0 for the owned node
    int jn = -1;
    for (int k = 0; k < DIM; ++k)
      if (pown[p * ND + k] >= 0) jn = pown[p * ND + k] / DIM;
    for (int t = tid; t < ND * npp; t += nt) {
      const int k = t / npp, q = t % npp, o = pown[p * ND + k];
      Z[t] = o < 0 ? 0.0 : (k < DIM ? W[(size_t)(k * npp + q) * nv + o / DIM] : (q == o - nvd ? 1.0 : 0.0));
    }
    for (int a = tid; a < nv; a += nt) U0[a] = a == jn ? 1.0 : 0.0;
    __syncthreads();
    cta_lu_solve_multi(S, npp, s_piv + nv, Z, ND);
    if (jn >= 0) cta_lu_solve_multi(Ah, nv, s_piv, U0, 1);
    double* out = rows + REC * s0;
    for (int t = tid; t < REC * n; t += nt) {
      const int j = t / REC, f = t % REC;
      if (f == 0) {
        out[t] = __longlong_as_double((long long)dof[j]);
        continue;
      }
      const int k = f - 1, o = pown[p * ND + k];
      if (o < 0) {
        out[t] = 0.0;
        continue;
      }
      const double* z = Z + (size_t)k * npp;
      const double sg = k < DIM ? 1.0 : -1.0;
      double v;
      if (j < nvd) {
        const int a = j / DIM, c = j % DIM;
        double acc = 0.0;
        for (int q = 0; q < npp; ++q) acc = fma(W[(size_t)(c * npp + q) * nv + a], z[q], acc);
        v = sg * acc + (k < DIM && c == k ? U0[a] : 0.0);
      } else {
        v = -sg * z[j - nvd];
      }
      out[t] = Dg[o] * v * Dg[j];
    }
    if (tid == 0 && s_flag) atomicOr(d_err, kErrSingularPatch);
    __syncthreads();  // the next patch reuses the workspace
  }
}

// 3D apply: a warp per vertex; lane l sums the 25 rows over the slots
// l, l + 32, ... (coalesced row loads, residual gathers from the padded
// copies), a reduce-scatter leaves row l's sum in lane l, and lanes 0..24
// write the restricted update of the owned DoFs.
__global__ void __launch_bounds__(256)
    q2_apply3_kernel(Q2Grid q, const double* __restrict__ coef, const unsigned char* __restrict__ mask,
                     const double* __restrict__ rpv, const double* __restrict__ rpp, double omega,
                     double* __restrict__ x) {
  using P = Q2P3;
  __shared__ int soff[P::SP];
  const int PX = q.nf[0] + 8, PY = q.nf[1] + 8, PXP = q.nv1[0] + 2, PYP = q.nv1[1] + 2;
  for (int j = threadIdx.x; j < P::SP; j += blockDim.x) {
    if (j < P::NSV) {
      const int pn = j / 3, c = j % 3;
      soff[j] = ((pn % 9 - 4) + PX * ((pn / 9) % 9 - 4 + PY * (pn / 81 - 4))) * 3 + c;
    } else if (j < P::NS) {
      const int pq = j - P::NSV;
      soff[j] = (pq % 3 - 1) + PXP * ((pq / 3) % 3 - 1 + PYP * (pq / 9 - 1));
    } else {
      soff[j] = 0;  // padding slots: zero coefficients
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long gv = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const bool valid = gv < q.np;
  const long long v = valid ? gv : q.np - 1;
  const int ax = (int)(v % q.nv1[0]), ay = (int)((v / q.nv1[0]) % q.nv1[1]),
            az = (int)(v / ((long long)q.nv1[0] * q.nv1[1]));
  const double* rv = rpv + (((long long)(2 * az + 4) * PY + (2 * ay + 4)) * PX + (2 * ax + 4)) * 3;
  const double* rp = rpp + ((long long)(az + 1) * PYP + (ay + 1)) * PXP + (ax + 1);
  const double* cf = coef + (size_t)v * P::NROW * P::SP;
  double y[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) y[k] = 0.0;
  for (int j = lane; j < P::SP; j += 32) {
    const double r = j < P::NSV ? rv[soff[j]] : rp[soff[j]];
#pragma unroll
    for (int k = 0; k < P::NROW; ++k) y[k] += __ldcs(cf + (size_t)k * P::SP + j) * r;
  }
  // reduce-scatter over the 32 lanes: after the step of width w each lane
  // keeps the half of its partial sums selected by bit w of its lane index
#pragma unroll
  for (int w = 16; w > 0; w >>= 1) {
    const bool hi = lane & w;
#pragma unroll
    for (int i = 0; i < w; ++i) {
      const double send = hi ? y[i] : y[i + w];
      const double keep = hi ? y[i + w] : y[i];
      y[i] = keep + __shfl_xor_sync(0xffffffffu, send, w);
    }
  }
  if (!valid || lane >= P::NROW) return;
  const double yk = y[0];
  if (lane < 24) {
    const int s = lane / 3, c = lane % 3;
    const int I = 2 * ax + (s & 1), J = 2 * ay + ((s >> 1) & 1), K = 2 * az + (s >> 2);
    if (I >= q.nf[0] || J >= q.nf[1] || K >= q.nf[2]) return;
    const long long i = I + (long long)q.nf[0] * (J + (long long)q.nf[1] * K);
    const double add = mask[i] ? rv[((s & 1) + PX * (((s >> 1) & 1) + PY * (s >> 2))) * 3 + c] : omega * yk;
    x[i * 3 + c] += add;
  } else {
    x[q.nq * 3 + v] += omega * yk;
  }
}

}  // namespace

size_t factor_doubles(int dim) { return dim == 3 ? (size_t)kBandRec : PatchDims<2>::REC; }
size_t factor_ints(int dim) { return dim == 3 ? (size_t)kBandRecI : PatchDims<2>::RECI; }
size_t dense_factor_doubles(int dim) { return dim == 3 ? PatchDims<3>::REC : PatchDims<2>::REC; }
size_t dense_factor_ints(int dim) { return dim == 3 ? PatchDims<3>::RECI : PatchDims<2>::RECI; }

cudaError_t launch_patch_build(const LevelGeom& g, const double* st, const unsigned char* mask, int mode,
                               double omega, double* coef64, double* fac, int* fpiv,
                               const double* rpad, double* x, unsigned* d_err, const int* work,
                               long long nwork, cudaStream_t s) {
  if (g.dim == 2) {
    if (mode == 0) return run_factor<2, 0>(g, st, mask, omega, coef64, fac, fpiv, rpad, x, d_err, work, nwork, s);
    if (mode == 1) return run_factor<2, 1>(g, st, mask, omega, coef64, fac, fpiv, rpad, x, d_err, work, nwork, s);
    return run_factor<2, 2>(g, st, mask, omega, coef64, fac, fpiv, rpad, x, d_err, nullptr, 0, s);
  }
  if (mode == 0) return run_factor<3, 0>(g, st, mask, omega, coef64, fac, fpiv, rpad, x, d_err, work, nwork, s);
  if (mode == 1) return run_factor<3, 1>(g, st, mask, omega, coef64, fac, fpiv, rpad, x, d_err, work, nwork, s);
  return run_factor<3, 2>(g, st, mask, omega, coef64, fac, fpiv, rpad, x, d_err, nullptr, 0, s);
}

cudaError_t launch_patch_rows_ldl(const LevelGeom& g, const double* st, const unsigned char* mask,
                                  double* coef64, unsigned* d_err, const int* work, long long nwork,
                                  int* redo_node, int* redo_out, int* nredo, cudaStream_t s) {
  if (g.dim != 3) return cudaErrorInvalidValue;
  const size_t sm = ldl_rows_smem<3>();
  cudaError_t e = cudaFuncSetAttribute(patch_rows_ldl_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const long long nb = work ? nwork : g.nnodes;
  if (nb <= 0) return cudaSuccess;
  patch_rows_ldl_kernel<0><<<(unsigned)nb, 256, sm, s>>>(g, st, mask, coef64, nullptr, d_err, work, redo_node, redo_out,
                                                         nredo, ldl_min_pivot_env(), nullptr, nullptr, 0.0);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_patch_rows_dense_redo(const LevelGeom& g, const double* st, const unsigned char* mask,
                                         double* coef64, unsigned* d_err, const int* redo_node,
                                         long long nredo, const int* redo_out, cudaStream_t s) {
  if (g.dim != 3) return cudaErrorInvalidValue;
  return run_factor<3, 0>(g, st, mask, 0.0, coef64, nullptr, nullptr, nullptr, nullptr, d_err, redo_node, nredo, s,
                          redo_out);
}

cudaError_t launch_patch_rows_ir(const LevelGeom& g, const double* st, const unsigned char* mask,
                                 double* coef64, unsigned* d_err, const int* work, long long nwork,
                                 int* redo_node, int* redo_out, int* nredo, cudaStream_t s) {
  if (g.dim == 2) return run_ir_factor<2>(g, st, mask, coef64, d_err, work, nwork, redo_node, redo_out, nredo, s);
  return run_ir_factor<3>(g, st, mask, coef64, d_err, work, nwork, redo_node, redo_out, nredo, s);
}

cudaError_t launch_patch_rows_pair(const LevelGeom& g, const double* st, const unsigned char* mask,
                                   double* coef64, unsigned* d_err, const int* work, long long nwork,
                                   const int* outidx, cudaStream_t s) {
  if (g.dim == 2) return run_pair_factor<2>(g, st, mask, coef64, d_err, work, nwork, outidx, s);
  return run_pair_factor<3>(g, st, mask, coef64, d_err, work, nwork, outidx, s);
}

cudaError_t launch_patch_apply(const LevelGeom& g, fc_prec prec, const void* coef,
                               const unsigned char* mask, const double* rpad, const float* rpad32,
                               double omega, double* x, const int* prow, cudaStream_t s) {
  const long long threads32 = g.nnodes * 32;
  const unsigned blocks = (unsigned)((threads32 + 255) / 256);
  // 2D: 4 lanes per patch (see apply_tpp); 3D: a warp per patch
  const unsigned blocks4 = (unsigned)((g.nnodes * 4 + 255) / 256);
  if (prec == FC_PREC_FP64) {
    const int t = apply64_tpp(g.dim);
    const unsigned bl = (unsigned)((g.nnodes * t + 255) / 256);
    const double* c = (const double*)coef;
    if (g.dim == 2) {
      apply_fp64_kernel<2, 4><<<bl, 256, 0, s>>>(g, c, mask, rpad, omega, x, prow);
    } else {
      switch (t) {
        case 4: apply_fp64_kernel<3, 4><<<bl, 256, 0, s>>>(g, c, mask, rpad, omega, x, prow); break;
        case 16: apply_fp64_kernel<3, 16><<<bl, 256, 0, s>>>(g, c, mask, rpad, omega, x, prow); break;
        case 32: apply_fp64_kernel<3, 32><<<bl, 256, 0, s>>>(g, c, mask, rpad, omega, x, prow); break;
        default: apply_fp64_kernel<3, 8><<<bl, 256, 0, s>>>(g, c, mask, rpad, omega, x, prow); break;
      }
    }
  } else if (prec == FC_PREC_FP32) {
    if (g.dim == 2) apply_lowp_kernel<2, float, 4><<<blocks4, 256, 0, s>>>(g, (const float*)coef, mask, rpad32, omega, x, prow);
    else apply_lowp_kernel<3, float, 32><<<blocks, 256, 0, s>>>(g, (const float*)coef, mask, rpad32, omega, x, prow);
  } else if (prec == FC_PREC_BF16) {
    if (g.dim == 2) apply_lowp_kernel<2, __nv_bfloat16, 4><<<blocks4, 256, 0, s>>>(g, (const __nv_bfloat16*)coef, mask, rpad32, omega, x, prow);
    else apply_lowp_kernel<3, __nv_bfloat16, 32><<<blocks, 256, 0, s>>>(g, (const __nv_bfloat16*)coef, mask, rpad32, omega, x, prow);
  } else {
    const float2 om2 = make_float2((float)omega, (float)(omega - (double)(float)omega));
    if (g.dim == 2) apply_df_kernel<2><<<blocks, 256, 0, s>>>(g, (const float2*)coef, mask, (const float2*)rpad32, omega, x, nullptr, om2, prow);
    else apply_df_kernel<3><<<blocks, 256, 0, s>>>(g, (const float2*)coef, mask, (const float2*)rpad32, omega, x, nullptr, om2, prow);
  }
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_patch_apply_df2(const LevelGeom& g, const void* coef, const unsigned char* mask,
                                   const float* rpad2, double omega, float2* xp2, const int* prow,
                                   const int* cls_blk, cudaStream_t s) {
  const float2 om2 = make_float2((float)omega, (float)(omega - (double)(float)omega));
  const int2 cls = make_int2(cls_blk ? cls_blk[0] : -1, cls_blk ? cls_blk[1] : -1);
  if (g.dim == 2)
    return run_df_persistent<2>(g, (const float2*)coef, mask, (const float2*)rpad2, xp2, om2, prow, cls, s);
  return run_df_persistent<3>(g, (const float2*)coef, mask, (const float2*)rpad2, xp2, om2, prow, cls, s);
}

cudaError_t launch_factor_apply(const LevelGeom& g, const double* st, const FactorStore& f,
                                const unsigned char* mask, const double* rpad, double omega, double* x,
                                const int* prow, cudaStream_t s) {
  if (g.dim == 2) {
    long long threads = g.nnodes * 32;
    unsigned blocks = (unsigned)((threads + 127) / 128);
    factor_apply_kernel<2><<<blocks, 128, 0, s>>>(g, f.fac, f.fpiv, mask, rpad, omega, x, prow, nullptr, nullptr, 0);
    note_launches(1);
    return cudaGetLastError();
  }
  band_factor_apply_kernel<<<(unsigned)g.nnodes, 96, 0, s>>>(g, st, f.fac, f.fpiv, mask, rpad, omega, x, prow);
  note_launches(1);
  if (f.nlist > 0) {
    const long long threads = f.nlist * 32;
    const unsigned blocks = (unsigned)((threads + 127) / 128);
    factor_apply_kernel<3><<<blocks, 128, 0, s>>>(g, f.facd, f.fpivd, mask, rpad, omega, x, nullptr, f.lnode, f.lrec,
                                                  f.nlist);
    note_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_band_factors(const LevelGeom& g, const double* st, const unsigned char* mask, double* fac,
                                int* fpiv, unsigned* d_err, const int* work, long long nwork, int* redo_node,
                                int* redo_out, int* nredo, cudaStream_t s) {
  if (g.dim != 3) return cudaErrorInvalidValue;
  const size_t sm = ldl_rows_smem<3>();
  cudaError_t e = cudaFuncSetAttribute(patch_rows_ldl_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const long long nb = work ? nwork : g.nnodes;
  if (nb <= 0) return cudaSuccess;
  patch_rows_ldl_kernel<1><<<(unsigned)nb, 256, sm, s>>>(g, st, mask, fac, fpiv, d_err, work, redo_node, redo_out,
                                                         nredo, ldl_min_pivot_env(), nullptr, nullptr, 0.0);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_none_check(const LevelGeom& g, const double* st, const unsigned char* mask, unsigned* d_err,
                              int* redo_node, int* redo_out, int* nredo, double dmin, cudaStream_t s) {
  if (g.dim != 3) return cudaErrorInvalidValue;
  const size_t sm = ldl_rows_smem<3>();
  cudaError_t e = cudaFuncSetAttribute(patch_rows_ldl_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  patch_rows_ldl_kernel<2><<<(unsigned)g.nnodes, 256, sm, s>>>(g, st, mask, nullptr, nullptr, d_err, nullptr, redo_node,
                                                               redo_out, nredo, dmin, nullptr, nullptr, 0.0);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_none_sweep(const LevelGeom& g, const double* st, const unsigned char* mask, double omega,
                              const double* rpad, double* x, unsigned* d_err, const int* dense_nodes,
                              long long ndense, double dmin, cudaStream_t s) {
  if (g.dim != 3) return launch_patch_build(g, st, mask, 2, omega, nullptr, nullptr, nullptr, rpad, x, d_err, nullptr, 0, s);
  const size_t sm = ldl_rows_smem<3>();
  cudaError_t e = cudaFuncSetAttribute(patch_rows_ldl_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  patch_rows_ldl_kernel<2><<<(unsigned)g.nnodes, 256, sm, s>>>(g, st, mask, nullptr, nullptr, d_err, nullptr, nullptr,
                                                               nullptr, nullptr, dmin, rpad, x, omega);
  note_launches(1);
  e = cudaGetLastError();
  if (e != cudaSuccess || ndense <= 0) return e;
  return run_factor<3, 2>(g, st, mask, omega, nullptr, nullptr, nullptr, rpad, x, d_err, dense_nodes, ndense, s);
}

cudaError_t launch_dense_factor_redo(const LevelGeom& g, const double* st, const unsigned char* mask, double* facd,
                                     int* fpivd, unsigned* d_err, const int* redo_node, const int* redo_out, int nredo,
                                     int* fpiv, cudaStream_t s) {
  if (g.dim != 3 || nredo <= 0) return cudaSuccess;
  cudaError_t e = run_factor<3, 1>(g, st, mask, 0.0, nullptr, facd, fpivd, nullptr, nullptr, d_err, redo_node, nredo, s);
  if (e != cudaSuccess) return e;
  mark_dense_records_kernel<<<(unsigned)((nredo + 255) / 256), 256, 0, s>>>(redo_out, nredo, fpiv);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_dense_list(const LevelGeom& g, const int* prow, const int* fpiv, int* lnode, int* lrec,
                              int* nlist, cudaStream_t s) {
  dense_list_kernel<<<(unsigned)((g.nnodes + 255) / 256), 256, 0, s>>>(g.nnodes, prow, fpiv, lnode, lrec, nlist);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_convert_rows(const LevelGeom& g, fc_prec prec, const double* coef64, void* out,
                                long long nblocks, cudaStream_t s) {
  long long n = nblocks * (long long)nslot(g.dim) * g.nd;
  unsigned blocks = (unsigned)std::min<long long>((n + 255) / 256, 152LL * 32);
  if (prec == FC_PREC_FP32) convert_kernel<float><<<blocks, 256, 0, s>>>(n, coef64, (float*)out);
  else if (prec == FC_PREC_BF16) convert_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>(n, coef64, (__nv_bfloat16*)out);
  else if (prec == FC_PREC_DF64) convert_kernel<float2><<<blocks, 256, 0, s>>>(n, coef64, (float2*)out);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace fc

namespace fc {

size_t q2_patch_rows_doubles(int dim) {
  return dim == 2 ? (size_t)Q2P::NS * Q2P::NROWP : (size_t)Q2P3::NROW * Q2P3::SP;
}

size_t q2_patch_rows_work_doubles(int dim, long long ctas) { return dim == 3 ? (size_t)ctas * Q2P3::WS : 0; }

int q2_patch_rows_ctas(int dim, long long np) {
  if (dim != 3) return 0;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    nsm = 1;
  return (int)std::min<long long>(np, std::min(nsm, kQ2Rows3MaxCtas));
}

cudaError_t launch_q2_patch_rows(int dim, const Q2Grid& q, const double* A, const double* B, const unsigned char* mask,
                                 double* coef, double* work, int ctas, unsigned* d_err, cudaStream_t s) {
  if (dim == 3) {
    q2_patch_rows3_kernel<<<(unsigned)ctas, 512, 0, s>>>(q, A, B, mask, coef, work, d_err);
    note_launches(1);
    return cudaGetLastError();
  }
  constexpr int NV = Q2P::NV, NP = Q2P::NP;
  const size_t smem = sizeof(double) * ((size_t)NV * NV + 2 * NV * NP + 2 * NP * NV + NP * NP + NV + NP + 4 * NV + 9 * NP) +
                      sizeof(int) * (2 * (NV + NP) + 1);
  cudaError_t e = cudaFuncSetAttribute(q2_patch_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  q2_patch_rows_kernel<<<(unsigned)q.np, 256, smem, s>>>(q, A, B, mask, coef, d_err);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_q2_apply(int dim, const Q2Grid& q, const double* coef, const unsigned char* mask, const double* rpv,
                            const double* rpp, double omega, double* x, cudaStream_t s) {
  if (dim == 3) {
    const long long threads = q.np * 32;
    q2_apply3_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(q, coef, mask, rpv, rpp, omega, x);
  } else {
    const long long threads = q.np * 8;
    q2_apply_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(q, coef, mask, rpv, rpp, omega, x);
  }
  note_launches(1);
  return cudaGetLastError();
}

namespace {
size_t amr_block_doubles(int dim, int n) { return (size_t)n * n + (size_t)(dim + 2) * n; }
size_t amr_schur_doubles(int dim, int nv, int np) {
  return (size_t)nv * nv + 2 * (size_t)dim * np * nv + (size_t)np * np + (size_t)dim * nv + np +
         (size_t)(dim + 1) * np + nv;
}
constexpr size_t kAmrSmemBytes = 216 * 1024;  // + 8 KB of pivots within the 227 KB per CTA
}  // namespace

double ldl_min_pivot() { return ldl_min_pivot_env(); }

bool amr_patch_rows_in_smem(int dim, int maxn) { return amr_block_doubles(dim, maxn) * 8 <= kAmrSmemBytes; }

int amr_patch_rows_ctas(const AmrLevel& A) {
  if (A.nfree == 0 || amr_patch_rows_in_smem(A.dim, A.maxn)) return 0;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return (int)std::min<long long>(A.nfree, std::max(nsm, 1));
}

size_t amr_patch_rows_work_doubles(const AmrLevel& A, int ctas) {
  return (size_t)ctas * amr_schur_doubles(A.dim, A.maxnv, A.maxnp);
}

cudaError_t launch_amr_patch_rows(const AmrLevel& A, double* work, int ctas, unsigned* d_err, cudaStream_t s) {
  if (A.nfree == 0) return cudaSuccess;
  if (A.maxn > kAmrMaxPatch) return cudaErrorInvalidValue;
  if (work == nullptr) {
    // dense block in shared memory, one CTA per patch
    if (!amr_patch_rows_in_smem(A.dim, A.maxn)) return cudaErrorInvalidValue;
    auto kern = A.dim == 2 ? amr_patch_rows_kernel<2> : amr_patch_rows_kernel<3>;
    const size_t smem = sizeof(double) * amr_block_doubles(A.dim, A.maxn);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)A.nfree, 256, smem, s>>>(A.nfree, A.pstart, A.pdof, A.pown, A.rowptr, A.col, A.val, A.rows,
                                               d_err);
  } else {
    // block elimination in the global workspace, persistent CTAs
    if (ctas <= 0) return cudaErrorInvalidValue;
    auto kern = A.dim == 2 ? amr_patch_rows_schur_kernel<2> : amr_patch_rows_schur_kernel<3>;
    kern<<<(unsigned)ctas, 512, 0, s>>>(A.nfree, A.pstart, A.pdof, A.pown, A.rowptr, A.col, A.val, A.rows, work,
                                        (long long)amr_schur_doubles(A.dim, A.maxnv, A.maxnp), A.maxnv, A.maxnp,
                                        d_err);
  }
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace fc
