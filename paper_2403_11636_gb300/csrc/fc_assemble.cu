// fc_assemble.cu -- global operator L and right-hand side b (paper Sec. 3,
// eq. linear_system) from the element data.
//
// The operator is kept as a compressed node stencil: for node a and each of
// its 3^d neighbours b the values A (velocity-velocity, equal for every
// component), B_c (row (a,c), column p_b), T_c (row p_a, column (b,c)) and
// C (pressure-pressure), summed over the cells that contain both nodes in
// the order of the 2^d cells around a.  C comes from the closed form of the
// stabilisation c(q,p) = -(1/eta)(q - Pi0 q, p - Pi0 p) on an axis-aligned
// cell (eq. stabilization_l2): -(1/eta)(M_ab - |K| / 4^d), M the Q1 mass.
// Strong Dirichlet DoFs are not baked in; the node masks turn their rows
// into identity rows and their columns into right-hand-side lifting.
#include "fc_internal.cuh"

namespace fc {

namespace {

template <int DIM>
__global__ void assemble_kernel(LevelGeom g, const double* __restrict__ eA,
                                const double* __restrict__ eB, double* __restrict__ st) {
  constexpr int NL = 1 << DIM, NB = DIM == 3 ? 27 : 9, SP = 2 * DIM + 2;
  long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= g.nnodes * NB) return;
  long long node = tid % g.nnodes;
  int nb = (int)(tid / g.nnodes);
  int ia[3] = {(int)(node % g.nn[0]), (int)((node / g.nn[0]) % g.nn[1]),
               DIM == 3 ? (int)(node / ((long long)g.nn[0] * g.nn[1])) : 0};
  int off[3] = {nb % 3 - 1, (nb / 3) % 3 - 1, DIM == 3 ? nb / 9 - 1 : 0};
  double vA = 0.0, vB[3] = {0, 0, 0}, vT[3] = {0, 0, 0}, vC = 0.0;
  // closed-form stabilisation block
  double vol = 1.0;
  for (int k = 0; k < DIM; ++k) vol = vol * g.h[k];
  for (int cc = 0; cc < NL; ++cc) {
    int ic[3] = {0, 0, 0};
    bool inside = true;
    for (int k = 0; k < DIM; ++k) {
      ic[k] = ia[k] - 1 + ((cc >> k) & 1);
      if (ic[k] < 0 || ic[k] >= g.n[k]) inside = false;
    }
    if (!inside) continue;
    int la = 0, lb = 0;
    bool shared = true;
    for (int k = 0; k < DIM; ++k) {
      la |= (ia[k] - ic[k]) << k;
      int d = ia[k] + off[k] - ic[k];
      if (d < 0 || d > 1) shared = false;
      lb |= (d & 1) << k;
    }
    if (!shared) continue;
    long long cell = ic[0] + (long long)g.n[0] * (ic[1] + (long long)g.n[1] * ic[2]);
    const double* A = eA + cell * NL * NL;
    const double* B = eB + cell * DIM * NL * NL;
    vA = vA + A[la * NL + lb];
    for (int c = 0; c < DIM; ++c) {
      vB[c] = vB[c] + B[(c * NL + la) * NL + lb];
      vT[c] = vT[c] + B[(c * NL + lb) * NL + la];
    }
    double m = 1.0;
    for (int k = 0; k < DIM; ++k) m = m * (((la >> k) & 1) == ((lb >> k) & 1) ? 1.0 / 3.0 : 1.0 / 6.0);
    double quarter = 1.0;
    for (int k = 0; k < DIM; ++k) quarter = quarter * 0.25;
    vC = vC + (-(1.0 / g.eta) * (vol * m - vol * quarter));
  }
  long long base = (long long)nb * SP;
  st[(base + 0) * g.nnodes + node] = vA;
  for (int c = 0; c < DIM; ++c) {
    st[(base + 1 + c) * g.nnodes + node] = vB[c];
    st[(base + 1 + DIM + c) * g.nnodes + node] = vT[c];
  }
  st[(base + 1 + 2 * DIM) * g.nnodes + node] = vC;
}

// Dirichlet data per boundary preset: 0 channel (inflow at x = lo with the
// parabolic profile of eq. cf_inflow, no-slip walls on the y (and z) faces),
// 1 porous (no-slip on the y (and z) faces), 2 none.  All velocity
// components of a node are constrained together.
__global__ void mask_kernel(LevelGeom g, unsigned char* __restrict__ mask, double* __restrict__ wfix) {
  long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g.nnodes) return;
  int i = (int)(node % g.nn[0]), j = (int)((node / g.nn[0]) % g.nn[1]);
  int k = g.dim == 3 ? (int)(node / ((long long)g.nn[0] * g.nn[1])) : 0;
  bool wall = (j == 0 || j == g.n[1]);
  if (g.dim == 3) wall = wall || k == 0 || k == g.n[2];
  bool fixed = false;
  double w0 = 0.0;
  if (g.preset == 0) {
    bool inflow = (i == 0);
    fixed = wall || inflow;
    if (!wall && inflow) {
      double y = g.lo[1] + (double)j * g.h[1];
      double H = g.hi[1] - g.lo[1];
      double s = (y - g.lo[1]) / H;
      double v = 4.0 * g.ubar * s * (1.0 - s);
      if (g.dim == 3) {
        double z = g.lo[2] + (double)k * g.h[2];
        double t = (z - g.lo[2]) / (g.hi[2] - g.lo[2]);
        v = v * 4.0 * t * (1.0 - t);
      }
      w0 = v;
    }
  } else if (g.preset == 1) {
    fixed = wall;
  }
  unsigned char mk = 0;
  if (fixed)
    for (int c = 0; c < g.dim; ++c) mk |= (unsigned char)(1u << c);
  mask[node] = mk;
  for (int c = 0; c < g.nd; ++c) wfix[node * g.nd + c] = (fixed && c == 0) ? w0 : 0.0;
}

// b = f gathered from the cells around each node, minus the lifted
// constrained columns; b = w on constrained DoFs.
template <int DIM>
__global__ void rhs_kernel(LevelGeom g, const double* __restrict__ eF, const double* __restrict__ st,
                           const unsigned char* __restrict__ mask, const double* __restrict__ wfix,
                           double* __restrict__ b) {
  constexpr int NL = 1 << DIM, NB = DIM == 3 ? 27 : 9, SP = 2 * DIM + 2, ND = DIM + 1;
  long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g.nnodes) return;
  int ia[3] = {(int)(node % g.nn[0]), (int)((node / g.nn[0]) % g.nn[1]),
               DIM == 3 ? (int)(node / ((long long)g.nn[0] * g.nn[1])) : 0};
  double f[DIM];
  for (int c = 0; c < DIM; ++c) f[c] = 0.0;
  for (int cc = 0; cc < NL; ++cc) {
    int ic[3] = {0, 0, 0};
    bool inside = true;
    for (int k = 0; k < DIM; ++k) {
      ic[k] = ia[k] - 1 + ((cc >> k) & 1);
      if (ic[k] < 0 || ic[k] >= g.n[k]) inside = false;
    }
    if (!inside) continue;
    int la = 0;
    for (int k = 0; k < DIM; ++k) la |= (ia[k] - ic[k]) << k;
    long long cell = ic[0] + (long long)g.n[0] * (ic[1] + (long long)g.n[1] * ic[2]);
    for (int c = 0; c < DIM; ++c) f[c] = f[c] + eF[cell * DIM * NL + c * NL + la];
  }
  unsigned char ma = mask[node];
  for (int ca = 0; ca < ND; ++ca) {
    if (ca < DIM && ((ma >> ca) & 1)) {
      b[node * ND + ca] = wfix[node * ND + ca];
      continue;
    }
    double rhs = ca < DIM ? f[ca] : 0.0;
    for (int nb = 0; nb < NB; ++nb) {
      int ib[3] = {ia[0] + nb % 3 - 1, ia[1] + (nb / 3) % 3 - 1, DIM == 3 ? ia[2] + nb / 9 - 1 : 0};
      bool inside = true;
      for (int k = 0; k < DIM; ++k)
        if (ib[k] < 0 || ib[k] > g.n[k]) inside = false;
      if (!inside) continue;
      long long bn = ib[0] + (long long)g.nn[0] * (ib[1] + (long long)g.nn[1] * ib[2]);
      unsigned char mb = mask[bn];
      for (int cb = 0; cb < DIM; ++cb) {
        if (!((mb >> cb) & 1)) continue;
        double v;
        if (ca < DIM) v = (ca == cb) ? st[((long long)nb * SP + 0) * g.nnodes + node] : 0.0;
        else v = st[((long long)nb * SP + 1 + DIM + cb) * g.nnodes + node];
        rhs = rhs - v * wfix[bn * ND + cb];
      }
    }
    b[node * ND + ca] = rhs;
  }
}

// Galerkin coarse operator L_c = R L_f P (the alternative to rediscretising
// the coarser grids of the hierarchy, Sec. 3), with the transfers of the
// V-cycle: P = Q1 interpolation per component, weight prod_k w(i_k - 2 I_k),
// w(0) = 1, w(+-1) = 1/2; constrained fine velocity DoFs have zero rows of P
// (the prolongation leaves them alone), so the product runs over free fine
// velocity DoFs only.  One thread per (coarse node I, neighbour offset):
// the fine nodes i = 2 I + e and j = 2 J + e' (e, e' in {-1, 0, 1}^d) with
// j - i within the fine 3^d stencil, summed in a fixed order, so equal fine
// neighbourhoods give bit-equal coarse entries.  The result is a raw coarse
// stencil like the rediscretised one: the coarse masks act where it is used.
template <int DIM>
__global__ void galerkin_kernel(LevelGeom gc, LevelGeom gf, const double* __restrict__ stf,
                                const unsigned char* __restrict__ maskf, double* __restrict__ stc) {
  constexpr int NB = DIM == 3 ? 27 : 9, SP = 2 * DIM + 2;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= gc.nnodes * NB) return;
  const long long node = tid % gc.nnodes;
  const int nb = (int)(tid / gc.nnodes);
  const int ia[3] = {(int)(node % gc.nn[0]), (int)((node / gc.nn[0]) % gc.nn[1]),
                     DIM == 3 ? (int)(node / ((long long)gc.nn[0] * gc.nn[1])) : 0};
  const int off[3] = {nb % 3 - 1, (nb / 3) % 3 - 1, DIM == 3 ? nb / 9 - 1 : 0};
  double vA = 0.0, vB[3] = {0, 0, 0}, vT[3] = {0, 0, 0}, vC = 0.0;
  for (int ti = 0; ti < NB; ++ti) {
    int fi[3] = {0, 0, 0};
    double wi = 1.0;
    bool in = true;
    for (int k = 0; k < DIM; ++k) {
      const int e = (k == 0 ? ti % 3 : (k == 1 ? (ti / 3) % 3 : ti / 9)) - 1;
      fi[k] = 2 * ia[k] + e;
      if (fi[k] < 0 || fi[k] > gf.n[k]) in = false;
      wi = wi * (e == 0 ? 1.0 : 0.5);
    }
    if (!in) continue;
    const long long i = fi[0] + (long long)gf.nn[0] * (fi[1] + (long long)gf.nn[1] * fi[2]);
    const bool fixi = maskf[i] != 0;
    for (int tj = 0; tj < NB; ++tj) {
      int fj[3] = {0, 0, 0}, d[3] = {0, 0, 0};
      double wj = 1.0;
      bool ok = true;
      for (int k = 0; k < DIM; ++k) {
        const int e = (k == 0 ? tj % 3 : (k == 1 ? (tj / 3) % 3 : tj / 9)) - 1;
        fj[k] = 2 * (ia[k] + off[k]) + e;
        d[k] = fj[k] - fi[k];
        if (fj[k] < 0 || fj[k] > gf.n[k] || d[k] < -1 || d[k] > 1) ok = false;
        wj = wj * (e == 0 ? 1.0 : 0.5);
      }
      if (!ok) continue;
      const long long j = fj[0] + (long long)gf.nn[0] * (fj[1] + (long long)gf.nn[1] * fj[2]);
      const bool fixj = maskf[j] != 0;
      const int fnb = (d[0] + 1) + 3 * (d[1] + 1) + (DIM == 3 ? 9 * (d[2] + 1) : 0);
      const double* sv = stf + (long long)fnb * SP * gf.nnodes + i;
      const double w = wi * wj;
      if (!fixi && !fixj) vA = vA + w * sv[0];
      for (int c = 0; c < DIM; ++c) {
        if (!fixi) vB[c] = vB[c] + w * sv[(1 + c) * gf.nnodes];
        if (!fixj) vT[c] = vT[c] + w * sv[(1 + DIM + c) * gf.nnodes];
      }
      vC = vC + w * sv[(1 + 2 * DIM) * gf.nnodes];
    }
  }
  const long long base = (long long)nb * SP;
  stc[(base + 0) * gc.nnodes + node] = vA;
  for (int c = 0; c < DIM; ++c) {
    stc[(base + 1 + c) * gc.nnodes + node] = vB[c];
    stc[(base + 1 + DIM + c) * gc.nnodes + node] = vT[c];
  }
  stc[(base + 1 + 2 * DIM) * gc.nnodes + node] = vC;
}

// cell data of a coarse level from its 2^d children on the finer level:
// the class is the children's common class (0 when they differ or any is
// cut), the cell statistics are the children's sums (fluid volume first)
template <int DIM>
__global__ void coarsen_cells_kernel(LevelGeom gc, LevelGeom gf, const unsigned char* __restrict__ cf,
                                     unsigned char* __restrict__ cc, const double* __restrict__ ef,
                                     double* __restrict__ ec) {
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= gc.ncell) return;
  const int ic[3] = {(int)(cell % gc.n[0]), (int)((cell / gc.n[0]) % gc.n[1]),
                     DIM == 3 ? (int)(cell / ((long long)gc.n[0] * gc.n[1])) : 0};
  int cls = -1;
  double st[4] = {0.0, 0.0, 0.0, 0.0};
  for (int ch = 0; ch < (1 << DIM); ++ch) {
    int f[3] = {0, 0, 0};
    for (int k = 0; k < DIM; ++k) f[k] = 2 * ic[k] + ((ch >> k) & 1);
    const long long fc = f[0] + (long long)gf.n[0] * (f[1] + (long long)gf.n[1] * f[2]);
    if (cf) {
      const int c = cf[fc];
      cls = cls < 0 ? c : (cls == c ? cls : 0);
    }
    if (ef)
      for (int t = 0; t < 4; ++t) st[t] = st[t] + ef[fc * 4 + t];
  }
  if (cc) cc[cell] = (unsigned char)(cls < 0 ? 0 : cls);
  if (ec)
    for (int t = 0; t < 4; ++t) ec[cell * 4 + t] = st[t];
}

}  // namespace

cudaError_t launch_assemble(const LevelGeom& g, const double* eA, const double* eB, double* st,
                            cudaStream_t s) {
  long long n = g.nnodes * (g.dim == 3 ? 27 : 9);
  unsigned blocks = (unsigned)((n + 255) / 256);
  if (g.dim == 2) assemble_kernel<2><<<blocks, 256, 0, s>>>(g, eA, eB, st);
  else assemble_kernel<3><<<blocks, 256, 0, s>>>(g, eA, eB, st);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_masks(const LevelGeom& g, unsigned char* mask, double* wfix, cudaStream_t s) {
  mask_kernel<<<(unsigned)((g.nnodes + 255) / 256), 256, 0, s>>>(g, mask, wfix);
  note_launches(1);
  return cudaGetLastError();
}

// a layer stays flagged only if every node in it has all velocity
// components constrained; any other node clears the flags of its x, y and z
// layers (every writer stores 0, so the races are benign)
__global__ void dead_layer_kernel(LevelGeom g, const unsigned char* __restrict__ mask, unsigned char* out) {
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g.nnodes) return;
  if ((mask[node] & 7) == 7) return;
  const unsigned u = (unsigned)node, nx = (unsigned)g.nn[0], ny = (unsigned)g.nn[1];
  const unsigned t = u / nx;
  out[u - t * nx] = 0;
  out[g.nn[0] + t % ny] = 0;
  out[g.nn[0] + g.nn[1] + t / ny] = 0;
}

cudaError_t launch_dead_layers(const LevelGeom& g, const unsigned char* mask, unsigned char* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 1, (size_t)g.nn[0] + g.nn[1] + g.nn[2], s);
  if (e != cudaSuccess) return e;
  dead_layer_kernel<<<(unsigned)((g.nnodes + 255) / 256), 256, 0, s>>>(g, mask, out);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_rhs(const LevelGeom& g, const double* eF, const double* st,
                       const unsigned char* mask, const double* wfix, double* b, cudaStream_t s) {
  unsigned blocks = (unsigned)((g.nnodes + 127) / 128);
  if (g.dim == 2) rhs_kernel<2><<<blocks, 128, 0, s>>>(g, eF, st, mask, wfix, b);
  else rhs_kernel<3><<<blocks, 128, 0, s>>>(g, eF, st, mask, wfix, b);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace fc

// ---------------------------------------------------------------------------
// Patch classes.  A node whose 2^d cells all exist and are plain with one
// alpha (cell class 1 fluid, 2 fictitious) has a stencil bit-identical to
// every other such node of the same class.  A patch whose 5^d nodes are all
// in the grid, unconstrained and of one node class therefore has a
// bit-identical block L_i: its rows of L_i^{-1} (or its factors) are those
// of the class representative (the lowest patch index of the class).  The
// work list holds the patches that are factored and stored -- every patch
// of class 0 and one representative per class -- in increasing patch order.
// prow[i] = stored block of patch i, encoded as -(block + 1) for blocks
// shared by a class (read through the cache) and block for unique patches.
namespace fc {
namespace {

template <int DIM>
__global__ void node_class_kernel(LevelGeom g, const unsigned char* __restrict__ cclass,
                                  unsigned char* __restrict__ nclass) {
  long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g.nnodes) return;
  const unsigned u = (unsigned)node, nx = (unsigned)g.nn[0], ny = (unsigned)g.nn[1];
  const unsigned q = u / nx;
  int ia[3] = {(int)(u - q * nx), DIM == 3 ? (int)(q % ny) : (int)q, DIM == 3 ? (int)(q / ny) : 0};
  int cls = -1;
  for (int cc = 0; cc < (1 << DIM); ++cc) {
    int ic[3] = {0, 0, 0};
    bool in = true;
    for (int k = 0; k < DIM; ++k) {
      ic[k] = ia[k] - 1 + ((cc >> k) & 1);
      if (ic[k] < 0 || ic[k] >= g.n[k]) in = false;
    }
    if (!in) { cls = 0; break; }
    int c = cclass[ic[0] + (long long)g.n[0] * (ic[1] + (long long)g.n[1] * ic[2])];
    if (cls < 0) cls = c;
    else if (c != cls) { cls = 0; break; }
  }
  nclass[node] = (unsigned char)(cls < 0 ? 0 : cls);
}

template <int DIM>
__global__ void patch_class_kernel(LevelGeom g, const unsigned char* __restrict__ nclass,
                                   const unsigned char* __restrict__ mask, int* __restrict__ pclass,
                                   int* __restrict__ rep, int dedup) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.nnodes) return;
  if (!dedup) { pclass[i] = 0; return; }
  const unsigned u = (unsigned)i, nx = (unsigned)g.nn[0], ny = (unsigned)g.nn[1];
  const unsigned q = u / nx;
  int ia[3] = {(int)(u - q * nx), DIM == 3 ? (int)(q % ny) : (int)q, DIM == 3 ? (int)(q / ny) : 0};
  int cls = nclass[i];
  const int r5 = DIM == 3 ? 5 : 1;
  for (int dz = 0; dz < r5 && cls; ++dz)
    for (int dy = 0; dy < 5 && cls; ++dy)
      for (int dx = 0; dx < 5 && cls; ++dx) {
        int b0 = ia[0] + dx - 2, b1 = ia[1] + dy - 2, b2 = DIM == 3 ? ia[2] + dz - 2 : 0;
        if (b0 < 0 || b0 > g.n[0] || b1 < 0 || b1 > g.n[1] || (DIM == 3 && (b2 < 0 || b2 > g.n[2]))) { cls = 0; break; }
        long long bn = b0 + (long long)g.nn[0] * (b1 + (long long)g.nn[1] * b2);
        if ((mask[bn] & 1) || nclass[bn] != cls) cls = 0;
      }
  pclass[i] = cls;
  if (cls) atomicMin(&rep[cls], (int)i);
}

constexpr int kScanBlock = 1024;

// flag: patch is stored (class 0 or a class representative)
__device__ __forceinline__ bool stored(const int* pclass, const int* rep, long long i) {
  int c = pclass[i];
  return c == 0 || rep[c] == (int)i;
}

__global__ void count_stored_kernel(long long n, const int* __restrict__ pclass, const int* __restrict__ rep,
                                    int* __restrict__ counts) {
  __shared__ int sm[32];
  long long i = (long long)blockIdx.x * kScanBlock + threadIdx.x;
  int f = (i < n && stored(pclass, rep, i)) ? 1 : 0;
  unsigned bal = __ballot_sync(0xffffffffu, f);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = __popc(bal);
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < kScanBlock / 32; ++w) t += sm[w];
    counts[blockIdx.x] = t;
  }
}

__global__ void scan_counts_kernel(int nb, int* __restrict__ counts, int* __restrict__ total) {
  // exclusive scan in one thread (nb is the number of 1024-patch blocks)
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int run = 0;
  for (int b = 0; b < nb; ++b) {
    int c = counts[b];
    counts[b] = run;
    run += c;
  }
  *total = run;
}

__global__ void place_stored_kernel(long long n, const int* __restrict__ pclass, const int* __restrict__ rep,
                                    const int* __restrict__ offs, int* __restrict__ work, int* __restrict__ prow) {
  __shared__ int sm[32];
  long long i = (long long)blockIdx.x * kScanBlock + threadIdx.x;
  int f = (i < n && stored(pclass, rep, i)) ? 1 : 0;
  unsigned bal = __ballot_sync(0xffffffffu, f);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sm[wid] = __popc(bal);
  __syncthreads();
  int before = 0;
  for (int w = 0; w < wid; ++w) before += sm[w];
  if (f) {
    int pos = offs[blockIdx.x] + before + __popc(bal & ((1u << lane) - 1u));
    work[pos] = (int)i;
    prow[i] = pclass[i] ? -(pos + 1) : pos;
  }
}

__global__ void class_rows_kernel(long long n, const int* __restrict__ pclass, const int* __restrict__ rep,
                                  int* __restrict__ prow) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = pclass[i];
  if (c && rep[c] != (int)i) prow[i] = prow[rep[c]];
}

}  // namespace

cudaError_t launch_patch_classes(const LevelGeom& g, const unsigned char* cclass, const unsigned char* mask,
                                 unsigned char* nclass, int* pclass, int* rep, int* work, int* nwork,
                                 int* prow, int dedup, cudaStream_t s) {
  const long long n = g.nnodes;
  const unsigned b256 = (unsigned)((n + 255) / 256);
  const int nb = (int)((n + kScanBlock - 1) / kScanBlock);
  int init[4] = {0x7fffffff, 0x7fffffff, 0x7fffffff, 0x7fffffff};
  cudaError_t e = cudaMemcpyAsync(rep, init, sizeof(init), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  if (g.dim == 2) {
    node_class_kernel<2><<<b256, 256, 0, s>>>(g, cclass, nclass);
    patch_class_kernel<2><<<b256, 256, 0, s>>>(g, nclass, mask, pclass, rep, dedup);
  } else {
    node_class_kernel<3><<<b256, 256, 0, s>>>(g, cclass, nclass);
    patch_class_kernel<3><<<b256, 256, 0, s>>>(g, nclass, mask, pclass, rep, dedup);
  }
  // block counts live in the tail of `work` scratch: work has n + nb ints
  int* counts = work + n;
  count_stored_kernel<<<nb, kScanBlock, 0, s>>>(n, pclass, rep, counts);
  scan_counts_kernel<<<1, 32, 0, s>>>(nb, counts, nwork);
  place_stored_kernel<<<nb, kScanBlock, 0, s>>>(n, pclass, rep, counts, work, prow);
  class_rows_kernel<<<b256, 256, 0, s>>>(n, pclass, rep, prow);
  note_launches(6);
  return cudaGetLastError();
}


cudaError_t launch_galerkin(const LevelGeom& gc, const LevelGeom& gf, const double* stf, const unsigned char* maskf,
                            double* stc, cudaStream_t s) {
  const long long n = gc.nnodes * (gc.dim == 3 ? 27 : 9);
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (gc.dim == 2) galerkin_kernel<2><<<blocks, 256, 0, s>>>(gc, gf, stf, maskf, stc);
  else galerkin_kernel<3><<<blocks, 256, 0, s>>>(gc, gf, stf, maskf, stc);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_coarsen_cells(const LevelGeom& gc, const LevelGeom& gf, const unsigned char* cclass_f,
                                 unsigned char* cclass_c, const double* estat_f, double* estat_c, cudaStream_t s) {
  const unsigned blocks = (unsigned)((gc.ncell + 255) / 256);
  if (gc.dim == 2) coarsen_cells_kernel<2><<<blocks, 256, 0, s>>>(gc, gf, cclass_f, cclass_c, estat_f, estat_c);
  else coarsen_cells_kernel<3><<<blocks, 256, 0, s>>>(gc, gf, cclass_f, cclass_c, estat_f, estat_c);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace fc
