// fc_mg.cu -- operator application (residual r = b - L x, paper eq.
// iteration), grid transfers R and P = R^T (eq. restriction_op), the dense
// coarse solve (Sec. 3), and the vector kernels of the FP64 FGMRES outer
// iteration (Sec. 4 remark on Krylov methods).
#include <math.h>

#include <algorithm>

#include "fc_internal.cuh"

namespace fc {

namespace {

// ---------------------------------------------------------------------------
// residual / apply: one thread per node, the 3^d neighbour blocks of the
// compressed stencil; constrained rows are identity rows and constrained
// columns are skipped (their values live in b).
// OUT: 0 -> r (unpadded, optional) and rpad (padded, optional) in float64,
//      1 -> rpad as float32 pairs (hi, lo), 2 -> rpad as float32.
template <int DIM, int OUT>
__global__ void __launch_bounds__(256)
    residual_kernel(LevelGeom g, const double* __restrict__ st, const unsigned char* __restrict__ mask,
                    const double* __restrict__ x, const double* __restrict__ b,
                    double* __restrict__ r, double* __restrict__ rpad, float* __restrict__ rpadf) {
  constexpr int NB = DIM == 3 ? 27 : 9, SP = 2 * DIM + 2, ND = DIM + 1;
  long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g.nnodes) return;
  // 32-bit decode: 64-bit division would run on the slow FP64 pipe
  int ia[3];
  {
    const unsigned u = (unsigned)node, nx = (unsigned)g.nn[0], ny = (unsigned)g.nn[1];
    const unsigned t = u / nx;
    ia[0] = (int)(u - t * nx);
    ia[1] = DIM == 3 ? (int)(t % ny) : (int)t;
    ia[2] = DIM == 3 ? (int)(t / ny) : 0;
  }
  double acc[ND];
#pragma unroll
  for (int c = 0; c < ND; ++c) acc[c] = 0.0;
#pragma unroll
  for (int nb = 0; nb < NB; ++nb) {
    int ib0 = ia[0] + nb % 3 - 1, ib1 = ia[1] + (nb / 3) % 3 - 1, ib2 = DIM == 3 ? ia[2] + nb / 9 - 1 : 0;
    if (ib0 < 0 || ib0 > g.n[0] || ib1 < 0 || ib1 > g.n[1]) continue;
    if (DIM == 3 && (ib2 < 0 || ib2 > g.n[2])) continue;
    long long bn = ib0 + (long long)g.nn[0] * (ib1 + (long long)g.nn[1] * ib2);
    unsigned char mb = mask[bn];
    double xb[ND];
#pragma unroll
    for (int c = 0; c < ND; ++c) xb[c] = x[bn * ND + c];
#pragma unroll
    for (int c = 0; c < DIM; ++c)
      if ((mb >> c) & 1) xb[c] = 0.0;
    const double* s = st + (long long)nb * SP * g.nnodes + node;
    double vA = s[0];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      acc[c] = acc[c] + vA * xb[c];
      acc[c] = acc[c] + s[(1 + c) * g.nnodes] * xb[DIM];
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) acc[DIM] = acc[DIM] + s[(1 + DIM + c) * g.nnodes] * xb[c];
    acc[DIM] = acc[DIM] + s[(1 + 2 * DIM) * g.nnodes] * xb[DIM];
  }
  unsigned char ma = mask[node];
  long long pn = pad_node(g, ia[0], ia[1], ia[2]);
#pragma unroll
  for (int c = 0; c < ND; ++c) {
    double y = (c < DIM && ((ma >> c) & 1)) ? x[node * ND + c] : acc[c];
    double v = b ? b[node * ND + c] - y : y;
    if (OUT == 0) {
      if (r) r[node * ND + c] = v;
      if (rpad) rpad[pn * ND + c] = v;
    } else if (OUT == 1) {
      float hi = (float)v;
      float lo = (float)(v - (double)hi);
      rpadf[(pn * ND + c) * 2 + 0] = hi;
      rpadf[(pn * ND + c) * 2 + 1] = lo;
    } else {
      rpadf[pn * ND + c] = (float)v;
    }
  }
}

// ---------------------------------------------------------------------------
// float-pair residual for the smoother (FC_PREC_DF64): the stencil, x and b
// as (hi, lo) pairs of float32, products by the exact FMA split plus cross
// terms, sums by two-sum of the high parts with the low parts collected
// apart (about 48-bit significand), all on the float32 pipes.
struct dfp { float hi, lo; };
__device__ __forceinline__ void dfacc(dfp& acc, float2 a, float2 b) {
  float p = a.x * b.x;
  float pe = fmaf(a.x, b.x, -p);
  float cross = fmaf(a.x, b.y, a.y * b.x);
  float s = acc.hi + p;
  float bb = s - acc.hi;
  float e = (acc.hi - (s - bb)) + (p - bb);
  acc.hi = s;
  acc.lo += e + (pe + cross);
}

// The operator is symmetric, so the pair stencil keeps half of the
// neighbour offsets: the zero offset and the NH - 1 offsets after it in
// lexicographic order (the "own" offsets).  The entries of node a for a
// mirrored offset -d are the transposed entries that its neighbour b = a - d
// stores for offset +d:  A(a,b) = A(b,a), B_c(a,b) = T_c(b,a),
// T_c(a,b) = B_c(b,a), C(a,b) = C(b,a).  Each node reads its own entries
// and those of its neighbours for the mirrored offsets (mostly from L2), so
// the stencil's DRAM bytes halve.
template <int DIM>
__device__ __forceinline__ constexpr int half_offsets() { return (DIM == 3 ? 27 : 9) - (DIM == 3 ? 13 : 4); }

// sum of two running pair sums (high parts by an exact two-sum, low parts
// plainly); symmetric in its arguments, so both lanes of a shuffle pair get
// the same result
__device__ __forceinline__ dfp dfp_join(dfp a, dfp b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb);
  return {s, e + (a.lo + b.lo)};
}

// float-pair residual on the half stencil, TPP lanes per node: lane l takes
// the half-stencil offsets l, l + TPP, ... (own and mirrored entries), the
// group adds its partial sums by shuffles.  TPP = 1 on large levels; small levels, where one
// thread per node leaves most SMs idle and each thread walks all 27
// neighbours' loads in turn, take a group.  Own entries of out-of-grid
// neighbours are stored as zero and x has a zero halo, mirrored entries are
// read only from neighbours inside the grid.
template <int DIM, int TPP>
__global__ void __launch_bounds__(256)
    residual_df2_kernel(LevelGeom g, const float2* __restrict__ sth, const unsigned char* __restrict__ mask,
                        const float2* __restrict__ xp2, const float2* __restrict__ b2,
                        float2* __restrict__ rpad2, double* __restrict__ r) {
  constexpr int CEN = DIM == 3 ? 13 : 4, NH = half_offsets<DIM>(), SP = 2 * DIM + 2, ND = DIM + 1;
  // a warp covers W = 32 / TPP consecutive nodes; warp lane w takes node
  // w % W and offset slot w / W, so the lanes of one slot read W consecutive
  // nodes of each stencil plane.  A node's group (the lanes w % W equal)
  // leaves as a whole past the last node and shuffles among its own lanes.
  constexpr int W = 32 / TPP;
  const int wl = threadIdx.x & 31;
  const int lane = wl / W;
  const long long node = ((long long)blockIdx.x * blockDim.x + (threadIdx.x - wl)) / TPP + wl % W;
  unsigned gmask = 0u;
#pragma unroll
  for (int j = 0; j < TPP; ++j) gmask |= 1u << (wl % W + W * j);
  if (node >= g.nnodes) return;
  int ia[3];
  {
    const unsigned u = (unsigned)node, nx = (unsigned)g.nn[0], ny = (unsigned)g.nn[1];
    const unsigned q = u / nx;
    ia[0] = (int)(u - q * nx);
    ia[1] = DIM == 3 ? (int)(q % ny) : (int)q;
    ia[2] = DIM == 3 ? (int)(q / ny) : 0;
  }
  const int px = g.nn[0] + 4, py = g.nn[1] + 4;
  const long long pn = pad_node(g, ia[0], ia[1], ia[2]);
  const float2* xc = xp2 + pn * ND;
  dfp acc[ND];
#pragma unroll
  for (int c = 0; c < ND; ++c) acc[c] = {0.0f, 0.0f};
  // every lane of a group runs the same iterations (offset k TPP + lane)
  constexpr int NIT = (NH + TPP - 1) / TPP;
#pragma unroll
  for (int k = 0; k < NIT; ++k) {
    const int h = TPP == 1 ? k : k * TPP + lane;
    if (TPP > 1 && h >= NH) break;
    const int nb = CEN + h;
    const int d0 = nb % 3 - 1, d1 = (nb / 3) % 3 - 1, d2 = DIM == 3 ? nb / 9 - 1 : 0;
    const int off = d0 + px * (d1 + (DIM == 3 ? py * d2 : 0));
    {  // own entries, neighbour a + d
      const float2* xb = xc + off * ND;
      const float2* sp = sth + (long long)h * SP * g.nnodes + node;
      const float2 vA = __ldcs(sp);
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        dfacc(acc[c], vA, xb[c]);
        dfacc(acc[c], __ldcs(sp + (1 + c) * g.nnodes), xb[DIM]);
      }
#pragma unroll
      for (int c = 0; c < DIM; ++c) dfacc(acc[DIM], __ldcs(sp + (1 + DIM + c) * g.nnodes), xb[c]);
      dfacc(acc[DIM], __ldcs(sp + (1 + 2 * DIM) * g.nnodes), xb[DIM]);
    }
    if (h > 0) {  // mirrored offset -d: transposed entries of b = a - d
      const int b0 = ia[0] - d0, b1 = ia[1] - d1, b2i = ia[2] - d2;
      const bool in = b0 >= 0 && b0 <= g.n[0] && b1 >= 0 && b1 <= g.n[1] && (DIM == 2 || (b2i >= 0 && b2i <= g.n[2]));
      if (in) {
        const long long bnode = node - (d0 + (long long)g.nn[0] * (d1 + (long long)g.nn[1] * d2));
        const float2* xm = xc - off * ND;
        const float2* sm = sth + (long long)h * SP * g.nnodes + bnode;
        const float2 vA = sm[0];
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          dfacc(acc[c], vA, xm[c]);
          dfacc(acc[c], sm[(1 + DIM + c) * g.nnodes], xm[DIM]);
        }
#pragma unroll
        for (int c = 0; c < DIM; ++c) dfacc(acc[DIM], sm[(1 + c) * g.nnodes], xm[c]);
        dfacc(acc[DIM], sm[(1 + 2 * DIM) * g.nnodes], xm[DIM]);
      }
    }
  }
#pragma unroll
  for (int o = TPP / 2; o > 0; o >>= 1)
#pragma unroll
    for (int c = 0; c < ND; ++c) {
      const dfp other = {__shfl_xor_sync(gmask, acc[c].hi, o * W), __shfl_xor_sync(gmask, acc[c].lo, o * W)};
      acc[c] = dfp_join(acc[c], other);
    }
  const unsigned char ma = mask[node];
#pragma unroll
  for (int c = 0; c < ND; ++c) {
    if (TPP > 1 && c % TPP != lane) continue;
    float yh = acc[c].hi + acc[c].lo;
    float yl = acc[c].lo - (yh - acc[c].hi);
    if (c < DIM && ((ma >> c) & 1)) {
      const float2 xv = xc[c];
      yh = xv.x; yl = xv.y;
    }
    const float2 bv = b2[node * ND + c];
    // (b - y) as a pair
    const float sh = bv.x - yh;
    const float bb = sh - bv.x;
    float e = (bv.x - (sh - bb)) + (-yh - bb);
    e += bv.y - yl;
    const float hh = sh + e;
    const float l = e - (hh - sh);
    if (rpad2) rpad2[pn * ND + c] = make_float2(hh, l);
    if (r) r[node * ND + c] = (double)hh + (double)l;
  }
}

// half pair stencil (own offsets only, see residual_df2_kernel) with the
// columns of constrained DoFs folded to zero.  A stored entry serves row a
// (column b) and, transposed, row b (column a); all velocity components of
// a node are constrained together and rows of constrained velocities are
// identity rows, so:  A is zero when a or b is constrained, B_c (also the
// T_c of row b) when a is, T_c (also the B_c of row b) when b is.
template <int DIM>
__global__ void fold_stencil_pairs_kernel(LevelGeom g, const double* __restrict__ st,
                                          const unsigned char* __restrict__ mask, float2* __restrict__ sth) {
  constexpr int CEN = DIM == 3 ? 13 : 4, NH = half_offsets<DIM>(), SP = 2 * DIM + 2;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.nnodes * NH) return;
  const long long node = t % g.nnodes;
  const int h = (int)(t / g.nnodes), nb = CEN + h;
  int ia[3];
  {
    const unsigned u = (unsigned)node, nx = (unsigned)g.nn[0], ny = (unsigned)g.nn[1];
    const unsigned q = u / nx;
    ia[0] = (int)(u - q * nx);
    ia[1] = DIM == 3 ? (int)(q % ny) : (int)q;
    ia[2] = DIM == 3 ? (int)(q / ny) : 0;
  }
  const int ib0 = ia[0] + nb % 3 - 1, ib1 = ia[1] + (nb / 3) % 3 - 1, ib2 = DIM == 3 ? ia[2] + nb / 9 - 1 : 0;
  const bool inside = !(ib0 < 0 || ib0 > g.n[0] || ib1 < 0 || ib1 > g.n[1]) &&
                      !(DIM == 3 && (ib2 < 0 || ib2 > g.n[2]));
  const bool own_fixed = mask[node] & 1;
  const bool nb_fixed = inside && (mask[ib0 + (long long)g.nn[0] * (ib1 + (long long)g.nn[1] * ib2)] & 1);
  for (int e = 0; e < SP; ++e) {
    double v = inside ? st[((long long)nb * SP + e) * g.nnodes + node] : 0.0;
    if (e == 0 && (own_fixed || nb_fixed)) v = 0.0;
    else if (e >= 1 && e <= DIM && own_fixed) v = 0.0;
    else if (e >= 1 + DIM && e < 1 + 2 * DIM && nb_fixed) v = 0.0;
    const float hi = (float)v;
    sth[((long long)h * SP + e) * g.nnodes + node] = make_float2(hi, (float)(v - (double)hi));
  }
}

// float32 half stencil for the float32 correction-form V-cycle: the same
// own offsets and folding rules as the pair stencil above
template <int DIM>
__global__ void fold_stencil_f32_kernel(LevelGeom g, const double* __restrict__ st,
                                        const unsigned char* __restrict__ mask, float* __restrict__ st32) {
  constexpr int CEN = DIM == 3 ? 13 : 4, NH = half_offsets<DIM>(), SP = 2 * DIM + 2;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.nnodes * NH) return;
  const long long node = t % g.nnodes;
  const int h = (int)(t / g.nnodes), nb = CEN + h;
  int ia[3];
  {
    const unsigned u = (unsigned)node, nx = (unsigned)g.nn[0], ny = (unsigned)g.nn[1];
    const unsigned q = u / nx;
    ia[0] = (int)(u - q * nx);
    ia[1] = DIM == 3 ? (int)(q % ny) : (int)q;
    ia[2] = DIM == 3 ? (int)(q / ny) : 0;
  }
  const int ib0 = ia[0] + nb % 3 - 1, ib1 = ia[1] + (nb / 3) % 3 - 1, ib2 = DIM == 3 ? ia[2] + nb / 9 - 1 : 0;
  const bool inside = !(ib0 < 0 || ib0 > g.n[0] || ib1 < 0 || ib1 > g.n[1]) &&
                      !(DIM == 3 && (ib2 < 0 || ib2 > g.n[2]));
  const bool own_fixed = mask[node] & 1;
  const bool nb_fixed = inside && (mask[ib0 + (long long)g.nn[0] * (ib1 + (long long)g.nn[1] * ib2)] & 1);
  for (int e = 0; e < SP; ++e) {
    double v = inside ? st[((long long)nb * SP + e) * g.nnodes + node] : 0.0;
    if (e == 0 && (own_fixed || nb_fixed)) v = 0.0;
    else if (e >= 1 && e <= DIM && own_fixed) v = 0.0;
    else if (e >= 1 + DIM && e < 1 + 2 * DIM && nb_fixed) v = 0.0;
    st32[((long long)h * SP + e) * g.nnodes + node] = (float)v;
  }
}

template <int DIM>
__global__ void split_x_padded_kernel(LevelGeom g, const double* __restrict__ x, float2* __restrict__ xp2) {
  constexpr int ND = DIM + 1;
  long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g.nnodes) return;
  const unsigned u = (unsigned)node, nx = (unsigned)g.nn[0], ny = (unsigned)g.nn[1];
  const unsigned q = u / nx;
  const long long pn = pad_node(g, (int)(u - q * nx), DIM == 3 ? (int)(q % ny) : (int)q, DIM == 3 ? (int)(q / ny) : 0);
#pragma unroll
  for (int c = 0; c < ND; ++c) {
    double v = x[node * ND + c];
    float hi = (float)v;
    xp2[pn * ND + c] = make_float2(hi, (float)(v - (double)hi));
  }
}

template <int DIM>
__global__ void merge_x_padded_kernel(LevelGeom g, const float2* __restrict__ xp2, double* __restrict__ x) {
  constexpr int ND = DIM + 1;
  long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g.nnodes) return;
  const unsigned u = (unsigned)node, nx = (unsigned)g.nn[0], ny = (unsigned)g.nn[1];
  const unsigned q = u / nx;
  const long long pn = pad_node(g, (int)(u - q * nx), DIM == 3 ? (int)(q % ny) : (int)q, DIM == 3 ? (int)(q / ny) : 0);
#pragma unroll
  for (int c = 0; c < ND; ++c) {
    float2 v = xp2[pn * ND + c];
    x[node * ND + c] = (double)v.x + (double)v.y;
  }
}

__global__ void split_pairs_kernel(long long n, const double* __restrict__ in, float2* __restrict__ out) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double v = in[t];
    float hi = (float)v;
    out[t] = make_float2(hi, (float)(v - (double)hi));
  }
}

// ---------------------------------------------------------------------------
// transfers: Q1 interpolation between nested uniform grids (fine n = 2 nc)
__device__ __forceinline__ double pw(int d) { return d == 0 ? 1.0 : 0.5; }

template <int DIM>
__global__ void restrict_kernel(LevelGeom f, LevelGeom c, const unsigned char* __restrict__ cmask,
                                const double* __restrict__ rf, double* __restrict__ bc) {
  constexpr int ND = DIM + 1;
  long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= c.nnodes) return;
  int I[3] = {(int)(node % c.nn[0]), (int)((node / c.nn[0]) % c.nn[1]),
              DIM == 3 ? (int)(node / ((long long)c.nn[0] * c.nn[1])) : 0};
  double acc[ND];
  for (int q = 0; q < ND; ++q) acc[q] = 0.0;
  for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int i = 2 * I[0] + dx, j = 2 * I[1] + dy, k = DIM == 3 ? 2 * I[2] + dz : 0;
        if (i < 0 || i > f.n[0] || j < 0 || j > f.n[1]) continue;
        if (DIM == 3 && (k < 0 || k > f.n[2])) continue;
        double w = pw(dx) * pw(dy) * (DIM == 3 ? pw(dz) : 1.0);
        long long fn = i + (long long)f.nn[0] * (j + (long long)f.nn[1] * k);
        for (int q = 0; q < ND; ++q) acc[q] = acc[q] + w * rf[fn * ND + q];
      }
  unsigned char m = cmask[node];
  for (int q = 0; q < ND; ++q) bc[node * ND + q] = (q < DIM && ((m >> q) & 1)) ? 0.0 : acc[q];
}

template <int DIM>
__global__ void prolong_kernel(LevelGeom f, LevelGeom c, const unsigned char* __restrict__ fmask,
                               const double* __restrict__ ec, double* __restrict__ xf) {
  constexpr int ND = DIM + 1;
  long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= f.nnodes) return;
  int ia[3] = {(int)(node % f.nn[0]), (int)((node / f.nn[0]) % f.nn[1]),
               DIM == 3 ? (int)(node / ((long long)f.nn[0] * f.nn[1])) : 0};
  int lo[3], hi[3];
  for (int k = 0; k < 3; ++k) { lo[k] = ia[k] / 2; hi[k] = (ia[k] + 1) / 2; }
  double acc[ND];
  for (int q = 0; q < ND; ++q) acc[q] = 0.0;
  for (int t = 0; t < (1 << DIM); ++t) {
    int ic[3] = {0, 0, 0};
    double w = 1.0;
    bool dup = false;
    for (int k = 0; k < DIM; ++k) {
      int bit = (t >> k) & 1;
      if (lo[k] == hi[k] && bit) dup = true;
      ic[k] = bit ? hi[k] : lo[k];
      w = w * (lo[k] == hi[k] ? 1.0 : 0.5);
    }
    if (dup) continue;
    long long cn = ic[0] + (long long)c.nn[0] * (ic[1] + (long long)c.nn[1] * ic[2]);
    for (int q = 0; q < ND; ++q) acc[q] = acc[q] + w * ec[cn * ND + q];
  }
  unsigned char m = fmask[node];
  for (int q = 0; q < ND; ++q)
    if (!(q < DIM && ((m >> q) & 1))) xf[node * ND + q] = xf[node * ND + q] + acc[q];
}

// ---------------------------------------------------------------------------
// coarse operator: dense matrix of the coarsest level, equilibrated LU with
// partial pivoting in one CTA, then the explicit inverse (columns solved
// from the identity) so that each V-cycle applies one dense GEMV.
template <int DIM>
__global__ void coarse_dense_kernel(LevelGeom g, const double* __restrict__ st,
                                    const unsigned char* __restrict__ mask, double* __restrict__ A) {
  constexpr int NB = DIM == 3 ? 27 : 9, SP = 2 * DIM + 2, ND = DIM + 1;
  long long n = g.ndof;
  long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  long long node = row / ND;
  int ca = (int)(row % ND);
  for (long long c2 = 0; c2 < n; ++c2) A[row * n + c2] = 0.0;
  unsigned char ma = mask[node];
  if (ca < DIM && ((ma >> ca) & 1)) { A[row * n + row] = 1.0; return; }
  int ia[3] = {(int)(node % g.nn[0]), (int)((node / g.nn[0]) % g.nn[1]),
               DIM == 3 ? (int)(node / ((long long)g.nn[0] * g.nn[1])) : 0};
  for (int nb = 0; nb < NB; ++nb) {
    int ib[3] = {ia[0] + nb % 3 - 1, ia[1] + (nb / 3) % 3 - 1, DIM == 3 ? ia[2] + nb / 9 - 1 : 0};
    bool inside = true;
    for (int k = 0; k < DIM; ++k)
      if (ib[k] < 0 || ib[k] > g.n[k]) inside = false;
    if (!inside) continue;
    long long bn = ib[0] + (long long)g.nn[0] * (ib[1] + (long long)g.nn[1] * ib[2]);
    unsigned char mb = mask[bn];
    const double* s = st + (long long)nb * SP * g.nnodes + node;
    for (int cb = 0; cb < ND; ++cb) {
      if (cb < DIM && ((mb >> cb) & 1)) continue;
      double v;
      if (ca < DIM && cb < DIM) v = ca == cb ? s[0] : 0.0;
      else if (ca < DIM) v = s[(1 + ca) * g.nnodes];
      else if (cb < DIM) v = s[(1 + DIM + cb) * g.nnodes];
      else v = s[(1 + 2 * DIM) * g.nnodes];
      A[row * n + bn * ND + cb] = v;
    }
  }
}

// Explicit inverse of the equilibrated coarsest operator by Gauss-Jordan
// elimination with partial pivoting (max |a|, lowest row on ties) on the
// pair [D A D | I], D = |diag A|^{-1/2}: after the n steps the right half is
// (D A D)^{-1}, and A^{-1} = D (D A D)^{-1} D.  Each step is one pivot
// launch (one CTA: pivot search, row swap, pivot row scaled, the column's
// factors saved) and one elimination launch over the whole GPU, so the
// O(n^3) work spreads over every SM.
__global__ void gj_scale_kernel(int n, const double* __restrict__ A, double* __restrict__ dsc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double v = fabs(A[(long long)j * n + j]);
  dsc[j] = v > 0.0 ? 1.0 / sqrt(v) : 1.0;
}

// A <- D A D, R <- I (a block per row)
__global__ void gj_init_kernel(int n, double* __restrict__ A, double* __restrict__ R, const double* __restrict__ dsc) {
  for (int rr = blockIdx.x; rr < n; rr += gridDim.x) {
    const double dr = dsc[rr];
    double* ar = A + (long long)rr * n;
    double* rw = R + (long long)rr * n;
    for (int cc = threadIdx.x; cc < n; cc += blockDim.x) {
      ar[cc] = dr * ar[cc] * dsc[cc];
      rw[cc] = rr == cc ? 1.0 : 0.0;
    }
  }
}

__global__ void __launch_bounds__(1024)
    gj_pivot_kernel(int n, int k, double* __restrict__ A, double* __restrict__ R, double* __restrict__ col,
                    int* __restrict__ piv, unsigned* __restrict__ d_err) {
  __shared__ double sval[32];
  __shared__ int sidx[32];
  __shared__ int s_p;
  __shared__ double s_d;
  const int tid = threadIdx.x, nt = blockDim.x;
  double best = -1.0;
  int bi = k;
  for (int rr = k + tid; rr < n; rr += nt) {
    const double v = fabs(A[(long long)rr * n + k]);
    if (v > best) { best = v; bi = rr; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_down_sync(0xffffffffu, best, o);
    const int oi = __shfl_down_sync(0xffffffffu, bi, o);
    if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
  }
  if ((tid & 31) == 0) { sval[tid >> 5] = best; sidx[tid >> 5] = bi; }
  __syncthreads();
  if (tid == 0) {
    const int nw = (nt + 31) / 32;
    double bv = sval[0];
    int bidx = sidx[0];
    for (int w = 1; w < nw; ++w)
      if (sval[w] > bv || (sval[w] == bv && sidx[w] < bidx)) { bv = sval[w]; bidx = sidx[w]; }
    s_p = bidx;
    piv[k] = bidx;
    if (bv == 0.0) atomicOr(d_err, kErrSingularCoarse);
  }
  __syncthreads();
  const int p = s_p;
  if (p != k) {
    for (int cc = k + tid; cc < n; cc += nt) {
      const double t0 = A[(long long)k * n + cc];
      A[(long long)k * n + cc] = A[(long long)p * n + cc];
      A[(long long)p * n + cc] = t0;
    }
    for (int cc = tid; cc < n; cc += nt) {
      const double t0 = R[(long long)k * n + cc];
      R[(long long)k * n + cc] = R[(long long)p * n + cc];
      R[(long long)p * n + cc] = t0;
    }
  }
  __syncthreads();
  if (tid == 0) s_d = A[(long long)k * n + k];
  __syncthreads();
  const double d = s_d;
  // the factors of column k (taken before the pivot row is scaled)
  for (int rr = tid; rr < n; rr += nt) col[rr] = rr == k ? 0.0 : A[(long long)rr * n + k];
  __syncthreads();
  if (d != 0.0) {
    for (int cc = k + 1 + tid; cc < n; cc += nt) A[(long long)k * n + cc] = A[(long long)k * n + cc] / d;
    for (int cc = tid; cc < n; cc += nt) R[(long long)k * n + cc] = R[(long long)k * n + cc] / d;
  }
  if (tid == 0) A[(long long)k * n + k] = 1.0;
}

// rows r != k: row_r -= col[r] * row_k on the columns still live (left part
// beyond k, all of the right part); a block per row, rows with a zero factor
// skip the step
__global__ void gj_eliminate_kernel(int n, int k, double* __restrict__ A, double* __restrict__ R,
                                    const double* __restrict__ col) {
  const double* ak = A + (long long)k * n;
  const double* rk = R + (long long)k * n;
  for (int rr = blockIdx.x; rr < n; rr += gridDim.x) {
    const double f = col[rr];
    if (rr == k || f == 0.0) continue;
    double* ar = A + (long long)rr * n;
    double* rw = R + (long long)rr * n;
    for (int cc = k + 1 + threadIdx.x; cc < n; cc += blockDim.x) ar[cc] -= f * ak[cc];
    for (int cc = threadIdx.x; cc < n; cc += blockDim.x) rw[cc] -= f * rk[cc];
  }
}

// inv = D R D (in place, a block per row)
__global__ void gj_finish_kernel(int n, double* __restrict__ R, const double* __restrict__ dsc) {
  for (int rr = blockIdx.x; rr < n; rr += gridDim.x) {
    const double dr = dsc[rr];
    double* rw = R + (long long)rr * n;
    for (int cc = threadIdx.x; cc < n; cc += blockDim.x) rw[cc] = dr * rw[cc] * dsc[cc];
  }
}

// y = A x, one warp per row
__global__ void gemv_kernel(int n, const double* __restrict__ A, const double* __restrict__ x,
                            double* __restrict__ y) {
  int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (row >= n) return;
  double s = 0.0;
  for (int c = lane; c < n; c += 32) s += A[(long long)row * n + c] * x[c];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) y[row] = s;
}

// ---------------------------------------------------------------------------
// deterministic reductions: a fixed grid of partial sums, then one block
constexpr int kRedBlocks = 1024;

__global__ void dot_partial_kernel(long long n, const double* __restrict__ a, const double* __restrict__ b,
                                   double* __restrict__ partial) {
  __shared__ double sm[32];
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += a[i] * b[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
  }
}

__global__ void sum_partial_kernel(int np, const double* __restrict__ partial, double* __restrict__ out) {
  __shared__ double sm[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += partial[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) out[0] = t;
  }
}

// Fused modified Gram-Schmidt step.  Every block first reduces, in one fixed
// order, the block partials of the previous dot product (so all blocks hold
// the same h), subtracts h v_prev from w, and accumulates its partial of the
// next dot product (w . v_next, or w . w for the norm).  Block 0 stores h.
// With finish != 0 the kernel instead takes the norm from the partials,
// stores it and writes v_next = w / norm.
__device__ __forceinline__ double reduce_partials(const double* __restrict__ partial, int np, double* sm) {
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += partial[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) sm[32] = t;
  }
  __syncthreads();
  t = sm[32];
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(256)
    mgs_fused_kernel(long long n, double* __restrict__ w, const double* __restrict__ v_prev,
                     const double* __restrict__ part_in, double* __restrict__ h_out,
                     const double* __restrict__ v_next, double* __restrict__ part_out, int finish,
                     double* __restrict__ v_out, double* __restrict__ hn_copy) {
  __shared__ double sm[33];
  double h = 0.0;
  if (part_in) {
    h = reduce_partials(part_in, gridDim.x, sm);
    if (finish) h = sqrt(h);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      *h_out = h;
      if (hn_copy) *hn_copy = h;
    }
  }
  if (finish) {
    const double f = h != 0.0 ? 1.0 / h : 0.0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
      v_out[t] = w[t] * f;
    return;
  }
  double acc = 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double wv = w[t];
    if (v_prev) {
      wv = wv - h * v_prev[t];
      w[t] = wv;
    }
    acc += wv * (v_next ? v_next[t] : wv);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t2 = threadIdx.x < (blockDim.x >> 5) ? sm[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t2 += __shfl_down_sync(0xffffffffu, t2, o);
    if (threadIdx.x == 0) part_out[blockIdx.x] = t2;
  }
}

__global__ void axpy_kernel(long long n, double alpha, const double* __restrict__ x, double* __restrict__ y) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = y[i] + alpha * x[i];
}

// y = x * s[sidx] (or / s[sidx] when invert), s a device scalar array
__global__ void scale_copy_kernel(long long n, const double* __restrict__ s, int sidx, int invert,
                                  const double* __restrict__ x, double* __restrict__ y) {
  double f = s[sidx];
  if (invert) f = f != 0.0 ? 1.0 / f : 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i] * f;
}

// w -= h * v with h a device scalar
__global__ void mgs_step_kernel(long long n, double* __restrict__ w, const double* __restrict__ v,
                                const double* __restrict__ h) {
  double hv = h[0];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    w[i] = w[i] - hv * v[i];
}

// Small FGMRES state (device, one thread):
//   H[(m+1) x m] row-major at small[0], cs[m], sn[m], g[m+1], y[m],
//   scalars at the end: [est, hn, beta, ...]
__global__ void givens_kernel(double* small, int m, int j, double bnorm) {
  double* H = small;
  double* cs = H + (m + 1) * m;
  double* sn = cs + m;
  double* g = sn + m;
  double* sc = g + (m + 1) + m;  // after y
  // H[j+1][j] was written from the norm scalar
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
  sc[0] = fabs(g[j + 1]) / bnorm;
}

// y = H^{-1} g (k x k upper triangular), then x += sum_i y_i Z_i
__global__ void solve_y_kernel(double* small, int m, int k) {
  double* H = small;
  double* cs = H + (m + 1) * m;
  double* sn = cs + m;
  double* g = sn + m;
  double* y = g + (m + 1);
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int t = i + 1; t < k; ++t) s = s - H[i * m + t] * y[t];
    y[i] = s / H[i * m + i];
  }
}

__global__ void update_x_kernel(long long n, int k, int m, const double* __restrict__ small,
                                const double* __restrict__ Z, double* __restrict__ x) {
  const double* y = small + (m + 1) * m + m + m + (m + 1);
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double s = x[t];
    for (int i = 0; i < k; ++i) s = s + y[i] * Z[(long long)i * n + t];
    x[t] = s;
  }
}

__global__ void zero_kernel(double* p, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) p[i] = 0.0;
}

inline unsigned grid_for(long long n, int bs) {
  long long b = (n + bs - 1) / bs;
  if (b > 152LL * 16) b = 152LL * 16;
  if (b < 1) b = 1;
  return (unsigned)b;
}

}  // namespace

cudaError_t launch_residual(const LevelGeom& g, const double* st, const unsigned char* mask,
                            const double* x, const double* b, double* r, double* rpad,
                            cudaStream_t s) {
  unsigned blocks = (unsigned)((g.nnodes + 255) / 256);
  if (g.dim == 2) residual_kernel<2, 0><<<blocks, 256, 0, s>>>(g, st, mask, x, b, r, rpad, nullptr);
  else residual_kernel<3, 0><<<blocks, 256, 0, s>>>(g, st, mask, x, b, r, rpad, nullptr);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_residual_df(const LevelGeom& g, const double* st, const unsigned char* mask,
                               const double* x, const double* b, float* rpad2, cudaStream_t s) {
  unsigned blocks = (unsigned)((g.nnodes + 255) / 256);
  if (g.dim == 2) residual_kernel<2, 1><<<blocks, 256, 0, s>>>(g, st, mask, x, b, nullptr, nullptr, rpad2);
  else residual_kernel<3, 1><<<blocks, 256, 0, s>>>(g, st, mask, x, b, nullptr, nullptr, rpad2);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_residual_f32(const LevelGeom& g, const double* st, const unsigned char* mask,
                                const double* x, const double* b, float* rpad, cudaStream_t s) {
  unsigned blocks = (unsigned)((g.nnodes + 255) / 256);
  if (g.dim == 2) residual_kernel<2, 2><<<blocks, 256, 0, s>>>(g, st, mask, x, b, nullptr, nullptr, rpad);
  else residual_kernel<3, 2><<<blocks, 256, 0, s>>>(g, st, mask, x, b, nullptr, nullptr, rpad);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_split_pairs(long long n, const double* in, float2* out, cudaStream_t s) {
  split_pairs_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, in, out);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_residual_df2(const LevelGeom& g, const float2* st2, const unsigned char* mask,
                                const float2* xp2, const float2* b2, float2* rpad2, double* r,
                                cudaStream_t s) {
  // lanes per node by level size (3D, GB300, ms per launch for 1 / 8 / 16
  // lanes): 64^3 nodes 0.087 / 0.131 / 0.170, 32^3 0.029 / 0.021 / 0.026,
  // 16^3 0.029 / 0.012 / 0.010.  One thread per node where the level fills
  // the GPU, a group where it leaves most SMs idle.
  const long long nn = g.nnodes;
  const int tpp = nn >= 152LL * 512 ? 1 : g.dim == 2 ? 8 : nn >= 152LL * 128 ? 8 : 16;
  const unsigned blocks = (unsigned)((nn * tpp + 255) / 256);
  if (g.dim == 2) {
    if (tpp == 1) residual_df2_kernel<2, 1><<<blocks, 256, 0, s>>>(g, st2, mask, xp2, b2, rpad2, r);
    else residual_df2_kernel<2, 8><<<blocks, 256, 0, s>>>(g, st2, mask, xp2, b2, rpad2, r);
  } else if (tpp == 1) {
    residual_df2_kernel<3, 1><<<blocks, 256, 0, s>>>(g, st2, mask, xp2, b2, rpad2, r);
  } else if (tpp == 8) {
    residual_df2_kernel<3, 8><<<blocks, 256, 0, s>>>(g, st2, mask, xp2, b2, rpad2, r);
  } else {
    residual_df2_kernel<3, 16><<<blocks, 256, 0, s>>>(g, st2, mask, xp2, b2, rpad2, r);
  }
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_fold_stencil_pairs(const LevelGeom& g, const double* st, const unsigned char* mask,
                                      float2* st2, cudaStream_t s) {
  long long n = g.nnodes * (g.dim == 3 ? 14 : 5);  // own (half) offsets
  unsigned blocks = (unsigned)((n + 255) / 256);
  if (g.dim == 2) fold_stencil_pairs_kernel<2><<<blocks, 256, 0, s>>>(g, st, mask, st2);
  else fold_stencil_pairs_kernel<3><<<blocks, 256, 0, s>>>(g, st, mask, st2);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_fold_stencil_f32(const LevelGeom& g, const double* st, const unsigned char* mask, float* st32,
                                    cudaStream_t s) {
  long long n = g.nnodes * (g.dim == 3 ? 14 : 5);  // own (half) offsets
  unsigned blocks = (unsigned)((n + 255) / 256);
  if (g.dim == 2) fold_stencil_f32_kernel<2><<<blocks, 256, 0, s>>>(g, st, mask, st32);
  else fold_stencil_f32_kernel<3><<<blocks, 256, 0, s>>>(g, st, mask, st32);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_split_x_padded(const LevelGeom& g, const double* x, float2* xp2, cudaStream_t s) {
  unsigned blocks = (unsigned)((g.nnodes + 255) / 256);
  if (g.dim == 2) split_x_padded_kernel<2><<<blocks, 256, 0, s>>>(g, x, xp2);
  else split_x_padded_kernel<3><<<blocks, 256, 0, s>>>(g, x, xp2);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_merge_x_padded(const LevelGeom& g, const float2* xp2, double* x, cudaStream_t s) {
  unsigned blocks = (unsigned)((g.nnodes + 255) / 256);
  if (g.dim == 2) merge_x_padded_kernel<2><<<blocks, 256, 0, s>>>(g, xp2, x);
  else merge_x_padded_kernel<3><<<blocks, 256, 0, s>>>(g, xp2, x);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_restrict(const LevelGeom& f, const LevelGeom& c, const unsigned char* cmask,
                            const double* rf, double* bc, cudaStream_t s) {
  unsigned blocks = (unsigned)((c.nnodes + 255) / 256);
  if (f.dim == 2) restrict_kernel<2><<<blocks, 256, 0, s>>>(f, c, cmask, rf, bc);
  else restrict_kernel<3><<<blocks, 256, 0, s>>>(f, c, cmask, rf, bc);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_prolong_add(const LevelGeom& f, const LevelGeom& c, const unsigned char* fmask,
                               const double* ec, double* xf, cudaStream_t s) {
  unsigned blocks = (unsigned)((f.nnodes + 255) / 256);
  if (f.dim == 2) prolong_kernel<2><<<blocks, 256, 0, s>>>(f, c, fmask, ec, xf);
  else prolong_kernel<3><<<blocks, 256, 0, s>>>(f, c, fmask, ec, xf);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_zero_pad_halo(double* p, long long n, cudaStream_t s) {
  zero_kernel<<<grid_for(n, 256), 256, 0, s>>>(p, n);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_coarse_factor(const LevelGeom& g, const double* st, const unsigned char* mask,
                                 double* work, double* inv, int* piv, double* dsc, unsigned* d_err,
                                 cudaStream_t s) {
  unsigned blocks = (unsigned)((g.ndof + 127) / 128);
  if (g.dim == 2) coarse_dense_kernel<2><<<blocks, 128, 0, s>>>(g, st, mask, work);
  else coarse_dense_kernel<3><<<blocks, 128, 0, s>>>(g, st, mask, work);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  note_launches(1);
  return launch_dense_inverse((int)g.ndof, work, inv, piv, dsc, d_err, s);
}

cudaError_t launch_dense_inverse(int n, double* work, double* inv, int* piv, double* dsc, unsigned* d_err,
                                 cudaStream_t s) {
  // dsc holds 2 n doubles: the scaling, then the factors of the current column
  double* col = dsc + n;
  const unsigned gb = (unsigned)std::min(n, 152 * 16);
  gj_scale_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, work, dsc);
  gj_init_kernel<<<gb, 256, 0, s>>>(n, work, inv, dsc);
  for (int k = 0; k < n; ++k) {
    gj_pivot_kernel<<<1, 1024, 0, s>>>(n, k, work, inv, col, piv, d_err);
    gj_eliminate_kernel<<<gb, 256, 0, s>>>(n, k, work, inv, col);
  }
  gj_finish_kernel<<<gb, 256, 0, s>>>(n, inv, dsc);
  note_launches(3 + 2 * n);
  return cudaGetLastError();
}

cudaError_t launch_dense_gemv(int n, const double* A, const double* x, double* y, cudaStream_t s) {
  long long threads = (long long)n * 32;
  gemv_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(n, A, x, y);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_dot(long long n, const double* a, const double* b, double* partial, double* out,
                       cudaStream_t s) {
  dot_partial_kernel<<<kRedBlocks, 256, 0, s>>>(n, a, b, partial);
  sum_partial_kernel<<<1, 1024, 0, s>>>(kRedBlocks, partial, out);
  note_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_mgs_fused(long long n, double* w, const double* v_prev, const double* part_in,
                             double* h_out, const double* v_next, double* part_out, int finish,
                             double* v_out, double* hn_copy, cudaStream_t s) {
  mgs_fused_kernel<<<kRedBlocks, 256, 0, s>>>(n, w, v_prev, part_in, h_out, v_next, part_out, finish, v_out,
                                              hn_copy);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_axpy(long long n, double alpha, const double* x, double* y, cudaStream_t s) {
  axpy_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, alpha, x, y);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_scale_copy(long long n, const double* sc, int sidx, int invert, const double* x,
                              double* y, cudaStream_t s) {
  scale_copy_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, sc, sidx, invert, x, y);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_mgs_step(long long n, double* w, const double* vi, const double* hij, cudaStream_t s) {
  mgs_step_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, w, vi, hij);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_givens(double* small, int m, int j, double bnorm, cudaStream_t s) {
  givens_kernel<<<1, 1, 0, s>>>(small, m, j, bnorm);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_update_x(long long n, int k, int m, const double* small, const double* Z, double* x,
                            cudaStream_t s) {
  solve_y_kernel<<<1, 1, 0, s>>>(const_cast<double*>(small), m, k);
  update_x_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, k, m, small, Z, x);
  note_launches(2);
  return cudaGetLastError();
}

}  // namespace fc
