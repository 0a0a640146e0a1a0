// fc_batch.cu -- many independent finite cell problems smoothed, cycled and
// solved together on one GPU.
//
// A batch groups handles set up one by one (fc_setup: each keeps its own
// operator, patch cache and coarse inverse) and runs their work as one set
// of launches: every (problem, level) pair is a segment, every segment is
// cut into chunks of 256 nodes, and each batched kernel is a persistent grid
// that walks the chunk list of one phase (all problems' levels at the same
// depth from the coarsest grid) -- patches of uneven problems share a launch
// instead of one launch per problem and level.  The smoother is the paper's
// restricted additive sweep (Sec. 3.1: residual, local solves with the
// cached owned rows of L_i^{-1}, restricted update), the V-cycle is Sec. 3's
// with the coarse direct solve, and the outer FGMRES (Sec. 4 remark on
// Krylov methods) runs per problem with its own Krylov basis, Hessenberg
// matrix, Givens rotations and stopping test, each problem's vector work on
// one thread-block cluster.
//
// The patch-apply tile (lanes per patch, threads per CTA, CTAs per SM) is
// picked at creation by timing every candidate on the batch's own finest
// levels; the pick changes rounding order only.  Each Arnoldi step (pointer
// update, V-cycle, operator application, Gram-Schmidt, Givens) of the solve
// is one CUDA graph, captured once and replayed.  Problems are coupled by
// nothing but the launches: a problem's arithmetic, and hence its result,
// does not depend on the other members of the batch.
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <unordered_set>
#include <vector>

#include "fc_internal.cuh"

namespace cg = cooperative_groups;

namespace fc {
namespace {

constexpr int kChunk = kChunkNodes;   // nodes per chunk
constexpr int kCL = 8;        // CTAs per cluster in the Krylov kernels
constexpr int kKThreads = 256;

struct BGeom {
  int n[3], nn[3];
  long long nnodes;
};

// one (problem, level) pair
struct BSeg {
  BGeom g;
  int prob, li;
  double omega;
  const double* st;
  const unsigned char* mask;
  const void* coef;
  const int* prow;
  double* x;           // level correction (finest level: set per call)
  double* b;           // right-hand side (finest level: the caller's, read only)
  double* r;           // unpadded float64 residual
  double* rpad;        // padded float64 residual (float64 rows)
  float* rpadf;        // padded float32 residual (float32 / bfloat16 rows)
  const double* cinv;  // coarse inverse (level 0)
  int cn;
  // float32 correction form (float32 / bfloat16 rows): folded float32 half
  // stencil, padded correction d and right-hand side b32 of the level
  const float* st32;
  float* d32;
  float* b32;
  float omega_f;
  // tensor-core apply of the shared class blocks: the stored blocks of the
  // classes 1 and 2 (-1: none) and their rows as the MMA tile (see
  // f_apply_tc_kernel; null when the batch does not use tensor cores)
  int cls[2];
  const void* tcA;
};

struct Chunk {
  int seg, node0;
};

__device__ __forceinline__ void decode(const BGeom& g, int dim, unsigned u, int* ia) {
  const unsigned nx = (unsigned)g.nn[0], ny = (unsigned)g.nn[1];
  const unsigned t = u / nx;
  ia[0] = (int)(u - t * nx);
  if (dim == 3) {
    ia[1] = (int)(t % ny);
    ia[2] = (int)(t / ny);
  } else {
    ia[1] = (int)t;
    ia[2] = 0;
  }
}

__device__ __forceinline__ long long padded(const BGeom& g, int dim, const int* ia) {
  const long long px = g.nn[0] + 4, py = g.nn[1] + 4;
  const int kk = dim == 3 ? ia[2] + 2 : 0;
  return ((long long)kk * py + (ia[1] + 2)) * px + (ia[0] + 2);
}

// ---------------------------------------------------------------------------
// operator application on the chunks of one phase.
// OUT 0: r (unpadded float64), 1: rpad (padded float64), 2: rpadf (padded
// float32).  use_b = 0 gives L x instead of b - L x.  With a state array
// only problems whose state equals `gate` are processed.
// v = b - L x (or L x when b is null) at one node, float64
template <int DIM>
__device__ __forceinline__ void residual64(const BSeg* S, const BGeom& g, long long node, const int* ia,
                                           const double* b, double* v) {
  constexpr int NB = DIM == 3 ? 27 : 9, SP = 2 * DIM + 2, ND = DIM + 1;
  const double* __restrict__ st = S->st;
  const unsigned char* __restrict__ mask = S->mask;
  const double* x = S->x;
  double acc[ND];
#pragma unroll
  for (int q = 0; q < ND; ++q) acc[q] = 0.0;
#pragma unroll
  for (int nb = 0; nb < NB; ++nb) {
    const int ib0 = ia[0] + nb % 3 - 1, ib1 = ia[1] + (nb / 3) % 3 - 1, ib2 = DIM == 3 ? ia[2] + nb / 9 - 1 : 0;
    if (ib0 < 0 || ib0 > g.n[0] || ib1 < 0 || ib1 > g.n[1]) continue;
    if (DIM == 3 && (ib2 < 0 || ib2 > g.n[2])) continue;
    const long long bn = ib0 + (long long)g.nn[0] * (ib1 + (long long)g.nn[1] * ib2);
    const unsigned char mb = mask[bn];
    double xb[ND];
#pragma unroll
    for (int q = 0; q < ND; ++q) xb[q] = x[bn * ND + q];
#pragma unroll
    for (int q = 0; q < DIM; ++q)
      if ((mb >> q) & 1) xb[q] = 0.0;
    const double* s = st + (long long)nb * SP * g.nnodes + node;
    const double vA = s[0];
#pragma unroll
    for (int q = 0; q < DIM; ++q) {
      acc[q] = acc[q] + vA * xb[q];
      acc[q] = acc[q] + s[(1 + q) * g.nnodes] * xb[DIM];
    }
#pragma unroll
    for (int q = 0; q < DIM; ++q) acc[DIM] = acc[DIM] + s[(1 + DIM + q) * g.nnodes] * xb[q];
    acc[DIM] = acc[DIM] + s[(1 + 2 * DIM) * g.nnodes] * xb[DIM];
  }
  const unsigned char ma = mask[node];
#pragma unroll
  for (int q = 0; q < ND; ++q) {
    const double y = (q < DIM && ((ma >> q) & 1)) ? x[node * ND + q] : acc[q];
    v[q] = b ? b[node * ND + q] - y : y;
  }
}

template <int DIM, int OUT>
__global__ void __launch_bounds__(256)
    b_residual_kernel(const BSeg* __restrict__ segs, const Chunk* __restrict__ ch, int nch, int use_b,
                      const int* __restrict__ state, int gate) {
  constexpr int ND = DIM + 1;
  for (int c = blockIdx.x; c < nch; c += gridDim.x) {
    const Chunk k = ch[c];
    const BSeg* S = segs + k.seg;
    if (state && state[S->prob] != gate) continue;
    const BGeom g = S->g;
    const long long node = (long long)k.node0 + threadIdx.x;
    if (node >= g.nnodes) continue;
    int ia[3];
    decode(g, DIM, (unsigned)node, ia);
    double v[ND];
    residual64<DIM>(S, g, node, ia, use_b ? S->b : nullptr, v);
    const long long pn = padded(g, DIM, ia);
#pragma unroll
    for (int q = 0; q < ND; ++q) {
      if (OUT == 0) S->r[node * ND + q] = v[q];
      else if (OUT == 1) S->rpad[pn * ND + q] = v[q];
      else S->rpadf[pn * ND + q] = (float)v[q];
    }
  }
}

// ---------------------------------------------------------------------------
// restricted additive patch apply (Sec. 3.1.2, cache_inverse): a group of
// TPP lanes takes one patch, gathers the padded residual through the slot
// table, multiplies by the (d+1) owned rows and updates the owned DoFs.
// PT 0: float64 rows/residual/sums; 1: float32; 2: bfloat16 rows with
// float32 residual and sums.
template <typename V>
__device__ __forceinline__ V ldr(const V* p, bool cached) {
  return cached ? __ldg(p) : __ldcs(p);
}

template <int PT, int ND>
struct RowLoad;
template <int ND>
struct RowLoad<0, ND> {
  using T = double;
  using A = double;
  static __device__ __forceinline__ void load(const double* p, bool c, double* v) {
    if (ND == 4) {
      const double2* q = reinterpret_cast<const double2*>(p);
      const double2 a = ldr(q, c), b = ldr(q + 1, c);
      v[0] = a.x; v[1] = a.y; v[2] = b.x; v[ND - 1] = b.y;
    } else {
#pragma unroll
      for (int k = 0; k < ND; ++k) v[k] = ldr(p + k, c);
    }
  }
};
template <int ND>
struct RowLoad<1, ND> {
  using T = float;
  using A = float;
  static __device__ __forceinline__ void load(const float* p, bool c, float* v) {
    if (ND == 4) {
      const float4 a = ldr(reinterpret_cast<const float4*>(p), c);
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[ND - 1] = a.w;
    } else {
#pragma unroll
      for (int k = 0; k < ND; ++k) v[k] = ldr(p + k, c);
    }
  }
};
template <int ND>
struct RowLoad<2, ND> {
  using T = __nv_bfloat16;
  using A = float;
  static __device__ __forceinline__ void load(const __nv_bfloat16* p, bool c, float* v) {
    if (ND == 4) {
      const uint2 a = ldr(reinterpret_cast<const uint2*>(p), c);
      v[0] = __uint_as_float(a.x << 16); v[1] = __uint_as_float(a.x & 0xffff0000u);
      v[2] = __uint_as_float(a.y << 16); v[ND - 1] = __uint_as_float(a.y & 0xffff0000u);
    } else {
      const unsigned short* q = reinterpret_cast<const unsigned short*>(p);
#pragma unroll
      for (int k = 0; k < ND; ++k) v[k] = __uint_as_float((unsigned)ldr(q + k, c) << 16);
    }
  }
};

// slot j of a patch -> offset (in values) of its DoF in the padded vector:
// velocity slots (5^d nodes, component inner) first, then the 3^d pressures
template <int DIM>
__device__ __forceinline__ int slot_offset(int j, int px, int py) {
  constexpr int NU = DIM == 3 ? 125 : 25, ND = DIM + 1;
  int o0, o1, o2, c;
  if (j < NU * DIM) {
    const int v = j / DIM;
    c = j - v * DIM;
    o0 = v % 5 - 2;
    o1 = (v / 5) % 5 - 2;
    o2 = DIM == 3 ? v / 25 - 2 : 0;
  } else {
    const int p = j - NU * DIM;
    c = DIM;
    o0 = p % 3 - 1;
    o1 = (p / 3) % 3 - 1;
    o2 = DIM == 3 ? p / 9 - 1 : 0;
  }
  return (o0 + px * (o1 + py * o2)) * ND + c;
}

template <int DIM, int PT, int TPP>
__global__ void __launch_bounds__(512)
    b_apply_kernel(const BSeg* __restrict__ segs, const Chunk* __restrict__ ch, int nch,
                   const int* __restrict__ state, int gate) {
  constexpr int ND = DIM + 1, NSLOT = DIM == 3 ? 402 : 59;
  using RL = RowLoad<PT, ND>;
  using T = typename RL::T;
  using A = typename RL::A;
  __shared__ int soff[NSLOT];
  int cur_px = -1, cur_py = -1;
  const int lane = threadIdx.x % TPP, grp = threadIdx.x / TPP, ngrp = blockDim.x / TPP;
  for (int c = blockIdx.x; c < nch; c += gridDim.x) {
    const Chunk k = ch[c];
    const BSeg* S = segs + k.seg;
    if (state && state[S->prob] != gate) continue;  // uniform over the CTA
    const BGeom g = S->g;
    const int px = g.nn[0] + 4, py = g.nn[1] + 4;
    if (px != cur_px || py != cur_py) {
      __syncthreads();
      for (int j = threadIdx.x; j < NSLOT; j += blockDim.x) soff[j] = slot_offset<DIM>(j, px, py);
      __syncthreads();
      cur_px = px;
      cur_py = py;
    }
    const T* __restrict__ coef = static_cast<const T*>(S->coef);
    const int* __restrict__ prow = S->prow;
    const unsigned char* __restrict__ mask = S->mask;
    const A* __restrict__ rpad = PT == 0 ? reinterpret_cast<const A*>(S->rpad) : reinterpret_cast<const A*>(S->rpadf);
    double* x = S->x;
    const double omega = S->omega;
    // every group of a warp runs the same number of passes (blockDim is a
    // multiple of TPP and kChunk of the group count), so the shuffles below
    // always see full warps
    for (int q = grp; q < kChunk; q += ngrp) {
      const long long node = (long long)k.node0 + q;
      const bool valid = node < g.nnodes;
      const unsigned i = (unsigned)(valid ? node : g.nnodes - 1);
      int ia[3];
      decode(g, DIM, i, ia);
      const A* rp = rpad + padded(g, DIM, ia) * ND;
      const int pr = prow ? prow[i] : (int)i;
      const bool shared_rows = pr < 0;
      const T* cf = coef + (size_t)(shared_rows ? -pr - 1 : pr) * NSLOT * ND;
      A y[ND];
#pragma unroll
      for (int t = 0; t < ND; ++t) y[t] = A(0);
#pragma unroll 4
      for (int j = lane; j < NSLOT; j += TPP) {
        const A rv = rp[soff[j]];
        A cv[ND];
        RL::load(cf + (size_t)j * ND, shared_rows, cv);
#pragma unroll
        for (int t = 0; t < ND; ++t) y[t] = fma(cv[t], rv, y[t]);
      }
#pragma unroll
      for (int t = 0; t < ND; ++t)
#pragma unroll
        for (int o = TPP / 2; o > 0; o >>= 1) y[t] += __shfl_xor_sync(0xffffffffu, y[t], o);
      if (valid) {
        const unsigned char mi = mask[i];
        // lane t of the group updates component t (all of them when TPP = 1)
#pragma unroll
        for (int t0 = 0; t0 < ND; t0 += TPP) {
          const int t = t0 + lane;
          if (t >= ND) break;
          A yl = y[0];
#pragma unroll
          for (int u = 1; u < ND; ++u)
            if (t == u) yl = y[u];
          const size_t xi = (size_t)i * ND + t;
          const bool fixed = t < DIM && ((mi >> t) & 1);
          x[xi] = x[xi] + (fixed ? (double)rp[t] : omega * (double)yl);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// transfers (Sec. 3, Q1 full weighting R = P^T and Q1 interpolation P)
__device__ __forceinline__ double pw(int d) { return d == 0 ? 1.0 : 0.5; }

// b_c <- R r_f and x_c <- 0 on the chunks of coarse segments; the fine
// segment of a problem follows its coarse one in the table
template <int DIM>
__global__ void __launch_bounds__(256)
    b_restrict_kernel(const BSeg* __restrict__ segs, const Chunk* __restrict__ ch, int nch,
                      const int* __restrict__ state, int gate) {
  constexpr int ND = DIM + 1;
  for (int c = blockIdx.x; c < nch; c += gridDim.x) {
    const Chunk k = ch[c];
    const BSeg* C = segs + k.seg;
    const BSeg* F = C + 1;
    if (state && state[C->prob] != gate) continue;
    const BGeom cg_ = C->g, fg = F->g;
    const long long node = (long long)k.node0 + threadIdx.x;
    if (node >= cg_.nnodes) continue;
    int I[3];
    decode(cg_, DIM, (unsigned)node, I);
    const double* rf = F->r;
    double acc[ND];
#pragma unroll
    for (int q = 0; q < ND; ++q) acc[q] = 0.0;
    for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int i = 2 * I[0] + dx, j = 2 * I[1] + dy, kk = DIM == 3 ? 2 * I[2] + dz : 0;
          if (i < 0 || i > fg.n[0] || j < 0 || j > fg.n[1]) continue;
          if (DIM == 3 && (kk < 0 || kk > fg.n[2])) continue;
          const double w = pw(dx) * pw(dy) * (DIM == 3 ? pw(dz) : 1.0);
          const long long fn = i + (long long)fg.nn[0] * (j + (long long)fg.nn[1] * kk);
#pragma unroll
          for (int q = 0; q < ND; ++q) acc[q] = acc[q] + w * rf[fn * ND + q];
        }
    const unsigned char m = C->mask[node];
#pragma unroll
    for (int q = 0; q < ND; ++q) {
      C->b[node * ND + q] = (q < DIM && ((m >> q) & 1)) ? 0.0 : acc[q];
      C->x[node * ND + q] = 0.0;
    }
  }
}

// x_f += P x_c on the chunks of fine segments
template <int DIM>
__global__ void __launch_bounds__(256)
    b_prolong_kernel(const BSeg* __restrict__ segs, const Chunk* __restrict__ ch, int nch,
                     const int* __restrict__ state, int gate) {
  constexpr int ND = DIM + 1;
  for (int c = blockIdx.x; c < nch; c += gridDim.x) {
    const Chunk k = ch[c];
    const BSeg* F = segs + k.seg;
    const BSeg* C = F - 1;
    if (state && state[F->prob] != gate) continue;
    const BGeom fg = F->g, cg_ = C->g;
    const long long node = (long long)k.node0 + threadIdx.x;
    if (node >= fg.nnodes) continue;
    int ia[3];
    decode(fg, DIM, (unsigned)node, ia);
    int lo[3], hi[3];
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      lo[t] = ia[t] / 2;
      hi[t] = (ia[t] + 1) / 2;
    }
    const double* ec = C->x;
    double acc[ND];
#pragma unroll
    for (int q = 0; q < ND; ++q) acc[q] = 0.0;
    for (int t = 0; t < (1 << DIM); ++t) {
      int ic[3] = {0, 0, 0};
      double w = 1.0;
      bool dup = false;
      for (int d = 0; d < DIM; ++d) {
        const int bit = (t >> d) & 1;
        if (lo[d] == hi[d] && bit) dup = true;
        ic[d] = bit ? hi[d] : lo[d];
        w = w * (lo[d] == hi[d] ? 1.0 : 0.5);
      }
      if (dup) continue;
      const long long cn = ic[0] + (long long)cg_.nn[0] * (ic[1] + (long long)cg_.nn[1] * ic[2]);
#pragma unroll
      for (int q = 0; q < ND; ++q) acc[q] = acc[q] + w * ec[cn * ND + q];
    }
    const unsigned char m = F->mask[node];
    double* xf = F->x;
#pragma unroll
    for (int q = 0; q < ND; ++q)
      if (!(q < DIM && ((m >> q) & 1))) xf[node * ND + q] = xf[node * ND + q] + acc[q];
  }
}

// x <- A^{-1} b on each problem's coarsest level (one CTA per problem, one
// warp per row of the dense inverse)
__global__ void __launch_bounds__(256)
    b_coarse_kernel(const BSeg* __restrict__ segs, const int* __restrict__ cseg, const int* __restrict__ state,
                    int gate) {
  const BSeg* S = segs + cseg[blockIdx.x];
  if (state && state[S->prob] != gate) return;
  const int n = S->cn, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double* A = S->cinv;
  const double* b = S->b;
  double* x = S->x;
  for (int row = warp; row < n; row += nw) {
    double s = 0.0;
    for (int c = lane; c < n; c += 32) s += A[(long long)row * n + c] * b[c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) x[row] = s;
  }
}

// x <- 0 on the chunks (finest levels before a V-cycle from a zero guess)
template <int ND>
__global__ void __launch_bounds__(256)
    b_zero_kernel(const BSeg* __restrict__ segs, const Chunk* __restrict__ ch, int nch,
                  const int* __restrict__ state, int gate) {
  for (int c = blockIdx.x; c < nch; c += gridDim.x) {
    const Chunk k = ch[c];
    const BSeg* S = segs + k.seg;
    if (state && state[S->prob] != gate) continue;
    const long long node = (long long)k.node0 + threadIdx.x;
    if (node >= S->g.nnodes) continue;
#pragma unroll
    for (int q = 0; q < ND; ++q) S->x[node * ND + q] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// Float32 correction form (float32 / bfloat16 rows).  A V-cycle or a
// smoothing phase on (x, b) runs on the correction d with d = 0 at the start
// and right-hand side b32 = b - L x (float64 residual, skipped when x is
// known to be zero), entirely in float32: residual r = b32 - L32 d with the
// float32 half stencil (constrained columns folded to zero), patch
// solves d += omega L_i^{-1} r on the owned DoFs, transfers and prolongation
// on d; the coarse solve reads b32 and sums in float64.  At the end x += d
// in float64.  In exact arithmetic this is the same iteration as on x.

// b32 = b - L x (float64) or b, d = 0, on the finest levels
template <int DIM>
__global__ void __launch_bounds__(256)
    f_enter_kernel(const BSeg* __restrict__ segs, const Chunk* __restrict__ ch, int nch, int xzero,
                   const int* __restrict__ state, int gate) {
  constexpr int ND = DIM + 1;
  for (int c = blockIdx.x; c < nch; c += gridDim.x) {
    const Chunk k = ch[c];
    const BSeg* S = segs + k.seg;
    if (state && state[S->prob] != gate) continue;
    const BGeom g = S->g;
    const long long node = (long long)k.node0 + threadIdx.x;
    if (node >= g.nnodes) continue;
    int ia[3];
    decode(g, DIM, (unsigned)node, ia);
    double v[ND];
    if (xzero) {
#pragma unroll
      for (int q = 0; q < ND; ++q) v[q] = S->b[node * ND + q];
    } else {
      residual64<DIM>(S, g, node, ia, S->b, v);
    }
    const long long pn = padded(g, DIM, ia);
#pragma unroll
    for (int q = 0; q < ND; ++q) {
      S->b32[node * ND + q] = (float)v[q];
      S->d32[pn * ND + q] = 0.0f;
    }
  }
}

// x = x + d (or x = d when x was zero), float64, on the finest levels
template <int DIM>
__global__ void __launch_bounds__(256)
    f_exit_kernel(const BSeg* __restrict__ segs, const Chunk* __restrict__ ch, int nch, int xzero,
                  const int* __restrict__ state, int gate) {
  constexpr int ND = DIM + 1;
  for (int c = blockIdx.x; c < nch; c += gridDim.x) {
    const Chunk k = ch[c];
    const BSeg* S = segs + k.seg;
    if (state && state[S->prob] != gate) continue;
    const BGeom g = S->g;
    const long long node = (long long)k.node0 + threadIdx.x;
    if (node >= g.nnodes) continue;
    int ia[3];
    decode(g, DIM, (unsigned)node, ia);
    const long long pn = padded(g, DIM, ia);
    double* x = S->x;
#pragma unroll
    for (int q = 0; q < ND; ++q) {
      const double dv = (double)S->d32[pn * ND + q];
      x[node * ND + q] = xzero ? dv : x[node * ND + q] + dv;
    }
  }
}

// r = b32 - L32 d into the padded float32 residual
template <int DIM>
__global__ void __launch_bounds__(256)
    f_residual_kernel(const BSeg* __restrict__ segs, const Chunk* __restrict__ ch, int nch,
                      const int* __restrict__ state, int gate) {
  // half stencil: the zero offset and the offsets after it are the node's
  // own entries; a mirrored offset -d takes the transposed entries of the
  // neighbour b = a - d (A(a,b) = A(b,a), B_c(a,b) = T_c(b,a),
  // T_c(a,b) = B_c(b,a), C(a,b) = C(b,a))
  constexpr int CEN = DIM == 3 ? 13 : 4, NH = (DIM == 3 ? 27 : 9) - CEN, SP = 2 * DIM + 2, ND = DIM + 1;
  for (int c = blockIdx.x; c < nch; c += gridDim.x) {
    const Chunk k = ch[c];
    const BSeg* S = segs + k.seg;
    if (state && state[S->prob] != gate) continue;
    const BGeom g = S->g;
    const long long node = (long long)k.node0 + threadIdx.x;
    if (node >= g.nnodes) continue;
    int ia[3];
    decode(g, DIM, (unsigned)node, ia);
    const int px = g.nn[0] + 4, py = g.nn[1] + 4;
    const long long pn = padded(g, DIM, ia);
    const float* __restrict__ d = S->d32;
    const float* __restrict__ st = S->st32;
    float acc[ND];
#pragma unroll
    for (int q = 0; q < ND; ++q) acc[q] = 0.0f;
#pragma unroll
    for (int h = 0; h < NH; ++h) {
      const int nb = CEN + h;
      const int d0 = nb % 3 - 1, d1 = (nb / 3) % 3 - 1, d2 = DIM == 3 ? nb / 9 - 1 : 0;
      const int off = d0 + px * (d1 + (DIM == 3 ? py * d2 : 0));
      {
        const float* db = d + (pn + off) * ND;
        const float* sp = st + (long long)h * SP * g.nnodes + node;
        float dv[ND];
#pragma unroll
        for (int q = 0; q < ND; ++q) dv[q] = db[q];
        const float vA = __ldcs(sp);
#pragma unroll
        for (int q = 0; q < DIM; ++q) {
          acc[q] = fmaf(vA, dv[q], acc[q]);
          acc[q] = fmaf(__ldcs(sp + (1 + q) * g.nnodes), dv[DIM], acc[q]);
        }
#pragma unroll
        for (int q = 0; q < DIM; ++q) acc[DIM] = fmaf(__ldcs(sp + (1 + DIM + q) * g.nnodes), dv[q], acc[DIM]);
        acc[DIM] = fmaf(__ldcs(sp + (1 + 2 * DIM) * g.nnodes), dv[DIM], acc[DIM]);
      }
      if (h > 0) {
        const int b0 = ia[0] - d0, b1 = ia[1] - d1, b2 = ia[2] - d2;
        const bool in = b0 >= 0 && b0 <= g.n[0] && b1 >= 0 && b1 <= g.n[1] && (DIM == 2 || (b2 >= 0 && b2 <= g.n[2]));
        if (in) {
          const long long bnode = node - (d0 + (long long)g.nn[0] * (d1 + (long long)g.nn[1] * d2));
          const float* db = d + (pn - off) * ND;
          const float* sm = st + (long long)h * SP * g.nnodes + bnode;
          float dv[ND];
#pragma unroll
          for (int q = 0; q < ND; ++q) dv[q] = db[q];
          const float vA = sm[0];
#pragma unroll
          for (int q = 0; q < DIM; ++q) {
            acc[q] = fmaf(vA, dv[q], acc[q]);
            acc[q] = fmaf(sm[(1 + DIM + q) * g.nnodes], dv[DIM], acc[q]);
          }
#pragma unroll
          for (int q = 0; q < DIM; ++q) acc[DIM] = fmaf(sm[(1 + q) * g.nnodes], dv[q], acc[DIM]);
          acc[DIM] = fmaf(sm[(1 + 2 * DIM) * g.nnodes], dv[DIM], acc[DIM]);
        }
      }
    }
    const unsigned char ma = S->mask[node];
    const float* dc = d + pn * ND;
#pragma unroll
    for (int q = 0; q < ND; ++q) {
      const float y = (q < DIM && ((ma >> q) & 1)) ? dc[q] : acc[q];
      S->rpadf[pn * ND + q] = S->b32[node * ND + q] - y;
    }
  }
}

// d += omega L_i^{-1} r on the owned DoFs (PT 1: float32 rows, 2: bfloat16).
// The 2D loop is bound by the latency of its loads (rows from the cache for
// the shared class blocks, residual gathers): three 512-thread CTAs per SM
// (40 registers, a few per-chunk values in local memory) keep more loads in
// flight than the 64 registers the compiler picks unbounded (0.170 against
// 0.200 ms per launch on 256 uneven problems; capping the registers with a
// shallower unroll instead of spilling ran 0.32 ms).
template <int DIM, int PT, int TPP>
__global__ void __launch_bounds__(512, DIM == 2 ? 3 : 1)
    f_apply_kernel(const BSeg* __restrict__ segs, const Chunk* __restrict__ ch, int nch,
                   const int* __restrict__ state, int gate) {
  constexpr int ND = DIM + 1, NSLOT = DIM == 3 ? 402 : 59;
  using RL = RowLoad<PT, ND>;
  using T = typename RL::T;
  __shared__ int soff[NSLOT];
  int cur_px = -1, cur_py = -1;
  const int lane = threadIdx.x % TPP, grp = threadIdx.x / TPP, ngrp = blockDim.x / TPP;
  for (int c = blockIdx.x; c < nch; c += gridDim.x) {
    const Chunk k = ch[c];
    const BSeg* S = segs + k.seg;
    if (state && state[S->prob] != gate) continue;  // uniform over the CTA
    const BGeom g = S->g;
    const int px = g.nn[0] + 4, py = g.nn[1] + 4;
    if (px != cur_px || py != cur_py) {
      __syncthreads();
      for (int j = threadIdx.x; j < NSLOT; j += blockDim.x) soff[j] = slot_offset<DIM>(j, px, py);
      __syncthreads();
      cur_px = px;
      cur_py = py;
    }
    const T* __restrict__ coef = static_cast<const T*>(S->coef);
    const int* __restrict__ prow = S->prow;
    const unsigned char* __restrict__ mask = S->mask;
    const float* __restrict__ rpad = S->rpadf;
    float* d = S->d32;
    const float omega = S->omega_f;
    for (int q = grp; q < kChunk; q += ngrp) {
      const long long node = (long long)k.node0 + q;
      const bool valid = node < g.nnodes;
      const unsigned i = (unsigned)(valid ? node : g.nnodes - 1);
      int ia[3];
      decode(g, DIM, i, ia);
      const long long pb = padded(g, DIM, ia) * ND;
      const float* rp = rpad + pb;
      const int pr = prow ? prow[i] : (int)i;
      const bool shared_rows = pr < 0;
      const T* cf = coef + (size_t)(shared_rows ? -pr - 1 : pr) * NSLOT * ND;
      float y[ND];
#pragma unroll
      for (int t = 0; t < ND; ++t) y[t] = 0.0f;
#pragma unroll 4
      for (int j = lane; j < NSLOT; j += TPP) {
        const float rv = rp[soff[j]];
        float cv[ND];
        RL::load(cf + (size_t)j * ND, shared_rows, cv);
#pragma unroll
        for (int t = 0; t < ND; ++t) y[t] = fmaf(cv[t], rv, y[t]);
      }
#pragma unroll
      for (int t = 0; t < ND; ++t)
#pragma unroll
        for (int o = TPP / 2; o > 0; o >>= 1) y[t] += __shfl_xor_sync(0xffffffffu, y[t], o);
      if (valid) {
        const unsigned char mi = mask[i];
#pragma unroll
        for (int t0 = 0; t0 < ND; t0 += TPP) {
          const int t = t0 + lane;
          if (t >= ND) break;
          float yl = y[0];
#pragma unroll
          for (int u = 1; u < ND; ++u)
            if (t == u) yl = y[u];
          const bool fixed = t < DIM && ((mi >> t) & 1);
          d[pb + t] += fixed ? rp[t] : omega * yl;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Tensor-core apply of the shared class blocks (float32 correction form).
// Patches of a class (bit-identical L_i: uncut, one alpha, away from
// constraints) share one row block Inv_k ((d+1) x nslot), so their updates
// are one dense product (Sec. 3.1.2 cache_inverse, applied to many patches
// at once): the rows of both class blocks, stacked as rows 4k + c (class k,
// component c) of the M = 16 side of an m16n8 MMA tile (rows 8-15 zero),
// times the gathered residuals of 8 patches (N = 8, one column per patch)
// over K = the patch slots (zero rows past nslot).  A patch keeps the rows of
// its own class.  Cut patches (blocks of their own) take the CUDA cores with
// 8 lanes each.  A warp owns 32 consecutive nodes of a 256-node chunk.
//   MODE 1: rows and residual rounded to TF32, one m16n8k8 product per step;
//   MODE 2: both split into a TF32 head and a TF32 tail, three products
//           (head x head, head x tail, tail x head): float32-class accuracy;
//   MODE 3: rows and residual in BF16, one m16n8k16 product per step.
// FP32 accumulation in every mode.
template <int DIM>
struct TcDims {
  static constexpr int NSLOT = DIM == 3 ? 402 : 59;
  static constexpr int KP = DIM == 3 ? 416 : 64;   // slots padded to the MMA K steps
  // row strides of the staged tile (in elements): 32-bit rows at 4 mod 32
  // words, bf16 rows at 20 mod 32 words, so the 8 fragment rows fall on
  // distinct banks
  static constexpr int KS32 = KP + 4;
  static constexpr int KS16 = DIM == 3 ? 424 : 104;
};

template <int DIM, int MODE>
__host__ __device__ constexpr size_t tc_tile_bytes() {
  return MODE == 3 ? (size_t)8 * TcDims<DIM>::KS16 * 2 : (size_t)(MODE == 2 ? 2 : 1) * 8 * TcDims<DIM>::KS32 * 4;
}

__device__ __forceinline__ unsigned to_tf32(float v) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}

__device__ __forceinline__ void mma_tf32(float* d, unsigned a0, unsigned a2, unsigned b0, unsigned b1) {
  // rows 8-15 of the A tile are zero (a1 = a3 = 0)
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(0u), "r"(a2), "r"(0u), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_bf16(float* d, unsigned a0, unsigned a2, unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(0u), "r"(a2), "r"(0u), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const unsigned*>(&v);
}

// the staged tile of a segment: rows 4k + c of the class blocks, written
// once per batch from the stored rows (float32 or bfloat16) of the blocks
template <int DIM, int MODE, typename T>
__global__ void tc_prepare_kernel(const T* __restrict__ coef, int cls0, int cls1, void* out) {
  using D = TcDims<DIM>;
  constexpr int ND = DIM + 1;
  for (int t = threadIdx.x + blockIdx.x * blockDim.x; t < 8 * D::KP; t += blockDim.x * gridDim.x) {
    const int row = t / D::KP, j = t % D::KP, k = row >> 2, c = row & 3;
    const int blk = k == 0 ? cls0 : cls1;
    float v = 0.0f;
    if (blk >= 0 && c < ND && j < D::NSLOT) v = (float)coef[((size_t)blk * D::NSLOT + j) * ND + c];
    if (MODE == 3) {
      reinterpret_cast<__nv_bfloat16*>(out)[row * D::KS16 + j] = __float2bfloat16_rn(v);
    } else {
      const unsigned head = to_tf32(v);
      reinterpret_cast<unsigned*>(out)[row * D::KS32 + j] = head;
      if (MODE == 2) reinterpret_cast<unsigned*>(out)[8 * D::KS32 + row * D::KS32 + j] = to_tf32(v - __uint_as_float(head));
    }
  }
}

template <int DIM, int PT, int MODE>
__global__ void __launch_bounds__(256)
    f_apply_tc_kernel(const BSeg* __restrict__ segs, const Chunk* __restrict__ ch, int nch,
                      const int* __restrict__ state, int gate) {
  using D = TcDims<DIM>;
  constexpr int ND = DIM + 1, NSLOT = D::NSLOT, KP = D::KP;
  using RL = RowLoad<PT, ND>;
  using T = typename RL::T;
  extern __shared__ __align__(16) unsigned char tc_shm[];
  int* soff = reinterpret_cast<int*>(tc_shm);                 // KP slot offsets (0 past nslot)
  unsigned* sA = reinterpret_cast<unsigned*>(tc_shm + KP * 4);  // the staged tile
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t4 = lane & 3;
  const BSeg* cur = nullptr;
  for (int c = blockIdx.x; c < nch; c += gridDim.x) {
    const Chunk k = ch[c];
    const BSeg* S = segs + k.seg;
    if (state && state[S->prob] != gate) continue;  // uniform over the CTA
    const BGeom gm = S->g;
    if (S != cur) {
      __syncthreads();
      const int px = gm.nn[0] + 4, py = gm.nn[1] + 4;
      for (int j = threadIdx.x; j < KP; j += blockDim.x) soff[j] = j < NSLOT ? slot_offset<DIM>(j, px, py) : 0;
      if (S->tcA) {
        const uint4* src = reinterpret_cast<const uint4*>(S->tcA);
        uint4* dst = reinterpret_cast<uint4*>(sA);
        for (int t = threadIdx.x; t < (int)(tc_tile_bytes<DIM, MODE>() / 16); t += blockDim.x) dst[t] = src[t];
      }
      __syncthreads();
      cur = S;
    }
    const T* __restrict__ coef = static_cast<const T*>(S->coef);
    const int* __restrict__ prow = S->prow;
    const unsigned char* __restrict__ mask = S->mask;
    const float* __restrict__ rpad = S->rpadf;
    float* d = S->d32;
    const float omega = S->omega_f;
    const long long node = (long long)k.node0 + warp * 32 + lane;
    const bool valid = node < gm.nnodes;
    const unsigned i = (unsigned)(valid ? node : gm.nnodes - 1);
    int ia[3];
    decode(gm, DIM, i, ia);
    const long long pb = padded(gm, DIM, ia) * ND;
    const int pr = prow ? prow[i] : (int)i;
    int cls = -1;
    if (S->tcA && pr < 0) {
      const int blk = -pr - 1;
      cls = blk == S->cls[0] ? 0 : (blk == S->cls[1] ? 1 : -1);
    }
    const unsigned mc = __ballot_sync(0xffffffffu, valid && cls >= 0);
    const unsigned mu = __ballot_sync(0xffffffffu, valid && cls < 0);
    // ---- class patches: up to 4 tiles of 8 patches on the tensor cores
    const int ncls = __popc(mc);
    if (ncls) {
      const int ntile = (ncls + 7) >> 3;
      long long tb[4];   // padded base of patch g of each tile
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int idx = min(8 * t + g, ncls - 1);
        const int src = __fns(mc, 0, idx + 1);
        tb[t] = __shfl_sync(0xffffffffu, pb, src);
      }
      float acc[4][4];
#pragma unroll
      for (int t = 0; t < 4; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.0f;
      if (MODE == 3) {
        const unsigned* arow = sA + g * (D::KS16 / 2);
#pragma unroll 2
        for (int k0 = 0; k0 < KP; k0 += 16) {
          const unsigned a0 = arow[k0 / 2 + t4], a2 = arow[k0 / 2 + t4 + 4];
          const int o0 = soff[k0 + 2 * t4], o1 = soff[k0 + 2 * t4 + 1];
          const int o2 = soff[k0 + 2 * t4 + 8], o3 = soff[k0 + 2 * t4 + 9];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            if (t >= ntile) break;
            const float* rp = rpad + tb[t];
            mma_bf16(acc[t], a0, a2, pack_bf16(rp[o0], rp[o1]), pack_bf16(rp[o2], rp[o3]));
          }
        }
      } else {
        const unsigned* ah = sA + g * D::KS32;
        const unsigned* al = sA + 8 * D::KS32 + g * D::KS32;
#pragma unroll 2
        for (int k0 = 0; k0 < KP; k0 += 8) {
          const unsigned a0 = ah[k0 + t4], a2 = ah[k0 + t4 + 4];
          unsigned l0 = 0u, l2 = 0u;
          if (MODE == 2) {
            l0 = al[k0 + t4];
            l2 = al[k0 + t4 + 4];
          }
          const int o0 = soff[k0 + t4], o1 = soff[k0 + t4 + 4];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            if (t >= ntile) break;
            const float* rp = rpad + tb[t];
            const float r0 = rp[o0], r1 = rp[o1];
            const unsigned h0 = to_tf32(r0), h1 = to_tf32(r1);
            if (MODE == 2) {
              const unsigned e0 = to_tf32(r0 - __uint_as_float(h0)), e1 = to_tf32(r1 - __uint_as_float(h1));
              mma_tf32(acc[t], a0, a2, e0, e1);
              mma_tf32(acc[t], l0, l2, h0, h1);
            }
            mma_tf32(acc[t], a0, a2, h0, h1);
          }
        }
      }
      // thread (g, t4) holds row g (class g / 4, component g % 4) of the
      // patches 2 t4 and 2 t4 + 1 of every tile
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (t >= ntile) break;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int idx = 8 * t + 2 * t4 + e;
          const int src = __fns(mc, 0, min(idx, ncls - 1) + 1);
          const int cn = __shfl_sync(0xffffffffu, cls, src);
          const long long pbn = __shfl_sync(0xffffffffu, pb, src);
          const int comp = g & 3;
          if (idx < ncls && cn == (g >> 2) && comp < ND) d[pbn + comp] += omega * acc[t][e];
        }
      }
    }
    // ---- patches with their own rows: 8 lanes per patch, 4 at a time
    const int nu = __popc(mu);
    const int q = lane >> 3, l8 = lane & 7;
    for (int base = 0; base < nu; base += 4) {
      const int idx = base + q;
      const int src = __fns(mu, 0, min(idx, nu - 1) + 1);
      const long long pbq = __shfl_sync(0xffffffffu, pb, src);
      const int prq = __shfl_sync(0xffffffffu, pr, src);
      const unsigned iq = __shfl_sync(0xffffffffu, i, src);
      const bool shared_rows = prq < 0;
      const T* cf = coef + (size_t)(shared_rows ? -prq - 1 : prq) * NSLOT * ND;
      const float* rp = rpad + pbq;
      float y[ND];
#pragma unroll
      for (int u = 0; u < ND; ++u) y[u] = 0.0f;
#pragma unroll 4
      for (int j = l8; j < NSLOT; j += 8) {
        const float rv = rp[soff[j]];
        float cv[ND];
        RL::load(cf + (size_t)j * ND, shared_rows, cv);
#pragma unroll
        for (int u = 0; u < ND; ++u) y[u] = fmaf(cv[u], rv, y[u]);
      }
#pragma unroll
      for (int u = 0; u < ND; ++u)
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) y[u] += __shfl_xor_sync(0xffffffffu, y[u], o);
      if (idx < nu && l8 < ND) {
        float yl = y[0];
#pragma unroll
        for (int u = 1; u < ND; ++u)
          if (l8 == u) yl = y[u];
        const bool fixed = l8 < DIM && ((mask[iq] >> l8) & 1);
        d[pbq + l8] += fixed ? rp[l8] : omega * yl;
      }
    }
  }
}

// coarse b32 = R r (fine padded residual), coarse d = 0
template <int DIM>
__global__ void __launch_bounds__(256)
    f_restrict_kernel(const BSeg* __restrict__ segs, const Chunk* __restrict__ ch, int nch,
                      const int* __restrict__ state, int gate) {
  constexpr int ND = DIM + 1;
  for (int c = blockIdx.x; c < nch; c += gridDim.x) {
    const Chunk k = ch[c];
    const BSeg* C = segs + k.seg;
    const BSeg* F = C + 1;
    if (state && state[C->prob] != gate) continue;
    const BGeom cg_ = C->g, fg = F->g;
    const long long node = (long long)k.node0 + threadIdx.x;
    if (node >= cg_.nnodes) continue;
    int I[3];
    decode(cg_, DIM, (unsigned)node, I);
    const float* rf = F->rpadf;
    float acc[ND];
#pragma unroll
    for (int q = 0; q < ND; ++q) acc[q] = 0.0f;
    for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          int fi[3] = {2 * I[0] + dx, 2 * I[1] + dy, DIM == 3 ? 2 * I[2] + dz : 0};
          if (fi[0] < 0 || fi[0] > fg.n[0] || fi[1] < 0 || fi[1] > fg.n[1]) continue;
          if (DIM == 3 && (fi[2] < 0 || fi[2] > fg.n[2])) continue;
          const float w = (dx == 0 ? 1.0f : 0.5f) * (dy == 0 ? 1.0f : 0.5f) * (dz == 0 ? 1.0f : 0.5f);
          const long long fp = padded(fg, DIM, fi);
#pragma unroll
          for (int q = 0; q < ND; ++q) acc[q] = fmaf(w, rf[fp * ND + q], acc[q]);
        }
    const unsigned char m = C->mask[node];
    const long long pc = padded(cg_, DIM, I);
#pragma unroll
    for (int q = 0; q < ND; ++q) {
      C->b32[node * ND + q] = (q < DIM && ((m >> q) & 1)) ? 0.0f : acc[q];
      C->d32[pc * ND + q] = 0.0f;
    }
  }
}

// fine d += P (coarse d)
template <int DIM>
__global__ void __launch_bounds__(256)
    f_prolong_kernel(const BSeg* __restrict__ segs, const Chunk* __restrict__ ch, int nch,
                     const int* __restrict__ state, int gate) {
  constexpr int ND = DIM + 1;
  for (int c = blockIdx.x; c < nch; c += gridDim.x) {
    const Chunk k = ch[c];
    const BSeg* F = segs + k.seg;
    const BSeg* C = F - 1;
    if (state && state[F->prob] != gate) continue;
    const BGeom fg = F->g, cg_ = C->g;
    const long long node = (long long)k.node0 + threadIdx.x;
    if (node >= fg.nnodes) continue;
    int ia[3];
    decode(fg, DIM, (unsigned)node, ia);
    int lo[3], hi[3];
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      lo[t] = ia[t] / 2;
      hi[t] = (ia[t] + 1) / 2;
    }
    const float* ec = C->d32;
    float acc[ND];
#pragma unroll
    for (int q = 0; q < ND; ++q) acc[q] = 0.0f;
    for (int t = 0; t < (1 << DIM); ++t) {
      int ic[3] = {0, 0, 0};
      float w = 1.0f;
      bool dup = false;
      for (int dd = 0; dd < DIM; ++dd) {
        const int bit = (t >> dd) & 1;
        if (lo[dd] == hi[dd] && bit) dup = true;
        ic[dd] = bit ? hi[dd] : lo[dd];
        w = w * (lo[dd] == hi[dd] ? 1.0f : 0.5f);
      }
      if (dup) continue;
      const long long cp = padded(cg_, DIM, ic);
#pragma unroll
      for (int q = 0; q < ND; ++q) acc[q] = fmaf(w, ec[cp * ND + q], acc[q]);
    }
    const unsigned char m = F->mask[node];
    float* df = F->d32 + padded(fg, DIM, ia) * ND;
#pragma unroll
    for (int q = 0; q < ND; ++q)
      if (!(q < DIM && ((m >> q) & 1))) df[q] += acc[q];
  }
}

// coarse d = A^{-1} b32 (float64 inverse and sums), one CTA per problem
template <int DIM>
__global__ void __launch_bounds__(256)
    f_coarse_kernel(const BSeg* __restrict__ segs, const int* __restrict__ cseg, const int* __restrict__ state,
                    int gate) {
  constexpr int ND = DIM + 1;
  const BSeg* S = segs + cseg[blockIdx.x];
  if (state && state[S->prob] != gate) return;
  const BGeom g = S->g;
  const int n = S->cn, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double* A = S->cinv;
  const float* b = S->b32;
  for (int row = warp; row < n; row += nw) {
    double s = 0.0;
    for (int c = lane; c < n; c += 32) s += A[(long long)row * n + c] * (double)b[c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) {
      int ia[3];
      decode(g, DIM, (unsigned)(row / ND), ia);
      S->d32[padded(g, DIM, ia) * ND + row % ND] = (float)s;
    }
  }
}

// finest-level vectors of every problem: x = xb + j*xstep + off[p] (j from
// the device counter dj when given), likewise b; r = rb + off[p]
__global__ void b_point_kernel(BSeg* segs, const int* __restrict__ fin, const long long* __restrict__ off,
                               int nprob, double* xb, long long xstep, const double* bb, long long bstep,
                               double* rb, const int* dj) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nprob) return;
  const long long j = dj ? *dj : 0;
  BSeg* S = segs + fin[p];
  S->x = xb + j * xstep + off[p];
  if (bb) S->b = const_cast<double*>(bb) + j * bstep + off[p];
  if (rb) S->r = rb + off[p];
}

__global__ void b_bump_kernel(int* dj) { *dj += 1; }

// ---------------------------------------------------------------------------
// Krylov kernels: one cluster of kCL CTAs per problem; CTA `rank` owns a
// contiguous slice of the problem's finest-level vector.  Sums are reduced
// in a fixed order (warp shuffles, warps in order, CTAs in rank order), so
// a problem's result does not depend on the rest of the batch.
struct KrylovArgs {
  int nprob, m, maxit;
  double rtol;
  long long ntot;
  const long long* off;
  double* V;       // (m+1) packed vectors
  double* Z;       // m packed vectors
  double* R;       // packed work vector
  double* small;   // per problem: H (m+1) x m, cs m, sn m, g m+1, y m
  double* bn;      // ||b||
  double* rel;     // last true relative residual
  int* state;      // 0 done, 1 in a cycle, 2 cycle ended, 3 residual due
  int* its;        // preconditioner applications
  int* kk;         // Krylov dimension of the ended cycle
  int* count;      // problems in a cycle after the kernel
  const int* dj;   // Arnoldi step of the cycle
};

__host__ __device__ inline long long small_stride(int m) { return (long long)(m + 1) * m + 3LL * m + (m + 1); }

struct ClusterSum {
  double warp[32];
  double part[2];
  double bcast;
};

// sum of v over the cluster (every thread passes its partial)
__device__ double cluster_sum(double v, ClusterSum& sm, int& parity, cg::cluster_group& cl) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sm.warp[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm.warp[w];
    sm.part[parity] = t;
  }
  cl.sync();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int r = 0; r < kCL; ++r) t += *cl.map_shared_rank(&sm.part[parity], r);
    sm.bcast = t;
  }
  __syncthreads();
  const double t = sm.bcast;
  parity ^= 1;
  return t;
}

__device__ __forceinline__ void slice(long long n, int rank, long long* lo, long long* hi) {
  *lo = n * rank / kCL;
  *hi = n * (rank + 1) / kCL;
}

// ||b||: state 3 (residual due) or, for b = 0, x = 0 and done
__global__ void __cluster_dims__(kCL, 1, 1) __launch_bounds__(kKThreads)
    k_init_kernel(KrylovArgs a, const double* __restrict__ b, double* __restrict__ x) {
  __shared__ ClusterSum sm;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), p = blockIdx.x / kCL;
  int parity = 0;
  const long long o = a.off[p];
  long long lo, hi;
  slice(a.off[p + 1] - o, rank, &lo, &hi);
  double s = 0.0;
  for (long long t = lo + threadIdx.x; t < hi; t += blockDim.x) s += b[o + t] * b[o + t];
  const double bn = sqrt(cluster_sum(s, sm, parity, cl));
  if (bn == 0.0)
    for (long long t = lo + threadIdx.x; t < hi; t += blockDim.x) x[o + t] = 0.0;
  if (rank == 0 && threadIdx.x == 0) {
    a.bn[p] = bn;
    a.its[p] = 0;
    a.rel[p] = 0.0;
    a.state[p] = bn == 0.0 ? 0 : 3;
  }
  cl.sync();
}

// start of a cycle for problems with state 3: beta = ||r||, stop or
// g = beta e_1 and v_0 = r / beta
__global__ void __cluster_dims__(kCL, 1, 1) __launch_bounds__(kKThreads) k_start_kernel(KrylovArgs a) {
  __shared__ ClusterSum sm;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), p = blockIdx.x / kCL;
  const int st = a.state[p];
  if (st != 3) return;  // the same decision in every CTA of the cluster
  int parity = 0;
  const long long o = a.off[p];
  long long lo, hi;
  slice(a.off[p + 1] - o, rank, &lo, &hi);
  const double* w = a.R + o;
  double s = 0.0;
  for (long long t = lo + threadIdx.x; t < hi; t += blockDim.x) s += w[t] * w[t];
  const double beta = sqrt(cluster_sum(s, sm, parity, cl));
  const double bn = a.bn[p];
  const bool stop = beta <= a.rtol * bn || a.its[p] >= a.maxit;
  if (!stop) {
    const double f = beta != 0.0 ? 1.0 / beta : 0.0;
    double* v0 = a.V + o;
    for (long long t = lo + threadIdx.x; t < hi; t += blockDim.x) v0[t] = w[t] * f;
  }
  cl.sync();  // every CTA has read the state before it changes
  if (rank == 0 && threadIdx.x == 0) {
    a.rel[p] = beta / bn;
    if (stop) {
      a.state[p] = 0;
    } else {
      double* g = a.small + p * small_stride(a.m) + (long long)(a.m + 1) * a.m + 2LL * a.m;
      for (int t = 0; t <= a.m; ++t) g[t] = t == 0 ? beta : 0.0;
      a.state[p] = 1;
      atomicAdd(a.count, 1);
    }
  }
}

// Arnoldi step j for problems in a cycle: w = R (= L z_j), modified
// Gram-Schmidt against v_0..v_j (subtraction of v_i fused with the dot with
// v_{i+1}), h_{j+1,j} = ||w||, v_{j+1} = w / h, Givens update of the
// Hessenberg column and of g, stopping test on |g_{j+1}| / ||b||
__global__ void __cluster_dims__(kCL, 1, 1) __launch_bounds__(kKThreads) k_arnoldi_kernel(KrylovArgs a) {
  __shared__ ClusterSum sm;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), p = blockIdx.x / kCL;
  if (a.state[p] != 1) return;
  const int j = *a.dj, m = a.m;
  int parity = 0;
  const long long o = a.off[p];
  long long lo, hi;
  slice(a.off[p + 1] - o, rank, &lo, &hi);
  double* w = a.R + o;
  double* H = a.small + p * small_stride(m);
  double s = 0.0;
  {
    const double* v0 = a.V + o;
    for (long long t = lo + threadIdx.x; t < hi; t += blockDim.x) s += w[t] * v0[t];
  }
  for (int i = 0; i <= j; ++i) {
    const double h = cluster_sum(s, sm, parity, cl);
    if (rank == 0 && threadIdx.x == 0) H[(long long)i * m + j] = h;
    const double* vi = a.V + (long long)i * a.ntot + o;
    const double* vn = i < j ? a.V + (long long)(i + 1) * a.ntot + o : nullptr;
    s = 0.0;
    for (long long t = lo + threadIdx.x; t < hi; t += blockDim.x) {
      const double wv = w[t] - h * vi[t];
      w[t] = wv;
      s += wv * (vn ? vn[t] : wv);
    }
  }
  const double hn = sqrt(cluster_sum(s, sm, parity, cl));
  {
    const double f = hn != 0.0 ? 1.0 / hn : 0.0;
    double* vj1 = a.V + (long long)(j + 1) * a.ntot + o;
    for (long long t = lo + threadIdx.x; t < hi; t += blockDim.x) vj1[t] = w[t] * f;
  }
  cl.sync();
  if (rank == 0 && threadIdx.x == 0) {
    double* cs = H + (long long)(m + 1) * m;
    double* sn = cs + m;
    double* g = sn + m;
    H[(long long)(j + 1) * m + j] = hn;
    for (int i = 0; i < j; ++i) {
      const double x0 = H[(long long)i * m + j], x1 = H[(long long)(i + 1) * m + j];
      H[(long long)i * m + j] = cs[i] * x0 + sn[i] * x1;
      H[(long long)(i + 1) * m + j] = -sn[i] * x0 + cs[i] * x1;
    }
    const double x0 = H[(long long)j * m + j], x1 = H[(long long)(j + 1) * m + j];
    const double den = sqrt(x0 * x0 + x1 * x1);
    cs[j] = den == 0.0 ? 1.0 : x0 / den;
    sn[j] = den == 0.0 ? 0.0 : x1 / den;
    H[(long long)j * m + j] = den;
    H[(long long)(j + 1) * m + j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    const double est = fabs(g[j + 1]) / a.bn[p];
    const int its = a.its[p] + 1;
    a.its[p] = its;
    if (est <= a.rtol || hn == 0.0 || its >= a.maxit || j + 1 == m) {
      a.kk[p] = j + 1;
      a.state[p] = 2;
    } else {
      atomicAdd(a.count, 1);
    }
  }
}

// end of a cycle (state 2): y = H_k^{-1} g, x += sum_i y_i z_i, state 3
__global__ void __cluster_dims__(kCL, 1, 1) __launch_bounds__(kKThreads)
    k_update_kernel(KrylovArgs a, double* __restrict__ x) {
  __shared__ double y[256];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), p = blockIdx.x / kCL;
  if (a.state[p] != 2) return;
  const int m = a.m, k = a.kk[p];
  const double* H = a.small + p * small_stride(m);
  const double* g = H + (long long)(m + 1) * m + 2LL * m;
  if (threadIdx.x == 0) {
    for (int i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int t = i + 1; t < k; ++t) s = s - H[(long long)i * m + t] * y[t];
      y[i] = s / H[(long long)i * m + i];
    }
  }
  __syncthreads();
  const long long o = a.off[p];
  long long lo, hi;
  slice(a.off[p + 1] - o, rank, &lo, &hi);
  for (long long t = lo + threadIdx.x; t < hi; t += blockDim.x) {
    double s = x[o + t];
    for (int i = 0; i < k; ++i) s = s + y[i] * a.Z[(long long)i * a.ntot + o + t];
    x[o + t] = s;
  }
  cl.sync();  // every CTA has read the state before it changes
  if (rank == 0 && threadIdx.x == 0) a.state[p] = 3;
}

// ---------------------------------------------------------------------------
// host side
struct Plan {
  int first = 0, count = 0;
};

struct Tile {
  int tpp = 16, threads = 256, ctas_per_sm = 8;
};

typedef void (*ApplyFn)(const BSeg*, const Chunk*, int, const int*, int);

template <int DIM, int PT>
ApplyFn apply_fn(int tpp) {
  switch (tpp) {
    case 1: return b_apply_kernel<DIM, PT, 1>;
    case 2: return b_apply_kernel<DIM, PT, 2>;
    case 4: return b_apply_kernel<DIM, PT, 4>;
    case 8: return b_apply_kernel<DIM, PT, 8>;
    case 16: return b_apply_kernel<DIM, PT, 16>;
    default: return b_apply_kernel<DIM, PT, 32>;
  }
}

template <int DIM, int PT>
ApplyFn fapply_fn(int tpp) {
  switch (tpp) {
    case 1: return f_apply_kernel<DIM, PT, 1>;
    case 2: return f_apply_kernel<DIM, PT, 2>;
    case 4: return f_apply_kernel<DIM, PT, 4>;
    case 8: return f_apply_kernel<DIM, PT, 8>;
    case 16: return f_apply_kernel<DIM, PT, 16>;
    default: return f_apply_kernel<DIM, PT, 32>;
  }
}

template <int DIM, int PT>
ApplyFn tcapply_fn(int mode) {
  if (mode == 1) return f_apply_tc_kernel<DIM, PT, 1>;
  if (mode == 2) return f_apply_tc_kernel<DIM, PT, 2>;
  return f_apply_tc_kernel<DIM, PT, 3>;
}

size_t tc_bytes(int dim, int mode) {
  if (dim == 2) return mode == 1 ? tc_tile_bytes<2, 1>() : mode == 2 ? tc_tile_bytes<2, 2>() : tc_tile_bytes<2, 3>();
  return mode == 1 ? tc_tile_bytes<3, 1>() : mode == 2 ? tc_tile_bytes<3, 2>() : tc_tile_bytes<3, 3>();
}

size_t tc_smem(int dim, int mode) { return (size_t)(dim == 3 ? TcDims<3>::KP : TcDims<2>::KP) * 4 + tc_bytes(dim, mode); }

ApplyFn pick_apply(int dim, fc_prec prec, int tpp) {
  if (prec == FC_PREC_FP32) return dim == 2 ? fapply_fn<2, 1>(tpp) : fapply_fn<3, 1>(tpp);
  if (prec == FC_PREC_BF16) return dim == 2 ? fapply_fn<2, 2>(tpp) : fapply_fn<3, 2>(tpp);
  const int pt = prec == FC_PREC_FP64 ? 0 : prec == FC_PREC_FP32 ? 1 : 2;
  if (dim == 2) return pt == 0 ? apply_fn<2, 0>(tpp) : pt == 1 ? apply_fn<2, 1>(tpp) : apply_fn<2, 2>(tpp);
  return pt == 0 ? apply_fn<3, 0>(tpp) : pt == 1 ? apply_fn<3, 1>(tpp) : apply_fn<3, 2>(tpp);
}

}  // namespace
}  // namespace fc

struct fc_batch_s {
  int nprob = 0, dim = 0, maxl = 0, m = 30, nu_pre = 0, nu_post = 0;
  fc_prec prec = FC_PREC_FP32;
  bool f32 = false;  // float32 correction form (float32 / bfloat16 rows)
  int tc = 0;        // tensor-core apply of the class blocks (fc_options.tc), float32 form only
  std::vector<void*> tcbuf;  // staged MMA tiles of the segments
  cudaStream_t user = nullptr, s = nullptr;
  cudaEvent_t ev = nullptr;
  std::vector<fc_handle> hs;
  std::vector<long long> off;
  long long ntot = 0;
  int nseg = 0;
  fc::BSeg* segs = nullptr;
  int* fin = nullptr;
  int* cseg = nullptr;
  long long* doff = nullptr;
  fc::Chunk* chunks = nullptr;
  std::vector<fc::Plan> pn, prc;
  fc::Plan pfin;  // finest levels
  fc::Plan psm;   // finest levels that are smoothed (more than one level)
  long long fin_patches = 0;
  int nsm = 152;
  fc::Tile tile;
  double* V = nullptr;
  double* Z = nullptr;
  double* R = nullptr;
  double* small = nullptr;
  double* bn = nullptr;
  double* rel = nullptr;
  int* state = nullptr;
  int* its = nullptr;
  int* kk = nullptr;
  int* dj = nullptr;
  int* count = nullptr;
  int* hcount = nullptr;  // pinned
  // per-launch timing of the finest-level smoothing (fc_batch_smooth):
  // kind 0 patch apply, 1 residual
  bool prof_on = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof[2];
  double apply_bytes = 0.0;  // algorithmic bytes of one finest-level apply
  double* bh = nullptr;  // device staging of fc_batch_solve_host
  double* xh = nullptr;
  cudaGraphExec_t step_graph = nullptr;
  int step_kernels = 0;
  cudaGraphExec_t vgraph[2] = {nullptr, nullptr};  // float32 V-cycle (handle path)
  int vgraph_kernels = 0;
  double graph_rtol = -1.0;  // the captured step bakes these in
  int graph_maxit = -1;
  std::string err;
};

namespace {

using namespace fc;

cudaError_t prepare_tc_tile(int dim, int mode, fc_prec prec, const void* coef, int c0, int c1, void* out,
                            cudaStream_t s) {
  const bool f = prec == FC_PREC_FP32;
  const float* cf = static_cast<const float*>(coef);
  const __nv_bfloat16* cb = static_cast<const __nv_bfloat16*>(coef);
  if (dim == 2) {
    if (mode == 1) f ? tc_prepare_kernel<2, 1><<<4, 256, 0, s>>>(cf, c0, c1, out) : tc_prepare_kernel<2, 1><<<4, 256, 0, s>>>(cb, c0, c1, out);
    else if (mode == 2) f ? tc_prepare_kernel<2, 2><<<4, 256, 0, s>>>(cf, c0, c1, out) : tc_prepare_kernel<2, 2><<<4, 256, 0, s>>>(cb, c0, c1, out);
    else f ? tc_prepare_kernel<2, 3><<<4, 256, 0, s>>>(cf, c0, c1, out) : tc_prepare_kernel<2, 3><<<4, 256, 0, s>>>(cb, c0, c1, out);
  } else {
    if (mode == 1) f ? tc_prepare_kernel<3, 1><<<16, 256, 0, s>>>(cf, c0, c1, out) : tc_prepare_kernel<3, 1><<<16, 256, 0, s>>>(cb, c0, c1, out);
    else if (mode == 2) f ? tc_prepare_kernel<3, 2><<<16, 256, 0, s>>>(cf, c0, c1, out) : tc_prepare_kernel<3, 2><<<16, 256, 0, s>>>(cb, c0, c1, out);
    else f ? tc_prepare_kernel<3, 3><<<16, 256, 0, s>>>(cf, c0, c1, out) : tc_prepare_kernel<3, 3><<<16, 256, 0, s>>>(cb, c0, c1, out);
  }
  note_launches(1);
  return cudaGetLastError();
}

fc_status bfail(fc_batch b, fc_status st, const std::string& msg) {
  if (b) b->err = msg;
  return st;
}

#define BK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) return bfail(B, FC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

unsigned grid_of(const fc_batch B, const Plan& p, int per_sm) {
  long long g = std::min<long long>(p.count, (long long)B->nsm * per_sm);
  return (unsigned)std::max<long long>(g, 1);
}

fc_status residual(fc_batch B, const Plan& p, int out, int use_b, const int* state, int gate) {
  if (p.count == 0) return FC_OK;
  const unsigned grid = grid_of(B, p, 8);
  const Chunk* c = B->chunks + p.first;
  if (B->dim == 2) {
    if (out == 0) b_residual_kernel<2, 0><<<grid, kChunk, 0, B->s>>>(B->segs, c, p.count, use_b, state, gate);
    else if (out == 1) b_residual_kernel<2, 1><<<grid, kChunk, 0, B->s>>>(B->segs, c, p.count, use_b, state, gate);
    else b_residual_kernel<2, 2><<<grid, kChunk, 0, B->s>>>(B->segs, c, p.count, use_b, state, gate);
  } else {
    if (out == 0) b_residual_kernel<3, 0><<<grid, kChunk, 0, B->s>>>(B->segs, c, p.count, use_b, state, gate);
    else if (out == 1) b_residual_kernel<3, 1><<<grid, kChunk, 0, B->s>>>(B->segs, c, p.count, use_b, state, gate);
    else b_residual_kernel<3, 2><<<grid, kChunk, 0, B->s>>>(B->segs, c, p.count, use_b, state, gate);
  }
  note_launches(1);
  BK(cudaGetLastError());
  return FC_OK;
}

fc_status apply(fc_batch B, const Plan& p, const Tile& t, const int* state, int gate) {
  if (p.count == 0) return FC_OK;
  if (B->f32 && B->tc) {
    const int pt = B->prec == FC_PREC_FP32 ? 1 : 2;
    ApplyFn fn = B->dim == 2 ? (pt == 1 ? tcapply_fn<2, 1>(B->tc) : tcapply_fn<2, 2>(B->tc))
                             : (pt == 1 ? tcapply_fn<3, 1>(B->tc) : tcapply_fn<3, 2>(B->tc));
    const size_t smem = tc_smem(B->dim, B->tc);
    int per_sm = 0, nsm = 0;
    BK(persistent_ctas((const void*)fn, 256, smem, &per_sm, &nsm));
    fn<<<grid_of(B, p, per_sm), 256, smem, B->s>>>(B->segs, B->chunks + p.first, p.count, state, gate);
    note_launches(1);
    BK(cudaGetLastError());
    return FC_OK;
  }
  ApplyFn fn = pick_apply(B->dim, B->prec, t.tpp);
  const unsigned grid = grid_of(B, p, t.ctas_per_sm);
  fn<<<grid, t.threads, 0, B->s>>>(B->segs, B->chunks + p.first, p.count, state, gate);
  note_launches(1);
  BK(cudaGetLastError());
  return FC_OK;
}

// float32 correction-form phases: 0 enter (xzero), 1 exit (xzero),
// 2 residual, 3 restrict, 4 prolong
fc_status fphase(fc_batch B, int kind, const Plan& p, int xzero, const int* state, int gate) {
  if (p.count == 0) return FC_OK;
  const unsigned grid = grid_of(B, p, 8);
  const Chunk* c = B->chunks + p.first;
  const int n = p.count;
  if (B->dim == 2) {
    switch (kind) {
      case 0: f_enter_kernel<2><<<grid, kChunk, 0, B->s>>>(B->segs, c, n, xzero, state, gate); break;
      case 1: f_exit_kernel<2><<<grid, kChunk, 0, B->s>>>(B->segs, c, n, xzero, state, gate); break;
      case 2: f_residual_kernel<2><<<grid, kChunk, 0, B->s>>>(B->segs, c, n, state, gate); break;
      case 3: f_restrict_kernel<2><<<grid, kChunk, 0, B->s>>>(B->segs, c, n, state, gate); break;
      default: f_prolong_kernel<2><<<grid, kChunk, 0, B->s>>>(B->segs, c, n, state, gate); break;
    }
  } else {
    switch (kind) {
      case 0: f_enter_kernel<3><<<grid, kChunk, 0, B->s>>>(B->segs, c, n, xzero, state, gate); break;
      case 1: f_exit_kernel<3><<<grid, kChunk, 0, B->s>>>(B->segs, c, n, xzero, state, gate); break;
      case 2: f_residual_kernel<3><<<grid, kChunk, 0, B->s>>>(B->segs, c, n, state, gate); break;
      case 3: f_restrict_kernel<3><<<grid, kChunk, 0, B->s>>>(B->segs, c, n, state, gate); break;
      default: f_prolong_kernel<3><<<grid, kChunk, 0, B->s>>>(B->segs, c, n, state, gate); break;
    }
  }
  note_launches(1);
  BK(cudaGetLastError());
  return FC_OK;
}

fc_status sweeps(fc_batch B, const Plan& p, int n, const int* state, int gate) {
  const int out = B->prec == FC_PREC_FP64 ? 1 : 2;
  for (int s = 0; s < n; ++s) {
    fc_status st = B->f32 ? fphase(B, 2, p, 0, state, gate) : residual(B, p, out, 1, state, gate);
    if (st == FC_OK) st = apply(B, p, B->tile, state, gate);
    if (st != FC_OK) return st;
  }
  return FC_OK;
}

fc_status transfer(fc_batch B, int kind, const Plan& p, const int* state, int gate) {
  if (p.count == 0) return FC_OK;
  const unsigned grid = grid_of(B, p, 8);
  const Chunk* c = B->chunks + p.first;
  if (kind == 0) {
    if (B->dim == 2) b_restrict_kernel<2><<<grid, kChunk, 0, B->s>>>(B->segs, c, p.count, state, gate);
    else b_restrict_kernel<3><<<grid, kChunk, 0, B->s>>>(B->segs, c, p.count, state, gate);
  } else {
    if (B->dim == 2) b_prolong_kernel<2><<<grid, kChunk, 0, B->s>>>(B->segs, c, p.count, state, gate);
    else b_prolong_kernel<3><<<grid, kChunk, 0, B->s>>>(B->segs, c, p.count, state, gate);
  }
  note_launches(1);
  BK(cudaGetLastError());
  return FC_OK;
}

// V(nu_pre, nu_post) in the float32 correction form (x known zero: xzero)
fc_status vcycle_f32(fc_batch B, int xzero, const int* state, int gate) {
  fc_status st = fphase(B, 0, B->pfin, xzero, state, gate);
  for (int li = B->maxl - 1; li >= 1 && st == FC_OK; --li) {
    st = sweeps(B, B->pn[li], B->nu_pre, state, gate);
    if (st == FC_OK) st = fphase(B, 2, B->pn[li], 0, state, gate);
    if (st == FC_OK) st = fphase(B, 3, B->prc[li - 1], 0, state, gate);
  }
  if (st != FC_OK) return st;
  if (B->dim == 2) f_coarse_kernel<2><<<B->nprob, 256, 0, B->s>>>(B->segs, B->cseg, state, gate);
  else f_coarse_kernel<3><<<B->nprob, 256, 0, B->s>>>(B->segs, B->cseg, state, gate);
  note_launches(1);
  BK(cudaGetLastError());
  for (int li = 1; li < B->maxl && st == FC_OK; ++li) {
    st = fphase(B, 4, B->pn[li], 0, state, gate);
    if (st == FC_OK) st = sweeps(B, B->pn[li], B->nu_post, state, gate);
  }
  if (st == FC_OK) st = fphase(B, 1, B->pfin, xzero, state, gate);
  return st;
}

// V(nu_pre, nu_post) on every problem at once: levels aligned at the
// coarsest grid, so each phase holds the problems deep enough for it
fc_status vcycle_all(fc_batch B, const int* state, int gate) {
  fc_status st = FC_OK;
  for (int li = B->maxl - 1; li >= 1 && st == FC_OK; --li) {
    st = sweeps(B, B->pn[li], B->nu_pre, state, gate);
    if (st == FC_OK) st = residual(B, B->pn[li], 0, 1, state, gate);
    if (st == FC_OK) st = transfer(B, 0, B->prc[li - 1], state, gate);
  }
  if (st != FC_OK) return st;
  b_coarse_kernel<<<B->nprob, 256, 0, B->s>>>(B->segs, B->cseg, state, gate);
  note_launches(1);
  BK(cudaGetLastError());
  for (int li = 1; li < B->maxl && st == FC_OK; ++li) {
    st = transfer(B, 1, B->pn[li], state, gate);
    if (st == FC_OK) st = sweeps(B, B->pn[li], B->nu_post, state, gate);
  }
  return st;
}

fc_status point(fc_batch B, double* x, long long xstep, const double* b, long long bstep, double* r,
                const int* dj) {
  b_point_kernel<<<(B->nprob + 127) / 128, 128, 0, B->s>>>(B->segs, B->fin, B->doff, B->nprob, x, xstep, b, bstep,
                                                           r, dj);
  note_launches(1);
  BK(cudaGetLastError());
  return FC_OK;
}

fc_status zero_finest(fc_batch B, const int* state, int gate) {
  const Plan& p = B->pfin;
  if (p.count == 0) return FC_OK;
  const unsigned grid = grid_of(B, p, 8);
  if (B->dim == 2) b_zero_kernel<3><<<grid, kChunk, 0, B->s>>>(B->segs, B->chunks + p.first, p.count, state, gate);
  else b_zero_kernel<4><<<grid, kChunk, 0, B->s>>>(B->segs, B->chunks + p.first, p.count, state, gate);
  note_launches(1);
  BK(cudaGetLastError());
  return FC_OK;
}

// Patch-apply tile autotuner: every (lanes per patch, threads per CTA, CTAs
// per SM) candidate runs the finest-level apply of the batch (x pointed at
// scratch), best of three timed launches after one warm-up; the fastest
// candidate is kept.
fc_status autotune(fc_batch B) {
  if (B->psm.count == 0) return FC_OK;
  fc_status st = point(B, B->R, 0, nullptr, 0, nullptr, nullptr);
  if (st != FC_OK) return st;
  BK(cudaMemsetAsync(B->R, 0, sizeof(double) * B->ntot, B->s));
  cudaEvent_t e0, e1;
  BK(cudaEventCreate(&e0));
  BK(cudaEventCreate(&e1));
  float best = 1e30f;
  Tile bt = B->tile;
  const int tpps[6] = {1, 2, 4, 8, 16, 32};
  const int thr[3] = {128, 256, 512};
  const int cps[4] = {2, 4, 8, 16};
  for (int a = 0; a < 6 && st == FC_OK; ++a)
    for (int t = 0; t < 3 && st == FC_OK; ++t)
      for (int c = 0; c < 4 && st == FC_OK; ++c) {
        if (thr[t] * cps[c] > 2048 || thr[t] / tpps[a] > kChunk) continue;
        Tile cand{tpps[a], thr[t], cps[c]};
        float tmin = 1e30f;
        for (int rep = 0; rep < 4 && st == FC_OK; ++rep) {
          if (cudaEventRecord(e0, B->s) != cudaSuccess) st = FC_ERR_CUDA;
          if (st == FC_OK) st = apply(B, B->psm, cand, nullptr, 0);
          if (st == FC_OK && cudaEventRecord(e1, B->s) != cudaSuccess) st = FC_ERR_CUDA;
          if (st == FC_OK && cudaEventSynchronize(e1) != cudaSuccess) st = FC_ERR_CUDA;
          float ms = 0.0f;
          if (st == FC_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = FC_ERR_CUDA;
          if (rep > 0) tmin = std::min(tmin, ms);
        }
        if (st == FC_OK && tmin < best) {
          best = tmin;
          bt = cand;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != FC_OK) return st == FC_ERR_CUDA ? bfail(B, st, "autotune: CUDA error") : st;
  B->tile = bt;
  return FC_OK;
}

void prof_clear(fc_batch B, int kind) {
  for (auto& pr : B->prof[kind]) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  B->prof[kind].clear();
}

void free_batch(fc_batch B) {
  if (!B) return;
  if (B->s) cudaStreamSynchronize(B->s);
  prof_clear(B, 0);
  prof_clear(B, 1);
  if (B->step_graph) cudaGraphExecDestroy(B->step_graph);
  for (auto& g : B->vgraph)
    if (g) cudaGraphExecDestroy(g);
  void* ptrs[] = {B->segs, B->fin, B->cseg, B->doff, B->chunks, B->V, B->Z, B->R, B->small, B->bn, B->rel,
                  B->state, B->its, B->kk, B->dj, B->count, B->bh, B->xh};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (void* p : B->tcbuf)
    if (p) cudaFree(p);
  if (B->hcount) cudaFreeHost(B->hcount);
  if (B->ev) cudaEventDestroy(B->ev);
  if (B->s) cudaStreamDestroy(B->s);
}

// order the batch stream after the caller's stream (entry) and the
// caller's stream after the batch stream (exit)
fc_status krylov_alloc(fc_batch B) {
  if (B->V) return FC_OK;
  const size_t nt = (size_t)B->ntot;
  const int nprob = B->nprob;
  BK(cudaMalloc(&B->V, sizeof(double) * nt * (B->m + 1)));
  BK(cudaMalloc(&B->Z, sizeof(double) * nt * B->m));
  BK(cudaMalloc(&B->small, sizeof(double) * small_stride(B->m) * nprob));
  BK(cudaMalloc(&B->bn, sizeof(double) * nprob));
  BK(cudaMalloc(&B->rel, sizeof(double) * nprob));
  BK(cudaMalloc(&B->state, sizeof(int) * nprob));
  BK(cudaMalloc(&B->its, sizeof(int) * nprob));
  BK(cudaMalloc(&B->kk, sizeof(int) * nprob));
  BK(cudaMalloc(&B->dj, sizeof(int)));
  BK(cudaMalloc(&B->count, sizeof(int)));
  BK(cudaMallocHost(&B->hcount, sizeof(int)));
  BK(cudaMemsetAsync(B->state, 0, sizeof(int) * nprob, B->s));
  return FC_OK;
}

fc_status enter(fc_batch B) {
  BK(cudaEventRecord(B->ev, B->user));
  BK(cudaStreamWaitEvent(B->s, B->ev, 0));
  return FC_OK;
}
fc_status leave(fc_batch B, fc_status st) {
  if (cudaEventRecord(B->ev, B->s) == cudaSuccess) cudaStreamWaitEvent(B->user, B->ev, 0);
  return st;
}

fc_status step_graph(fc_batch B, KrylovArgs& ka) {
  if (B->step_graph) return FC_OK;
  cudaGraph_t graph = nullptr;
  BK(cudaStreamBeginCapture(B->s, cudaStreamCaptureModeThreadLocal));
  set_capturing(true);
  fc_status st = point(B, B->Z, B->ntot, B->V, B->ntot, B->R, B->dj);
  if (st == FC_OK && cudaMemsetAsync(B->count, 0, sizeof(int), B->s) != cudaSuccess) st = FC_ERR_CUDA;
  if (B->f32) {
    if (st == FC_OK) st = vcycle_f32(B, 1, B->state, 1);
  } else {
    if (st == FC_OK) st = zero_finest(B, B->state, 1);
    if (st == FC_OK) st = vcycle_all(B, B->state, 1);
  }
  if (st == FC_OK) st = residual(B, B->pfin, 0, 0, B->state, 1);  // R = L z_j
  if (st == FC_OK) {
    k_arnoldi_kernel<<<B->nprob * kCL, kKThreads, 0, B->s>>>(ka);
    b_bump_kernel<<<1, 1, 0, B->s>>>(B->dj);
    note_launches(2);
    if (cudaGetLastError() != cudaSuccess) st = FC_ERR_CUDA;
  }
  cudaError_t e = cudaStreamEndCapture(B->s, &graph);
  set_capturing(false);
  if (e != cudaSuccess || st != FC_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st != FC_OK ? st : bfail(B, FC_ERR_CUDA, std::string("step graph capture: ") + cudaGetErrorString(e));
  }
  size_t nn = 0;
  cudaGraphGetNodes(graph, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn) cudaGraphGetNodes(graph, nodes.data(), &nn);
  int kernels = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) kernels++;
  }
  e = cudaGraphInstantiate(&B->step_graph, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    B->step_graph = nullptr;
    return bfail(B, FC_ERR_CUDA, std::string("step graph instantiate: ") + cudaGetErrorString(e));
  }
  B->step_kernels = kernels;
  return FC_OK;
}

}  // namespace

namespace {
fc_status create_batch(fc_batch* out, const fc_handle* handles, int nprob, void* cuda_stream, const Tile* fixed);
}

namespace fc {

// V-cycle of one handle with float32 / bfloat16 rows in the float32
// correction form, through a batch holding that handle alone (created on
// first use; the tile tuned on the handle's finest level).  The V-cycle
// after the pointer update is captured once per x-is-zero flag as a CUDA
// graph.
// Tiles of the single-handle V-cycles, one per (dimension, row precision,
// size class = log2 of the finest patch count), tuned by the first handle of
// a class and reused by every later one: a problem's rounding then does not
// depend on what else ran while its tile was timed (serving runs problems
// side by side).
std::mutex g_tile_mu;
std::map<long long, Tile> g_tiles;

fc_status handle_vcycle_f32(fc_handle h, double* x, const double* b, bool xzero) {
  if (!h->self_batch) {
    fc_handle one = h;
    const long long np = h->lev[h->nlev - 1].g.nnodes;
    int cls = 0;
    while ((1LL << (cls + 1)) <= np) ++cls;
    const long long key = (((long long)h->dim * 8 + (long long)h->opt.prec) * 4 + h->opt.tc) * 64 + cls;
    std::lock_guard<std::mutex> lk(g_tile_mu);
    auto it = g_tiles.find(key);
    fc_status st = create_batch(&h->self_batch, &one, 1, h->stream, it == g_tiles.end() ? nullptr : &it->second);
    if (st == FC_OK && it == g_tiles.end()) g_tiles[key] = h->self_batch->tile;
    if (st != FC_OK) {
      h->err = std::string("float32 V-cycle: ") + fc_batch_last_error(h->self_batch);
      fc_batch_destroy(h->self_batch);
      h->self_batch = nullptr;
      return st;
    }
  }
  fc_batch B = h->self_batch;
  fc_status st = enter(B);
  if (st == FC_OK) st = point(B, x, 0, b, 0, B->R, nullptr);
  cudaGraphExec_t& gx = B->vgraph[xzero ? 1 : 0];
  if (st == FC_OK && !gx) {
    cudaGraph_t graph = nullptr;
    BK(cudaStreamBeginCapture(B->s, cudaStreamCaptureModeThreadLocal));
    set_capturing(true);
    st = vcycle_f32(B, xzero ? 1 : 0, nullptr, 0);
    cudaError_t e = cudaStreamEndCapture(B->s, &graph);
    set_capturing(false);
    if (e == cudaSuccess && st == FC_OK) {
      size_t nn = 0;
      cudaGraphGetNodes(graph, nullptr, &nn);
      B->vgraph_kernels = (int)nn;
      e = cudaGraphInstantiate(&gx, graph, 0);
    }
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      gx = nullptr;
      st = bfail(B, FC_ERR_CUDA, std::string("V-cycle graph: ") + cudaGetErrorString(e));
    }
  }
  if (st == FC_OK) {
    BK(cudaGraphLaunch(gx, B->s));
    note_launches(B->vgraph_kernels);
  }
  st = leave(B, st);
  if (st != FC_OK) h->err = std::string("float32 V-cycle: ") + B->err;
  return st;
}

void handle_batch_free(fc_handle h) {
  if (h->self_batch) {
    fc_batch_destroy(h->self_batch);
    h->self_batch = nullptr;
  }
}

}  // namespace fc

extern "C" {

fc_status fc_batch_create(fc_batch* out, const fc_handle* handles, int nprob, void* cuda_stream) {
  return create_batch(out, handles, nprob, cuda_stream, nullptr);
}

fc_status fc_batch_create_tiled(fc_batch* out, const fc_handle* handles, int nprob, void* cuda_stream, int tpp,
                                int threads, int ctas_per_sm) {
  if (!out) return FC_ERR_INVALID;
  const bool ok_tpp = tpp == 1 || tpp == 2 || tpp == 4 || tpp == 8 || tpp == 16 || tpp == 32;
  const bool ok_thr = threads == 128 || threads == 256 || threads == 512;
  if (!ok_tpp || !ok_thr || threads / tpp > fc::kChunkNodes || ctas_per_sm < 1 || ctas_per_sm > 64) {
    *out = nullptr;
    return FC_ERR_INVALID;
  }
  const Tile t{tpp, threads, ctas_per_sm};
  return create_batch(out, handles, nprob, cuda_stream, &t);
}

}  // extern "C"

namespace {

fc_status create_batch(fc_batch* out, const fc_handle* handles, int nprob, void* cuda_stream, const Tile* fixed) {
  if (!out) return FC_ERR_INVALID;
  *out = nullptr;
  fc_batch B = new (std::nothrow) fc_batch_s();
  if (!B) return FC_ERR_OOM;
  *out = B;
  B->user = (cudaStream_t)cuda_stream;
  if (!handles || nprob < 1) return bfail(B, FC_ERR_INVALID, "empty batch");
  const fc_handle h0 = handles[0];
  if (!h0) return bfail(B, FC_ERR_INVALID, "null handle");
  B->nprob = nprob;
  B->dim = h0->dim;
  B->prec = h0->opt.prec;
  B->f32 = B->prec == FC_PREC_FP32 || B->prec == FC_PREC_BF16;
  B->tc = B->f32 ? h0->opt.tc : 0;
  B->m = h0->restart;
  B->nu_pre = h0->opt.nu_pre;
  B->nu_post = h0->opt.nu_post;
  // each problem's level vectors are the batch's workspace for it
  std::unordered_set<const void*> seen;
  for (int p = 0; p < nprob; ++p) {
    if (!handles[p]) return bfail(B, FC_ERR_INVALID, "null handle");
    if (!seen.insert(handles[p]).second) return bfail(B, FC_ERR_INVALID, "a handle appears twice in the batch");
  }
  for (int p = 0; p < nprob; ++p) {
    const fc_handle h = handles[p];
    if (!h->ready) return bfail(B, FC_ERR_INVALID, "handle not set up (fc_setup failed)");
    if (h->dim != B->dim) return bfail(B, FC_ERR_INVALID, "all problems of a batch must have the same dimension");
    if (h->opt.cache != FC_CACHE_INVERSE || h->opt.prec == FC_PREC_DF64)
      return bfail(B, FC_ERR_INVALID, "batches take cache_inverse handles with fp64, fp32 or bf16 rows");
    if (h->opt.element != 0 || h->opt.amr_uniform >= 0)
      return bfail(B, FC_ERR_INVALID, "batches take Q1-Q1 handles on uniform grids");
    if (h->opt.prec != B->prec || h->restart != B->m || h->opt.nu_pre != B->nu_pre || h->opt.nu_post != B->nu_post)
      return bfail(B, FC_ERR_INVALID, "row precision, FGMRES restart and sweep counts must agree across the batch");
    if (B->f32 && h->opt.tc != B->tc)
      return bfail(B, FC_ERR_INVALID, "the tensor-core mode (fc_options.tc) must agree across the batch");
    B->hs.push_back(h);
    B->maxl = std::max(B->maxl, h->nlev);
  }
  int dev = 0;
  BK(cudaGetDevice(&dev));
  BK(cudaDeviceGetAttribute(&B->nsm, cudaDevAttrMultiProcessorCount, dev));
  BK(cudaStreamCreateWithFlags(&B->s, cudaStreamNonBlocking));
  BK(cudaEventCreateWithFlags(&B->ev, cudaEventDisableTiming));
  for (fc_handle h : B->hs) BK(cudaStreamSynchronize(h->stream));

  // segments: problem p's levels li = 0..L_p-1 in order
  std::vector<BSeg> segs;
  std::vector<int> first(nprob), fin(nprob), cseg(nprob);
  B->off.assign(nprob + 1, 0);
  for (int p = 0; p < nprob; ++p) {
    const fc_handle h = B->hs[p];
    first[p] = (int)segs.size();
    for (int li = 0; li < h->nlev; ++li) {
      const Level& L = h->lev[li];
      BSeg S{};
      for (int k = 0; k < 3; ++k) {
        S.g.n[k] = L.g.n[k];
        S.g.nn[k] = L.g.nn[k];
      }
      S.g.nnodes = L.g.nnodes;
      S.prob = p;
      S.li = li;
      S.omega = h->opt.omega;
      S.st = L.st;
      S.mask = L.mask;
      S.coef = L.coef;
      S.prow = L.prow;
      S.x = L.x;
      S.b = L.b;
      S.r = L.r;
      S.rpad = L.rpad;
      S.rpadf = L.rpad32;
      S.cinv = li == 0 ? h->coarse_inv : nullptr;
      S.cn = li == 0 ? h->coarse_n : 0;
      S.st32 = L.st32;
      S.d32 = L.d32;
      S.b32 = L.b32;
      S.omega_f = (float)h->opt.omega;
      S.cls[0] = L.cls_blk[0];
      S.cls[1] = L.cls_blk[1];
      S.tcA = nullptr;
      if (B->tc && li > 0 && L.coef && (L.cls_blk[0] >= 0 || L.cls_blk[1] >= 0)) {
        void* buf = nullptr;
        BK(cudaMalloc(&buf, tc_bytes(B->dim, B->tc)));
        B->tcbuf.push_back(buf);
        BK(prepare_tc_tile(B->dim, B->tc, B->prec, L.coef, L.cls_blk[0], L.cls_blk[1], buf, B->s));
        S.tcA = buf;
      }
      if (B->f32 && (!L.d32 || !L.b32 || (li > 0 && !L.st32)))
        return bfail(B, FC_ERR_INVALID, "handle without float32 level vectors");
      if (li > 0 && !L.coef) return bfail(B, FC_ERR_INVALID, "handle without a patch cache");
      if (li > 0 && B->prec != FC_PREC_FP64 && !L.rpad32) return bfail(B, FC_ERR_INVALID, "handle without float residual");
      segs.push_back(S);
    }
    fin[p] = first[p] + h->nlev - 1;
    cseg[p] = first[p];
    B->off[p + 1] = B->off[p] + h->lev[h->nlev - 1].g.ndof;
  }
  B->ntot = B->off[nprob];
  B->nseg = (int)segs.size();
  // chunk plans
  std::vector<Chunk> chunks;
  auto add_seg = [&](int sid) {
    const long long nn = segs[sid].g.nnodes;
    for (long long n0 = 0; n0 < nn; n0 += kChunk) chunks.push_back(Chunk{sid, (int)n0});
  };
  B->pn.assign(B->maxl, Plan{});
  B->prc.assign(B->maxl, Plan{});
  for (int li = 0; li < B->maxl; ++li) {
    B->pn[li].first = (int)chunks.size();
    for (int p = 0; p < nprob; ++p)
      if (B->hs[p]->nlev > li) add_seg(first[p] + li);
    B->pn[li].count = (int)chunks.size() - B->pn[li].first;
    B->prc[li].first = (int)chunks.size();
    for (int p = 0; p < nprob; ++p)
      if (B->hs[p]->nlev > li + 1) add_seg(first[p] + li);
    B->prc[li].count = (int)chunks.size() - B->prc[li].first;
  }
  B->pfin.first = (int)chunks.size();
  for (int p = 0; p < nprob; ++p) add_seg(fin[p]);
  B->pfin.count = (int)chunks.size() - B->pfin.first;
  // smoothed finest levels: problems with more than one level (the only
  // level of a one-level problem is the coarse solve's)
  B->psm.first = (int)chunks.size();
  {
    const double cb = B->prec == FC_PREC_FP64 ? 8.0 : B->prec == FC_PREC_FP32 ? 4.0 : 2.0;
    const double rb = B->prec == FC_PREC_FP64 ? 8.0 : 4.0;
    for (int p = 0; p < nprob; ++p)
      if (B->hs[p]->nlev > 1) {
        add_seg(fin[p]);
        const Level& L = B->hs[p]->lev[B->hs[p]->nlev - 1];
        B->fin_patches += L.g.nnodes;
        // stored rows streamed once, residual gathered once, x read and written
        // (float32 correction form: d read and written in float32)
        B->apply_bytes += (double)L.active_work * L.g.nd * cb + (double)L.g.nnodes * L.g.nd * (rb + (B->f32 ? 8.0 : 16.0));
      }
  }
  B->psm.count = (int)chunks.size() - B->psm.first;

  BK(cudaMalloc(&B->segs, sizeof(BSeg) * segs.size()));
  BK(cudaMalloc(&B->fin, sizeof(int) * nprob));
  BK(cudaMalloc(&B->cseg, sizeof(int) * nprob));
  BK(cudaMalloc(&B->doff, sizeof(long long) * (nprob + 1)));
  BK(cudaMalloc(&B->chunks, sizeof(Chunk) * std::max<size_t>(chunks.size(), 1)));
  BK(cudaMemcpyAsync(B->segs, segs.data(), sizeof(BSeg) * segs.size(), cudaMemcpyHostToDevice, B->s));
  BK(cudaMemcpyAsync(B->fin, fin.data(), sizeof(int) * nprob, cudaMemcpyHostToDevice, B->s));
  BK(cudaMemcpyAsync(B->cseg, cseg.data(), sizeof(int) * nprob, cudaMemcpyHostToDevice, B->s));
  BK(cudaMemcpyAsync(B->doff, B->off.data(), sizeof(long long) * (nprob + 1), cudaMemcpyHostToDevice, B->s));
  if (!chunks.empty())
    BK(cudaMemcpyAsync(B->chunks, chunks.data(), sizeof(Chunk) * chunks.size(), cudaMemcpyHostToDevice, B->s));
  // packed work vector (the Krylov basis is allocated by the first solve)
  BK(cudaMalloc(&B->R, sizeof(double) * (size_t)B->ntot));
  if (fixed) {
    B->tile = *fixed;
  } else if (B->tc) {
    // the tensor-core apply has a fixed tile (a warp per 32 nodes of a chunk)
  } else {
    fc_status st = autotune(B);
    if (st != FC_OK) return st;
  }
  BK(cudaStreamSynchronize(B->s));
  return FC_OK;
}

}  // namespace

extern "C" {

fc_status fc_batch_offsets(fc_batch B, long long* offsets) {
  if (!B || !offsets) return FC_ERR_INVALID;
  if (B->off.empty()) return bfail(B, FC_ERR_INVALID, "batch not created");
  for (int p = 0; p <= B->nprob; ++p) offsets[p] = B->off[p];
  return FC_OK;
}

fc_status fc_batch_tile(fc_batch B, int* tpp, int* threads, int* ctas_per_sm) {
  if (!B) return FC_ERR_INVALID;
  if (tpp) *tpp = B->tile.tpp;
  if (threads) *threads = B->tile.threads;
  if (ctas_per_sm) *ctas_per_sm = B->tile.ctas_per_sm;
  return FC_OK;
}

fc_status fc_batch_set_tile(fc_batch B, int tpp, int threads, int ctas_per_sm) {
  if (!B) return FC_ERR_INVALID;
  if ((tpp != 1 && tpp != 2 && tpp != 4 && tpp != 8 && tpp != 16 && tpp != 32) ||
      (threads != 128 && threads != 256 && threads != 512) || threads / tpp > kChunk || ctas_per_sm < 1 ||
      ctas_per_sm > 64)
    return bfail(B, FC_ERR_INVALID,
                 "tile: lanes per patch in {1,2,4,8,16,32}, threads in {128,256,512} with at most 256 patches "
                 "per pass, 1..64 CTAs per SM");
  cudaStreamSynchronize(B->s);
  if (B->step_graph) {
    cudaGraphExecDestroy(B->step_graph);
    B->step_graph = nullptr;
  }
  for (auto& g : B->vgraph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  B->tile = Tile{tpp, threads, ctas_per_sm};
  return FC_OK;
}

fc_status fc_batch_smooth(fc_batch B, double* x, const double* b, int nsweeps) {
  if (!B || !x || !b || nsweeps < 0) return B ? bfail(B, FC_ERR_INVALID, "bad smoother arguments") : FC_ERR_INVALID;
  fc_status st = enter(B);
  if (st == FC_OK) st = point(B, x, 0, b, 0, B->R, nullptr);
  if (st == FC_OK && B->f32) st = fphase(B, 0, B->psm, 0, nullptr, 0);
  if (!B->prof_on) {
    if (st == FC_OK) st = sweeps(B, B->psm, nsweeps, nullptr, 0);
  } else {
    const int out = B->prec == FC_PREC_FP64 ? 1 : 2;
    for (int k = 0; k < nsweeps && st == FC_OK; ++k)
      for (int kind = 1; kind >= 0 && st == FC_OK; --kind) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
          st = bfail(B, FC_ERR_CUDA, "profile event");
          break;
        }
        B->prof[kind].push_back({e0, e1});
        cudaEventRecord(e0, B->s);
        if (kind == 0) st = apply(B, B->psm, B->tile, nullptr, 0);
        else st = B->f32 ? fphase(B, 2, B->psm, 0, nullptr, 0) : residual(B, B->psm, out, 1, nullptr, 0);
        cudaEventRecord(e1, B->s);
      }
  }
  if (st == FC_OK && B->f32) st = fphase(B, 1, B->psm, 0, nullptr, 0);
  return leave(B, st);
}

fc_status fc_batch_vcycle(fc_batch B, double* x, const double* b) {
  if (!B || !x || !b) return B ? bfail(B, FC_ERR_INVALID, "bad V-cycle arguments") : FC_ERR_INVALID;
  fc_status st = enter(B);
  if (st == FC_OK) st = point(B, x, 0, b, 0, B->R, nullptr);
  if (st == FC_OK) st = B->f32 ? vcycle_f32(B, 0, nullptr, 0) : vcycle_all(B, nullptr, 0);
  return leave(B, st);
}

fc_status fc_batch_solve(fc_batch B, const double* b, double* x, double rtol, int maxit, int* iters,
                         double* relres) {
  if (!B || !b || !x || !(rtol > 0.0) || maxit < 0)
    return B ? bfail(B, FC_ERR_INVALID, "bad solve arguments") : FC_ERR_INVALID;
  fc_status st = krylov_alloc(B);
  if (st == FC_OK) st = enter(B);
  if (st != FC_OK) return st;
  KrylovArgs ka{};
  ka.nprob = B->nprob;
  ka.m = B->m;
  ka.maxit = maxit;
  ka.rtol = rtol;
  ka.ntot = B->ntot;
  ka.off = B->doff;
  ka.V = B->V;
  ka.Z = B->Z;
  ka.R = B->R;
  ka.small = B->small;
  ka.bn = B->bn;
  ka.rel = B->rel;
  ka.state = B->state;
  ka.its = B->its;
  ka.kk = B->kk;
  ka.count = B->count;
  ka.dj = B->dj;
  // the captured step bakes in rtol and maxit: recapture when they change
  if (B->step_graph && (B->graph_rtol != rtol || B->graph_maxit != maxit)) {
    cudaGraphExecDestroy(B->step_graph);
    B->step_graph = nullptr;
  }
  st = step_graph(B, ka);
  if (st != FC_OK) return leave(B, st);
  B->graph_rtol = rtol;
  B->graph_maxit = maxit;
  const unsigned kgrid = (unsigned)(B->nprob * kCL);
  k_init_kernel<<<kgrid, kKThreads, 0, B->s>>>(ka, b, x);
  note_launches(1);
  BK(cudaGetLastError());
  while (st == FC_OK) {
    st = point(B, x, 0, b, 0, B->R, nullptr);
    if (st == FC_OK) st = residual(B, B->pfin, 0, 1, B->state, 3);  // R = b - L x
    if (st != FC_OK) break;
    BK(cudaMemsetAsync(B->count, 0, sizeof(int), B->s));
    k_start_kernel<<<kgrid, kKThreads, 0, B->s>>>(ka);
    note_launches(1);
    BK(cudaGetLastError());
    BK(cudaMemcpyAsync(B->hcount, B->count, sizeof(int), cudaMemcpyDeviceToHost, B->s));
    BK(cudaStreamSynchronize(B->s));
    if (*B->hcount == 0) break;
    BK(cudaMemsetAsync(B->dj, 0, sizeof(int), B->s));
    for (int j = 0; j < B->m; ++j) {
      BK(cudaGraphLaunch(B->step_graph, B->s));
      note_launches(B->step_kernels);
      BK(cudaMemcpyAsync(B->hcount, B->count, sizeof(int), cudaMemcpyDeviceToHost, B->s));
      BK(cudaStreamSynchronize(B->s));
      if (*B->hcount == 0) break;
    }
    k_update_kernel<<<kgrid, kKThreads, 0, B->s>>>(ka, x);
    note_launches(1);
    BK(cudaGetLastError());
  }
  if (st != FC_OK) return leave(B, st);
  std::vector<int> hi(B->nprob);
  std::vector<double> hr(B->nprob);
  BK(cudaMemcpyAsync(hi.data(), B->its, sizeof(int) * B->nprob, cudaMemcpyDeviceToHost, B->s));
  BK(cudaMemcpyAsync(hr.data(), B->rel, sizeof(double) * B->nprob, cudaMemcpyDeviceToHost, B->s));
  BK(cudaStreamSynchronize(B->s));
  bool conv = true;
  for (int p = 0; p < B->nprob; ++p) {
    if (iters) iters[p] = hi[p];
    if (relres) relres[p] = hr[p];
    if (hr[p] > rtol) conv = false;
  }
  if (!conv) return leave(B, bfail(B, FC_ERR_NOT_CONVERGED, "some problems reached maxit above rtol"));
  return leave(B, FC_OK);
}

fc_status fc_batch_solve_host(fc_batch B, const double* b_host, double* x_host, double rtol, int maxit,
                              int* iters, double* relres) {
  if (!B || !b_host || !x_host) return B ? bfail(B, FC_ERR_INVALID, "bad solve arguments") : FC_ERR_INVALID;
  if (!B->bh) {
    BK(cudaMalloc(&B->bh, sizeof(double) * B->ntot));
    BK(cudaMalloc(&B->xh, sizeof(double) * B->ntot));
  }
  BK(cudaMemcpyAsync(B->bh, b_host, sizeof(double) * B->ntot, cudaMemcpyHostToDevice, B->user));
  BK(cudaMemcpyAsync(B->xh, x_host, sizeof(double) * B->ntot, cudaMemcpyHostToDevice, B->user));
  fc_status st = fc_batch_solve(B, B->bh, B->xh, rtol, maxit, iters, relres);
  if (st != FC_OK && st != FC_ERR_NOT_CONVERGED) return st;
  BK(cudaMemcpyAsync(x_host, B->xh, sizeof(double) * B->ntot, cudaMemcpyDeviceToHost, B->user));
  BK(cudaStreamSynchronize(B->user));
  return st;
}

fc_status fc_batch_info(fc_batch B, int* nprob, long long* ndof_total, long long* npatch_finest, int* levels_max) {
  if (!B) return FC_ERR_INVALID;
  if (nprob) *nprob = B->nprob;
  if (ndof_total) *ndof_total = B->ntot;
  if (npatch_finest) *npatch_finest = B->fin_patches;
  if (levels_max) *levels_max = B->maxl;
  return FC_OK;
}

fc_status fc_batch_profile_enable(fc_batch B, int on) {
  if (!B) return FC_ERR_INVALID;
  B->prof_on = on != 0;
  return FC_OK;
}

fc_status fc_batch_profile_read(fc_batch B, int kind, long long* launches, double* total_ms,
                                double* bytes_per_launch) {
  if (!B || kind < 0 || kind > 1) return B ? bfail(B, FC_ERR_INVALID, "profile kind is 0 or 1") : FC_ERR_INVALID;
  BK(cudaStreamSynchronize(B->s));
  double ms = 0.0;
  for (auto& pr : B->prof[kind]) {
    float t = 0.0f;
    BK(cudaEventElapsedTime(&t, pr.first, pr.second));
    ms += t;
  }
  if (launches) *launches = (long long)B->prof[kind].size();
  if (total_ms) *total_ms = ms;
  if (bytes_per_launch) *bytes_per_launch = kind == 0 ? B->apply_bytes : 0.0;
  prof_clear(B, kind);
  return FC_OK;
}

fc_status fc_batch_sync(fc_batch B) {
  if (!B) return FC_ERR_INVALID;
  BK(cudaStreamSynchronize(B->s));
  return FC_OK;
}

const char* fc_batch_last_error(fc_batch B) { return B ? B->err.c_str() : "null batch"; }

fc_status fc_batch_destroy(fc_batch B) {
  if (!B) return FC_ERR_INVALID;
  free_batch(B);
  delete B;
  return FC_OK;
}

}  // extern "C"
