// fc_api.cu -- the C-ABI of libfc: handle lifecycle, GPU setup of the
// multigrid hierarchy, smoother / V-cycle / FGMRES drivers, profiling.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "fc_internal.cuh"

using namespace fc;

namespace fc {
static std::atomic<long long> g_launches{0};
static thread_local bool g_capturing = false;
void note_launches(int n) {
  if (!g_capturing) g_launches.fetch_add(n, std::memory_order_relaxed);
}
void set_capturing(bool on) { g_capturing = on; }

cudaError_t persistent_ctas(const void* kern, int threads, size_t smem, int* per_sm, int* nsm) {
  struct Key {
    const void* k;
    int dev, threads;
    size_t smem;
  };
  struct Val {
    int per_sm, nsm;
  };
  static std::mutex mu;
  static std::vector<std::pair<Key, Val>> known;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  for (const auto& kv : known)
    if (kv.first.k == kern && kv.first.dev == dev && kv.first.threads == threads && kv.first.smem == smem) {
      *per_sm = kv.second.per_sm;
      *nsm = kv.second.nsm;
      return cudaSuccess;
    }
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int ps = 0, ns = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, kern, threads, smem);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&ns, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (ps < 1) ps = 1;
  known.push_back({{kern, dev, threads, smem}, {ps, ns}});
  *per_sm = ps;
  *nsm = ns;
  return cudaSuccess;
}
}  // namespace fc

namespace {

constexpr int kSmallScalars = 8;

fc_status fail(fc_handle h, fc_status st, const std::string& msg) {
  if (h) h->err = msg;
  return st;
}

fc_status cuda_fail(fc_handle h, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return fail(h, e == cudaErrorMemoryAllocation ? FC_ERR_OOM : FC_ERR_CUDA, m);
}

#define CK(call)                                         \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

template <typename T>
cudaError_t dalloc(fc_handle h, T** p, size_t count, int part) {
  size_t bytes = count * sizeof(T);
  if (bytes == 0) bytes = sizeof(T);
  // stream-ordered allocation: setup and teardown of one handle do not
  // synchronise the device, so handles on other streams keep running
  cudaError_t e = cudaMallocAsync((void**)p, bytes, h->stream);
  if (e == cudaSuccess && part >= 0) h->bytes[part] += bytes;
  return e;
}

// stream-ordered free of a possibly null pointer
void dfree(fc_handle h, void* p) {
  if (p) cudaFreeAsync(p, h->stream);
}

long long small_len(int m) { return (long long)(m + 1) * m + m + m + (m + 1) + m + kSmallScalars; }
long long small_sc(int m) { return (long long)(m + 1) * m + m + m + (m + 1) + m; }

size_t coef_elem_bytes(fc_prec p) {
  switch (p) {
    case FC_PREC_FP64: return 8;
    case FC_PREC_FP32: return 4;
    case FC_PREC_BF16: return 2;
    case FC_PREC_DF64: return 8;
  }
  return 8;
}

bool need_r32(fc_prec p) { return p != FC_PREC_FP64; }

// ---- profiling helpers --------------------------------------------------
cudaEvent_t prof_event(fc_handle h) {
  if (!h->prof.pool.empty()) {
    cudaEvent_t e = h->prof.pool.back();
    h->prof.pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

struct ProfScope {
  fc_handle h;
  int kind;
  double bytes;
  cudaEvent_t a = nullptr;
  ProfScope(fc_handle hh, int k, double b) : h(hh), kind(k), bytes(b) {
    if (h->prof.on && k >= 0 && !h->capturing) {
      a = prof_event(h);
      cudaEventRecord(a, h->stream);
    }
  }
  ~ProfScope() {
    if (a) {
      cudaEvent_t b = prof_event(h);
      cudaEventRecord(b, h->stream);
      h->prof.recs.push_back({a, b, kind, bytes});
    }
  }
};

}  // namespace

namespace {

__global__ void count_active_kernel(LevelGeom g, const unsigned char* __restrict__ mask,
                                    unsigned long long* __restrict__ out, const int* __restrict__ list,
                                    long long nlist) {
  // number of active (in-grid, unconstrained) patch DoFs summed over the
  // patches of `list` (all patches when list is null) into out[0], and the
  // same count times the patch's free owned DoFs (the rows a patch solve
  // needs: the pressure and the unconstrained velocities of its node) into
  // out[1]
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (list ? nlist : g.nnodes)) return;
  long long i = list ? list[t] : t;
  int ia[3] = {(int)(i % g.nn[0]), (int)((i / g.nn[0]) % g.nn[1]),
               g.dim == 3 ? (int)(i / ((long long)g.nn[0] * g.nn[1])) : 0};
  unsigned long long cnt = 0;
  int r5 = g.dim == 3 ? 5 : 1;
  for (int dz = 0; dz < r5; ++dz)
    for (int dy = 0; dy < 5; ++dy)
      for (int dx = 0; dx < 5; ++dx) {
        int b0 = ia[0] + dx - 2, b1 = ia[1] + dy - 2, b2 = g.dim == 3 ? ia[2] + dz - 2 : 0;
        if (b0 < 0 || b0 > g.n[0] || b1 < 0 || b1 > g.n[1]) continue;
        if (g.dim == 3 && (b2 < 0 || b2 > g.n[2])) continue;
        if (!(mask[b0 + (long long)g.nn[0] * (b1 + (long long)g.nn[1] * b2)] & 1)) cnt += g.dim;
      }
  int r3 = g.dim == 3 ? 3 : 1;
  for (int dz = 0; dz < r3; ++dz)
    for (int dy = 0; dy < 3; ++dy)
      for (int dx = 0; dx < 3; ++dx) {
        int b0 = ia[0] + dx - 1, b1 = ia[1] + dy - 1, b2 = g.dim == 3 ? ia[2] + dz - 1 : 0;
        if (b0 < 0 || b0 > g.n[0] || b1 < 0 || b1 > g.n[1]) continue;
        if (g.dim == 3 && (b2 < 0 || b2 > g.n[2])) continue;
        cnt += 1;
      }
  atomicAdd(out, cnt);
  const unsigned long long owned = (mask[i] & 1) ? 1 : (unsigned long long)(g.dim + 1);
  atomicAdd(out + 1, cnt * owned);
}

// Badly cut patches (fc_options.badcut_frac): among the work-list patches,
// those whose smallest cut-cell fluid fraction over the 4^d cells between
// their velocity nodes (cells i-2 .. i+1 per direction: the cells whose
// element matrices enter L_i) lies below `frac`.  A cell is cut when its
// fluid fraction (fluid volume from the cell quadrature / cell volume) is
// strictly between 0 and 1.  Appends (patch, row block) to the lists.
__global__ void badcut_kernel(LevelGeom g, const double* __restrict__ estat, const int* __restrict__ work,
                              long long nwork, double frac, int* __restrict__ bad_node, int* __restrict__ bad_out,
                              int* __restrict__ nbad) {
  const long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nwork) return;
  const long long i = work ? work[w] : w;
  const int ia[3] = {(int)(i % g.nn[0]), (int)((i / g.nn[0]) % g.nn[1]),
                     g.dim == 3 ? (int)(i / ((long long)g.nn[0] * g.nn[1])) : 0};
  const double vol = g.h[0] * g.h[1] * (g.dim == 3 ? g.h[2] : 1.0);
  double fmin = 2.0;
  const int r = g.dim == 3 ? 4 : 1;
  for (int dz = 0; dz < r; ++dz)
    for (int dy = 0; dy < 4; ++dy)
      for (int dx = 0; dx < 4; ++dx) {
        const int c0 = ia[0] + dx - 2, c1 = ia[1] + dy - 2, c2 = g.dim == 3 ? ia[2] + dz - 2 : 0;
        if (c0 < 0 || c0 >= g.n[0] || c1 < 0 || c1 >= g.n[1]) continue;
        if (g.dim == 3 && (c2 < 0 || c2 >= g.n[2])) continue;
        const long long cell = c0 + (long long)g.n[0] * (c1 + (long long)g.n[1] * c2);
        const double f = estat[cell * 4] / vol;
        if (f > 0.0 && f < 1.0 && f < fmin) fmin = f;
      }
  if (fmin < frac) {
    const int k = atomicAdd(nbad, 1);
    bad_node[k] = (int)i;
    bad_out[k] = (int)w;
  }
}

}  // namespace

namespace {

fc_status check_err(fc_handle h) {
  unsigned e = 0;
  CK(cudaMemcpyAsync(&e, h->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (e & kErrSingularCoarse) return fail(h, FC_ERR_SINGULAR, "coarse operator is singular");
  if (e & kErrSingularPatch) return fail(h, FC_ERR_SINGULAR, "a patch block is singular");
  if (e & kErrTooManyShapes) return fail(h, FC_ERR_INVALID, "more than 64 obstacles meet one cell");
  if (e & kErrBadIndex) return fail(h, FC_ERR_CUDA, "device index check failed");
  return FC_OK;
}

LevelGeom make_geom(const fc_grid* g, int nshape, const Shape* d_shapes, double alpha,
                    const fc_options* o, int coarsen) {
  LevelGeom G;
  memset(&G, 0, sizeof(G));
  G.dim = g->dim;
  G.nd = g->dim + 1;
  G.hmin = 1e300;
  G.ncell = 1;
  G.nnodes = 1;
  for (int k = 0; k < 3; ++k) {
    if (k < g->dim) {
      G.n[k] = g->n[k] >> coarsen;
      G.nn[k] = G.n[k] + 1;
      G.lo[k] = g->lo[k];
      G.hi[k] = g->hi[k];
      G.h[k] = (g->hi[k] - g->lo[k]) / (double)G.n[k];
      if (G.h[k] < G.hmin) G.hmin = G.h[k];
      G.ncell *= G.n[k];
      G.nnodes *= G.nn[k];
    } else {
      G.n[k] = 1;
      G.nn[k] = 1;
      G.lo[k] = 0.0;
      G.hi[k] = 1.0;
      G.h[k] = 1.0;
    }
  }
  G.ndof = G.nnodes * G.nd;
  G.nshape = nshape;
  G.shapes = d_shapes;
  G.alpha = alpha;
  G.eta = o->eta;
  G.lambda = o->nitsche_beta * o->eta / G.hmin;
  G.ubar = o->ubar;
  G.qdepth = o->quad_depth;
  G.preset = o->bc_preset;
  G.force_kind = o->force_kind;
  for (int k = 0; k < 3; ++k) G.force[k] = o->force[k];
  return G;
}

}  // namespace

namespace {

double level_apply_bytes(fc_handle h, int li) {
  const Level& L = h->lev[li];
  double cb = (double)coef_elem_bytes(h->opt.prec);
  double rb = (h->opt.prec == FC_PREC_FP32 || h->opt.prec == FC_PREC_BF16) ? 4.0 : 8.0;
  double act = (double)L.active_work;  // rows streamed: stored blocks, each once
  return act * L.g.nd * cb + (double)L.g.nnodes * L.g.nd * (rb + 16.0);
}

// residual into the smoother's input buffer (format per precision)
fc_status smoother_residual(fc_handle h, int li, const double* x, const double* b) {
  Level& L = h->lev[li];
  ProfScope ps(h, 1, 0.0);
  if (h->opt.cache == FC_CACHE_INVERSE && h->opt.prec == FC_PREC_DF64) {
    CK(launch_residual_df(L.g, L.st, L.mask, x, b, L.rpad32, h->stream));
  } else if (h->opt.cache == FC_CACHE_INVERSE && (h->opt.prec == FC_PREC_FP32 || h->opt.prec == FC_PREC_BF16)) {
    CK(launch_residual_f32(L.g, L.st, L.mask, x, b, L.rpad32, h->stream));
  } else {
    CK(launch_residual(L.g, L.st, L.mask, x, b, nullptr, L.rpad, h->stream));
  }
  return FC_OK;
}

bool pair_path(fc_handle h) { return h->opt.cache == FC_CACHE_INVERSE && h->opt.prec == FC_PREC_DF64; }

// float32 / bfloat16 rows: V-cycles in the float32 correction form
bool f32_path(fc_handle h) {
  return h->opt.cache == FC_CACHE_INVERSE && (h->opt.prec == FC_PREC_FP32 || h->opt.prec == FC_PREC_BF16);
}

// Float-pair smoothing: x and (unless already current) b are split into
// pairs once, then every sweep is a pair residual and a pair apply that
// keeps the pair copy of x current.
fc_status smooth_level_pairs(fc_handle h, int li, double* x, const double* b, int nsweeps, bool b_current) {
  Level& L = h->lev[li];
  if (nsweeps <= 0) return FC_OK;
  CK(launch_split_x_padded(L.g, x, L.xp2, h->stream));
  if (!b_current) CK(launch_split_pairs(L.g.ndof, b, L.bp2, h->stream));
  for (int s = 0; s < nsweeps; ++s) {
    {
      ProfScope ps(h, 1, 0.0);
      CK(launch_residual_df2(L.g, L.st2, L.mask, L.xp2, L.bp2, (float2*)L.rpad32, nullptr, h->stream));
    }
    ProfScope ps(h, 0, level_apply_bytes(h, li));
    ProfScope pf(h, li == h->nlev - 1 ? 4 : -1, level_apply_bytes(h, li));
    CK(launch_patch_apply_df2(L.g, L.coef, L.mask, L.rpad32, h->opt.omega, L.xp2, L.prow, L.cls_blk,
                              h->stream));
  }
  CK(launch_merge_x_padded(L.g, L.xp2, x, h->stream));
  return FC_OK;
}

bool q2_path(fc_handle h);
bool amr_path(fc_handle h);
cudaError_t level_residual(fc_handle h, int li, const double* x, const double* b, double* r);
cudaError_t level_restrict(fc_handle h, int li, const double* rf, double* bc);
cudaError_t level_prolong_add(fc_handle h, int li, const double* ec, double* xf);

fc_status smooth_level(fc_handle h, int li, double* x, const double* b, int nsweeps) {
  Level& L = h->lev[li];
  if (pair_path(h)) return smooth_level_pairs(h, li, x, b, nsweeps, false);
  if (amr_path(h)) {
    for (int s = 0; s < nsweeps; ++s) {
      {
        ProfScope ps(h, 1, 0.0);
        CK(launch_amr_residual(L.amr, x, b, L.r, h->stream));
      }
      ProfScope ps(h, 0, (double)L.coef_bytes);
      ProfScope pf(h, li == h->nlev - 1 ? 4 : -1, (double)L.coef_bytes);
      CK(launch_amr_apply(L.amr, L.r, h->opt.omega, x, h->stream));
    }
    return FC_OK;
  }
  if (q2_path(h)) {
    for (int s = 0; s < nsweeps; ++s) {
      {
        ProfScope ps(h, 1, 0.0);
        CK(launch_q2_residual(h->dim, L.q2, L.q2A, L.q2B, L.q2T, L.q2mask, x, b, nullptr, L.q2rpv, L.q2rpp,
                              h->stream));
      }
      ProfScope ps(h, 0, (double)L.coef_bytes);
      ProfScope pf(h, li == h->nlev - 1 ? 4 : -1, (double)L.coef_bytes);
      CK(launch_q2_apply(h->dim, L.q2, (const double*)L.coef, L.q2mask, L.q2rpv, L.q2rpp, h->opt.omega, x,
                         h->stream));
    }
    return FC_OK;
  }
  for (int s = 0; s < nsweeps; ++s) {
    fc_status st = smoother_residual(h, li, x, b);
    if (st != FC_OK) return st;
    if (h->opt.cache == FC_CACHE_INVERSE) {
      ProfScope ps(h, 0, level_apply_bytes(h, li));
      ProfScope pf(h, li == h->nlev - 1 ? 4 : -1, level_apply_bytes(h, li));
      CK(launch_patch_apply(L.g, h->opt.prec, L.coef, L.mask, L.rpad, L.rpad32, h->opt.omega, x, L.prow,
                            h->stream));
    } else if (h->opt.cache == FC_CACHE_MATRIX) {
      ProfScope ps(h, 0, (double)L.fac_bytes);
      CK(launch_factor_apply(L.g, L.st, factor_store(L), L.mask, L.rpad, h->opt.omega, x, L.prow, h->stream));
    } else {
      ProfScope ps(h, 0, 0.0);
      CK(launch_none_sweep(L.g, L.st, L.mask, h->opt.omega, L.rpad, x, h->d_err, L.lnode, L.nlist, L.ldl_dmin,
                           h->stream));
    }
  }
  return FC_OK;
}

fc_status vcycle_level(fc_handle h, int li, double* x, const double* b);

// Restriction of the finest residual buffer and the whole coarser V-cycle,
// all on buffers fixed per handle: captured once into a CUDA graph (one
// launch per V-cycle instead of one per kernel), replayed afterwards.
fc_status coarse_part(fc_handle h) {
  const int li = h->nlev - 1;
  Level& L = h->lev[li];
  Level& C = h->lev[li - 1];
  if (!h->coarse_graph) {
    cudaGraph_t graph = nullptr;
    h->capturing = true;
    fc::g_capturing = true;
    cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
    fc_status st = FC_OK;
    if (e == cudaSuccess) {
      if (level_restrict(h, li, L.r, C.b) != cudaSuccess ||
          cudaMemsetAsync(C.x, 0, sizeof(double) * C.g.ndof, h->stream) != cudaSuccess)
        st = FC_ERR_CUDA;
      if (st == FC_OK) st = vcycle_level(h, li - 1, C.x, C.b);
      e = cudaStreamEndCapture(h->stream, &graph);
    }
    h->capturing = false;
    fc::g_capturing = false;
    if (e != cudaSuccess || st != FC_OK) {
      if (graph) cudaGraphDestroy(graph);
      return e != cudaSuccess ? cuda_fail(h, e, "V-cycle graph capture") : st;
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
    e = cudaGraphInstantiate(&h->coarse_graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      h->coarse_graph = nullptr;
      return cuda_fail(h, e, "V-cycle graph instantiate");
    }
    h->coarse_graph_kernels = kernels;
  }
  CK(cudaGraphLaunch(h->coarse_graph, h->stream));
  note_launches(h->coarse_graph_kernels);
  return FC_OK;
}

fc_status vcycle_level(fc_handle h, int li, double* x, const double* b) {
  Level& L = h->lev[li];
  if (li == 0) {
    CK(launch_dense_gemv(h->coarse_n, h->coarse_inv, b, x, h->stream));
    return FC_OK;
  }
  Level& C = h->lev[li - 1];
  fc_status st;
  if (pair_path(h)) {
    // b is split once per level visit; x after the pre-sweeps is current in
    // pairs, so the residual for the restriction is a pair residual too
    CK(launch_split_pairs(L.g.ndof, b, L.bp2, h->stream));
    if (h->opt.nu_pre > 0) {
      st = smooth_level_pairs(h, li, x, b, h->opt.nu_pre, true);
      if (st != FC_OK) return st;
    } else {
      CK(launch_split_x_padded(L.g, x, L.xp2, h->stream));
    }
    CK(launch_residual_df2(L.g, L.st2, L.mask, L.xp2, L.bp2, nullptr, L.r, h->stream));
  } else {
    st = smooth_level(h, li, x, b, h->opt.nu_pre);
    if (st != FC_OK) return st;
    CK(level_residual(h, li, x, b, L.r));
  }
  if (li == h->nlev - 1 && h->stream != nullptr && h->stream != cudaStreamLegacy &&
      h->stream != cudaStreamPerThread) {
    // (the legacy default stream cannot be captured; it runs the launches directly)
    st = coarse_part(h);
  } else {
    CK(level_restrict(h, li, L.r, C.b));
    CK(cudaMemsetAsync(C.x, 0, sizeof(double) * C.g.ndof, h->stream));
    st = vcycle_level(h, li - 1, C.x, C.b);
  }
  if (st != FC_OK) return st;
  CK(level_prolong_add(h, li, C.x, x));
  if (pair_path(h)) return smooth_level_pairs(h, li, x, b, h->opt.nu_post, true);
  return smooth_level(h, li, x, b, h->opt.nu_post);
}

// a handle whose fc_setup failed holds partial data: no kernel may run on it
fc_status ready_ok(fc_handle h) {
  if (!h) return FC_ERR_INVALID;
  if (!h->ready) return fail(h, FC_ERR_INVALID, "handle not set up (fc_setup failed)");
  return FC_OK;
}

fc_status level_ok(fc_handle h, int level, int min_level) {
  fc_status st = ready_ok(h);
  if (st != FC_OK) return st;
  if (level < min_level || level > h->nlev) return fail(h, FC_ERR_INVALID, "level out of range");
  return FC_OK;
}

fc_status read_scalar(fc_handle h, const double* dptr, double* out) {
  CK(cudaMemcpyAsync(h->host_small, dptr, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *out = h->host_small[0];
  return FC_OK;
}

bool q2_path(fc_handle h) { return h->opt.element == 1; }
bool amr_path(fc_handle h) { return h->opt.amr_uniform >= 0; }

// ---- operator pieces that depend on the element pair
// r = b - L x (L x when b is null) on level li, unpadded
cudaError_t level_residual(fc_handle h, int li, const double* x, const double* b, double* r) {
  Level& L = h->lev[li];
  if (amr_path(h)) return launch_amr_residual(L.amr, x, b, r, h->stream);
  if (q2_path(h))
    return launch_q2_residual(h->dim, L.q2, L.q2A, L.q2B, L.q2T, L.q2mask, x, b, r, nullptr, nullptr, h->stream);
  return launch_residual(L.g, L.st, L.mask, x, b, r, nullptr, h->stream);
}

cudaError_t level_restrict(fc_handle h, int li, const double* rf, double* bc) {
  Level& L = h->lev[li];
  Level& C = h->lev[li - 1];
  if (amr_path(h)) return launch_amr_restrict(L.amr, C.amr, rf, bc, h->stream);
  if (q2_path(h)) return launch_q2_restrict(h->dim, L.q2, C.q2, C.q2mask, rf, bc, h->stream);
  return launch_restrict(L.g, C.g, C.mask, rf, bc, h->stream);
}

cudaError_t level_prolong_add(fc_handle h, int li, const double* ec, double* xf) {
  Level& L = h->lev[li];
  Level& C = h->lev[li - 1];
  if (amr_path(h)) return launch_amr_prolong_add(L.amr, ec, xf, h->stream);
  if (q2_path(h)) return launch_q2_prolong_add(h->dim, L.q2, C.q2, L.q2mask, ec, xf, h->stream);
  return launch_prolong_add(L.g, C.g, L.mask, ec, xf, h->stream);
}

// FGMRES workspace of the finest level
fc_status alloc_krylov(fc_handle h) {
  const long long n = h->lev[h->nlev - 1].g.ndof;
  const int m = h->restart;
  CK(dalloc(h, &h->V, (size_t)n * (m + 1), 2));
  CK(dalloc(h, &h->Z, (size_t)n * m, 2));
  CK(dalloc(h, &h->w, (size_t)n, 2));
  CK(dalloc(h, &h->red, 2048, 2));
  CK(dalloc(h, &h->small, (size_t)small_len(m), 2));
  CK(dalloc(h, &h->bh, (size_t)n, 2));
  CK(dalloc(h, &h->xh, (size_t)n, 2));
  CK(cudaMallocHost((void**)&h->host_small, sizeof(double) * (size_t)small_len(m)));
  return FC_OK;
}

// Q2-Q1 hierarchy (fc_q2.cu): element data with the Q2 basis, node masks,
// stencil blocks, right-hand side on the finest level, patch rows on every
// level above the coarsest, dense inverse of the coarsest operator
fc_status setup_q2(fc_handle h, const fc_grid* g, const fc_options* o, int nshape, double alpha, int depth) {
  const int dim = g->dim;
  const int nv = dim == 3 ? 27 : 9, np = 1 << dim;
  for (int li = 0; li < depth; ++li) {
    Level& L = h->lev[li];
    L.g = make_geom(g, nshape, h->d_shapes, alpha, o, depth - 1 - li);
    L.q2 = make_q2grid(L.g);
    const Q2Grid& q = L.q2;
    L.g.ndof = q.nq * dim + q.np;
    const LevelGeom& G = L.g;
    const int w5 = dim == 3 ? 125 : 25, w3 = dim == 3 ? 27 : 9;
    double *eA = nullptr, *eB = nullptr, *eF = nullptr;
    CK(dalloc(h, &eA, (size_t)G.ncell * nv * nv, -1));
    CK(dalloc(h, &eB, (size_t)G.ncell * dim * nv * np, -1));
    CK(dalloc(h, &eF, (size_t)G.ncell * dim * nv, -1));
    h->bytes[4] = std::max(h->bytes[4], (size_t)G.ncell * (nv * nv + dim * nv * np + dim * nv) * 8);
    CK(launch_cell_elements_q2(G, eA, eB, eF, nullptr, h->d_err, h->stream));
    CK(dalloc(h, &L.q2mask, (size_t)q.nq, 0));
    CK(dalloc(h, &L.wfix, (size_t)q.nq * dim, 0));
    CK(launch_q2_masks(G, q, L.q2mask, L.wfix, h->stream));
    CK(dalloc(h, &L.q2A, (size_t)w5 * q.nq, 0));
    CK(dalloc(h, &L.q2B, (size_t)w3 * dim * q.nq, 0));
    CK(dalloc(h, &L.q2T, (size_t)w5 * dim * q.np, 0));
    CK(dalloc(h, &L.x, (size_t)G.ndof, 2));
    CK(dalloc(h, &L.b, (size_t)G.ndof, 2));
    CK(dalloc(h, &L.r, (size_t)G.ndof, 2));
    CK(launch_q2_assemble(G, q, eA, eB, eF, L.q2mask, L.wfix, L.q2A, L.q2B, L.q2T,
                          li == depth - 1 ? L.b : nullptr, h->stream));
    long long pv = dim, pp = 1;
    for (int k = 0; k < dim; ++k) {
      pv *= q.nf[k] + 8;
      pp *= q.nv1[k] + 2;
    }
    CK(dalloc(h, &L.q2rpv, (size_t)pv, 2));
    CK(dalloc(h, &L.q2rpp, (size_t)pp, 2));
    CK(cudaMemsetAsync(L.q2rpv, 0, sizeof(double) * pv, h->stream));
    CK(cudaMemsetAsync(L.q2rpp, 0, sizeof(double) * pp, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    dfree(h, eA);
    dfree(h, eB);
    dfree(h, eF);
    fc_status st = check_err(h);
    if (st != FC_OK) return st;
    if (li > 0) {
      const size_t n = (size_t)q.np * q2_patch_rows_doubles(dim);
      double* c64 = nullptr;
      CK(dalloc(h, &c64, n, 1));
      const int ctas = q2_patch_rows_ctas(dim, q.np);
      double* work = nullptr;
      if (ctas > 0) CK(dalloc(h, &work, q2_patch_rows_work_doubles(dim, ctas), -1));
      {
        ProfScope ps(h, 3, 0.0);
        CK(launch_q2_patch_rows(dim, q, L.q2A, L.q2B, L.q2mask, c64, work, ctas, h->d_err, h->stream));
      }
      L.coef = c64;
      L.coef_bytes = n * 8;
      CK(cudaStreamSynchronize(h->stream));
      dfree(h, work);
      st = check_err(h);
      if (st != FC_OK) return st;
    }
  }
  // coarse solve: dense inverse of the coarsest operator
  {
    Level& C = h->lev[0];
    const long long n = C.g.ndof;
    if (n > 4096) return fail(h, FC_ERR_INVALID, "coarsest level too large for the dense solve; increase depth");
    h->coarse_n = (int)n;
    double *work = nullptr, *dsc = nullptr;
    int* piv = nullptr;
    CK(dalloc(h, &work, (size_t)n * n, -1));
    CK(dalloc(h, &dsc, (size_t)2 * n, -1));
    CK(dalloc(h, &piv, (size_t)n, -1));
    CK(dalloc(h, &h->coarse_inv, (size_t)n * n, 3));
    CK(launch_q2_dense(dim, C.q2, C.q2A, C.q2B, C.q2T, C.q2mask, work, h->stream));
    CK(launch_dense_inverse((int)n, work, h->coarse_inv, piv, dsc, h->d_err, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    dfree(h, work);
    dfree(h, dsc);
    dfree(h, piv);
    fc_status st = check_err(h);
    if (st != FC_OK) return st;
  }
  fc_status st = alloc_krylov(h);
  if (st != FC_OK) return st;
  CK(cudaStreamSynchronize(h->stream));
  return FC_OK;
}

// Adaptive hierarchy, quadtrees in 2D and octrees in 3D (fc_amr.cu): trees
// from the finest down (Algorithm 1), per level the nodes and leaves on the
// host, the element data of the leaves on the GPU (the element kernel on the
// uniform grid of each leaf level), the constrained assembly, patches and
// transfers on the host, then the device arrays, the patch rows (levels
// above the coarsest) and the dense inverse of the coarsest operator.
fc_status setup_amr(fc_handle h, const fc_grid* g, const fc_options* o, const std::vector<Shape>& hs, int nshape,
                    double alpha, int depth) {
  const int R = depth - 1, dim = g->dim, NC = 1 << dim;
  const int nroot[3] = {g->n[0] >> R, g->n[1] >> R, dim == 3 ? g->n[2] >> R : 1};
  std::vector<AmrTree> trees(depth);
  trees[depth - 1] = amr_tree_fine(hs, dim, g->lo, g->hi, nroot, o->amr_uniform, R);
  for (int li = depth - 2; li >= 0; --li) trees[li] = amr_tree_coarsen(trees[li + 1]);
  std::vector<AmrHost> H(depth);
  std::vector<std::vector<std::vector<long long>>> adj(depth);
  for (int li = 0; li < depth; ++li)
    if (!amr_structure(trees[li], H[li], adj[li]))
      return fail(h, FC_ERR_INVALID, "adaptive tree with a hanging parent of a hanging node");
  std::vector<int> maxn(depth, 0);
  const size_t wa = (size_t)NC * NC, wb = (size_t)dim * NC * NC, wf = (size_t)dim * NC;
  for (int li = 0; li < depth; ++li) {
    Level& L = h->lev[li];
    L.g = make_geom(g, nshape, h->d_shapes, alpha, o, 0);
    AmrHost& Hl = H[li];
    const size_t nleaf = Hl.leaf.size() / 4;
    std::vector<double> eA(nleaf * wa), eB(nleaf * wb), eF(nleaf * wf);
    for (int r = 0; r <= R; ++r) {
      std::vector<long long> slots;
      std::vector<long long> cells = amr_leaf_cells(trees[li], Hl, r, &slots);
      if (cells.empty()) continue;
      const long long n = (long long)cells.size();
      const LevelGeom Gr = make_geom(g, nshape, h->d_shapes, alpha, o, R - r);
      long long* dcells = nullptr;
      double *dA = nullptr, *dB = nullptr, *dF = nullptr;
      CK(dalloc(h, &dcells, (size_t)n, -1));
      CK(dalloc(h, &dA, (size_t)n * wa, -1));
      CK(dalloc(h, &dB, (size_t)n * wb, -1));
      CK(dalloc(h, &dF, (size_t)n * wf, -1));
      CK(cudaMemcpyAsync(dcells, cells.data(), sizeof(long long) * n, cudaMemcpyHostToDevice, h->stream));
      CK(launch_cell_elements_list(Gr, dcells, n, dA, dB, dF, h->d_err, h->stream));
      std::vector<double> tA((size_t)n * wa), tB((size_t)n * wb), tF((size_t)n * wf);
      CK(cudaMemcpyAsync(tA.data(), dA, sizeof(double) * tA.size(), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaMemcpyAsync(tB.data(), dB, sizeof(double) * tB.size(), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaMemcpyAsync(tF.data(), dF, sizeof(double) * tF.size(), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      for (long long q = 0; q < n; ++q) {
        std::copy(&tA[q * wa], &tA[q * wa] + wa, &eA[slots[q] * wa]);
        std::copy(&tB[q * wb], &tB[q * wb] + wb, &eB[slots[q] * wb]);
        std::copy(&tF[q * wf], &tF[q * wf] + wf, &eF[slots[q] * wf]);
      }
      dfree(h, dcells); dfree(h, dA); dfree(h, dB); dfree(h, dF);
    }
    fc_status st = check_err(h);
    if (st != FC_OK) return st;
    maxn[li] = amr_assemble(trees[li], L.g, eA, eB, eF, adj[li], Hl);
    if (li > 0) amr_transfers(trees[li], Hl, trees[li - 1], H[li - 1]);
    if (maxn[li] > kAmrMaxPatch) return fail(h, FC_ERR_INVALID, "adaptive patch larger than 2048 DoFs");
  }
  for (int li = 0; li < depth; ++li) {
    Level& L = h->lev[li];
    AmrHost& Hl = H[li];
    AmrLevel& A = L.amr;
    A.dim = dim;
    A.nfree = Hl.nfree;
    A.maxn = maxn[li];
    const int nd = dim + 1;
    for (long long i = 0; i < Hl.nfree; ++i) {
      int nvd = 0;
      for (long long t = Hl.pstart[i]; t < Hl.pstart[i + 1]; ++t) nvd += Hl.pdof[t] % nd != dim;
      A.maxnv = std::max(A.maxnv, nvd / dim);
      A.maxnp = std::max(A.maxnp, (int)(Hl.pstart[i + 1] - Hl.pstart[i]) - nvd);
    }
    const long long ndof = Hl.nfree * nd;
    L.g.ndof = ndof;
    L.g.nnodes = Hl.nfree;
    auto up = [&](auto** dst, const auto& v, int part) -> cudaError_t {
      cudaError_t e = dalloc(h, dst, std::max<size_t>(v.size(), 1), part);
      if (e != cudaSuccess || v.empty()) return e;
      return cudaMemcpyAsync(*dst, v.data(), sizeof(v[0]) * v.size(), cudaMemcpyHostToDevice, h->stream);
    };
    CK(up(&A.rowptr, Hl.rowptr, 0));
    CK(up(&A.col, Hl.col, 0));
    CK(up(&A.val, Hl.val, 0));
    CK(up(&A.fixed, Hl.fixed, 0));
    CK(up(&A.pstart, Hl.pstart, 1));
    CK(up(&A.pdof, Hl.pdof, 1));
    CK(up(&A.pown, Hl.pown, 1));
    CK(up(&A.nbp, Hl.nbp, 0));
    CK(up(&A.nbc, Hl.nbc, 0));
    CK(up(&A.nbv, Hl.nbv, 0));
    if (li > 0) {
      CK(up(&A.prp, Hl.prp, 0));
      CK(up(&A.pcl, Hl.pcl, 0));
      CK(up(&A.pvl, Hl.pvl, 0));
      CK(up(&A.rrp, Hl.rrp, 0));
      CK(up(&A.rcl, Hl.rcl, 0));
      CK(up(&A.rvl, Hl.rvl, 0));
    }
    CK(dalloc(h, &L.x, (size_t)ndof, 2));
    CK(dalloc(h, &L.b, (size_t)ndof, 2));
    CK(dalloc(h, &L.r, (size_t)ndof, 2));
    if (li == depth - 1)
      CK(cudaMemcpyAsync(L.b, Hl.rhs.data(), sizeof(double) * ndof, cudaMemcpyHostToDevice, h->stream));
    if (li > 0) {
      const size_t nrows = (size_t)(nd + 1) * Hl.pstart[Hl.nfree];  // slot records of d + 2 doubles
      CK(dalloc(h, &A.rows, nrows, 1));
      const int ctas = amr_patch_rows_ctas(A);
      double* work = nullptr;
      if (ctas > 0) CK(dalloc(h, &work, amr_patch_rows_work_doubles(A, ctas), -1));
      {
        ProfScope ps(h, 3, 0.0);
        CK(launch_amr_patch_rows(A, work, ctas, h->d_err, h->stream));
      }
      L.coef = A.rows;
      L.coef_bytes = nrows * 8;
      unsigned long long act = 0;
      for (long long i = 0; i < Hl.nfree; ++i) {
        int nown = 0;
        for (int c = 0; c < nd; ++c) nown += Hl.pown[i * nd + c] >= 0;
        act += (unsigned long long)(Hl.pstart[i + 1] - Hl.pstart[i]) * nown;
      }
      L.active_rows = act;
      CK(cudaStreamSynchronize(h->stream));
      dfree(h, work);
      fc_status st = check_err(h);
      if (st != FC_OK) return st;
    }
  }
  {
    Level& C = h->lev[0];
    const long long n = C.g.ndof;
    if (n > 4096) return fail(h, FC_ERR_INVALID, "coarsest level too large for the dense solve; increase depth");
    h->coarse_n = (int)n;
    double *work = nullptr, *dsc = nullptr;
    int* piv = nullptr;
    CK(dalloc(h, &work, (size_t)n * n, -1));
    CK(dalloc(h, &dsc, (size_t)2 * n, -1));
    CK(dalloc(h, &piv, (size_t)n, -1));
    CK(dalloc(h, &h->coarse_inv, (size_t)n * n, 3));
    CK(launch_amr_dense(C.amr, work, h->stream));
    CK(launch_dense_inverse((int)n, work, h->coarse_inv, piv, dsc, h->d_err, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    dfree(h, work);
    dfree(h, dsc);
    dfree(h, piv);
    fc_status st = check_err(h);
    if (st != FC_OK) return st;
  }
  fc_status st = alloc_krylov(h);
  if (st != FC_OK) return st;
  CK(cudaStreamSynchronize(h->stream));
  return FC_OK;
}

}  // namespace

extern "C" {

fc_status fc_options_default(fc_options* o) {
  if (!o) return FC_ERR_INVALID;
  memset(o, 0, sizeof(*o));
  o->eta = 1e-3;
  o->nitsche_beta = 100.0;
  o->omega = 0.8;
  o->nu_pre = 2;
  o->nu_post = 2;
  o->quad_depth = 4;
  o->cache = FC_CACHE_INVERSE;
  o->prec = FC_PREC_FP64;
  o->fgmres_restart = 30;
  o->bc_preset = 0;
  o->ubar = 0.3;
  o->force_kind = 0;
  o->dedup = 1;
  o->tc = 0;
  o->badcut_frac = 1e-3;
  o->element = 0;
  o->galerkin = 0;
  o->amr_uniform = -1;
  return FC_OK;
}

size_t fc_footprint_estimate(const fc_grid* g, int depth, const fc_options* o) {
  if (!g || !o || (g->dim != 2 && g->dim != 3) || depth < 1) return 0;
  if (o->element == 1) {
    // Q2-Q1: stencil blocks, masks and Dirichlet values, vectors and padded
    // residuals, patch rows (levels above the coarsest), the element data of
    // a level during setup, the coarse inverse and its elimination pair
    const int dim = g->dim, nv = dim == 3 ? 27 : 9, np = 1 << dim, w5 = dim == 3 ? 125 : 25, w3 = dim == 3 ? 27 : 9;
    size_t held = 0, transient = 0, coarse = 0, fine = 0;
    for (int l = 0; l < depth; ++l) {
      const int c = depth - 1 - l;
      size_t nq = 1, npv = 1, cells = 1, padv = 1, padp = 1;
      for (int k = 0; k < dim; ++k) {
        const size_t n = (size_t)(g->n[k] >> c);
        nq *= 2 * n + 1;
        npv *= n + 1;
        cells *= n;
        padv *= 2 * n + 9;
        padp *= n + 3;
      }
      const size_t ndof = nq * dim + npv;
      if (l == 0) coarse = ndof;
      if (l == depth - 1) fine = ndof;
      held += ((size_t)w5 + (size_t)w3 * dim) * nq * 8 + (size_t)w5 * dim * npv * 8 + nq + nq * dim * 8;
      held += 3 * ndof * 8 + padv * dim * 8 + padp * 8;
      if (l > 0) held += npv * q2_patch_rows_doubles(dim) * 8;
      transient = std::max(transient, cells * ((size_t)nv * nv + (size_t)dim * nv * np + (size_t)dim * nv) * 8);
    }
    held += coarse * coarse * 8;
    transient = std::max(transient, coarse * coarse * 8 + coarse * 24);
    transient = std::max(transient, q2_patch_rows_work_doubles(dim, kQ2Rows3MaxCtas) * 8);
    const int m = o->fgmres_restart > 0 ? o->fgmres_restart : 30;
    held += fine * 8 * (2 * (size_t)m + 4) + 2048 * 8 + (size_t)small_len(m) * 8;
    const size_t total = held + transient;
    return total + total / 50 + (8u << 20);
  }
  const int dim = g->dim, nd = dim + 1, nb = dim == 3 ? 27 : 9, nl = 1 << dim, sp = spn(dim);
  const bool inverse = o->cache == FC_CACHE_INVERSE;
  const bool pairs = inverse && o->prec == FC_PREC_DF64;
  const bool f32 = inverse && (o->prec == FC_PREC_FP32 || o->prec == FC_PREC_BF16);
  // held: what the handle keeps after setup; transient: the largest setup
  // temporary, which coexists with what is held at that point
  size_t held = 0, transient = 0;
  size_t coarse_dof = 0, fine_dof = 0;
  for (int l = 0; l < depth; ++l) {
    const int c = depth - 1 - l;
    size_t nodes = 1, pad = 1, cells = 1;
    for (int k = 0; k < dim; ++k) {
      const size_t n = (size_t)(g->n[k] >> c);
      nodes *= n + 1;
      pad *= n + 5;
      cells *= n;
    }
    const size_t dof = nodes * nd, pv = pad * nd;
    if (l == 0) coarse_dof = dof;
    if (l == depth - 1) fine_dof = dof;
    held += nodes * nb * sp * 8 + nodes + dof * 8;                  // stencil, mask, Dirichlet values
    held += 3 * dof * 8 + pv * 8;                                   // x, b, r, padded residual
    if (pairs && l > 0) held += nodes * (nb / 2 + 1) * sp * 8 + pv * 8 + dof * 8;  // pair half stencil, x, b
    if (need_r32(o->prec)) held += pv * 8;                          // pair / float32 padded residual
    if (f32) held += (l > 0 ? nodes * (nb / 2 + 1) * sp * 4 : 0) + pv * 4 + dof * 4;  // float32 V-cycle
    // class tables and the work list of the patches (every patch may be
    // cut: no sharing is assumed)
    const size_t classes = l > 0 && o->cache != FC_CACHE_NONE ? nodes * 9 + (nodes / 1024 + 1) * 4 : 0;
    // element matrices and cell classes of the level, which live until the
    // patch classes are known
    transient = std::max(transient, cells * ((size_t)nl * nl * (1 + dim) + (size_t)dim * nl) * 8 + cells + classes);
    if (l > 0 && o->cache != FC_CACHE_NONE) {
      held += nodes * 4;                                            // patch -> stored block
      size_t tmp = classes;
      if (inverse) {
        const size_t rows = nodes * nslot(dim) * nd;
        held += rows * coef_elem_bytes(o->prec);
        // reduced-precision rows are built in float64 and converted
        if (o->prec != FC_PREC_FP64) tmp += rows * 8 + nodes * 8;
      } else {
        held += nodes * (factor_doubles(dim) * 8 + factor_ints(dim) * 4);
        // 3D: dense records for the patches whose velocity block is not
        // positive definite (0.19 % at 64^3), counted for 1 % of the
        // patches, and their node list
        if (dim == 3)
          held += (nodes + 99) / 100 * (dense_factor_doubles(dim) * 8 + dense_factor_ints(dim) * 4) + nodes * 8;
      }
      transient = std::max(transient, tmp);
    }
  }
  held += coarse_dof * coarse_dof * 8;                              // coarse inverse
  transient = std::max(transient, coarse_dof * coarse_dof * 8 + coarse_dof * 12);  // its factorisation
  const int m = o->fgmres_restart > 0 ? o->fgmres_restart : 30;
  held += fine_dof * 8 * (2 * (size_t)m + 4) + 2048 * 8 + (size_t)small_len(m) * 8;  // FGMRES
  // error word, shapes, counters, the float32 V-cycle's batch tables and
  // allocator rounding
  const size_t total = held + transient;
  return total + total / 50 + (8u << 20);
}

fc_status fc_setup(fc_handle* out, const fc_grid* g, const fc_levelset* ls, double alpha, int depth,
                   const fc_options* o, void* cuda_stream) {
  if (!out || !g || !o) return FC_ERR_INVALID;
  *out = nullptr;
  fc_handle h = new (std::nothrow) fc_handle_s();
  if (!h) return FC_ERR_OOM;
  *out = h;
  h->opt = *o;
  h->alpha = alpha;
  h->stream = (cudaStream_t)cuda_stream;
  // ---- validation
  if (g->dim != 2 && g->dim != 3) return fail(h, FC_ERR_INVALID, "dim must be 2 or 3");
  if (depth < 1 || depth > kMaxLevels) return fail(h, FC_ERR_INVALID, "depth out of range");
  for (int k = 0; k < g->dim; ++k) {
    if (g->n[k] < 1 || (g->n[k] % (1 << (depth - 1))) != 0)
      return fail(h, FC_ERR_INVALID, "n must be a positive multiple of 2^(depth-1)");
    if (!(g->hi[k] > g->lo[k])) return fail(h, FC_ERR_INVALID, "empty box");
  }
  if (!(alpha > 0.0) || !(o->eta > 0.0) || !(o->omega > 0.0) || o->nu_pre < 0 || o->nu_post < 0 ||
      o->quad_depth < 0 || o->quad_depth > 6 || o->fgmres_restart < 1 || o->fgmres_restart > 256 ||
      o->bc_preset < 0 || o->bc_preset > 2 || o->force_kind < 0 || o->force_kind > 3 ||
      !(o->nitsche_beta >= 0.0) || o->dedup < 0 || o->dedup > 1 || o->tc < 0 || o->tc > 3 ||
      !(o->badcut_frac >= 0.0 && o->badcut_frac < 1.0))
    return fail(h, FC_ERR_INVALID, "invalid options");
  if (o->cache < FC_CACHE_INVERSE || o->cache > FC_CACHE_NONE || o->prec < FC_PREC_FP64 || o->prec > FC_PREC_DF64)
    return fail(h, FC_ERR_INVALID, "invalid cache policy or precision");
  if (o->prec != FC_PREC_FP64 && o->cache != FC_CACHE_INVERSE)
    return fail(h, FC_ERR_INVALID, "reduced-precision storage applies to cache_inverse only");
  if (o->element != 0 && o->element != 1) return fail(h, FC_ERR_INVALID, "invalid element pair");
  if (o->galerkin != 0 && o->galerkin != 1) return fail(h, FC_ERR_INVALID, "invalid coarse-operator choice");
  if (o->amr_uniform < -1 || o->amr_uniform > depth - 1)
    return fail(h, FC_ERR_INVALID, "amr_uniform must be -1 or a level of the hierarchy");
  if (o->amr_uniform >= 0 && (o->element != 0 || o->galerkin || o->cache != FC_CACHE_INVERSE ||
                              o->prec != FC_PREC_FP64))
    return fail(h, FC_ERR_INVALID, "adaptive grids run with the Q1-Q1 pair, cache_inverse and FP64 rows");
  if (o->galerkin && o->element != 0) return fail(h, FC_ERR_INVALID, "Galerkin coarse operators need the Q1-Q1 pair");
  if (o->element == 1 && (o->cache != FC_CACHE_INVERSE || o->prec != FC_PREC_FP64))
    return fail(h, FC_ERR_INVALID, "the Q2-Q1 pair runs with cache_inverse and FP64 rows");
  {
    long long nodes = 1;
    for (int k = 0; k < g->dim; ++k) nodes *= (long long)g->n[k] + 1;
    if (nodes >= (1LL << 30)) return fail(h, FC_ERR_INVALID, "grid too large (2^30 nodes at most)");
  }
  int nshape = ls ? ls->nshapes : 0;
  if (nshape < 0 || (nshape > 0 && !ls->shapes)) return fail(h, FC_ERR_INVALID, "bad level set");
  std::vector<Shape> hs(nshape);
  for (int s = 0; s < nshape; ++s) {
    const fc_shape& in = ls->shapes[s];
    if (in.type != 0 && !(in.type == 1 && g->dim == 2)) return fail(h, FC_ERR_INVALID, "unsupported shape type");
    if (!(in.r[0] > 0.0) || (in.type == 1 && !(in.r[1] > 0.0))) return fail(h, FC_ERR_INVALID, "bad radius");
    Shape& S = hs[s];
    S.type = in.type;
    for (int k = 0; k < 3; ++k) { S.c[k] = in.c[k]; S.r[k] = in.r[k]; }
    S.rot[0] = in.type == 1 ? in.rot[0] : 1.0;
    S.rot[1] = in.type == 1 ? in.rot[1] : 0.0;
    S.bbr = in.type == 0 ? in.r[0] : std::max(in.r[0], in.r[1]);
  }
  h->dim = g->dim;
  h->nlev = depth;
  h->restart = o->fgmres_restart;
  CK(cudaGetDevice(&h->device));
  h->nshape = nshape;

  CK(dalloc(h, &h->d_err, 1, 2));
  CK(cudaMemsetAsync(h->d_err, 0, sizeof(unsigned), h->stream));
  CK(dalloc(h, &h->d_shapes, (size_t)std::max(nshape, 1), 0));
  if (nshape) CK(cudaMemcpyAsync(h->d_shapes, hs.data(), sizeof(Shape) * nshape, cudaMemcpyHostToDevice, h->stream));
  if (o->element == 1) {
    fc_status st = setup_q2(h, g, o, nshape, alpha, depth);
    if (st != FC_OK) return st;
    h->ready = true;
    return FC_OK;
  }
  if (o->amr_uniform >= 0) {
    fc_status st = setup_amr(h, g, o, hs, nshape, alpha, depth);
    if (st != FC_OK) return st;
    h->ready = true;
    return FC_OK;
  }
  unsigned long long* d_count = nullptr;
  CK(dalloc(h, &d_count, 2, -1));

  const int dim = g->dim, nd = dim + 1, nb = dim == 3 ? 27 : 9, nl = 1 << dim;
  // Galerkin coarse operators: the levels are built from the finest down,
  // each coarser operator as R L P of the one above it (no quadrature on
  // the coarser grids); the finer level's cell classes and statistics are
  // kept for the next level's
  const bool galerkin = o->galerkin != 0;
  unsigned char* fine_cclass = nullptr;
  double* fine_estat = nullptr;
  for (int step = 0; step < depth; ++step) {
    const int li = galerkin ? depth - 1 - step : step;
    const bool gal = galerkin && li < depth - 1;
    Level& L = h->lev[li];
    L.g = make_geom(g, nshape, h->d_shapes, alpha, o, depth - 1 - li);
    const LevelGeom& G = L.g;
    // ---- element data and operator
    double *eA = nullptr, *eB = nullptr, *eF = nullptr;
    if (!gal) {
      CK(dalloc(h, &eA, (size_t)G.ncell * nl * nl, -1));
      CK(dalloc(h, &eB, (size_t)G.ncell * dim * nl * nl, -1));
      CK(dalloc(h, &eF, (size_t)G.ncell * dim * nl, -1));
      size_t tmp_bytes = (size_t)G.ncell * (nl * nl * (1 + dim) + dim * nl) * 8;
      h->bytes[4] = std::max(h->bytes[4], tmp_bytes);
    }
    // reference element matrices of an uncut cell of this level (alpha = 1,
    // same rule), then all cells; plain cells take alpha * reference
    double *rA = nullptr, *rB = nullptr, *rF = nullptr;
    unsigned char* cclass = nullptr;
    CK(dalloc(h, &cclass, (size_t)G.ncell, -1));
    if (!gal) {
      CK(dalloc(h, &rA, (size_t)nl * nl, -1));
      CK(dalloc(h, &rB, (size_t)dim * nl * nl, -1));
      CK(dalloc(h, &rF, (size_t)dim * nl, -1));
    }
    if (!gal) {
      LevelGeom R = G;
      R.ncell = 1;
      R.nnodes = 1;
      for (int k = 0; k < dim; ++k) {
        R.n[k] = 1;
        R.nn[k] = 2;
        R.lo[k] = 0.0;
        R.hi[k] = G.h[k];
        R.nnodes *= 2;
      }
      R.ndof = R.nnodes * nd;
      R.nshape = 0;
      R.force_kind = 0;
      R.force[0] = R.force[1] = R.force[2] = 0.0;
      CK(launch_cell_elements(R, rA, rB, rF, nullptr, h->d_err, nullptr, nullptr, nullptr, h->stream));
    }
    // cell fluid volumes for the bad-cut rule (float32 / bfloat16 rows)
    const bool badcut = li > 0 && o->cache == FC_CACHE_INVERSE && o->badcut_frac > 0.0 &&
                        (o->prec == FC_PREC_FP32 || o->prec == FC_PREC_BF16);
    double* estat = nullptr;
    if (badcut) CK(dalloc(h, &estat, (size_t)G.ncell * 4, -1));
    if (!gal)
      CK(launch_cell_elements(G, eA, eB, eF, estat, h->d_err, rA, rB, cclass, h->stream));
    else
      CK(launch_coarsen_cells(G, h->lev[li + 1].g, fine_cclass, cclass, estat ? fine_estat : nullptr, estat,
                              h->stream));
    CK(dalloc(h, &L.st, (size_t)G.nnodes * nb * spn(dim), 0));
    CK(dalloc(h, &L.mask, (size_t)G.nnodes, 0));
    CK(dalloc(h, &L.wfix, (size_t)G.ndof, 0));
    if (!gal) CK(launch_assemble(G, eA, eB, L.st, h->stream));
    else CK(launch_galerkin(G, h->lev[li + 1].g, h->lev[li + 1].st, h->lev[li + 1].mask, L.st, h->stream));
    CK(launch_masks(G, L.mask, L.wfix, h->stream));
    if (dim == 3 && li > 0) {
      CK(dalloc(h, &L.dead, (size_t)G.nn[0] + G.nn[1] + G.nn[2], 0));
      CK(launch_dead_layers(G, L.mask, L.dead, h->stream));
      L.g.dead_layer = L.dead;
    }
    // ---- vectors
    long long padn = pad_nodes(G);
    CK(dalloc(h, &L.x, (size_t)G.ndof, 2));
    CK(dalloc(h, &L.b, (size_t)G.ndof, 2));
    CK(dalloc(h, &L.r, (size_t)G.ndof, 2));
    CK(dalloc(h, &L.rpad, (size_t)padn * nd, 2));
    CK(cudaMemsetAsync(L.rpad, 0, sizeof(double) * padn * nd, h->stream));
    if (li > 0 && o->cache == FC_CACHE_INVERSE && o->prec == FC_PREC_DF64) {
      // half pair stencil: the zero offset and the offsets after it (the
      // operator is symmetric; the residual reads the others transposed)
      size_t nst = (size_t)G.nnodes * (nb / 2 + 1) * spn(dim);
      CK(dalloc(h, &L.st2, nst, 0));
      CK(launch_fold_stencil_pairs(G, L.st, L.mask, L.st2, h->stream));
      CK(dalloc(h, &L.xp2, (size_t)pad_nodes(G) * nd, 2));
      CK(cudaMemsetAsync(L.xp2, 0, sizeof(float2) * pad_nodes(G) * nd, h->stream));
      CK(dalloc(h, &L.bp2, (size_t)G.ndof, 2));
    }
    if (need_r32(o->prec)) {
      CK(dalloc(h, &L.rpad32, (size_t)padn * nd * 2, 2));
      CK(cudaMemsetAsync(L.rpad32, 0, sizeof(float) * padn * nd * 2, h->stream));
    }
    if (o->cache == FC_CACHE_INVERSE && (o->prec == FC_PREC_FP32 || o->prec == FC_PREC_BF16)) {
      // float32 correction-form V-cycle: folded float32 stencil, padded
      // correction (zero halo) and float32 right-hand side
      if (li > 0) {
        CK(dalloc(h, &L.st32, (size_t)G.nnodes * (nb / 2 + 1) * spn(dim), 0));  // half stencil
        CK(launch_fold_stencil_f32(G, L.st, L.mask, L.st32, h->stream));
      }
      CK(dalloc(h, &L.d32, (size_t)padn * nd, 2));
      CK(cudaMemsetAsync(L.d32, 0, sizeof(float) * padn * nd, h->stream));
      CK(dalloc(h, &L.b32, (size_t)G.ndof, 2));
    }
    if (li == depth - 1) {
      // finest right-hand side kept in L.b until fc_rhs; L.b is not used as a
      // V-cycle buffer on the finest level
      CK(launch_rhs(G, eF, L.st, L.mask, L.wfix, L.b, h->stream));
    }
    // ---- patch classes and the work list (patches factored and stored)
    int* work = nullptr;
    int* dnw = nullptr;
    if (li > 0 && o->cache != FC_CACHE_NONE) {
      unsigned char* nclass = nullptr;
      int* pclass = nullptr;
      int* rep = nullptr;
      const long long nbk = (G.nnodes + 1023) / 1024;
      CK(dalloc(h, &nclass, (size_t)G.nnodes, -1));
      CK(dalloc(h, &pclass, (size_t)G.nnodes, -1));
      CK(dalloc(h, &rep, 4, -1));
      CK(dalloc(h, &work, (size_t)(G.nnodes + nbk), -1));
      CK(dalloc(h, &dnw, 1, -1));
      CK(dalloc(h, &L.prow, (size_t)G.nnodes, 1));
      CK(launch_patch_classes(G, cclass, L.mask, nclass, pclass, rep, work, dnw, L.prow, o->dedup,
                              h->stream));
      CK(cudaMemcpyAsync(&L.nwork, dnw, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
      int reph[4] = {0, 0, 0, 0};
      CK(cudaMemcpyAsync(reph, rep, sizeof(reph), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      for (int c = 1; c <= 2; ++c) {
        if (reph[c] == 0x7fffffff) continue;
        int pr = 0;
        CK(cudaMemcpy(&pr, L.prow + reph[c], sizeof(int), cudaMemcpyDeviceToHost));
        L.cls_blk[c - 1] = pr < 0 ? -pr - 1 : -1;
      }
      dfree(h, nclass);
      dfree(h, pclass);
      dfree(h, rep);
    }
    CK(cudaStreamSynchronize(h->stream));
    dfree(h, eA);
    dfree(h, eB);
    dfree(h, eF);
    dfree(h, rA);
    dfree(h, rB);
    dfree(h, rF);
    if (galerkin) {
      dfree(h, fine_cclass);
      fine_cclass = cclass;
    } else {
      dfree(h, cclass);
    }
    fc_status st = check_err(h);
    if (st != FC_OK) return st;
    // ---- patch cache (every level above the coarsest)
    if (li > 0) {
      for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1 && !work) break;
        CK(cudaMemsetAsync(d_count, 0, 2 * sizeof(unsigned long long), h->stream));
        const long long cnt_n = pass == 0 ? G.nnodes : L.nwork;
        count_active_kernel<<<(unsigned)((cnt_n + 255) / 256), 256, 0, h->stream>>>(
            G, L.mask, d_count, pass == 0 ? nullptr : work, cnt_n);
        CK(cudaGetLastError());
        note_launches(1);
        unsigned long long cnt[2] = {0, 0};
        CK(cudaMemcpyAsync(cnt, d_count, sizeof(cnt), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        if (pass == 0) {
          L.active_slots = cnt[0];
          L.active_rows = cnt[1];
        } else {
          L.active_work = cnt[0];
        }
      }
      if (o->cache == FC_CACHE_INVERSE) {
        size_t n = (size_t)L.nwork * nslot(dim) * nd;
        double* c64 = nullptr;
        CK(dalloc(h, &c64, n, o->prec == FC_PREC_FP64 ? 1 : -1));
        {
          ProfScope ps(h, 3, 0.0);
          if (dim == 3) {
            // banded LDL^T of the velocity block in FP64; patches whose block
            // is not positive definite are redone by the pivoted dense LU.
            // Float-pair, float32 and bfloat16 rows are these FP64 rows split
            // or rounded: in 3D the FP64 band factorisation is cheaper per
            // patch than the float-pair elimination and than the float32
            // dense LU with refinement, so every patch, the badly cut ones
            // included, is factored in FP64.
            const long long nw = work ? L.nwork : G.nnodes;
            int *redo_node = nullptr, *redo_out = nullptr, *nredo = nullptr;
            CK(dalloc(h, &redo_node, (size_t)std::max(nw, 1LL), -1));
            CK(dalloc(h, &redo_out, (size_t)std::max(nw, 1LL), -1));
            CK(dalloc(h, &nredo, 1, -1));
            CK(cudaMemsetAsync(nredo, 0, sizeof(int), h->stream));
            CK(launch_patch_rows_ldl(G, L.st, L.mask, c64, h->d_err, work, L.nwork, redo_node, redo_out, nredo,
                                     h->stream));
            int nr = 0;
            CK(cudaMemcpyAsync(&nr, nredo, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            if (nr > 0)
              CK(launch_patch_rows_dense_redo(G, L.st, L.mask, c64, h->d_err, redo_node, nr, redo_out, h->stream));
            h->ldl_fallback += nr;
            if (estat) {
              // the bad-cut rule's patches, counted (their rows are FP64 already)
              CK(cudaMemsetAsync(nredo, 0, sizeof(int), h->stream));
              badcut_kernel<<<(unsigned)((nw + 255) / 256), 256, 0, h->stream>>>(G, estat, work, nw, o->badcut_frac,
                                                                               redo_node, redo_out, nredo);
              CK(cudaGetLastError());
              note_launches(1);
              int nb = 0;
              CK(cudaMemcpyAsync(&nb, nredo, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
              CK(cudaStreamSynchronize(h->stream));
              h->badcut += nb;
            }
            dfree(h, redo_node);
            dfree(h, redo_out);
            dfree(h, nredo);
          } else if (o->prec == FC_PREC_FP64)
            CK(launch_patch_build(G, L.st, L.mask, 0, o->omega, c64, nullptr, nullptr, nullptr, nullptr,
                                  h->d_err, work, L.nwork, h->stream));
          else if (o->prec == FC_PREC_DF64)  // rows kept as float pairs: float-pair factorisation
            CK(launch_patch_rows_pair(G, L.st, L.mask, c64, h->d_err, work, L.nwork, nullptr, h->stream));
          else {  // float32 / bfloat16 rows: float32 factors and iterative refinement
            const long long nw = work ? L.nwork : G.nnodes;
            int *redo_node = nullptr, *redo_out = nullptr, *nredo = nullptr;
            CK(dalloc(h, &redo_node, (size_t)std::max(nw, 1LL), -1));
            CK(dalloc(h, &redo_out, (size_t)std::max(nw, 1LL), -1));
            CK(dalloc(h, &nredo, 1, -1));
            CK(cudaMemsetAsync(nredo, 0, sizeof(int), h->stream));
            CK(launch_patch_rows_ir(G, L.st, L.mask, c64, h->d_err, work, L.nwork, redo_node, redo_out, nredo,
                                    h->stream));
            int nr = 0;
            CK(cudaMemcpyAsync(&nr, nredo, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            // patches whose float32 refinement did not converge: float pairs
            if (nr > 0)
              CK(launch_patch_rows_pair(G, L.st, L.mask, c64, h->d_err, redo_node, nr, redo_out, h->stream));
            h->pair_fallback += nr;
            if (estat) {
              // badly cut patches: float pairs whatever the refinement did
              CK(cudaMemsetAsync(nredo, 0, sizeof(int), h->stream));
              badcut_kernel<<<(unsigned)((nw + 255) / 256), 256, 0, h->stream>>>(G, estat, work, nw, o->badcut_frac,
                                                                               redo_node, redo_out, nredo);
              CK(cudaGetLastError());
              note_launches(1);
              int nb = 0;
              CK(cudaMemcpyAsync(&nb, nredo, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
              CK(cudaStreamSynchronize(h->stream));
              if (nb > 0)
                CK(launch_patch_rows_pair(G, L.st, L.mask, c64, h->d_err, redo_node, nb, redo_out, h->stream));
              h->badcut += nb;
            }
            dfree(h, redo_node);
            dfree(h, redo_out);
            dfree(h, nredo);
          }
        }
        if (o->prec == FC_PREC_FP64) {
          L.coef = c64;
          L.coef_bytes = n * 8;
        } else {
          size_t eb = coef_elem_bytes(o->prec);
          void* cv = nullptr;
          CK(cudaMallocAsync(&cv, n * eb, h->stream));
          h->bytes[1] += n * eb;
          CK(launch_convert_rows(G, o->prec, c64, cv, L.nwork, h->stream));
          CK(cudaStreamSynchronize(h->stream));
          dfree(h, c64);
          L.coef = cv;
          L.coef_bytes = n * eb;
        }
      } else if (o->cache == FC_CACHE_MATRIX) {
        CK(dalloc(h, &L.fac, (size_t)L.nwork * factor_doubles(dim), 1));
        CK(dalloc(h, &L.fpiv, (size_t)L.nwork * factor_ints(dim), 1));
        L.fac_bytes = (size_t)L.nwork * (factor_doubles(dim) * 8 + factor_ints(dim) * 4);
        ProfScope ps(h, 3, 0.0);
        if (dim == 3) {
          // band factor records by the banded LDL^T; the patches whose
          // velocity block is not positive definite get dense records
          const long long nw = work ? L.nwork : G.nnodes;
          int *rn = nullptr, *ro = nullptr, *nr_d = nullptr;
          CK(dalloc(h, &rn, (size_t)std::max(nw, 1LL), -1));
          CK(dalloc(h, &ro, (size_t)std::max(nw, 1LL), -1));
          CK(dalloc(h, &nr_d, 1, -1));
          CK(cudaMemsetAsync(nr_d, 0, sizeof(int), h->stream));
          CK(launch_band_factors(G, L.st, L.mask, L.fac, L.fpiv, h->d_err, work, L.nwork, rn, ro, nr_d, h->stream));
          int nr = 0;
          CK(cudaMemcpyAsync(&nr, nr_d, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
          CK(cudaStreamSynchronize(h->stream));
          if (nr > 0) {
            CK(dalloc(h, &L.facd, (size_t)nr * dense_factor_doubles(dim), 1));
            CK(dalloc(h, &L.fpivd, (size_t)nr * dense_factor_ints(dim), 1));
            L.fac_bytes += (size_t)nr * (dense_factor_doubles(dim) * 8 + dense_factor_ints(dim) * 4);
            CK(launch_dense_factor_redo(G, L.st, L.mask, L.facd, L.fpivd, h->d_err, rn, ro, nr, L.fpiv, h->stream));
            CK(dalloc(h, &L.lnode, (size_t)G.nnodes, 1));
            CK(dalloc(h, &L.lrec, (size_t)G.nnodes, 1));
            CK(cudaMemsetAsync(nr_d, 0, sizeof(int), h->stream));
            CK(launch_dense_list(G, L.prow, L.fpiv, L.lnode, L.lrec, nr_d, h->stream));
            int nl = 0;
            CK(cudaMemcpyAsync(&nl, nr_d, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
            CK(cudaStreamSynchronize(h->stream));
            L.nlist = nl;
          }
          h->ldl_fallback += nr;
          dfree(h, rn);
          dfree(h, ro);
          dfree(h, nr_d);
        } else {
          CK(launch_patch_build(G, L.st, L.mask, 1, o->omega, nullptr, L.fac, L.fpiv, nullptr, nullptr,
                                h->d_err, work, L.nwork, h->stream));
        }
      } else if (dim == 3) {
        // cache_none: list once the patches whose velocity block is not
        // positive definite; every sweep solves them by the dense LU
        int *rn = nullptr, *ro = nullptr, *nr_d = nullptr;
        CK(dalloc(h, &rn, (size_t)G.nnodes, -1));
        CK(dalloc(h, &ro, (size_t)G.nnodes, -1));
        CK(dalloc(h, &nr_d, 1, -1));
        CK(cudaMemsetAsync(nr_d, 0, sizeof(int), h->stream));
        L.ldl_dmin = ldl_min_pivot();
        CK(launch_none_check(G, L.st, L.mask, h->d_err, rn, ro, nr_d, L.ldl_dmin, h->stream));
        int nr = 0;
        CK(cudaMemcpyAsync(&nr, nr_d, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        if (nr > 0) {
          CK(dalloc(h, &L.lnode, (size_t)nr, 1));
          CK(cudaMemcpyAsync(L.lnode, rn, sizeof(int) * nr, cudaMemcpyDeviceToDevice, h->stream));
          L.nlist = nr;
        }
        h->ldl_fallback += nr;
        CK(cudaStreamSynchronize(h->stream));
        dfree(h, rn);
        dfree(h, ro);
        dfree(h, nr_d);
      }
      CK(cudaStreamSynchronize(h->stream));
      dfree(h, work);
      dfree(h, dnw);
      st = check_err(h);
      if (st != FC_OK) return st;
    }
    if (galerkin) {
      dfree(h, fine_estat);
      fine_estat = estat;
    } else {
      dfree(h, estat);
    }
  }
  dfree(h, fine_cclass);
  dfree(h, fine_estat);
  dfree(h, d_count);
  // ---- coarse solve
  {
    Level& C = h->lev[0];
    long long n = C.g.ndof;
    if (n > 4096) return fail(h, FC_ERR_INVALID, "coarsest level too large for the dense solve; increase depth");
    h->coarse_n = (int)n;
    double* work = nullptr;
    double* dsc = nullptr;
    int* piv = nullptr;
    CK(dalloc(h, &work, (size_t)n * n, -1));
    CK(dalloc(h, &dsc, (size_t)2 * n, -1));  // scaling and the elimination's column factors
    CK(dalloc(h, &piv, (size_t)n, -1));
    CK(dalloc(h, &h->coarse_inv, (size_t)n * n, 3));
    CK(launch_coarse_factor(C.g, C.st, C.mask, work, h->coarse_inv, piv, dsc, h->d_err, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    dfree(h, work);
    dfree(h, dsc);
    dfree(h, piv);
    fc_status st = check_err(h);
    if (st != FC_OK) return st;
  }
  // ---- FGMRES workspace
  {
    fc_status st = alloc_krylov(h);
    if (st != FC_OK) return st;
  }
  CK(cudaStreamSynchronize(h->stream));
  h->ready = true;
  return FC_OK;
}

fc_status fc_rhs(fc_handle h, double* b_dev) {
  fc_status st = ready_ok(h);
  if (st != FC_OK) return st;
  if (!b_dev) return fail(h, FC_ERR_INVALID, "null vector");
  Level& L = h->lev[h->nlev - 1];
  CK(cudaMemcpyAsync(b_dev, L.b, sizeof(double) * L.g.ndof, cudaMemcpyDeviceToDevice, h->stream));
  return FC_OK;
}

fc_status fc_residual(fc_handle h, int level, const double* x, const double* b, double* r) {
  fc_status st = level_ok(h, level, 1);
  if (st != FC_OK) return st;
  if (!x || !b || !r) return fail(h, FC_ERR_INVALID, "null vector");
  CK(level_residual(h, level - 1, x, b, r));
  return FC_OK;
}

fc_status fc_apply(fc_handle h, int level, const double* x, double* y) {
  fc_status st = level_ok(h, level, 1);
  if (st != FC_OK) return st;
  if (!x || !y) return fail(h, FC_ERR_INVALID, "null vector");
  CK(level_residual(h, level - 1, x, nullptr, y));
  return FC_OK;
}

fc_status fc_smooth(fc_handle h, int level, double* x, const double* b, int nsweeps) {
  fc_status st = level_ok(h, level, 2);
  if (st != FC_OK) return st;
  if (!x || !b || nsweeps < 0) return fail(h, FC_ERR_INVALID, "bad smoother arguments");
  return smooth_level(h, level - 1, x, b, nsweeps);
}

fc_status fc_restrict(fc_handle h, int level, const double* rf, double* bc) {
  fc_status st = level_ok(h, level, 2);
  if (st != FC_OK) return st;
  if (!rf || !bc) return fail(h, FC_ERR_INVALID, "null vector");
  CK(level_restrict(h, level - 1, rf, bc));
  return FC_OK;
}

fc_status fc_prolong_add(fc_handle h, int level, const double* ec, double* xf) {
  fc_status st = level_ok(h, level, 2);
  if (st != FC_OK) return st;
  if (!ec || !xf) return fail(h, FC_ERR_INVALID, "null vector");
  CK(level_prolong_add(h, level - 1, ec, xf));
  return FC_OK;
}

fc_status fc_coarse_solve(fc_handle h, const double* b, double* x) {
  fc_status st = ready_ok(h);
  if (st != FC_OK) return st;
  if (!b || !x) return fail(h, FC_ERR_INVALID, "null vector");
  CK(launch_dense_gemv(h->coarse_n, h->coarse_inv, b, x, h->stream));
  return FC_OK;
}

fc_status fc_vcycle(fc_handle h, double* x, const double* b) {
  fc_status st = ready_ok(h);
  if (st != FC_OK) return st;
  if (!x || !b) return fail(h, FC_ERR_INVALID, "null vector");
  ProfScope ps(h, 2, 0.0);
  if (f32_path(h)) return handle_vcycle_f32(h, x, b, false);
  return vcycle_level(h, h->nlev - 1, x, b);
}

fc_status fc_solve(fc_handle h, const double* b, double* x, double rtol, int maxit, int* iters,
                   double* relres) {
  const fc_status rs = ready_ok(h);
  if (rs != FC_OK) return rs;
  if (!b || !x || !(rtol > 0.0) || maxit < 0) return fail(h, FC_ERR_INVALID, "bad solve arguments");
  Level& F = h->lev[h->nlev - 1];
  const long long n = F.g.ndof;
  const int m = h->restart;
  cudaStream_t s = h->stream;
  double* H = h->small;
  double* g = H + (long long)(m + 1) * m + m + m;
  double* sc = H + small_sc(m);
  double bn2 = 0.0;
  CK(launch_dot(n, b, b, h->red, sc + 1, s));
  fc_status st = read_scalar(h, sc + 1, &bn2);
  if (st != FC_OK) return st;
  double bn = sqrt(bn2);
  int its = 0;
  double rel = 0.0;
  if (bn == 0.0) {
    CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    CK(cudaStreamSynchronize(s));
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    return FC_OK;
  }
  for (;;) {
    CK(level_residual(h, h->nlev - 1, x, b, h->w));
    double beta2 = 0.0;
    CK(launch_dot(n, h->w, h->w, h->red, sc + 1, s));
    st = read_scalar(h, sc + 1, &beta2);
    if (st != FC_OK) return st;
    double beta = sqrt(beta2);
    rel = beta / bn;
    if (beta <= rtol * bn || its >= maxit) break;
    // g = (beta, 0, ...); V_0 = w / beta
    for (int t = 0; t <= m; ++t) h->host_small[t] = t == 0 ? beta : 0.0;
    CK(cudaMemcpyAsync(g, h->host_small, sizeof(double) * (m + 1), cudaMemcpyHostToDevice, s));
    CK(launch_scale_copy(n, g, 0, 1, h->w, h->V, s));
    int k = 0;
    for (int j = 0; j < m && its < maxit; ++j) {
      double* Vj = h->V + (long long)j * n;
      double* Zj = h->Z + (long long)j * n;
      CK(cudaMemsetAsync(Zj, 0, sizeof(double) * n, s));
      {
        ProfScope ps(h, 2, 0.0);
        st = f32_path(h) ? handle_vcycle_f32(h, Zj, Vj, true) : vcycle_level(h, h->nlev - 1, Zj, Vj);
        if (st != FC_OK) return st;
      }
      its++;
      CK(level_residual(h, h->nlev - 1, Zj, nullptr, h->w));
      // modified Gram-Schmidt, one fused kernel per step: step i finishes
      // h_{i-1,j} from the block partials, subtracts it and starts the dot
      // with v_i; the last two steps give the norm and v_{j+1}
      double* pa = h->red;
      double* pb = h->red + 1024;
      CK(launch_mgs_fused(n, h->w, nullptr, nullptr, nullptr, h->V, pa, 0, nullptr, nullptr, s));
      for (int i = 1; i <= j + 1; ++i) {
        const double* vnext = i <= j ? h->V + (long long)i * n : nullptr;
        CK(launch_mgs_fused(n, h->w, h->V + (long long)(i - 1) * n, pa, H + (long long)(i - 1) * m + j, vnext,
                            pb, 0, nullptr, nullptr, s));
        std::swap(pa, pb);
      }
      double* hn = H + (long long)(j + 1) * m + j;
      CK(launch_mgs_fused(n, h->w, nullptr, pa, hn, nullptr, nullptr, 1, h->V + (long long)(j + 1) * n, sc + 2,
                          s));
      CK(launch_givens(H, m, j, bn, s));
      CK(cudaMemcpyAsync(h->host_small, sc, sizeof(double) * 3, cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      double est = h->host_small[0], hnv = h->host_small[2];
      k = j + 1;
      if (est <= rtol || hnv == 0.0) break;
    }
    CK(launch_update_x(n, k, m, H, h->Z, x, s));
  }
  CK(cudaStreamSynchronize(s));
  if (iters) *iters = its;
  if (relres) *relres = rel;
  if (rel > rtol) return fail(h, FC_ERR_NOT_CONVERGED, "FGMRES reached maxit above rtol");
  return FC_OK;
}

fc_status fc_gmg_solve(fc_handle h, const double* b, double* x, double reduction, int maxit, int* iters,
                       double* relred) {
  const fc_status rs = ready_ok(h);
  if (rs != FC_OK) return rs;
  if (!b || !x || !(reduction > 0.0) || maxit < 0) return fail(h, FC_ERR_INVALID, "bad GMG arguments");
  Level& F = h->lev[h->nlev - 1];
  const long long n = F.g.ndof;
  cudaStream_t s = h->stream;
  double* sc = h->small + small_sc(h->restart);
  double r0 = 0.0, rn = 0.0;
  CK(level_residual(h, h->nlev - 1, x, b, h->w));
  CK(launch_dot(n, h->w, h->w, h->red, sc + 1, s));
  fc_status st = read_scalar(h, sc + 1, &r0);
  if (st != FC_OK) return st;
  r0 = sqrt(r0);
  rn = r0;
  int it = 0;
  while (it < maxit && rn > reduction * r0) {
    {
      ProfScope ps(h, 2, 0.0);
      st = f32_path(h) ? handle_vcycle_f32(h, x, b, false) : vcycle_level(h, h->nlev - 1, x, b);
      if (st != FC_OK) return st;
    }
    CK(level_residual(h, h->nlev - 1, x, b, h->w));
    CK(launch_dot(n, h->w, h->w, h->red, sc + 1, s));
    st = read_scalar(h, sc + 1, &rn);
    if (st != FC_OK) return st;
    rn = sqrt(rn);
    it++;
  }
  if (iters) *iters = it;
  const double red = r0 > 0.0 ? rn / r0 : 0.0;
  if (relred) *relred = red;
  if (r0 > 0.0 && red > reduction) return fail(h, FC_ERR_NOT_CONVERGED, "GMG reached maxit above the reduction");
  return FC_OK;
}

fc_status fc_solve_host(fc_handle h, const double* b_host, double* x_host, double rtol, int maxit,
                        int* iters, double* relres) {
  const fc_status rs = ready_ok(h);
  if (rs != FC_OK) return rs;
  if (!b_host || !x_host) return fail(h, FC_ERR_INVALID, "null buffer");
  long long n = h->lev[h->nlev - 1].g.ndof;
  CK(cudaMemcpyAsync(h->bh, b_host, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->xh, x_host, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream));
  fc_status st = fc_solve(h, h->bh, h->xh, rtol, maxit, iters, relres);
  if (st != FC_OK && st != FC_ERR_NOT_CONVERGED) return st;
  CK(cudaMemcpyAsync(x_host, h->xh, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return st;
}

fc_status fc_info(fc_handle h, int level, long long* ndof, long long* npatch, size_t* bytes_by_part) {
  fc_status st = level_ok(h, level, 1);
  if (st != FC_OK) return st;
  const Level& L = h->lev[level - 1];
  if (ndof) *ndof = L.g.ndof;
  if (npatch) *npatch = level >= 2 ? L.g.nnodes : 0;
  if (bytes_by_part) {
    for (int k = 0; k < 8; ++k) bytes_by_part[k] = h->bytes[k];
    bytes_by_part[5] = (size_t)(h->pair_fallback + h->ldl_fallback);
    bytes_by_part[6] = level >= 2 ? (size_t)(2 * L.active_rows) : 0;
    bytes_by_part[7] = (size_t)h->badcut;
  }
  return FC_OK;
}

fc_status fc_patch_dofs(fc_handle h, int level, long long node, long long* dofs_host, int capacity, int* n) {
  fc_status st = level_ok(h, level, 2);
  if (st != FC_OK) return st;
  const Level& L = h->lev[level - 1];
  if (!amr_path(h)) return fail(h, FC_ERR_INVALID, "patch DoF lists are given for adaptive grids");
  if (!dofs_host || !n || node < 0 || node >= L.amr.nfree) return fail(h, FC_ERR_INVALID, "bad patch");
  long long se[2] = {0, 0};
  CK(cudaMemcpyAsync(se, L.amr.pstart + node, sizeof(se), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  const int cnt = (int)(se[1] - se[0]);
  if (cnt > capacity) return fail(h, FC_ERR_INVALID, "patch DoF buffer too short");
  std::vector<int> d((size_t)std::max(cnt, 1));
  CK(cudaMemcpyAsync(d.data(), L.amr.pdof + se[0], sizeof(int) * cnt, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (int t = 0; t < cnt; ++t) dofs_host[t] = d[t];
  *n = cnt;
  return FC_OK;
}

fc_status fc_patch_rows(fc_handle h, int level, long long node, double* rows_host) {
  fc_status st = level_ok(h, level, 2);
  if (st != FC_OK) return st;
  const Level& L = h->lev[level - 1];
  if (!rows_host || node < 0 || node >= L.g.nnodes) return fail(h, FC_ERR_INVALID, "bad patch");
  if (h->opt.cache != FC_CACHE_INVERSE || !L.coef) return fail(h, FC_ERR_INVALID, "no cached rows");
  if (amr_path(h)) {
    long long se[2] = {0, 0};
    CK(cudaMemcpyAsync(se, L.amr.pstart + node, sizeof(se), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    const size_t n = (size_t)(se[1] - se[0]), nd = (size_t)h->dim + 1, rec = nd + 1;
    std::vector<double> raw(rec * n);
    CK(cudaMemcpyAsync(raw.data(), L.amr.rows + rec * se[0], sizeof(double) * rec * n, cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (size_t k = 0; k < nd; ++k)
      for (size_t j = 0; j < n; ++j) rows_host[k * n + j] = raw[rec * j + 1 + k];
    return FC_OK;
  }
  if (q2_path(h)) {
    // 2D: 9 owned rows x 171 slots, stored [slot][10]; 3D: 25 x 2214, stored [row][2240]
    const bool d3 = h->dim == 3;
    const int NS = d3 ? 2214 : 171, NR = d3 ? 25 : 9;
    const size_t per = q2_patch_rows_doubles(h->dim);
    std::vector<double> raw(per);
    CK(cudaMemcpyAsync(raw.data(), (const double*)L.coef + (size_t)node * per, sizeof(double) * per,
                       cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int k = 0; k < NR; ++k)
      for (int j = 0; j < NS; ++j)
        rows_host[(size_t)k * NS + j] = d3 ? raw[(size_t)k * 2240 + j] : raw[(size_t)j * 10 + k];
    return FC_OK;
  }
  const int ns = nslot(h->dim), nd = h->dim + 1;
  const size_t cnt = (size_t)ns * nd;
  const size_t eb = coef_elem_bytes(h->opt.prec);
  std::vector<unsigned char> raw(cnt * eb);
  int pr = (int)node;
  if (L.prow) {
    CK(cudaMemcpyAsync(&pr, L.prow + node, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  const size_t blk = pr < 0 ? (size_t)(-(long long)pr - 1) : (size_t)pr;
  CK(cudaMemcpyAsync(raw.data(), (const char*)L.coef + blk * cnt * eb, cnt * eb,
                     cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (int j = 0; j < ns; ++j)
    for (int k = 0; k < nd; ++k) {
      size_t t = (size_t)j * nd + k;
      double v = 0.0;
      if (h->opt.prec == FC_PREC_FP64) memcpy(&v, raw.data() + t * 8, 8);
      else if (h->opt.prec == FC_PREC_FP32) { float f; memcpy(&f, raw.data() + t * 4, 4); v = f; }
      else if (h->opt.prec == FC_PREC_BF16) {
        unsigned short u; memcpy(&u, raw.data() + t * 2, 2);
        unsigned int w = (unsigned int)u << 16; float f; memcpy(&f, &w, 4); v = f;
      } else { float f2[2]; memcpy(f2, raw.data() + t * 8, 8); v = (double)f2[0] + (double)f2[1]; }
      rows_host[(size_t)k * ns + j] = v;
    }
  return FC_OK;
}

fc_status fc_profile_enable(fc_handle h, int on) {
  if (!h) return FC_ERR_INVALID;
  h->prof.on = on != 0;
  return FC_OK;
}

fc_status fc_profile_read(fc_handle h, int kind, long long* launches, double* total_ms,
                          double* bytes_per_launch) {
  if (!h) return FC_ERR_INVALID;
  CK(cudaStreamSynchronize(h->stream));
  long long cnt = 0;
  double ms = 0.0, bytes = 0.0;
  std::vector<Profile::Rec> keep;
  for (auto& r : h->prof.recs) {
    if (r.kind != kind) { keep.push_back(r); continue; }
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, r.a, r.b));
    ms += t;
    bytes += r.bytes;
    cnt++;
    h->prof.pool.push_back(r.a);
    h->prof.pool.push_back(r.b);
  }
  h->prof.recs.swap(keep);
  if (launches) *launches = cnt;
  if (total_ms) *total_ms = ms;
  if (bytes_per_launch) *bytes_per_launch = cnt ? bytes / cnt : 0.0;
  return FC_OK;
}

fc_status fc_sync(fc_handle h) {
  if (!h) return FC_ERR_INVALID;
  CK(cudaStreamSynchronize(h->stream));
  return FC_OK;
}

fc_status fc_launch_count(long long* count) {
  if (!count) return FC_ERR_INVALID;
  *count = g_launches.load();
  return FC_OK;
}

const char* fc_last_error(fc_handle h) { return h ? h->err.c_str() : "null handle"; }

fc_status fc_destroy(fc_handle h) {
  if (!h) return FC_ERR_INVALID;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  handle_batch_free(h);
  for (int l = 0; l < kMaxLevels; ++l) {
    Level& L = h->lev[l];
    dfree(h, L.st); dfree(h, L.mask); dfree(h, L.dead); dfree(h, L.wfix); dfree(h, L.coef); dfree(h, L.fac); dfree(h, L.fpiv);
    dfree(h, L.facd); dfree(h, L.fpivd); dfree(h, L.lnode); dfree(h, L.lrec);
    dfree(h, L.x); dfree(h, L.b); dfree(h, L.r); dfree(h, L.rpad); dfree(h, L.rpad32);
    dfree(h, L.st2); dfree(h, L.xp2); dfree(h, L.bp2); dfree(h, L.prow);
    dfree(h, L.st32); dfree(h, L.d32); dfree(h, L.b32);
    dfree(h, L.q2mask); dfree(h, L.q2A); dfree(h, L.q2B); dfree(h, L.q2T); dfree(h, L.q2rpv); dfree(h, L.q2rpp);
    dfree(h, L.amr.rowptr); dfree(h, L.amr.col); dfree(h, L.amr.val); dfree(h, L.amr.fixed);
    dfree(h, L.amr.pstart); dfree(h, L.amr.pdof); dfree(h, L.amr.pown);
    dfree(h, L.amr.nbp); dfree(h, L.amr.nbc); dfree(h, L.amr.nbv);
    dfree(h, L.amr.prp); dfree(h, L.amr.pcl); dfree(h, L.amr.pvl);
    dfree(h, L.amr.rrp); dfree(h, L.amr.rcl); dfree(h, L.amr.rvl);
  }
  if (h->coarse_graph) cudaGraphExecDestroy(h->coarse_graph);
  dfree(h, h->d_shapes); dfree(h, h->d_err); dfree(h, h->coarse_inv);
  dfree(h, h->V); dfree(h, h->Z); dfree(h, h->w); dfree(h, h->red); dfree(h, h->small);
  dfree(h, h->bh); dfree(h, h->xh);
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  if (h->host_small) cudaFreeHost(h->host_small);
  for (auto& r : h->prof.recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : h->prof.pool) cudaEventDestroy(e);
  delete h;
  return FC_OK;
}

}  // extern "C"
