// fc_internal.cuh -- shared declarations of the libfc translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fc.h"

namespace fc {

constexpr int kMaxLevels = 12;
constexpr int kChunkNodes = 256;  // nodes per chunk of the batched kernels (fc_batch.cu)
constexpr int kMaxShapesPerCell = 64;

// Device-side error word bits (set by kernels, read back at sync points).
enum DevErr : unsigned {
  kErrTooManyShapes = 1u,
  kErrSingularPatch = 2u,
  kErrSingularCoarse = 4u,
  kErrBadIndex = 8u,
};

struct Shape {
  int type;
  double c[3], r[3], rot[2];
  double bbr;  // bounding half-width (radius or max semi-axis)
};

// Geometry and discretisation parameters of one level (passed by value).
struct LevelGeom {
  int dim, nd;         // nd = dim + 1 DoFs per node
  int n[3], nn[3];     // cells / nodes per direction (1 beyond dim)
  double lo[3], hi[3], h[3], hmin;
  long long ncell, nnodes, ndof;
  int nshape;
  const Shape* shapes;  // device
  double alpha, eta, lambda, ubar;
  int qdepth, preset, force_kind;
  double force[3];
  // 3D levels with a patch cache: one flag per x layer (nn[0] entries), then
  // per y layer (nn[1]) and per z layer (nn[2]), set when every node of the
  // layer has all its velocity components constrained (a Dirichlet wall);
  // the FP64 patch apply skips such layers and out-of-grid ones.  Null: no
  // flags.
  const unsigned char* dead_layer;
};

// Compressed operator stencil: for node a and neighbour offset nb (3^d,
// lexicographic, x fastest) the values [A, B_0..B_{d-1}, T_0..T_{d-1}, C]
// (SPN = 2d + 2 per pair), stored structure-of-arrays:
// st[(nb * SPN + e) * nnodes + a].  A: velocity-velocity (same for every
// component), B_c: row (a, c) col (b, p), T_c: row (a, p) col (b, c),
// C: pressure-pressure.  Constrained DoFs are handled with the node masks.
inline __host__ __device__ int spn(int dim) { return 2 * dim + 2; }
inline __host__ __device__ int nbr_count(int dim) { return dim == 3 ? 27 : 9; }

// Padded vector with a zero halo of two nodes on each side (for the patch
// gathers): node (i,j,k) -> ((k+2)*(ny+5) + (j+2))*(nx+5) + (i+2).
inline __host__ __device__ long long pad_node(const LevelGeom& g, int i, int j, int k) {
  long long px = g.nn[0] + 4, py = g.nn[1] + 4;
  int kk = g.dim == 3 ? k + 2 : 0;
  return ((long long)kk * py + (j + 2)) * px + (i + 2);
}
inline long long pad_nodes(const LevelGeom& g) {
  long long px = g.nn[0] + 4, py = g.nn[1] + 4, pz = g.dim == 3 ? g.nn[2] + 4 : 1;
  return px * py * pz;
}

// Q2-Q1 grid sizes of a level: Q2 nodes nf_k = 2 n_k + 1, vertices n_k + 1
struct Q2Grid {
  int nf[3], nv1[3];
  long long nq, np;
};

// Slot layout of the cached rows: nslot = 5^d * d + 3^d.
inline __host__ __device__ int nslot_u(int dim) { return dim == 3 ? 375 : 50; }
// Sum of four per-lane partial sums over a group of TPP lanes (TPP >= 4, a
// power of two, groups aligned within the warp) as a reduce-scatter: the
// first exchange halves the values a lane carries, the second halves them
// again, the remaining ones add a single value.  A lane ends with the full
// sum of value *c (c = 2 * bit(TPP/2) + bit(TPP/4) of its group lane); every
// FP64 add counts on this part (FP64 at 1/64 of the FP32 rate), and this
// takes 3 + log2(TPP/4) adds per lane instead of 4 log2(TPP).
template <int TPP>
__device__ __forceinline__ double reduce_scatter4(const double* y, int lane, int* c) {
  static_assert(TPP >= 4 && (TPP & (TPP - 1)) == 0, "group of at least 4 lanes");
  const bool h1 = lane & (TPP / 2), h2 = lane & (TPP / 4);
  double k0 = h1 ? y[2] : y[0], k1 = h1 ? y[3] : y[1];
  const double s0 = h1 ? y[0] : y[2], s1 = h1 ? y[1] : y[3];
  k0 += __shfl_xor_sync(0xffffffffu, s0, TPP / 2);
  k1 += __shfl_xor_sync(0xffffffffu, s1, TPP / 2);
  double k = h2 ? k1 : k0;
  k += __shfl_xor_sync(0xffffffffu, h2 ? k0 : k1, TPP / 4);
#pragma unroll
  for (int o = TPP / 8; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
  *c = (h1 ? 2 : 0) + (h2 ? 1 : 0);
  return k;
}

inline __host__ __device__ int nslot(int dim) { return dim == 3 ? 402 : 59; }

// Adaptive space-tree grids, quadtrees in 2D and octrees in 3D (fc_amr.cu):
// the tree as the leaf level of every lattice cell (the cells of the finest
// level R), the host half of a level, and its device arrays.
struct AmrTree {
  int dim = 2, R = 0, nroot[3] = {0, 0, 1}, NX = 0, NY = 0, NZ = 1;
  std::vector<unsigned char> lev;  // [NZ][NY][NX]
};

struct AmrHost {
  int dim = 2;
  long long nfree = 0;
  std::vector<long long> fid, fvert;      // vertex -> free node or -1; free node -> vertex
  std::vector<long long> hp;              // 4 per vertex: parents of a hanging vertex
  std::vector<unsigned char> hn;          // per vertex: parents of a hanging vertex (2 or 4), 0 otherwise
  std::vector<int> leaf;                  // (X, Y, Z, level) per leaf, lattice order
  std::vector<int> rowptr, col;           // operator, node-interleaved (velocity components, p)
  std::vector<double> val, rhs, wfix;
  std::vector<unsigned char> fixed;
  std::vector<long long> pstart;          // patch DoF offsets
  std::vector<int> pdof, pown;            // patch DoFs; owned local index (dim + 1 per patch) or -1
  std::vector<int> prp, pcl, rrp, rcl;    // prolongation from the coarser level and its transpose
  std::vector<double> pvl, rvl;
  std::vector<int> nbp, nbc;              // node blocks: neighbours of each free node (CSR over nodes)
  std::vector<double> nbv;                // per neighbour pair: A, B_0 .. B_{d-1}, T_0 .. T_{d-1}, C
};

struct AmrLevel {
  int dim = 2;
  long long nfree = 0;
  int maxn = 0;                  // largest patch
  int maxnv = 0, maxnp = 0;      // most velocity nodes / pressures in a patch
  int* rowptr = nullptr;
  int* col = nullptr;
  double* val = nullptr;
  unsigned char* fixed = nullptr;
  long long* pstart = nullptr;
  int* pdof = nullptr;
  int* pown = nullptr;
  double* rows = nullptr;        // per patch slot (from (dim + 2) * pstart[p]): DoF index bits, dim + 1
                                 // owned-row coefficients
  int* nbp = nullptr;            // node-block operator for the residual (the velocity block is the same
  int* nbc = nullptr;            // scalar A for every component, as in the uniform stencil)
  double* nbv = nullptr;
  int *prp = nullptr, *pcl = nullptr, *rrp = nullptr, *rcl = nullptr;
  double *pvl = nullptr, *rvl = nullptr;
  unsigned long long rows_flop = 0;  // 2 x (patch DoFs x free owned DoFs) summed over the patches
};

struct Level {
  LevelGeom g;
  double* st = nullptr;         // stencil, SPN * 3^d * nnodes
  unsigned char* mask = nullptr;  // per node: bit c = velocity comp c constrained
  unsigned char* dead = nullptr;  // layer flags (LevelGeom::dead_layer), 3D levels above the coarsest
  double* wfix = nullptr;       // Dirichlet values per DoF (0 where free)
  // patch cache
  void* coef = nullptr;         // cache_inverse rows
  size_t coef_bytes = 0;
  double* fac = nullptr;        // cache_matrix factors (3D: band records)
  int* fpiv = nullptr;
  size_t fac_bytes = 0;
  // 3D cache_matrix: dense records of the patches whose velocity block was
  // not positive definite, and the nodes (with record index) that use them
  double* facd = nullptr;
  int* fpivd = nullptr;
  int* lnode = nullptr;
  int* lrec = nullptr;
  long long nlist = 0;
  double ldl_dmin = 1e-14;  // 3D cache_none: the pivot bound the list was made with
  // level vectors (device)
  double* x = nullptr;          // V-cycle correction on this level
  double* b = nullptr;          // right-hand side on this level
  double* r = nullptr;          // unpadded residual
  double* rpad = nullptr;       // padded residual (smoother)
  float* rpad32 = nullptr;      // padded residual in float32 / pairs (mixed paths)
  // float-pair smoother state (FC_PREC_DF64): the stencil as (hi, lo) pairs
  // for the zero offset and the offsets after it (the operator is
  // symmetric), with constrained columns folded in (zero), a padded pair copy
  // of x (zero halo) that a smoothing phase updates in place, and a pair
  // copy of b
  float2* st2 = nullptr;
  float2* xp2 = nullptr;
  float2* bp2 = nullptr;
  // float32 correction form of the V-cycle (float32 / bfloat16 rows): the
  // half stencil (zero offset and the offsets after it) in float32 with the
  // columns of constrained DoFs folded to zero (levels above the coarsest),
  // the padded correction and the right-hand side in float32 (every level)
  float* st32 = nullptr;
  float* d32 = nullptr;
  float* b32 = nullptr;
  size_t vec_bytes = 0;
  unsigned long long active_slots = 0;  // sum over patches of active patch DoFs
  unsigned long long active_rows = 0;   // sum over patches of active DoFs x free owned DoFs
  // patch classes (bit-identical L_i): prow[i] = row block of patch i;
  // nwork row blocks are factored and stored
  int* prow = nullptr;
  int nwork = 0;
  int cls_blk[2] = {-1, -1};            // stored blocks of the patch classes 1 and 2
  unsigned long long active_work = 0;   // active DoFs summed over the stored blocks
  // Q2-Q1 variant (fc_options.element = 1, see fc_q2.cu): grid sizes, node
  // masks, stencil blocks, padded residual copies (velocity halo 4 nodes,
  // pressure halo 1 vertex); the patch rows live in coef, Dirichlet values
  // in wfix, vectors in x, b, r
  Q2Grid q2{};
  unsigned char* q2mask = nullptr;
  double* q2A = nullptr;
  double* q2B = nullptr;
  double* q2T = nullptr;
  double* q2rpv = nullptr;
  double* q2rpp = nullptr;
  // adaptive grids (fc_options.amr_uniform >= 0, see fc_amr.cu)
  AmrLevel amr{};
};

AmrTree amr_tree_fine(const std::vector<Shape>& sh, int dim, const double* lo, const double* hi, const int* nroot, int U,
                      int R);
AmrTree amr_tree_coarsen(const AmrTree& F);
bool amr_structure(const AmrTree& T, AmrHost& H, std::vector<std::vector<long long>>& adj);
int amr_assemble(const AmrTree& T, const LevelGeom& g, const std::vector<double>& eA, const std::vector<double>& eB,
                 const std::vector<double>& eF, const std::vector<std::vector<long long>>& adj, AmrHost& H);
void amr_transfers(const AmrTree& T, AmrHost& H, const AmrTree& Tc, const AmrHost& Hc);
std::vector<long long> amr_leaf_cells(const AmrTree& T, const AmrHost& H, int level, std::vector<long long>* slots);
cudaError_t launch_amr_residual(const AmrLevel& A, const double* x, const double* b, double* r, cudaStream_t s);
cudaError_t launch_amr_apply(const AmrLevel& A, const double* r, double omega, double* x, cudaStream_t s);
cudaError_t launch_amr_prolong_add(const AmrLevel& F, const double* ec, double* xf, cudaStream_t s);
cudaError_t launch_amr_restrict(const AmrLevel& F, const AmrLevel& C, const double* rf, double* bc, cudaStream_t s);
cudaError_t launch_amr_dense(const AmrLevel& A, double* M, cudaStream_t s);
// owned rows of every patch of an adaptive level (fc_patch.cu): L_i gathered
// from the CSR, equilibrated, rows of the owned DoFs; a dense LU with
// partial pivoting in shared memory (a CTA per patch, work null) when the
// block fits, else block elimination of the velocity block in a global
// workspace of amr_patch_rows_work_doubles() (ctas persistent CTAs)
constexpr int kAmrMaxPatch = 2048;  // largest adaptive patch (DoFs)
bool amr_patch_rows_in_smem(int dim, int maxn);
int amr_patch_rows_ctas(const AmrLevel& A);
size_t amr_patch_rows_work_doubles(const AmrLevel& A, int ctas);
cudaError_t launch_amr_patch_rows(const AmrLevel& A, double* work, int ctas, unsigned* d_err, cudaStream_t s);

struct Profile {
  bool on = false;
  struct Rec { cudaEvent_t a, b; int kind; double bytes; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
};

}  // namespace fc

struct fc_handle_s {
  int dim = 0, nlev = 0;
  // set when fc_setup completed; a handle whose setup failed holds partial
  // data and only answers fc_last_error, fc_sync and fc_destroy
  bool ready = false;
  fc::Level lev[fc::kMaxLevels];  // index 0 = coarsest (paper level 1)
  fc_options opt;
  double alpha = 0;
  cudaStream_t stream = nullptr;
  int device = -1;  // CUDA device current at fc_setup (holds every buffer of the handle)
  fc::Shape* d_shapes = nullptr;
  int nshape = 0;
  unsigned* d_err = nullptr;
  // coarse solve: dense inverse of the coarsest operator
  double* coarse_inv = nullptr;
  int coarse_n = 0;
  // FGMRES workspace
  double* V = nullptr;
  double* Z = nullptr;
  double* w = nullptr;
  double* red = nullptr;    // reduction scratch
  double* small = nullptr;  // Hessenberg, Givens, g, y (device)
  double* host_small = nullptr;  // pinned
  double* bh = nullptr;     // device staging for fc_solve_host
  double* xh = nullptr;
  int restart = 30;
  size_t bytes[8] = {0};
  // coarse part of the V-cycle (restriction from the finest level's residual
  // buffer down to the coarse solve) captured once as a CUDA graph
  cudaGraphExec_t coarse_graph = nullptr;
  int coarse_graph_kernels = 0;
  // float32 / bfloat16 rows: the V-cycle runs in the float32 correction form
  // through a batch holding this handle alone (created on first use)
  struct fc_batch_s* self_batch = nullptr;
  // float32 / bfloat16 rows: patches rebuilt by the float-pair elimination
  // because float32 refinement did not converge (all levels)
  long long pair_fallback = 0;
  // FP64 rows (3D): patches whose velocity block was not positive definite
  // for the banded LDL^T and took the pivoted dense LU, all levels
  long long ldl_fallback = 0;
  // float32 / bfloat16 rows: patches given float-pair rows by the bad-cut
  // rule (fc_options.badcut_frac), all levels
  long long badcut = 0;
  bool capturing = false;
  fc::Profile prof;
  std::string err;
};

namespace fc {

// process-wide count of libfc kernel launches (fc_api.cu)
void note_launches(int n);
// resident CTAs per SM of a persistent kernel and the SM count, on the
// current device: computed once per (kernel, device) under a lock, after
// raising the kernel's dynamic shared-memory limit on that device (fc_api.cu)
cudaError_t persistent_ctas(const void* kern, int threads, size_t smem, int* per_sm, int* nsm);
// launches recorded while a stream capture is open are counted at replay
void set_capturing(bool on);
// float32 correction-form V-cycle of a handle (x known zero: xzero)
fc_status handle_vcycle_f32(fc_handle h, double* x, const double* b, bool xzero);
void handle_batch_free(fc_handle h);

// ---- Q2-Q1 variant (fc_q2.cu, fc_patch.cu) ----
Q2Grid make_q2grid(const LevelGeom& g);
cudaError_t launch_q2_masks(const LevelGeom& g, const Q2Grid& q, unsigned char* mask, double* wfix, cudaStream_t s);
// stencil blocks A, B, T from the element data; b (nullable) gets the
// right-hand side (load, lifted Dirichlet values)
cudaError_t launch_q2_assemble(const LevelGeom& g, const Q2Grid& q, const double* eA, const double* eB,
                               const double* eF, const unsigned char* mask, const double* wfix, double* A,
                               double* B, double* T, double* b, cudaStream_t s);
// r = b - L x (L x without b) into r and / or the padded copies (nullable)
cudaError_t launch_q2_residual(int dim, const Q2Grid& q, const double* A, const double* B, const double* T,
                               const unsigned char* mask, const double* x, const double* b, double* r, double* rpv,
                               double* rpp, cudaStream_t s);
cudaError_t launch_q2_prolong_add(int dim, const Q2Grid& f, const Q2Grid& c, const unsigned char* fmask,
                                  const double* ec, double* xf, cudaStream_t s);
cudaError_t launch_q2_restrict(int dim, const Q2Grid& f, const Q2Grid& c, const unsigned char* cmask,
                               const double* rf, double* bc, cudaStream_t s);
cudaError_t launch_q2_dense(int dim, const Q2Grid& q, const double* A, const double* B, const double* T,
                            const unsigned char* mask, double* M, cudaStream_t s);
// patch rows: 2D [vertex][171 slots][10] (9 owned rows, padded); 3D
// [vertex][25 rows][2240] (2214 slots, padded).  The 3D factorisation takes
// a global workspace of q2_patch_rows_work_doubles(3, ctas) for `ctas`
// persistent CTAs (q2_patch_rows_ctas: one per SM, at most kQ2Rows3MaxCtas).
constexpr int kQ2Rows3MaxCtas = 256;
size_t q2_patch_rows_doubles(int dim);
size_t q2_patch_rows_work_doubles(int dim, long long ctas);
int q2_patch_rows_ctas(int dim, long long np);
cudaError_t launch_q2_patch_rows(int dim, const Q2Grid& q, const double* A, const double* B, const unsigned char* mask,
                                 double* coef, double* work, int ctas, unsigned* d_err, cudaStream_t s);
cudaError_t launch_q2_apply(int dim, const Q2Grid& q, const double* coef, const unsigned char* mask, const double* rpv,
                            const double* rpp, double omega, double* x, cudaStream_t s);
// explicit inverse of a dense n x n matrix (rows in `work`, destroyed) by
// the equilibrated Gauss-Jordan elimination of the coarse solve (fc_mg.cu);
// dsc holds 2 n doubles
cudaError_t launch_dense_inverse(int n, double* work, double* inv, int* piv, double* dsc, unsigned* d_err,
                                 cudaStream_t s);

// ---- launchers (defined in the .cu files) ----
// geometry + element data (fc_geom.cu)
// refA/refB (nullable): reference element matrices of an uncut cell for
// alpha = 1; plain cells then store alpha * reference.  cclass (nullable):
// 0 cut or mixed, 1 plain fluid, 2 plain fictitious.
cudaError_t launch_cell_elements(const LevelGeom& g, double* eA, double* eB, double* eF,
                                 double* estat, unsigned* d_err, const double* refA, const double* refB,
                                 unsigned char* cclass, cudaStream_t s);
// Q2-Q1 element data: eA [cell][3^d][3^d], eB [cell][d][3^d][2^d],
// eF [cell][d][3^d]; estat as above (nullable)
// element data of the listed cells of g (adaptive grids: the leaves of one
// level), outputs in list order
cudaError_t launch_cell_elements_list(const LevelGeom& g, const long long* cells, long long ncells, double* eA,
                                      double* eB, double* eF, unsigned* d_err, cudaStream_t s);
cudaError_t launch_cell_elements_q2(const LevelGeom& g, double* eA, double* eB, double* eF, double* estat,
                                    unsigned* d_err, cudaStream_t s);
// patch classes: node class from its 2^d cells, patch class from its 5^d
// nodes (in grid, unconstrained, one class); representatives and the work
// list of patches to factor; prow maps every patch to its row block
cudaError_t launch_patch_classes(const LevelGeom& g, const unsigned char* cclass, const unsigned char* mask,
                                 unsigned char* nclass, int* pclass, int* rep, int* work, int* nwork,
                                 int* prow, int dedup, cudaStream_t s);
// assembly (fc_assemble.cu)
cudaError_t launch_assemble(const LevelGeom& g, const double* eA, const double* eB, double* st,
                            cudaStream_t s);
cudaError_t launch_masks(const LevelGeom& g, unsigned char* mask, double* wfix, cudaStream_t s);
// Galerkin coarse stencil R L_f P from the finer level's stencil and masks,
// and the coarse cell classes / statistics from the children's
cudaError_t launch_galerkin(const LevelGeom& gc, const LevelGeom& gf, const double* stf, const unsigned char* maskf,
                            double* stc, cudaStream_t s);
cudaError_t launch_coarsen_cells(const LevelGeom& gc, const LevelGeom& gf, const unsigned char* cclass_f,
                                 unsigned char* cclass_c, const double* estat_f, double* estat_c, cudaStream_t s);
// x / y / z layer flags of g.dead_layer from the node masks (3D); out holds
// nn[0] + nn[1] + nn[2] bytes
cudaError_t launch_dead_layers(const LevelGeom& g, const unsigned char* mask, unsigned char* out, cudaStream_t s);
cudaError_t launch_rhs(const LevelGeom& g, const double* eF, const double* st,
                       const unsigned char* mask, const double* wfix, double* b, cudaStream_t s);
// operator application (fc_mg.cu)
cudaError_t launch_residual(const LevelGeom& g, const double* st, const unsigned char* mask,
                            const double* x, const double* b, double* r, double* rpad,
                            cudaStream_t s);
cudaError_t launch_residual_df(const LevelGeom& g, const double* st, const unsigned char* mask,
                               const double* x, const double* b, float* rpad2, cudaStream_t s);
cudaError_t launch_residual_f32(const LevelGeom& g, const double* st, const unsigned char* mask,
                                const double* x, const double* b, float* rpad, cudaStream_t s);
cudaError_t launch_restrict(const LevelGeom& f, const LevelGeom& c, const unsigned char* cmask,
                            const double* rf, double* bc, cudaStream_t s);
cudaError_t launch_prolong_add(const LevelGeom& f, const LevelGeom& c, const unsigned char* fmask,
                               const double* ec, double* xf, cudaStream_t s);
cudaError_t launch_zero_pad_halo(double* p, long long n, cudaStream_t s);
// patches (fc_patch.cu)
// patch cache build (mode 0 rows, 1 factors) over the work list (block w
// stores patch work[w]); mode 2 (solve on the fly) runs over all patches
cudaError_t launch_patch_build(const LevelGeom& g, const double* st, const unsigned char* mask,
                               int mode, double omega, double* coef64, double* fac, int* fpiv,
                               const double* rpad, double* x, unsigned* d_err, const int* work,
                               long long nwork, cudaStream_t s);
// owned rows of the work-list patches by a float-pair factorisation (for
// rows stored in reduced precision); float64 output like mode 0
// owned rows of the work-list patches by a float32 factorisation with two
// steps of iterative refinement (rows stored in float32 / bfloat16);
// patches whose refinement did not converge are appended to redo_node
// (patch) / redo_out (row block), *nredo counting them
cudaError_t launch_patch_rows_ir(const LevelGeom& g, const double* st, const unsigned char* mask,
                                 double* coef64, unsigned* d_err, const int* work, long long nwork,
                                 int* redo_node, int* redo_out, int* nredo, cudaStream_t s);
// 3D FP64 owned rows by a banded LDL^T of the velocity block; patches whose
// block is not positive definite go to redo_node / redo_out (count nredo)
cudaError_t launch_patch_rows_ldl(const LevelGeom& g, const double* st, const unsigned char* mask,
                                  double* coef64, unsigned* d_err, const int* work, long long nwork,
                                  int* redo_node, int* redo_out, int* nredo, cudaStream_t s);
// 3D FP64 owned rows of the redo-list patches by the pivoted dense LU
cudaError_t launch_patch_rows_dense_redo(const LevelGeom& g, const double* st, const unsigned char* mask,
                                         double* coef64, unsigned* d_err, const int* redo_node,
                                         long long nredo, const int* redo_out, cudaStream_t s);
// float-pair elimination; outidx (nullable) maps a work entry to its row block
cudaError_t launch_patch_rows_pair(const LevelGeom& g, const double* st, const unsigned char* mask,
                                   double* coef64, unsigned* d_err, const int* work, long long nwork,
                                   const int* outidx, cudaStream_t s);
// prow (nullable = identity) maps a patch to its stored row / factor block
cudaError_t launch_patch_apply(const LevelGeom& g, fc_prec prec, const void* coef,
                               const unsigned char* mask, const double* rpad, const float* rpad32,
                               double omega, double* x, const int* prow, cudaStream_t s);
// cache_matrix factors of a level: band records (3D) or dense records (2D),
// plus the dense records and node list of the 3D patches that need them
struct FactorStore {
  const double* fac = nullptr;
  const int* fpiv = nullptr;
  const double* facd = nullptr;
  const int* fpivd = nullptr;
  const int* lnode = nullptr;
  const int* lrec = nullptr;
  long long nlist = 0;
};
cudaError_t launch_factor_apply(const LevelGeom& g, const double* st, const FactorStore& f,
                                const unsigned char* mask, const double* rpad, double omega, double* x,
                                const int* prow, cudaStream_t s);
inline FactorStore factor_store(const Level& L) {
  FactorStore f;
  f.fac = L.fac;
  f.fpiv = L.fpiv;
  f.facd = L.facd;
  f.fpivd = L.fpivd;
  f.lnode = L.lnode;
  f.lrec = L.lrec;
  f.nlist = L.nlist;
  return f;
}
// 3D band factor records (cache_matrix) by the banded LDL^T; non-positive-
// definite patches go to redo_node / redo_out and are marked pending
cudaError_t launch_band_factors(const LevelGeom& g, const double* st, const unsigned char* mask, double* fac,
                                int* fpiv, unsigned* d_err, const int* work, long long nwork, int* redo_node,
                                int* redo_out, int* nredo, cudaStream_t s);
// dense factor records (records 0 .. nredo-1 of facd / fpivd) of the redo
// patches, and their index in the band records' int field
cudaError_t launch_dense_factor_redo(const LevelGeom& g, const double* st, const unsigned char* mask, double* facd,
                                     int* fpivd, unsigned* d_err, const int* redo_node, const int* redo_out, int nredo,
                                     int* fpiv, cudaStream_t s);
// cache_none in 3D: at setup, list the patches whose velocity block is not
// positive definite (redo_node, count nredo); per sweep, the banded
// on-the-fly solve of every patch and the dense one of the listed patches
// (dmin: the smallest accepted pivot, the same at setup and in every sweep,
// so that a patch is solved by exactly one of the two kernels)
double ldl_min_pivot();
cudaError_t launch_none_check(const LevelGeom& g, const double* st, const unsigned char* mask, unsigned* d_err,
                              int* redo_node, int* redo_out, int* nredo, double dmin, cudaStream_t s);
cudaError_t launch_none_sweep(const LevelGeom& g, const double* st, const unsigned char* mask, double omega,
                              const double* rpad, double* x, unsigned* d_err, const int* dense_nodes,
                              long long ndense, double dmin, cudaStream_t s);
// nodes whose record (through prow) is dense
cudaError_t launch_dense_list(const LevelGeom& g, const int* prow, const int* fpiv, int* lnode, int* lrec,
                              int* nlist, cudaStream_t s);
cudaError_t launch_convert_rows(const LevelGeom& g, fc_prec prec, const double* coef64, void* out,
                                long long nblocks, cudaStream_t s);
// float-pair smoother pieces: split float64 into (hi, lo) pairs; pair
// stencil with constrained columns folded to zero; padded pair copy of x
// and its merge back; pair residual into the padded pair residual and/or an
// unpadded float64 residual; pair apply updating the padded pair copy of x
cudaError_t launch_split_pairs(long long n, const double* in, float2* out, cudaStream_t s);
cudaError_t launch_fold_stencil_f32(const LevelGeom& g, const double* st, const unsigned char* mask, float* st32,
                                    cudaStream_t s);
cudaError_t launch_fold_stencil_pairs(const LevelGeom& g, const double* st, const unsigned char* mask,
                                      float2* st2, cudaStream_t s);
cudaError_t launch_split_x_padded(const LevelGeom& g, const double* x, float2* xp2, cudaStream_t s);
cudaError_t launch_merge_x_padded(const LevelGeom& g, const float2* xp2, double* x, cudaStream_t s);
cudaError_t launch_residual_df2(const LevelGeom& g, const float2* st2, const unsigned char* mask,
                                const float2* xp2, const float2* b2, float2* rpad2, double* r,
                                cudaStream_t s);
// cls_blk: host array of the (up to two) stored blocks shared by the patch
// classes, -1 for none; those blocks are staged in shared memory
cudaError_t launch_patch_apply_df2(const LevelGeom& g, const void* coef, const unsigned char* mask,
                                   const float* rpad2, double omega, float2* xp2, const int* prow,
                                   const int* cls_blk, cudaStream_t s);
size_t factor_doubles(int dim);
size_t factor_ints(int dim);
size_t dense_factor_doubles(int dim);
size_t dense_factor_ints(int dim);
// coarse solve (fc_mg.cu)
cudaError_t launch_coarse_factor(const LevelGeom& g, const double* st, const unsigned char* mask,
                                 double* work, double* inv, int* piv, double* dsc, unsigned* d_err,
                                 cudaStream_t s);
cudaError_t launch_dense_gemv(int n, const double* A, const double* x, double* y, cudaStream_t s);
// vector ops (fc_mg.cu)
cudaError_t launch_dot(long long n, const double* a, const double* b, double* partial,
                       double* out, cudaStream_t s);
cudaError_t launch_axpy(long long n, double alpha, const double* x, double* y, cudaStream_t s);
cudaError_t launch_scale_copy(long long n, const double* s, int sidx, int invert, const double* x,
                              double* y, cudaStream_t st);
cudaError_t launch_mgs_step(long long n, double* w, const double* vi, const double* hij,
                            cudaStream_t s);
// one fused MGS step (see fc_mg.cu); partial arrays hold 1024 block sums
cudaError_t launch_mgs_fused(long long n, double* w, const double* v_prev, const double* part_in,
                             double* h_out, const double* v_next, double* part_out, int finish,
                             double* v_out, double* hn_copy, cudaStream_t s);
cudaError_t launch_givens(double* small, int m, int j, double bnorm, cudaStream_t s);
cudaError_t launch_update_x(long long n, int k, int m, const double* small, const double* Z,
                            double* x, cudaStream_t s);

}  // namespace fc
