// Internal declarations shared by the CUDA translation units of libcmg.
// Nothing here is part of the C ABI (include/cmg.h).
#pragma once

#include <utility>

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/cmg.h"

namespace cmg {

// Process-wide count of kernels launched by this library.
void count_launches(int k);

constexpr int kBlock = 256;        // threads per CTA of the node-sample kernels
constexpr int kMaxLevels = 16;
constexpr int kMaxSPL = 8;         // chunks of V samples per lane
constexpr int kMaxCoarseM = 49;    // nodes of the coarsest grid (7 x 7)

template <typename T>
struct Vec3 {
  T* y;
  T* u;
  T* p;
};
template <typename T>
struct Vec3c {
  const T* y;
  const T* u;
  const T* p;
};
template <typename T>
__host__ __device__ inline Vec3c<T> cview(const Vec3<T>& v) { return {v.y, v.u, v.p}; }

// Read-only view of one grid's operator for the kernels.  Face arrays:
// kx[iy][f][j], f = 0..n (face f separates columns f-1 and f; f = 0 and n
// touch the boundary); ky[f][ix][j], f = 0..n likewise for rows.
// Nodes of a grid that carry a control basis function (local control, the
// paper's control on a subregion): the inclusive index box [x0, x1] x
// [y0, y1] of (ix, iy); an empty box (x1 < x0) means no control node.  The
// default covers every node (distributed control).
struct CtlBox {
  int x0 = 0, x1 = 1 << 30, y0 = 0, y1 = 1 << 30;
  __host__ __device__ bool inside(int iy, int ix) const { return ix >= x0 && ix <= x1 && iy >= y0 && iy <= y1; }
  __host__ __device__ bool full(int n) const { return x0 <= 0 && y0 <= 0 && x1 >= n - 1 && y1 >= n - 1; }
};

template <typename T>
struct LevelView {
  int n;            // nodes per side
  int N;            // samples
  int ld;           // sample stride of node arrays (elements)
  const T* kx;
  const T* ky;
  const double* inva;   // 1/diag(A_j) per node-sample (FP64 path only)
  const double* isigma; // 1 / Schur denominator of Eq. (13) per node, FP64 (for an FP32 view: of the FP32 operator)
  double c, G, d, e;    // scalar blocks of Eq. (12): C_j = c I, G, D_j = d I, E_j = e I
  int spl_target;       // chunks per lane chosen by the autotuner (0 = size heuristic)
  int freeze_u;         // 1: keep u fixed (local solves of the state and adjoint rows only)
  const float* isigma32;  // 1/sigma rounded to FP32 (read only by the all-FP32 option, ctl32)
  const double* a64;      // diag(A_j) = sum of the four faces per node-sample (FP64, finest grid only, else null)
  CtlBox ctl{};           // nodes with a control basis function (elsewhere u_i = 0, no control row)
  const float* dw = nullptr;   // per-node factor on d (semismooth Newton active sets); null = 1
  // FP32 views: 0 (default) = the per-node Schur scalar of Eq. (13) (the sum
  // over samples for u_i, 1/sigma_i and u_i) in FP64 from the lanes' FP32
  // partial sums; 1 = that work in FP32 as well (all-FP32 option)
  int ctl32 = 0;
};

// d_i = d * dw[node] (the control row's coupling to the adjoint at node i).
template <typename T>
__host__ __device__ inline double d_of(const LevelView<T>& L, long node) {
  return L.dw ? L.d * (double)L.dw[node] : L.d;
}

// Sample mapping of a node's N samples: lanes-per-node (power of two <= 32),
// vector width V (elements per 16-byte or narrower load), chunks per lane.
struct SampleMap {
  int lpn;
  int V;
  int spl;
};
// Lanes per node for a launch over `items` nodes.  A lane takes up to 4
// chunks so that one warp covers several nodes and the per-node FP64 work
// (control-row sum, u) is shared by one warp instruction, as long as the
// launch keeps at least kMinLanes lanes (two 256-thread CTAs per SM);
// small grids are latency-bound and use more lanes per node.  items = 0
// asks for the most lanes (one chunk per lane where N allows).
constexpr long kMinLanes = 2L * 152 * 256;
SampleMap choose_map(int N, int elem_bytes, long items, int spl_target = 0);

// Coarsest-grid factors (FP64).
struct CoarseData {
  int n, m, N;
  CtlBox ctl;        // control nodes of the coarsest grid (the control Schur system lives on them)
  const float* dw;   // per-node factor on d of the coarsest grid (null = 1)
  double* Ainv;      // [N][m][m]
  float* Ainv32;     // [N][m][m] FP32 copy for the FP32 cycle's coarse solve (may be null)
  double* Minv;      // [m][m]   inverse of the control Schur system
  double* wz;        // scratch [2][N][m] (A_j^{-1} f_y,j and A_j^{-1} f_p,j)
  double* partial;   // scratch [blocks][m]
  int blocks;
};

// ---- launches ----
// Programmatic dependent launch for the kernels of the cycle and the
// refinement loop (every kernel launched this way starts with pdl_enter);
// CMG_PDL=0 in the environment turns the attribute off.
bool pdl_enabled();
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// ---- stencil kernels (cmg_stencil.cu) ----
// r = f - S x (or r = S x when f.y == nullptr); the y block of r is then
// multiplied by wy (wy = N gives the paper's row scaling).
template <typename T>
cudaError_t launch_residual(const LevelView<T>& L, Vec3c<T> x, Vec3c<T> f, Vec3<T> r, cudaStream_t s,
                            double wy = 1.0);
// Tuning target flag (FP32): the half-sweep stages its loads through
// shared memory (cmg_staged.cu); the low bits are the chunks per lane.
constexpr int kTuneStaged = 16;
// Tuning target flag (FP32, N even and at most 64): two samples per lane
// (8-byte loads), so a node takes N/2 lanes rounded up to a power of two and
// a warp holds one node at N = 64 -- twice the warps of the 16-byte layout,
// finer work for the last wave of a grid.  Low bits must be 1.
constexpr int kTuneWide = 32;
// Tuning target flag (FP32): the cycle on this grid prolongs the coarse
// correction in its own pass and then runs the plain post-smoothing
// half-sweeps, instead of fusing the prolongation into the first of them.
constexpr int kTuneUnfused = 64;
// Tuning target flag (FP32): the red-black sweeps on this grid run as one
// launch per sweep (launch_rbgs_fused) in pairs through a second buffer.
constexpr int kTuneFused = 128;
// Tuning target flag (FP32, N % 4 == 0 and N <= 256, with 1, 2 or 4 chunks
// per lane): the plain half-sweeps on this grid bring their rows into
// shared memory by TMA loads that gather every other node of a grid row
// (launch_rbgs_half_tma, cmg_tma_sweep.cu); the same bits as the direct
// half-sweep.
constexpr int kTuneTma = 256;
inline bool wide_supported(int N) { return N % 2 == 0 && N <= 64; }
bool staged_supported(int N, int spl);
cudaError_t launch_rbgs_half_staged(const LevelView<float>& L, Vec3<float> x, Vec3c<float> f, int colour,
                                    const SampleMap& m, cudaStream_t s);
// cudaErrorNotSupported (nothing enqueued) where the shape is not covered.
cudaError_t launch_rbgs_half_tma(const LevelView<float>& L, Vec3<float> x, Vec3c<float> f, int colour,
                                 const SampleMap& m, cudaStream_t s);
template <typename T>
cudaError_t launch_rbgs_half(const LevelView<T>& L, Vec3<T> x, Vec3c<T> f, int colour, cudaStream_t s);
// Colour-0 half-sweep of a cycle that starts from a zero iterate: x is not
// read (its neighbour terms are zero) and need not have been cleared.
template <typename T>
cudaError_t launch_rbgs_zero(const LevelView<T>& L, Vec3<T> x, Vec3c<T> f, cudaStream_t s);
template <typename T>
cudaError_t launch_jacobi_update(const LevelView<T>& L, Vec3<T> x, Vec3c<T> r, double theta, cudaStream_t s);
// r = f - S x at the colour-0 nodes only: after a red-black sweep whose
// last half-sweep updated colour 1, the residual at the colour-1 nodes
// vanishes (each local solve satisfied that node's equations given
// neighbours that did not change since), so the restriction reads only
// colour-0 points (launch_restrict with colour0 = 1).
template <typename T>
cudaError_t launch_residual_c0(const LevelView<T>& L, Vec3c<T> x, Vec3c<T> f, Vec3<T> r, cudaStream_t s);
// Colour-0 half-sweep with the prolongation of the coarse correction e
// fused in: the neighbours (colour 1) are read as x + P e.  The colour-0
// values of x + P e are never needed (this sweep overwrites them from the
// neighbours) and the colour-1 values are needed only here (the next
// half-sweep overwrites them), so the prolongation pass is not run.
template <typename T>
cudaError_t launch_rbgs_prolong(const LevelView<T>& L, Vec3<T> x, Vec3c<T> f, Vec3c<T> e, int nc, cudaStream_t s);
// One whole red-black sweep in one launch (FP32, cmg_fused.cu): the
// colour-0 and colour-1 half-sweeps over tiles of the grid, reading the old
// iterate from xa and writing the new one to xb (xb != xa; equal to the two
// half-sweeps bit for bit).  Modes: kFusedPlain, kFusedZero (xa is zero and
// not read), kFusedProlong (colour 0 reads xa + P e, e on the grid of nc
// nodes per side).  cudaErrorNotSupported where the shape is not covered
// (fused_plan) or the control is frozen.
enum { kFusedPlain = 0, kFusedZero = 1, kFusedProlong = 2 };
struct FusedPlan {
  bool ok = false;
  int lpn = 0, spl = 0;          // the half-sweeps' sample map (V = 4)
  int W = 0, BH = 0;             // tile width (columns) and band height (rows)
  int strips = 0, tiles = 0;     // tile columns; tiles in all
  int threads = 0, grid = 0;     // CTA size; CTAs (each walks tiles grid apart)
};
FusedPlan fused_plan(int n, int N, int spl_target);
cudaError_t launch_rbgs_fused(const LevelView<float>& L, Vec3c<float> xa, Vec3<float> xb, Vec3c<float> f,
                              int mode, Vec3c<float> e, int nc, cudaStream_t s);
template <typename T>
cudaError_t launch_restrict(int nf, int N, Vec3c<T> r, Vec3<T> c, cudaStream_t s,
                            Vec3<T> zx = Vec3<T>{nullptr, nullptr, nullptr}, int colour0 = 0);
template <typename T>
cudaError_t launch_prolong_add(int nf, int N, Vec3c<T> e, Vec3<T> x, cudaStream_t s, CtlBox ctl = CtlBox{});

// ---- semismooth Newton for the L1 + box problem (cmg_ssn.cu) ----
// out[i] = sum_j p[i][j] (FP64, fixed order)
cudaError_t launch_sum_samples(long nodes, int N, const double* p, double* out, cudaStream_t s);
// F = the optimality map of Sec. 4 at (u + g du, Tu + g Tdp) (du, Tdp may be
// null), chi = the active-set indicator there (may be null), per-CTA
// partial sums of F^2; returns the number of partials (<= max_partials) or -1.
int launch_ssn_map(long nodes, const double* u, const double* du, const double* Tu, const double* Tdp, double g,
                   double nu, double beta, double a, double b, double* F, float* chi, double* partial,
                   int max_partials, cudaStream_t s);
cudaError_t launch_axpy64(long n, double g, const double* x, double* y, cudaStream_t s);       // y += g x
cudaError_t launch_scale64(long n, double sc, const double* x, double* y, cudaStream_t s);     // y = sc x
cudaError_t launch_spread(long nodes, int N, double c, const double* yd, double* fy, cudaStream_t s);  // fy[i][j] = c yd[i]
cudaError_t launch_fill32(long n, float v, float* x, cudaStream_t s);
cudaError_t launch_scale32(long n, float sc, const float* x, float* y, cudaStream_t s);    // y = sc x
cudaError_t launch_inject32(int nf, const float* fine, float* coarse, cudaStream_t s);  // coarse = fine at coinciding nodes

// ---- cluster-resident coarse-grid cycle (cmg_tail.cuh, cmg_tail_f32/f64.cu) ----
constexpr int kTailMax = 8;        // grids handled inside one cluster launch
constexpr int kTailThreads = 512;  // threads per CTA of the cluster kernel

template <typename T>
struct TailLevel {
  LevelView<T> L;
  Vec3<T> x, f, r;   // iterate, right side, residual work vector of this grid
};

template <typename T>
struct TailParams {
  int nlev;                        // grids in the tail, the last is the coarsest
  TailLevel<T> lev[kTailMax];
  int smoother, n1, n2, gamma;
  double theta;
  int freeze_u;                    // coarsest solve with a zero control correction
  int lpn;                         // lanes per node (SampleMap of N)
  // coarsest grid (CoarseData) and its blocks c, d, e
  int cm, cN;
  const double* Ainv;
  const double* Minv;
  double* wz;
  double cc, cd, ce;
};

// One launch of a thread-block cluster running Algorithm 1 from grid lev[0]
// down to the coarsest.  Returns cudaErrorNotSupported (nothing launched)
// when the sample count or the cluster configuration is not covered.
template <typename T>
cudaError_t launch_tail_cycle(const TailParams<T>& P, cudaStream_t s);
bool tail_supported(int N, int elem_bytes, int coarse_m);

// FP64 refinement pass: r32 = s (f - S x) and per-CTA partial sums of
// ||W r32||^2 (W scales the state block by wy).  Returns the number of
// partials written, or -1 on error / if more than max_partials are needed.
// The scale is *sdev when sdev is given (graph replays), else s.
int launch_residual_cast(const LevelView<double>& L, Vec3c<double> x, Vec3c<double> f, Vec3<float> r, double s,
                         const double* sdev, double wy, double* partial, int max_partials, cudaStream_t st,
                         const double* gate = nullptr);
// x += a * e on the three blocks (ny elements in y and p, nu in u); a is
// *adev when adev is given.
// Residual replacement in FP32 refinement (cmg_stencil.cu): r <- r - S e in
// place, d += e, partials of ||W r||^2 (returns their count or -1); and the
// gated anchor fold x += (*adev) d, d = 0 (nothing when *gate == 0).
int launch_recur(const LevelView<float>& L, Vec3c<float> e, Vec3<float> r, Vec3<float> d, double wy, double* partial,
                 int max_partials, cudaStream_t s);
cudaError_t launch_fold(const double* adev, const double* gate, Vec3<float> d, Vec3<double> x, size_t ny, size_t nu,
                        cudaStream_t s);
cudaError_t launch_zero3(Vec3<float> v, size_t ny, size_t nu, cudaStream_t s);
cudaError_t launch_axpy3(double a, const double* adev, Vec3c<float> e, Vec3<double> x, size_t ny, size_t nu,
                         cudaStream_t st);

// State of the FP32 refinement loop of one instance (device doubles; see
// the refinement loop in cmg_api.cu):
enum IrState {
  kSc = 0,       // scale for the next FP64 pass (1 / latest norm)
  kInvSc = 1,    // 1 / scale of the current right side r^ (also of d)
  kRho = 2,      // latest residual norm (recursive between anchors, true at one)
  kIt = 3,       // cycles done
  kMaxit = 4,
  kTolAbs = 5,
  kRhoAnchor = 6,   // true norm at the last anchor
  kSince = 7,       // cycles since the last anchor
  kAnchor = 8,      // 1: the anchor kernels of this iteration run
  kGo = 9,          // 1: another iteration follows
  kDrop = 10,       // anchor once the recursive norm is below kDrop times the last true one
  kAmax = 11,       // ... or after kAmax cycles since the last anchor
  kIrStateSize = 12
};

// ---- batched persistent form (cmg_batch.cu, batched coarsest solve in cmg_coarse.cu) ----
// Many independent instances advance through the FP32 refinement loop in
// lockstep.  Their grids are aligned by depth (depth 0 = each instance's
// finest grid); a V-cycle is one persistent launch per depth for the
// down-leg (pre-smoothing, residual, restriction), one launch for every
// instance's coarsest solve, and one persistent launch per depth for the
// up-leg (prolongation fused into the first post-smoothing half-sweep, the
// remaining half-sweeps).  A persistent launch walks a work list of (instance,
// warp of nodes) items phase by phase, with a grid-wide barrier between
// phases; instances that have converged are skipped (act[i] = 0).

// Sample maps of the batched FP32 node kernels: on depths run one launch
// per phase and map class, 16 samples per lane (kBatchMapPhase: 16 / V chunks
// of V; measured faster than 4 samples or 4 chunks per lane); in the
// persistent kernels, whose map is chosen at run time, four samples per lane
// (kBatchMapCoop: the registers of the widest variant stay within two CTAs
// per SM).
constexpr int kBatchMapCoop = 0;
constexpr int kBatchMapPhase = 1;

// One grid of one instance as the batched kernels see it.
struct BatchLevel {
  LevelView<float> L;     // FP32 operator of this grid
  Vec3<float> x, f, r;    // iterate (a correction), right side, residual
  int lpn, V, spl;        // sample map (by the rule BatchTables::maps of this depth)
  int nc;                 // nodes per side of the next coarser grid (0 on the coarsest)
};

// Finest-grid data of one instance for the refinement steps.
struct BatchInst {
  LevelView<double> L64;  // FP64 operator (anchor residual)
  Vec3c<double> f64;      // right side
  Vec3<double> x64;       // solution
  Vec3<float> d32;        // FP32 sum of the corrections since the last anchor
  double* state;          // refinement state (the single-instance loop's layout)
  float wy2;              // weight of the state block in ||W r||^2
  int lpn64, V64, spl64;  // FP64 sample map
  int levels;             // grids of this instance
};

// Coarsest grid of one instance (FP32 cycle).
struct BatchCoarse {
  int m, N, nside;
  CtlBox ctl;
  const float* Ainv32;
  const double* Minv;
  double c, d, e;
  const float* dw;
  Vec3c<float> f;
  Vec3<float> x;
};

size_t batch_coarse_smem(int N_max, int m);
cudaError_t launch_batch_coarse(const BatchCoarse* bc, int count, int N_max, int m, const int* act, const int* err,
                                cudaStream_t s);

// Device tables of a batch: per instance, kMaxLevels BatchLevel entries and
// one BatchInst; item prefix counts per (depth, kind) of length count + 1.
enum BatchKind { kBkColour0 = 0, kBkColour1 = 1, kBkCoarse = 2, kBkAll32 = 3, kBkAll64 = 4, kBkKinds = 5 };
// Tables per map class: 0 = every instance, 1 / 2 / 3 = the instances whose
// FP32 vectors are 4 / 2 / 1 samples wide.
constexpr int kBkClasses = 4;
struct BatchTables {
  int count;
  int depths;                   // the deepest instance's grid count
  const BatchLevel* lev;        // [count][kMaxLevels]
  const BatchInst* inst;        // [count]
  const int* pre;               // [depths][kBkKinds][kBkClasses][count + 1]
  int cls_mask[kMaxLevels];     // per depth: bit c-1 set when map class c has instances there
  int maps[kMaxLevels];         // per depth: the map rule of its grids (kBatchMapCoop or kBatchMapPhase)
  int items[kMaxLevels][kBkKinds][kBkClasses];   // the prefix tables' totals (host copy: launch grids)
  // per (depth, kind, class): the instance of item 8 b (the first item of
  // CTA b of a one-item-per-warp launch), at first + first_off[..]
  const int* first;
  int first_off[kMaxLevels][kBkKinds][kBkClasses];
  const int* act;               // [count] 1 = instance iterating
  unsigned* bar;                // grid barrier words [2]
  int* err;                     // 0 = fine, 1 = a barrier wait ran out (all kernels then return)
  long long limit;              // polls per barrier wait before giving up
  double* partial;              // per-item partial sums of the refinement norms
  int n1, n2;                   // pre- and post-smoothing sweeps
};
// Item prefix counts of (depth, kind, map class) in a batch's tables.
__host__ __device__ inline const int* batch_prefix(const BatchTables& T, int depth, int kind, int cls) {
  return T.pre + (((size_t)depth * kBkKinds + kind) * kBkClasses + cls) * (T.count + 1);
}
// Largest persistent grid of the batched kernels (co-resident CTAs on this
// GPU); per_sm > 0 caps the CTAs per SM.
int batch_grid(int which, int per_sm);
cudaError_t launch_batch_down(const BatchTables& T, int depth, int grid, cudaStream_t s);
cudaError_t launch_batch_up(const BatchTables& T, int depth, int grid, cudaStream_t s);
// The same legs as one ordinary launch per phase (no barrier; for the grids
// with the most work, where the persistent kernel's registers would halve
// the resident warps).
cudaError_t launch_batch_down_phases(const BatchTables& T, int depth, cudaStream_t s);
cudaError_t launch_batch_up_phases(const BatchTables& T, int depth, cudaStream_t s);
cudaError_t launch_batch_recur(const BatchTables& T, cudaStream_t s);
cudaError_t launch_batch_anchor(const BatchTables& T, cudaStream_t s);
// Per-instance control of the refinement (same decisions as the single-
// instance loop): after the recursion and after the anchor.
cudaError_t launch_batch_recur_control(const BatchTables& T, cudaStream_t s);
cudaError_t launch_batch_anchor_control(const BatchTables& T, cudaStream_t s);


// ---- coarsest grid (cmg_coarse.cu) ----
template <typename T>
cudaError_t launch_coarse_solve(const CoarseData& C, double c, double d, double e,
                                Vec3c<T> f, Vec3<T> x, cudaStream_t s, int freeze_u = 0);
cudaError_t launch_coarse_setup(const CoarseData& C, const double* kx, const double* ky,
                                double c, double G, double d, double e, cudaStream_t s);

// ---- coefficients (cmg_setup.cu) ----
// Nodal field on the (n+2)^2 grid including boundary points, then faces,
// 1/diag and Schur denominators.  kap: scratch [(n+2)^2][N] doubles.
// a[node][j] = sum of the node's four faces (FP64).
cudaError_t launch_diag_sum(int n, int N, const double* kx, const double* ky, double* a, cudaStream_t s);
cudaError_t launch_level_setup(int n, int N, int K, double amp, const double* xi, double* kap,
                               double* kx64, double* ky64, float* kx32, float* ky32,
                               double* inva, double* isigma, double c, double G, double d,
                               double e, cudaStream_t s);

// Coarse grid (nf-1)/2 with faces averaged from the finer grid's faces, then
// 1/diag and Schur denominators.
cudaError_t launch_coarse_level_setup(int nf, int N, const double* kxf, const double* kyf, double* kx64,
                                      double* ky64, float* kx32, float* ky32, double* inva, double* isigma,
                                      double c, double G, double d, double e, cudaStream_t s);

// Split set-up used for the averaged coarse grids: the FP32 cycle's
// operators (finest FP32 faces rounded from FP64, coarse FP32 faces averaged
// in FP32, 1/sigma from those) are built with every new sample set; the FP64
// coarse operators only when an FP64 cycle needs them.
cudaError_t launch_field_faces(int n, int N, int K, double amp, const double* xi, double* kap, double* kx64,
                               double* ky64, float* kx32, float* ky32, cudaStream_t s);
cudaError_t launch_diag64(int n, int N, const double* kx64, const double* ky64, double* inva, double* isigma,
                          double dce, double G, cudaStream_t s, const float* dw = nullptr);
cudaError_t launch_coarse_faces64(int nf, int N, const double* kxf, const double* kyf, double* kx64, double* ky64,
                                  cudaStream_t s);
cudaError_t launch_coarse_faces32(int nf, int N, const float* kxf, const float* kyf, float* kx32, float* ky32,
                                  cudaStream_t s);
// 1/sigma of the FP32 operator (sum over samples in FP64): FP64 isigma_d and
// its FP32 rounding isigma32.
cudaError_t launch_diag32(int n, int N, const float* kx32, const float* ky32, float* isigma32, double* isigma_d,
                          double dce, double G, cudaStream_t s, const float* dw = nullptr);

// ---- vector kernels (cmg_blas.cu) ----
constexpr int kRedBlocks = 304;    // fixed partial count: deterministic reductions
// partial[0..kRedBlocks) (+)= w2 * per-block sums of squares; call finish to combine.
cudaError_t launch_sumsq(const double* a, size_t n, double* partial, int accumulate, double w2, cudaStream_t s);
cudaError_t launch_finish_sum(const double* partial, int count, double* out, cudaStream_t s);
// out[i] = sum_k V_i[k] w[k], i < nv; V_i = V + i*stride.  partial: [nv][kRedBlocks]
cudaError_t launch_mdot(const double* V, size_t stride, int nv, const double* w, size_t n,
                        double* partial, double* out, cudaStream_t s);
// w += sign * sum_i coef[i] V_i  (coef on device)
cudaError_t launch_maxpy(const double* V, size_t stride, int nv, const double* coef, double sign,
                         double* w, size_t n, cudaStream_t s);
// y = alpha * x (alpha read from device scalar: y = x / *den if inv)
cudaError_t launch_scale_by(const double* x, const double* den, double* y, size_t n, cudaStream_t s);
// y += a * x (host scalar)
template <typename Tx, typename Ty>
cudaError_t launch_axpy(double a, const Tx* x, Ty* y, size_t n, cudaStream_t s);
// y = (Ty)(a * x)
template <typename Tx, typename Ty>
cudaError_t launch_scale_cast(double a, const Tx* x, Ty* y, size_t n, cudaStream_t s);
// y = (h^2/N) yd broadcast over samples, u = 0, p = h^2 f broadcast
cudaError_t launch_rhs(int n, int N, double h, const double* yd, const double* fsrc, double* fy,
                       double* fu, double* fp, cudaStream_t s);

// ---- Galerkin coarse operators (cmg_galerkin.cu, cmg_coarse.cu) ----
// Sec. 3 builds the coarse matrices as S_l = P^T S_{l-1} P with the bilinear
// P.  On a coarse grid every block is then a 9-point stencil: A_j variable
// ([9][n*n][N], offset k = (dy+1)*3 + (dx+1)) and the mass M_l constant
// (Stencil9; M_0 = I), the blocks c M_l, G M_l, d M_l, e M_l with the finest
// grid's c, G, d, e.
struct Stencil9 {
  double w[9];
};
// M_l from M_{l-1} (the same triple product with a constant stencil).
Stencil9 galerkin_mass(const Stencil9& fine);
// out9 = P^T A P on the (nf-1)/2 grid, from the finest grid's faces (in9 ==
// nullptr) or from the 9-point A of the nf grid.
cudaError_t launch_galerkin_setup(int nf, int N, const double* kx, const double* ky, const double* in9, double* out9,
                                  cudaStream_t s);
// inva = 1 / (A_j)_ii, isigma = 1 / (G + dce sum_j inva^2) (the Schur
// denominator of Eq. (13) with the diagonal entries of the blocks).
cudaError_t launch_galerkin_diag(int n, int N, const double* a9, double* inva, double* isigma, double dce, double G,
                                 cudaStream_t s);
// r = f - S_l x (r = S_l x when f.y == nullptr) with 9-point blocks: one
// launch on small grids; on larger ones three, with psum (scratch [2 n*n]
// FP64) holding the sums over samples of x.p, then (M u)_i.  T = double, or
// float for the FP32 cycle on FP32 copies of the planes (the control row
// and the sums over samples stay FP64).
template <typename T>
cudaError_t launch_residual9(int n, int N, const T* a9, const Stencil9& M, double c, double G, double d, double e,
                             Vec3c<T> x, Vec3c<T> f, Vec3<T> r, double* psum, cudaStream_t s);
// One collective Gauss-Seidel sweep in four colours (iy mod 2, ix mod 2) on
// a 9-point grid (Eq. (13) per node with the Galerkin diagonal entries):
// four launches for N <= 256; above, psum (scratch [n*n], the sums over
// samples of p) is filled first and kept current by the sweep.
// FP32: per-sample work in FP32, the Schur scalar of Eq. (13) in FP64.
template <typename T>
cudaError_t launch_gs4_sweep(int n, int N, const T* a9, const Stencil9& M, double c, double G, double d, double e,
                             const T* inva, const double* isigma, Vec3<T> x, Vec3c<T> f, double* psum,
                             cudaStream_t s);
// Damped collective Jacobi update x += theta S~^{-1} r on a 9-point grid
// (FP32; the FP64 cycle uses the 5-point update with the stored 1/a).
template <typename T>
cudaError_t launch_galerkin_jacobi(int n, int N, const Stencil9& M, double c, double d, double e, double theta,
                                   const T* inva, const double* isigma, Vec3<T> x, Vec3c<T> r, cudaStream_t s);
// Coarsest grid: A_j^{-1} per sample from the 9-point stencil, and the
// inverse of the control Schur matrix G M + d c e M (sum_j A_j^{-1} M A_j^{-1}) M.
cudaError_t launch_galerkin_coarse_setup(const CoarseData& C, const double* a9, const Stencil9& M, double c,
                                         double G, double d, double e, cudaStream_t s);
// x = S_L^{-1} f on the coarsest grid by block elimination with the
// non-diagonal mass (x and f must not overlap), in FP64 whatever T (the
// cycle's precision) f and x are stored in.
template <typename T>
cudaError_t launch_galerkin_coarse_solve(const CoarseData& C, const Stencil9& M, double c, double d, double e,
                                         Vec3c<T> f, Vec3<T> x, cudaStream_t s);

// ---- warm-start network kernels (cmg_nn_*.cu) ----
// mean over samples of log kappa_j at the n x n interior nodes of the finest grid.
cudaError_t launch_mean_log_kappa(int n, int N, int K, double amp, const double* xi, double* out, cudaStream_t s);

// C[M][N] = A[M][K] * B[N][K]^T (+ bias, ReLU) on tcgen05; row strides lda,
// ldb; K % 8 == 0.
// ksplit > 1: K is the slice length, slice z reads columns z*K.. and writes
// C32 + z*M*ldc (FP32 partials, no bias / ReLU / C16).
// Poll limit of the tensor-core GEMM's waits for work (0 = the default).
void set_gemm_wait_limit(long long polls);
// 3x3 convolution with zero padding 1 as an implicit GEMM on the tensor cores:
// Y[p][co] = sum_{t, c} X(pixel p shifted by tap t)[c] Wt[co][t C + c] (+
// bias, ReLU), X NHWC BF16 [B][H][W][C], Wt [Cout][9 C], Y [B H W][Cout] BF16
// (the im2col + GEMM result, bit for bit).  cudaErrorNotSupported where it
// does not apply (C neither a multiple of 32 nor 8, 16 or 24; Cout > 64; no
// tensor map; CMG_GEMM_TMA=0).
cudaError_t launch_conv3x3_bf16(const void* X, int B, int H, int W, int C, const void* Wt, int Cout,
                                const float* bias, int relu, void* Y16, int* status, cudaStream_t s);
cudaError_t launch_gemm_bf16_tn(const void* A, long lda, const void* B, long ldb, int M, int N, int K,
                                const float* bias, int relu, float* C32, void* C16, int ldc, int* status,
                                cudaStream_t s, int ksplit = 1);

}  // namespace cmg
