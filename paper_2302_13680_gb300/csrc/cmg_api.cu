// C ABI of libcmg (include/cmg.h): handle, grid hierarchy, cycles and
// outer solvers.  All device work is enqueued on the handle's stream.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <algorithm>
#include <atomic>

#include "cmg_common.cuh"

using namespace cmg;

namespace cmg {
static std::atomic<long long> g_launches{0};
void count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
}  // namespace cmg

namespace {

struct Lev {
  int n = 0;
  CtlBox ctl;                            // nodes with a control basis function (local control)
  int spl_target[2] = {0, 0};            // autotuned chunks per lane: [FP64, FP32]
  double h = 0, c = 0, G = 0, d = 0, e = 0;
  size_t nodes = 0;                      // n*n
  double *kx64 = nullptr, *ky64 = nullptr, *inva = nullptr, *isigma = nullptr;
  float* isigma32 = nullptr;             // 1/sigma in FP32 (the FP32 cycle's all-FP32 option)
  double* isigd32 = nullptr;             // 1/sigma of the FP32 operator in FP64 (the FP32 cycle's Schur scalar)
  double* a64 = nullptr;                 // finest grid: diag(A_j) for the FP64 refinement residual
  float *kx32 = nullptr, *ky32 = nullptr;
  double* x64[3] = {nullptr, nullptr, nullptr};
  double* f64[3] = {nullptr, nullptr, nullptr};
  double* r64[3] = {nullptr, nullptr, nullptr};
  float* x32[3] = {nullptr, nullptr, nullptr};
  float* xs32[3] = {nullptr, nullptr, nullptr};  // second FP32 iterate for the one-launch sweeps (N % 4 == 0)
  float* d32[3] = {nullptr, nullptr, nullptr};   // finest grid: FP32 correction since the last refinement anchor
  float* dw = nullptr;                   // per-node factor on d (1; semismooth Newton: active-set indicator)
  // Galerkin coarse operators (grids below the finest): 9-point A_j planes
  // [9][n*n][N], the mass stencil M_l, and a scratch [2 n*n] for the
  // 9-point residual (sums over samples, then M u).
  // c, G, d, e above then hold the diagonal entries (times M_l's centre).
  double* a9 = nullptr;
  double* psum = nullptr;
  Stencil9 m9{};
  float* a9f = nullptr;     // FP32 copies of the planes and of 1/(A_j)_ii for the FP32 cycle
  float* invaf = nullptr;
  float* f32[3] = {nullptr, nullptr, nullptr};
  float* r32[3] = {nullptr, nullptr, nullptr};
};

template <typename T> struct Work;
template <> struct Work<double> {
  static Vec3<double> x(Lev& l) { return {l.x64[0], l.x64[1], l.x64[2]}; }
  static Vec3<double> f(Lev& l) { return {l.f64[0], l.f64[1], l.f64[2]}; }
  static Vec3<double> r(Lev& l) { return {l.r64[0], l.r64[1], l.r64[2]}; }
};
template <> struct Work<float> {
  static Vec3<float> x(Lev& l) { return {l.x32[0], l.x32[1], l.x32[2]}; }
  static Vec3<float> f(Lev& l) { return {l.f32[0], l.f32[1], l.f32[2]}; }
  static Vec3<float> r(Lev& l) { return {l.r32[0], l.r32[1], l.r32[2]}; }
};

constexpr int kMaxRestart = 60;
constexpr int kMaxProf = 4096;   // event pairs recorded per profiling window

}  // namespace

struct cmg_handle {
  cmg_problem prob{};
  cudaStream_t stream = nullptr;
  int L = 0;
  Lev lv[kMaxLevels];
  CoarseData coarse{};     // coarsest-grid inverses from the FP64 operators (FP64 cycles)
  CoarseData coarse32{};   // from the FP32 operators (FP32 cycles; averaged coarse grids only)
  double* cface64 = nullptr;   // coarsest FP32 faces promoted to FP64 for coarse32's set-up
  bool fp64_ready = false;     // FP64 operators below the finest faces are current
  bool g32_ready = false;      // Galerkin handles: the FP32 copies of the coarse planes are current
  CoarseData& c32() { return prob.coarse_coeff == CMG_COARSE_NODAL ? coarse : coarse32; }
  bool galerkin() const { return prob.coarse_coeff == CMG_COARSE_GALERKIN; }
  double* xi = nullptr;       // [N][K] device
  double* kap = nullptr;      // setup scratch
  double* red = nullptr;      // reduction partials
  double* dsc = nullptr;      // device scalars
  double* hsc = nullptr;      // pinned host scalars
  double* part = nullptr;     // per-CTA partial sums of the fused refinement pass
  int part_cap = 0;
  double* ssn = nullptr;      // semismooth Newton work vectors (allocated on first use)
  double gscale = 1.0;        // factor on every grid's G (1/nu: the Newton systems' control row form)
  bool dw_on = false;         // the per-node factors on d are in use (else the views carry none: factor 1)
  // FP32 refinement loop as a CUDA graph with a device-side while node
  cudaStream_t cap = nullptr;            // non-blocking stream used for capture
  cudaGraph_t ir_graph = nullptr;
  cudaGraphExec_t ir_exec = nullptr;
  const void* ir_key[6] = {};
  double ir_gscale = 1.0;                // gscale the captured loop was built with (its kernels hold G by value)
  cmg_cycle ir_opts{};
  double* ir_state = nullptr;            // device refinement state, see IrState
  double anchor_drop = 1e-3;             // anchor policy of FP32 refinement (see IrState)
  int anchor_max = 8;
  long long ir_body_kernels = 0;         // kernels in one iteration of the captured loop body
  bool graphs = true;                    // false: CMG_GRAPHS=0 in the environment at creation
  // FGMRES workspace
  int gm_cap = 0;
  double* gm = nullptr;       // [2*cap + 2][nt_pad]
  size_t nt = 0, nt_pad = 0;
  std::vector<void*> allocs;
  std::string err;
  // kernel timing window (cmg_profile_begin / end)
  int prof_kinds = 0, prof_level = -1, prof_n = 0;
  std::vector<cudaEvent_t> prof_ev;
};

namespace {

cmg_status fail(cmg_handle* h, cmg_status st, const std::string& msg) {
  if (h) h->err = msg;
  return st;
}

cmg_status cuda_fail(cmg_handle* h, cudaError_t e, const char* what) {
  const cmg_status st = (e == cudaErrorMemoryAllocation) ? CMG_ERR_OOM : CMG_ERR_CUDA;
  (void)cudaGetLastError();  // clear a sticky launch error so the handle stays usable
  return fail(h, st, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                          \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

template <typename T>
cudaError_t dalloc(cmg_handle* h, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, (count ? count : 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  h->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return cudaSuccess;
}

// Brackets one launch of `kind` on grid `level` with CUDA events when the
// profiling window asks for it.
struct ProfScope {
  cmg_handle* h;
  int idx = -1;
  ProfScope(cmg_handle* hh, int kind, int level) : h(hh) {
    if ((h->prof_kinds & kind) && level == h->prof_level && h->prof_n < kMaxProf) {
      idx = h->prof_n++;
      (void)cudaEventRecord(h->prof_ev[2 * idx], h->stream);
    }
  }
  ~ProfScope() {
    if (idx >= 0) (void)cudaEventRecord(h->prof_ev[2 * idx + 1], h->stream);
  }
};

// ctl32: the FP32 cycle's all-FP32 option (cmg_cycle.ctl32); FP64 views ignore it.
template <typename T>
LevelView<T> view(const cmg_handle* h, int l, int freeze_u = 0, int ctl32 = 0);
template <>
LevelView<double> view<double>(const cmg_handle* h, int l, int freeze_u, int) {
  const Lev& v = h->lv[l];
  return {v.n, h->prob.N, h->prob.N, v.kx64, v.ky64, v.inva, v.isigma, v.c, v.G * h->gscale, v.d, v.e,
          v.spl_target[0], freeze_u, nullptr, v.a64, v.ctl, h->dw_on ? v.dw : nullptr, 0};
}
template <>
LevelView<float> view<float>(const cmg_handle* h, int l, int freeze_u, int ctl32) {
  const Lev& v = h->lv[l];
  // nodal coarse grids round the FP64 operator's 1/sigma; averaged ones have
  // their own FP32 operator with its FP64 1/sigma
  const double* isd = h->prob.coarse_coeff == CMG_COARSE_NODAL ? v.isigma : v.isigd32;
  return {v.n, h->prob.N, h->prob.N, v.kx32, v.ky32, v.inva, isd, v.c, v.G * h->gscale, v.d, v.e,
          v.spl_target[1], freeze_u, v.isigma32, nullptr, v.ctl, h->dw_on ? v.dw : nullptr, ctl32 ? 1 : 0};
}

// The coarsest-grid data for a cycle of precision T; its per-node factor on d
// is passed only while the factors are in use (else the kernels skip it).
template <typename T>
CoarseData coarse_for(cmg_handle* h) {
  CoarseData c = sizeof(T) == 4 ? h->c32() : h->coarse;
  if (!h->dw_on) c.dw = nullptr;
  return c;
}

bool level_ok(const cmg_handle* h, int l) { return h && l >= 0 && l < h->L; }

template <typename T>
bool vec_ok(const T* y, const T* u, const T* p) {
  // the node kernels move 16-byte vectors: a misaligned pointer is refused
  // here instead of faulting on the device
  const auto a16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
  return y && u && p && a16(y) && a16(u) && a16(p);
}

// Operators for a new sample set.  Averaged coarse grids (default): the
// finest FP64 + FP32 faces and diag(A) (the FP64 refinement residual needs
// them), then the FP32 cycle's operators on every grid, built in FP32; the
// FP64 operators below the finest faces wait for ensure_fp64.  Nodal coarse
// grids: everything at once, as each grid samples the field itself.
cudaError_t setup_coefficients(cmg_handle* h) {
  const cmg_problem& P = h->prob;
  if (P.coarse_coeff == CMG_COARSE_NODAL) {
    for (int l = 0; l < h->L; ++l) {
      Lev& v = h->lv[l];
      cudaError_t e = launch_level_setup(v.n, P.N, P.K, P.amp, h->xi, h->kap, v.kx64, v.ky64, v.kx32, v.ky32, v.inva,
                                         v.isigma, v.c, v.G, v.d, v.e, h->stream);
      if (e == cudaSuccess) e = launch_scale_cast<double, float>(1.0, v.isigma, v.isigma32, v.nodes, h->stream);
      if (e == cudaSuccess && v.a64) e = launch_diag_sum(v.n, P.N, v.kx64, v.ky64, v.a64, h->stream);
      if (e != cudaSuccess) return e;
    }
    const Lev& cl = h->lv[h->L - 1];
    h->fp64_ready = true;
    return launch_coarse_setup(h->coarse, cl.kx64, cl.ky64, cl.c, cl.G, cl.d, cl.e, h->stream);
  }
  h->fp64_ready = false;
  h->g32_ready = false;
  Lev& v0 = h->lv[0];
  cudaError_t e = launch_field_faces(v0.n, P.N, P.K, P.amp, h->xi, h->kap, v0.kx64, v0.ky64, v0.kx32, v0.ky32,
                                     h->stream);
  if (e == cudaSuccess) e = launch_diag_sum(v0.n, P.N, v0.kx64, v0.ky64, v0.a64, h->stream);
  for (int l = 0; l < h->L && e == cudaSuccess; ++l) {
    Lev& v = h->lv[l];
    if (l > 0) {
      const Lev& f = h->lv[l - 1];
      e = launch_coarse_faces32(f.n, P.N, f.kx32, f.ky32, v.kx32, v.ky32, h->stream);
    }
    if (e == cudaSuccess)
      e = launch_diag32(v.n, P.N, v.kx32, v.ky32, v.isigma32, v.isigd32, v.d * v.c * v.e, v.G * h->gscale, h->stream, v.dw);
  }
  if (e != cudaSuccess) return e;
  const Lev& cl = h->lv[h->L - 1];
  const size_t cf = (size_t)cl.n * (cl.n + 1) * P.N;
  e = launch_scale_cast<float, double>(1.0, cl.kx32, h->cface64, cf, h->stream);
  if (e == cudaSuccess) e = launch_scale_cast<float, double>(1.0, cl.ky32, h->cface64 + cf, cf, h->stream);
  if (e != cudaSuccess) return e;
  return launch_coarse_setup(h->coarse32, h->cface64, h->cface64 + cf, cl.c, cl.G * h->gscale, cl.d, cl.e,
                             h->stream);
}

// The FP64 operators below the finest faces (1/diag, 1/sigma on every grid,
// the averaged coarse faces, the coarsest inverses), built on the handle's
// stream the first time an FP64 cycle, smoother or coarse solve needs them
// after a new sample set.
cudaError_t ensure_fp64(cmg_handle* h) {
  if (h->fp64_ready) return cudaSuccess;
  const cmg_problem& P = h->prob;
  cudaError_t e = cudaSuccess;
  if (h->galerkin()) {
    // finest grid as for the rediscretised hierarchy; below it S_l = P^T S_{l-1} P
    const Lev& f0 = h->lv[0];
    e = launch_diag64(f0.n, P.N, f0.kx64, f0.ky64, f0.inva, f0.isigma, f0.d * f0.c * f0.e, f0.G, h->stream);
    for (int l = 1; l < h->L && e == cudaSuccess; ++l) {
      Lev& v = h->lv[l];
      const Lev& f = h->lv[l - 1];
      e = launch_galerkin_setup(f.n, P.N, f0.kx64, f0.ky64, l == 1 ? nullptr : f.a9, v.a9, h->stream);
      if (e == cudaSuccess) e = launch_galerkin_diag(v.n, P.N, v.a9, v.inva, v.isigma, v.d * v.c * v.e, v.G, h->stream);
    }
    if (e != cudaSuccess) return e;
    const Lev& cl = h->lv[h->L - 1];
    e = launch_galerkin_coarse_setup(h->coarse, cl.a9, cl.m9, f0.c, f0.G, f0.d, f0.e, h->stream);
    if (e == cudaSuccess) h->fp64_ready = true;
    return e;
  }
  for (int l = 0; l < h->L && e == cudaSuccess; ++l) {
    Lev& v = h->lv[l];
    if (l > 0) {
      const Lev& f = h->lv[l - 1];
      e = launch_coarse_faces64(f.n, P.N, f.kx64, f.ky64, v.kx64, v.ky64, h->stream);
    }
    if (e == cudaSuccess)
      e = launch_diag64(v.n, P.N, v.kx64, v.ky64, v.inva, v.isigma, v.d * v.c * v.e, v.G * h->gscale, h->stream,
                        v.dw);
  }
  if (e != cudaSuccess) return e;
  const Lev& cl = h->lv[h->L - 1];
  e = launch_coarse_setup(h->coarse, cl.kx64, cl.ky64, cl.c, cl.G * h->gscale, cl.d, cl.e, h->stream);
  if (e == cudaSuccess) h->fp64_ready = true;
  return e;
}

// Galerkin handles, FP32 cycles: FP32 copies of the coarse grids' planes and
// 1/(A_j)_ii, from the FP64 operators (built first); 1/sigma and the coarsest
// solve stay FP64.
cudaError_t ensure_galerkin32(cmg_handle* h) {
  if (!h->galerkin() || h->g32_ready) return cudaSuccess;
  cudaError_t e = ensure_fp64(h);
  const size_t N = (size_t)h->prob.N;
  for (int l = 1; l < h->L && e == cudaSuccess; ++l) {
    Lev& v = h->lv[l];
    e = launch_scale_cast<double, float>(1.0, v.a9, v.a9f, 9 * v.nodes * N, h->stream);
    if (e == cudaSuccess) e = launch_scale_cast<double, float>(1.0, v.inva, v.invaf, v.nodes * N, h->stream);
  }
  if (e == cudaSuccess) h->g32_ready = true;
  return e;
}

// The operators a call in precision T reads.
template <typename T>
cudaError_t ensure_ops(cmg_handle* h) {
  if constexpr (sizeof(T) == 8) return ensure_fp64(h);
  else return ensure_galerkin32(h);
}

// After the finest grid's per-node factor on d changed: inject it to the
// coarse grids and rebuild what depends on it (1/sigma on every grid, the
// coarsest control Schur inverse), for the FP32 operators and, where built,
// the FP64 ones.
cudaError_t refresh_dw(cmg_handle* h) {
  const cmg_problem& P = h->prob;
  const bool nodal = P.coarse_coeff == CMG_COARSE_NODAL;
  cudaError_t e = cudaSuccess;
  for (int l = 1; l < h->L && e == cudaSuccess; ++l)
    e = launch_inject32(h->lv[l - 1].n, h->lv[l - 1].dw, h->lv[l].dw, h->stream);
  for (int l = 0; l < h->L && e == cudaSuccess; ++l) {
    Lev& v = h->lv[l];
    const double G = v.G * h->gscale;
    if (nodal || h->fp64_ready)
      e = launch_diag64(v.n, P.N, v.kx64, v.ky64, v.inva, v.isigma, v.d * v.c * v.e, G, h->stream, v.dw);
    if (e != cudaSuccess) break;
    e = nodal ? launch_scale_cast<double, float>(1.0, v.isigma, v.isigma32, v.nodes, h->stream)
              : launch_diag32(v.n, P.N, v.kx32, v.ky32, v.isigma32, v.isigd32, v.d * v.c * v.e, G, h->stream, v.dw);
  }
  if (e != cudaSuccess) return e;
  const Lev& cl = h->lv[h->L - 1];
  if (!nodal) {
    const size_t cf = (size_t)cl.n * (cl.n + 1) * P.N;
    e = launch_coarse_setup(h->coarse32, h->cface64, h->cface64 + cf, cl.c, cl.G * h->gscale, cl.d, cl.e,
                            h->stream);
  }
  if (e == cudaSuccess && (nodal || h->fp64_ready))
    e = launch_coarse_setup(h->coarse, cl.kx64, cl.ky64, cl.c, cl.G * h->gscale, cl.d, cl.e, h->stream);
  return e;
}

// ---- smoothing and cycles --------------------------------------------------

// r = f - S_l x (r = S_l x when f.y == nullptr): the 9-point Galerkin
// operator on the coarse grids of a Galerkin hierarchy, else the 5-point one.
template <typename T>
cudaError_t level_residual(cmg_handle* h, int l, Vec3c<T> x, Vec3c<T> f, Vec3<T> r) {
  if (h->galerkin() && l > 0) {
    const Lev& v = h->lv[l];
    const Lev& f0 = h->lv[0];
    const T* a9 = nullptr;
    if constexpr (sizeof(T) == 8) a9 = v.a9;
    else a9 = v.a9f;
    return launch_residual9<T>(v.n, h->prob.N, a9, v.m9, f0.c, f0.G, f0.d, f0.e, x, f, r, v.psum, h->stream);
  }
  return launch_residual<T>(view<T>(h, l), x, f, r, h->stream);
}

// The red-black sweeps on grid l run as one launch each (launch_rbgs_fused),
// in pairs through the level's second iterate: FP32 cycles with the control
// updated on grids tuned for it (kTuneFused) whose shape the kernel covers.
bool fused_on(cmg_handle* h, const cmg_cycle& o, int l) {
  const Lev& v = h->lv[l];
  if (o.smoother != CMG_SMOOTH_RBGS || o.freeze_u || !(v.spl_target[1] & kTuneFused) || !v.xs32[0]) return false;
  if (h->galerkin() && l > 0) return false;
  return fused_plan(v.n, h->prob.N, v.spl_target[1]).ok;
}

Vec3<float> second_iterate(Lev& v) { return {v.xs32[0], v.xs32[1], v.xs32[2]}; }

// One pair of one-launch sweeps: the first (mode) from x into the second
// iterate, the second (plain) back into x.
cudaError_t fused_pair(cmg_handle* h, const cmg_cycle& o, int l, Vec3<float> x, Vec3c<float> f, int mode,
                       Vec3c<float> e = Vec3c<float>{nullptr, nullptr, nullptr}, int nc = 0) {
  Lev& v = h->lv[l];
  const LevelView<float> L = view<float>(h, l, o.freeze_u, o.ctl32);
  const Vec3<float> s = second_iterate(v);
  cudaError_t err;
  {
    ProfScope ps(h, mode == kFusedProlong ? CMG_KERNEL_PROLONG : CMG_KERNEL_SMOOTH, l);
    err = launch_rbgs_fused(L, cview(x), s, f, mode, e, nc, h->stream);
  }
  if (err != cudaSuccess) return err;
  ProfScope ps(h, CMG_KERNEL_SMOOTH, l);
  return launch_rbgs_fused(L, cview(s), x, f, kFusedPlain, e, nc, h->stream);
}

template <typename T>
cudaError_t smooth(cmg_handle* h, const cmg_cycle& o, int l, int sweeps, Vec3<T> x, Vec3c<T> f) {
  if constexpr (sizeof(T) == 4) {
    if (sweeps >= 2 && fused_on(h, o, l)) {
      for (; sweeps >= 2; sweeps -= 2) {
        const cudaError_t e = fused_pair(h, o, l, x, f, kFusedPlain);
        if (e != cudaSuccess) return e;
      }
    }
  }
  if (h->galerkin() && l > 0) {
    const Lev& v = h->lv[l];
    const Lev& f0 = h->lv[0];
    const T *a9 = nullptr, *inva = nullptr;
    if constexpr (sizeof(T) == 8) {
      a9 = v.a9;
      inva = v.inva;
    } else {
      a9 = v.a9f;
      inva = v.invaf;
    }
    if (o.smoother == CMG_SMOOTH_RBGS) {
      // Gauss-Seidel on a 9-point grid: four colours instead of two
      for (int s = 0; s < sweeps; ++s) {
        ProfScope ps(h, CMG_KERNEL_SMOOTH, l);
        const cudaError_t e = launch_gs4_sweep<T>(v.n, h->prob.N, a9, v.m9, f0.c, f0.G, f0.d, f0.e, inva, v.isigma,
                                                  x, f, v.psum, h->stream);
        if (e != cudaSuccess) return e;
      }
      return cudaSuccess;
    }
    if constexpr (sizeof(T) == 4) {
      // damped Jacobi with the 9-point diagonal entries (the FP64 cycle takes
      // the 5-point update below, which reads the stored 1/a)
      Vec3<T> r = Work<T>::r(h->lv[l]);
      for (int s = 0; s < sweeps; ++s) {
        cudaError_t e;
        {
          ProfScope ps(h, CMG_KERNEL_RESIDUAL, l);
          e = level_residual<T>(h, l, cview(x), f, r);
        }
        if (e != cudaSuccess) return e;
        ProfScope ps(h, CMG_KERNEL_SMOOTH, l);
        e = launch_galerkin_jacobi<T>(v.n, h->prob.N, v.m9, f0.c, f0.d, f0.e, o.theta, inva, v.isigma, x, cview(r),
                                      h->stream);
        if (e != cudaSuccess) return e;
      }
      return cudaSuccess;
    }
  }
  const LevelView<T> L = view<T>(h, l, o.freeze_u, o.ctl32);
  for (int s = 0; s < sweeps; ++s) {
    if (o.smoother == CMG_SMOOTH_RBGS) {
      for (int colour = 0; colour < 2; ++colour) {
        ProfScope ps(h, CMG_KERNEL_SMOOTH, l);
        const cudaError_t e = launch_rbgs_half<T>(L, x, f, colour, h->stream);
        if (e != cudaSuccess) return e;
      }
    } else {
      Vec3<T> r = Work<T>::r(h->lv[l]);
      cudaError_t e;
      {
        ProfScope ps(h, CMG_KERNEL_RESIDUAL, l);
        e = level_residual<T>(h, l, cview(x), f, r);
      }
      if (e != cudaSuccess) return e;
      ProfScope ps(h, CMG_KERNEL_SMOOTH, l);
      e = launch_jacobi_update<T>(L, x, cview(r), o.theta, h->stream);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t zero_vec(cmg_handle* h, int l, Vec3<T> x) {
  const size_t nodes = h->lv[l].nodes, N = (size_t)h->prob.N;
  cudaError_t e = cudaMemsetAsync(x.y, 0, nodes * N * sizeof(T), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(x.u, 0, nodes * sizeof(T), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(x.p, 0, nodes * N * sizeof(T), h->stream);
  return e;
}

// Algorithm 1 on grid l: smoothing, residual, restriction, gamma recursive
// calls from a zero guess, prolongation, smoothing; direct solve on the
// coarsest grid.
// The coarse-grid part of the cycle from grid l down as one cluster launch
// (cmg_tail.cuh).  Returns cudaErrorNotSupported when not applicable.
template <typename T>
cudaError_t tail_cycle(cmg_handle* h, const cmg_cycle& o, int l, Vec3<T> x, Vec3c<T> f) {
  const int nlev = h->L - l;
  if (nlev > kTailMax || !tail_supported(h->prob.N, sizeof(T), h->coarse.m)) return cudaErrorNotSupported;
  TailParams<T> P{};
  P.nlev = nlev;
  for (int k = 0; k < nlev; ++k) {
    Lev& v = h->lv[l + k];
    P.lev[k].L = view<T>(h, l + k, o.freeze_u, o.ctl32);
    P.lev[k].r = Work<T>::r(v);
    if (k == 0) {
      P.lev[k].x = x;
      P.lev[k].f = Vec3<T>{const_cast<T*>(f.y), const_cast<T*>(f.u), const_cast<T*>(f.p)};
    } else {
      P.lev[k].x = Work<T>::x(v);
      P.lev[k].f = Work<T>::f(v);
    }
  }
  P.smoother = o.smoother;
  P.n1 = o.n1;
  P.n2 = o.n2;
  P.gamma = o.gamma;
  P.theta = o.theta;
  P.freeze_u = o.freeze_u;
  P.lpn = choose_map(h->prob.N, sizeof(T), 0).lpn;
  const CoarseData& cd = sizeof(T) == 4 ? h->c32() : h->coarse;
  P.cm = cd.m;
  P.cN = cd.N;
  P.Ainv = cd.Ainv;
  P.Minv = cd.Minv;
  P.wz = cd.wz;
  const Lev& cl = h->lv[h->L - 1];
  P.cc = cl.c;
  P.cd = cl.d;
  P.ce = cl.e;
  ProfScope ps(h, CMG_KERNEL_TAIL, l);
  return launch_tail_cycle<T>(P, h->stream);
}

// True when a cycle on grid l from a zero iterate never reads that iterate,
// so it need not be cleared first: the coarsest direct solve forms x from f
// alone, and red-black pre-smoothing starts with the zero-guess colour-0
// half-sweep (launch_rbgs_zero).  Not with a frozen control (the sweeps and
// the direct solve read u) nor for grids handed to the cluster tail.
bool zero_guess_ok(const cmg_handle* h, const cmg_cycle& o, int l) {
  if (o.freeze_u) return false;
  if (h->galerkin() && l > 0 && l < h->L - 1) return false;   // the zero-guess sweep is the 5-point red-black one
  if (o.tail_n > 0 && h->lv[l].n <= o.tail_n) return false;
  if (l == h->L - 1) return true;
  return o.smoother == CMG_SMOOTH_RBGS && o.n1 >= 1;
}

// zg: x is logically zero on entry but its memory has not been cleared
// (callers pass it only where zero_guess_ok holds).
template <typename T>
cudaError_t cycle(cmg_handle* h, const cmg_cycle& o, int l, Vec3<T> x, Vec3c<T> f, bool zg = false) {
  Lev& v = h->lv[l];
  const int N = h->prob.N;
  if (o.tail_n > 0 && v.n <= o.tail_n && !h->galerkin()) {
    const cudaError_t e = tail_cycle<T>(h, o, l, x, f);
    if (e != cudaErrorNotSupported) return e;
  }
  if (l == h->L - 1) {
    ProfScope ps(h, CMG_KERNEL_COARSE, l);
    if (h->galerkin()) {
      const Lev& f0 = h->lv[0];
      return launch_galerkin_coarse_solve<T>(h->coarse, v.m9, f0.c, f0.d, f0.e, f, x, h->stream);
    }
    return launch_coarse_solve<T>(coarse_for<T>(h), v.c, v.d, v.e, f, x, h->stream, o.freeze_u);
  }
  cudaError_t e = cudaSuccess;
  bool fz = false;   // one-launch sweeps on this grid
  if constexpr (sizeof(T) == 4) fz = fused_on(h, o, l);
  if (zg && fz && o.n1 >= 2) {
    // the first pre-smoothing sweep from the zero iterate and the next one,
    // one launch each
    if constexpr (sizeof(T) == 4) e = fused_pair(h, o, l, x, f, kFusedZero);
    if (e == cudaSuccess) e = smooth<T>(h, o, l, o.n1 - 2, x, f);
  } else if (zg) {
    // first pre-smoothing sweep from the zero iterate
    const LevelView<T> L = view<T>(h, l, o.freeze_u, o.ctl32);
    {
      ProfScope ps(h, CMG_KERNEL_SMOOTH, l);
      e = launch_rbgs_zero<T>(L, x, f, h->stream);
    }
    if (e == cudaSuccess) {
      ProfScope ps(h, CMG_KERNEL_SMOOTH, l);
      e = launch_rbgs_half<T>(L, x, f, 1, h->stream);
    }
    if (e == cudaSuccess) e = smooth<T>(h, o, l, o.n1 - 1, x, f);
  } else {
    e = smooth<T>(h, o, l, o.n1, x, f);
  }
  if (e != cudaSuccess) return e;
  Vec3<T> r = Work<T>::r(v);
  // after red-black pre-smoothing (last half-sweep: colour 1) with the control
  // updated, the residual vanishes at colour 1: compute and restrict colour 0
  const int c0 = (o.smoother == CMG_SMOOTH_RBGS && o.n1 >= 1 && !o.freeze_u && !(h->galerkin() && l > 0)) ? 1 : 0;
  {
    ProfScope ps(h, CMG_KERNEL_RESIDUAL, l);
    e = c0 ? launch_residual_c0<T>(view<T>(h, l), cview(x), f, r, h->stream)
           : level_residual<T>(h, l, cview(x), f, r);
  }
  if (e != cudaSuccess) return e;
  Lev& cl = h->lv[l + 1];
  Vec3<T> fc = Work<T>::f(cl), xc = Work<T>::x(cl);
  // the coarse iterate starts at zero: cleared by the restriction unless the
  // coarse cycle's first visit does not read it
  const bool czg = zero_guess_ok(h, o, l + 1);
  {
    ProfScope ps(h, CMG_KERNEL_RESTRICT, l);
    e = launch_restrict<T>(v.n, N, cview(r), fc, h->stream, czg ? Vec3<T>{nullptr, nullptr, nullptr} : xc, c0);
  }
  for (int g = 0; g < o.gamma && e == cudaSuccess; ++g) e = cycle<T>(h, o, l + 1, xc, cview(fc), czg && g == 0);
  if (e != cudaSuccess) return e;
  if (fz && o.n2 >= 2 && !(v.spl_target[1] & kTuneUnfused)) {
    // the first post-smoothing sweep reads its colour-1 neighbours as x + P e
    // (see below), then the next sweep, one launch each
    if constexpr (sizeof(T) == 4) e = fused_pair(h, o, l, x, f, kFusedProlong, cview(xc), cl.n);
    if (e == cudaSuccess) e = smooth<T>(h, o, l, o.n2 - 2, x, f);
    return e;
  }
  if (sizeof(T) == 4 && o.smoother == CMG_SMOOTH_RBGS && o.n2 >= 1 && !o.freeze_u &&
      !(v.spl_target[1] & kTuneUnfused) && !(h->galerkin() && l > 0)) {
    // FP32: prolongation fused into the first post-smoothing half-sweep
    // (colour 0); identical results, one pass over x fewer.  (In FP64 the
    // fused sweep is bound by the FP64 pipe and costs more than the pass.)
    const LevelView<T> L = view<T>(h, l, o.freeze_u, o.ctl32);
    {
      ProfScope ps(h, CMG_KERNEL_PROLONG, l);
      e = launch_rbgs_prolong<T>(L, x, f, cview(xc), cl.n, h->stream);
    }
    if (e == cudaSuccess) {
      ProfScope ps(h, CMG_KERNEL_SMOOTH, l);
      e = launch_rbgs_half<T>(L, x, f, 1, h->stream);
    }
    if (e == cudaSuccess) e = smooth<T>(h, o, l, o.n2 - 1, x, f);
    return e;
  }
  {
    ProfScope ps(h, CMG_KERNEL_PROLONG, l);
    e = launch_prolong_add<T>(v.n, N, cview(xc), x, h->stream, v.ctl);
  }
  if (e == cudaSuccess) e = smooth<T>(h, o, l, o.n2, x, f);
  return e;
}

cmg_status check_cycle(cmg_handle* h, const cmg_cycle* o) {
  if (!o) return fail(h, CMG_ERR_INVALID_ARG, "null cycle options");
  if (o->smoother != CMG_SMOOTH_RBGS && o->smoother != CMG_SMOOTH_JACOBI)
    return fail(h, CMG_ERR_INVALID_ARG, "unknown smoother");
  if (o->n1 < 0 || o->n2 < 0 || o->n1 > 64 || o->n2 > 64) return fail(h, CMG_ERR_INVALID_ARG, "n1/n2 out of range");
  if (o->gamma < 1 || o->gamma > 2) return fail(h, CMG_ERR_INVALID_ARG, "gamma must be 1 or 2");
  if (o->precision != CMG_FP64 && o->precision != CMG_FP32) return fail(h, CMG_ERR_INVALID_ARG, "unknown precision");
  if (o->tail_n < 0) return fail(h, CMG_ERR_INVALID_ARG, "tail_n must be >= 0");
  if (o->freeze_u != 0 && o->freeze_u != 1) return fail(h, CMG_ERR_INVALID_ARG, "freeze_u must be 0 or 1");
  if (o->freeze_u && h && h->L < 2) return fail(h, CMG_ERR_INVALID_ARG, "freeze_u needs at least two grids");
  if (o->ctl32 != 0 && o->ctl32 != 1) return fail(h, CMG_ERR_INVALID_ARG, "ctl32 must be 0 or 1");
  if (o->smoother == CMG_SMOOTH_JACOBI && !(o->theta > 0.0 && o->theta <= 1.0))
    return fail(h, CMG_ERR_INVALID_ARG, "theta must be in (0, 1]");
  if (h && h->galerkin() && o->freeze_u)
    return fail(h, CMG_ERR_UNSUPPORTED, "Galerkin coarse operators: the control is updated in every sweep");
  if (h && h->galerkin() && o->precision != CMG_FP64 && o->ctl32)
    return fail(h, CMG_ERR_UNSUPPORTED, "Galerkin coarse operators: the control row is FP64");
  return CMG_OK;
}

// ---- norms -------------------------------------------------------------------

// wy2 * ||y||^2 + ||u||^2 + ||p||^2 of a level vector into *out (device), not
// synchronised.  wy2 = N^2 gives the norm in the paper's row scaling.
cudaError_t sumsq3(cmg_handle* h, int l, const double* y, const double* u, const double* p, double* out,
                   double wy2 = 1.0) {
  const size_t nodes = h->lv[l].nodes, N = (size_t)h->prob.N;
  cudaError_t e = launch_sumsq(y, nodes * N, h->red, 0, wy2, h->stream);
  if (e == cudaSuccess) e = launch_sumsq(u, nodes, h->red, 1, 1.0, h->stream);
  if (e == cudaSuccess) e = launch_sumsq(p, nodes * N, h->red, 1, 1.0, h->stream);
  if (e == cudaSuccess) e = launch_finish_sum(h->red, kRedBlocks, out, h->stream);
  return e;
}

cudaError_t fetch(cmg_handle* h, const double* dev, int count) {
  cudaError_t e = cudaMemcpyAsync(h->hsc, dev, count * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e;
}

}  // namespace

// ============================================================================
extern "C" {

// Local control region: all zero (or x1 <= x0) = control everywhere; else
// a box inside the unit square.
bool control_box_full(const double* b) { return !(b[1] > b[0]) || !(b[3] > b[2]); }
bool control_box_ok(const double* b) {
  for (int i = 0; i < 4; ++i)
    if (!std::isfinite(b[i])) return false;
  if (control_box_full(b)) return b[0] == 0.0 && b[1] == 0.0 && b[2] == 0.0 && b[3] == 0.0;
  return b[0] >= 0.0 && b[1] <= 1.0 && b[2] >= 0.0 && b[3] <= 1.0;
}
// Index box of the n x n grid's nodes ((ix+1) h, (iy+1) h) inside the
// closed region (a rounding tolerance keeps nodes on its edges).
CtlBox control_nodes(int n, const double* b) {
  CtlBox c;
  if (control_box_full(b)) return c;
  const double s = n + 1.0, eps = 1e-9;
  c.x0 = std::max(0, (int)std::ceil(b[0] * s - eps) - 1);
  c.x1 = std::min(n - 1, (int)std::floor(b[1] * s + eps) - 1);
  c.y0 = std::max(0, (int)std::ceil(b[2] * s - eps) - 1);
  c.y1 = std::min(n - 1, (int)std::floor(b[3] * s + eps) - 1);
  return c;
}

cmg_status cmg_create(const cmg_problem* prob, const double* xi_host, void* stream, cmg_handle** out) {
  if (!out) return CMG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!prob) return CMG_ERR_INVALID_ARG;
  const cmg_problem P = *prob;
  const auto pow2m1 = [](int v) { return v >= 1 && ((v + 1) & v) == 0; };
  if (!pow2m1(P.n) || P.n < 3 || P.n > 4095) return CMG_ERR_INVALID_ARG;
  if (!(P.coarsest_n == 1 || P.coarsest_n == 3 || P.coarsest_n == 7) || P.coarsest_n > P.n) return CMG_ERR_INVALID_ARG;
  if (P.N < 1 || P.K < 0 || P.K > 64 || !(P.nu > 0.0) || !std::isfinite(P.amp)) return CMG_ERR_INVALID_ARG;
  if (P.coarse_coeff != CMG_COARSE_AVERAGED && P.coarse_coeff != CMG_COARSE_NODAL &&
      P.coarse_coeff != CMG_COARSE_GALERKIN)
    return CMG_ERR_INVALID_ARG;
  if (P.K > 0 && !xi_host) return CMG_ERR_INVALID_ARG;
  if (!control_box_ok(P.ctl_box)) return CMG_ERR_INVALID_ARG;
  if (P.coarse_coeff == CMG_COARSE_GALERKIN && !control_box_full(P.ctl_box)) return CMG_ERR_UNSUPPORTED;
  const SampleMap m64 = choose_map(P.N, 8, 0), m32 = choose_map(P.N, 4, 0);   // most chunks per lane
  if (m64.spl > kMaxSPL || m32.spl > kMaxSPL) return CMG_ERR_UNSUPPORTED;

  cmg_handle* h = new (std::nothrow) cmg_handle();
  if (!h) return CMG_ERR_OOM;
  h->prob = P;
  h->stream = static_cast<cudaStream_t>(stream);
  const char* graphs_env = std::getenv("CMG_GRAPHS");
  h->graphs = !(graphs_env && std::strcmp(graphs_env, "0") == 0);
  if (const char* v = std::getenv("CMG_ANCHOR_DROP")) {
    const double d = std::atof(v);
    if (d > 0.0 && d < 1.0) h->anchor_drop = d;
  }
  if (const char* v = std::getenv("CMG_ANCHOR_MAX")) {
    const int m = std::atoi(v);
    if (m >= 1 && m <= 1000) h->anchor_max = m;
  }
  int n = P.n, L = 0;
  while (true) {
    Lev& v = h->lv[L];
    v.n = n;
    v.h = 1.0 / (n + 1);
    v.nodes = (size_t)n * n;
    v.c = v.h * v.h / P.N;
    v.G = P.nu * v.h * v.h;
    v.d = -v.h * v.h;
    v.e = -v.h * v.h;
    v.ctl = control_nodes(n, P.ctl_box);
    ++L;
    if (n == P.coarsest_n) break;
    n = (n - 1) / 2;
  }
  h->L = L;
  h->lv[0].m9.w[4] = 1.0;   // fine mass: the identity (times c, G, d, e)
  if (P.coarse_coeff == CMG_COARSE_GALERKIN) {
    const Lev& f0 = h->lv[0];
    for (int l = 1; l < L; ++l) {
      Lev& v = h->lv[l];
      v.m9 = galerkin_mass(h->lv[l - 1].m9);
      const double mii = v.m9.w[4];
      v.c = f0.c * mii;
      v.G = f0.G * mii;
      v.d = f0.d * mii;
      v.e = f0.e * mii;
    }
  }
  const size_t N = (size_t)P.N;
  cudaError_t e = cudaSuccess;
#define AL(ptr, cnt)                        \
  do {                                      \
    if (e == cudaSuccess) e = dalloc(h, &(ptr), (cnt)); \
  } while (0)
  for (int l = 0; l < L; ++l) {
    Lev& v = h->lv[l];
    const size_t faces = (size_t)v.n * (v.n + 1) * N;
    AL(v.kx64, faces); AL(v.ky64, faces); AL(v.kx32, faces); AL(v.ky32, faces);
    AL(v.inva, v.nodes * N); AL(v.isigma, v.nodes); AL(v.isigma32, v.nodes); AL(v.isigd32, v.nodes);
    for (int b = 0; b < 3; ++b) {
      const size_t cnt = (b == 1) ? v.nodes : v.nodes * N;
      AL(v.r64[b], cnt); AL(v.x32[b], cnt); AL(v.f32[b], cnt); AL(v.r32[b], cnt); AL(v.f64[b], cnt);
      AL(v.x64[b], cnt);
      if (P.N % 4 == 0 && l + 1 < L) AL(v.xs32[b], cnt);
    }
  }
  AL(h->lv[0].a64, h->lv[0].nodes * N);
  if (P.coarse_coeff == CMG_COARSE_GALERKIN)
    for (int l = 1; l < L; ++l) {
      AL(h->lv[l].a9, 9 * h->lv[l].nodes * N);
      AL(h->lv[l].psum, 2 * h->lv[l].nodes);
      AL(h->lv[l].a9f, 9 * h->lv[l].nodes * N);
      AL(h->lv[l].invaf, h->lv[l].nodes * N);
    }
  const size_t g = (size_t)P.n + 2;
  AL(h->kap, g * g * N + g * N);
  AL(h->xi, (size_t)N * (P.K > 0 ? P.K : 1));
  AL(h->red, (size_t)kRedBlocks * 8 * 16);
  AL(h->dsc, 1024);
  h->part_cap = (int)(((size_t)P.n * P.n * 32 + kBlock - 1) / kBlock + 16);
  AL(h->part, (size_t)h->part_cap);
  AL(h->ir_state, 16);
  {
    Lev& l0 = h->lv[0];
    AL(l0.d32[0], l0.nodes * N); AL(l0.d32[1], l0.nodes); AL(l0.d32[2], l0.nodes * N);
  }
  const int cn = h->lv[L - 1].n;
  h->coarse.n = cn;
  h->coarse.m = cn * cn;
  h->coarse.N = P.N;
  h->coarse.blocks = (P.N + 31) / 32;
  h->coarse.ctl = h->lv[L - 1].ctl;
  for (int l = 0; l < L; ++l) AL(h->lv[l].dw, h->lv[l].nodes);
  for (int l = 0; l < L && e == cudaSuccess; ++l) e = launch_fill32((long)h->lv[l].nodes, 1.f, h->lv[l].dw, h->stream);
  h->coarse.dw = h->lv[L - 1].dw;
  AL(h->coarse.Ainv, N * h->coarse.m * h->coarse.m);
  AL(h->coarse.Ainv32, N * h->coarse.m * h->coarse.m);
  AL(h->coarse.Minv, (size_t)h->coarse.m * h->coarse.m);
  AL(h->coarse.wz, std::max(2 * N * h->coarse.m, (size_t)h->coarse.m * h->coarse.m));
  AL(h->coarse.partial, (size_t)h->coarse.blocks * h->coarse.m);
  if (P.coarse_coeff != CMG_COARSE_NODAL) {
    h->coarse32.n = h->coarse.n;
    h->coarse32.m = h->coarse.m;
    h->coarse32.N = h->coarse.N;
    h->coarse32.blocks = h->coarse.blocks;
    h->coarse32.ctl = h->coarse.ctl;
    h->coarse32.dw = h->coarse.dw;
    AL(h->coarse32.Ainv, N * h->coarse.m * h->coarse.m);
    AL(h->coarse32.Ainv32, N * h->coarse.m * h->coarse.m);
    AL(h->coarse32.Minv, (size_t)h->coarse.m * h->coarse.m);
    AL(h->coarse32.wz, std::max(2 * N * h->coarse.m, (size_t)h->coarse.m * h->coarse.m));
    AL(h->coarse32.partial, (size_t)h->coarse.blocks * h->coarse.m);
    AL(h->cface64, 2 * (size_t)cn * (cn + 1) * N);
  }
#undef AL
  if (e == cudaSuccess) {
    void* hp = nullptr;
    e = cudaMallocHost(&hp, 1024 * sizeof(double));
    h->hsc = static_cast<double*>(hp);
  }
  if (e == cudaSuccess && P.K > 0)
    e = cudaMemcpyAsync(h->xi, xi_host, N * P.K * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = setup_coefficients(h);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    const cmg_status st = (e == cudaErrorMemoryAllocation) ? CMG_ERR_OOM : CMG_ERR_CUDA;
    (void)cudaGetLastError();
    cmg_destroy(h);
    return st;
  }
  *out = h;
  return CMG_OK;
}

cmg_status cmg_set_samples(cmg_handle* h, const double* xi_dev) {
  if (!h) return CMG_ERR_INVALID_ARG;
  if (h->prob.K > 0) {
    if (!xi_dev) return fail(h, CMG_ERR_INVALID_ARG, "null xi");
    CK(cudaMemcpyAsync(h->xi, xi_dev, (size_t)h->prob.N * h->prob.K * sizeof(double), cudaMemcpyDeviceToDevice,
                       h->stream));
  }
  CK(setup_coefficients(h));
  return CMG_OK;
}

void cmg_destroy(cmg_handle* h) {
  if (!h) return;
  if (h->stream) (void)cudaStreamSynchronize(h->stream);
  else (void)cudaDeviceSynchronize();
  if (h->ir_exec) (void)cudaGraphExecDestroy(h->ir_exec);
  if (h->ir_graph) (void)cudaGraphDestroy(h->ir_graph);
  if (h->cap) (void)cudaStreamDestroy(h->cap);
  for (void* p : h->allocs) (void)cudaFree(p);
  for (auto& ev : h->prof_ev) (void)cudaEventDestroy(ev);
  if (h->gm) (void)cudaFree(h->gm);
  if (h->hsc) (void)cudaFreeHost(h->hsc);
  delete h;
}

const char* cmg_last_error(const cmg_handle* h) { return h ? h->err.c_str() : "null handle"; }
int cmg_num_levels(const cmg_handle* h) { return h ? h->L : 0; }
int cmg_level_n(const cmg_handle* h, int level) { return level_ok(h, level) ? h->lv[level].n : -1; }

cmg_status cmg_rhs(cmg_handle* h, const double* yd, const double* fsrc, double* fy, double* fu, double* fp) {
  if (!h) return CMG_ERR_INVALID_ARG;
  if (!yd || !vec_ok(fy, fu, fp)) return fail(h, CMG_ERR_INVALID_ARG, "null pointer");
  CK(launch_rhs(h->prob.n, h->prob.N, h->lv[0].h, yd, fsrc, fy, fu, fp, h->stream));
  return CMG_OK;
}

#define CMG_LEVEL_OPS(SUF, T)                                                                                  \
  cmg_status cmg_residual##SUF(cmg_handle* h, int level, const T* y, const T* u, const T* p, const T* fy,       \
                               const T* fu, const T* fp, T* ry, T* ru, T* rp) {                                 \
    if (!h) return CMG_ERR_INVALID_ARG;                                                                         \
    if (!level_ok(h, level)) return fail(h, CMG_ERR_INVALID_ARG, "level out of range");                        \
    if (!vec_ok(y, u, p) || !vec_ok(ry, ru, rp)) return fail(h, CMG_ERR_INVALID_ARG, "null pointer");          \
    if ((fy || fu || fp) && !vec_ok(fy, fu, fp)) return fail(h, CMG_ERR_INVALID_ARG, "partial rhs");           \
    CK(ensure_ops<T>(h));                                                                                       \
    CK(level_residual<T>(h, level, Vec3c<T>{y, u, p}, Vec3c<T>{fy, fu, fp}, Vec3<T>{ry, ru, rp}));             \
    return CMG_OK;                                                                                              \
  }                                                                                                             \
  cmg_status cmg_smooth##SUF(cmg_handle* h, int level, const cmg_cycle* opts, int sweeps, T* y, T* u, T* p,     \
                             const T* fy, const T* fu, const T* fp) {                                           \
    if (!h) return CMG_ERR_INVALID_ARG;                                                                         \
    if (!level_ok(h, level)) return fail(h, CMG_ERR_INVALID_ARG, "level out of range");                        \
    if (!vec_ok(y, u, p) || !vec_ok(fy, fu, fp)) return fail(h, CMG_ERR_INVALID_ARG, "null pointer");          \
    if (sweeps < 0) return fail(h, CMG_ERR_INVALID_ARG, "negative sweeps");                                    \
    cmg_cycle o = *opts;                                                                                        \
    o.n1 = o.n2 = 0; o.gamma = 1; o.precision = sizeof(T) == 8 ? CMG_FP64 : CMG_FP32;                           \
    const cmg_status st = check_cycle(h, &o);                                                                   \
    if (st != CMG_OK) return st;                                                                                \
    CK(ensure_ops<T>(h));                                                                                       \
    CK(smooth<T>(h, o, level, sweeps, Vec3<T>{y, u, p}, Vec3c<T>{fy, fu, fp}));                                \
    return CMG_OK;                                                                                              \
  }                                                                                                             \
  cmg_status cmg_restrict##SUF(cmg_handle* h, int level, const T* ry, const T* ru, const T* rp, T* cy, T* cu,   \
                               T* cp) {                                                                         \
    if (!h) return CMG_ERR_INVALID_ARG;                                                                         \
    if (!level_ok(h, level) || level == h->L - 1) return fail(h, CMG_ERR_INVALID_ARG, "level out of range");   \
    if (!vec_ok(ry, ru, rp) || !vec_ok(cy, cu, cp)) return fail(h, CMG_ERR_INVALID_ARG, "null pointer");       \
    CK(launch_restrict<T>(h->lv[level].n, h->prob.N, Vec3c<T>{ry, ru, rp}, Vec3<T>{cy, cu, cp}, h->stream));   \
    return CMG_OK;                                                                                              \
  }                                                                                                             \
  cmg_status cmg_prolong_add##SUF(cmg_handle* h, int level, const T* ey, const T* eu, const T* ep, T* y, T* u,  \
                                  T* p) {                                                                       \
    if (!h) return CMG_ERR_INVALID_ARG;                                                                         \
    if (!level_ok(h, level) || level == h->L - 1) return fail(h, CMG_ERR_INVALID_ARG, "level out of range");   \
    if (!vec_ok(ey, eu, ep) || !vec_ok(y, u, p)) return fail(h, CMG_ERR_INVALID_ARG, "null pointer");          \
    CK(launch_prolong_add<T>(h->lv[level].n, h->prob.N, Vec3c<T>{ey, eu, ep}, Vec3<T>{y, u, p}, h->stream,          \
                             h->lv[level].ctl));   \
    return CMG_OK;                                                                                              \
  }                                                                                                             \
  cmg_status cmg_coarse_solve##SUF(cmg_handle* h, const T* fy, const T* fu, const T* fp, T* y, T* u, T* p) {    \
    if (!h) return CMG_ERR_INVALID_ARG;                                                                         \
    if (!vec_ok(fy, fu, fp) || !vec_ok(y, u, p)) return fail(h, CMG_ERR_INVALID_ARG, "null pointer");          \
    const Lev& v = h->lv[h->L - 1];                                                                             \
    if (h->galerkin()) {                                                                                        \
      CK(ensure_fp64(h));                                                                                       \
      const Lev& f0 = h->lv[0];                                                                                 \
      CK(launch_galerkin_coarse_solve<T>(h->coarse, v.m9, f0.c, f0.d, f0.e, Vec3c<T>{fy, fu, fp},              \
                                         Vec3<T>{y, u, p}, h->stream));                                         \
      return CMG_OK;                                                                                            \
    }                                                                                                           \
    if (sizeof(T) == 8) CK(ensure_fp64(h));                                                                     \
    CK(launch_coarse_solve<T>(coarse_for<T>(h), v.c, v.d, v.e, Vec3c<T>{fy, fu, fp},                           \
                              Vec3<T>{y, u, p}, h->stream));                                                    \
    return CMG_OK;                                                                                              \
  }                                                                                                             \
  cmg_status cmg_cycle_apply##SUF(cmg_handle* h, const cmg_cycle* opts, T* y, T* u, T* p, const T* fy,          \
                                  const T* fu, const T* fp) {                                                   \
    if (!h) return CMG_ERR_INVALID_ARG;                                                                         \
    const cmg_status st = check_cycle(h, opts);                                                                 \
    if (st != CMG_OK) return st;                                                                                \
    if (opts->precision != (sizeof(T) == 8 ? CMG_FP64 : CMG_FP32))                                              \
      return fail(h, CMG_ERR_INVALID_ARG, "precision does not match the vector type");                         \
    if (!vec_ok(y, u, p) || !vec_ok(fy, fu, fp)) return fail(h, CMG_ERR_INVALID_ARG, "null pointer");          \
    CK(ensure_ops<T>(h));                                                                                       \
    CK(cycle<T>(h, *opts, 0, Vec3<T>{y, u, p}, Vec3c<T>{fy, fu, fp}));                                          \
    return CMG_OK;                                                                                              \
  }

CMG_LEVEL_OPS(, double)
CMG_LEVEL_OPS(_f32, float)

cmg_status cmg_norm(cmg_handle* h, int level, const double* y, const double* u, const double* p, double* out_host) {
  if (!h) return CMG_ERR_INVALID_ARG;
  if (!level_ok(h, level)) return fail(h, CMG_ERR_INVALID_ARG, "level out of range");
  if (!vec_ok(y, u, p) || !out_host) return fail(h, CMG_ERR_INVALID_ARG, "null pointer");
  CK(sumsq3(h, level, y, u, p, h->dsc));
  CK(fetch(h, h->dsc, 1));
  *out_host = std::sqrt(h->hsc[0]);
  return CMG_OK;
}

cmg_status cmg_mean_log_kappa(cmg_handle* h, double* out) {
  if (!h) return CMG_ERR_INVALID_ARG;
  if (!out) return fail(h, CMG_ERR_INVALID_ARG, "null pointer");
  CK(launch_mean_log_kappa(h->prob.n, h->prob.N, h->prob.K, h->prob.amp, h->xi, out, h->stream));
  return CMG_OK;
}

cmg_status cmg_sync(cmg_handle* h) {
  if (!h) return CMG_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize(h->stream));
  return CMG_OK;
}

cmg_status cmg_profile_begin(cmg_handle* h, int kinds, int level) {
  if (!h) return CMG_ERR_INVALID_ARG;
  if (!level_ok(h, level)) return fail(h, CMG_ERR_INVALID_ARG, "level out of range");
  if (h->prof_ev.empty()) {
    h->prof_ev.resize(2 * kMaxProf);
    for (auto& ev : h->prof_ev) CK(cudaEventCreate(&ev));
  }
  h->prof_kinds = kinds;
  h->prof_level = level;
  h->prof_n = 0;
  return CMG_OK;
}

cmg_status cmg_profile_end(cmg_handle* h, double* total_ms, int* launches) {
  if (!h) return CMG_ERR_INVALID_ARG;
  h->prof_kinds = 0;
  CK(cudaStreamSynchronize(h->stream));
  double tot = 0.0;
  for (int i = 0; i < h->prof_n; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->prof_ev[2 * i], h->prof_ev[2 * i + 1]));
    tot += ms;
  }
  if (total_ms) *total_ms = tot;
  if (launches) *launches = h->prof_n;
  h->prof_n = 0;
  return CMG_OK;
}

long long cmg_kernel_launches(void) { return cmg::g_launches.load(); }

}  // extern "C"

namespace {

// Time `reps` red+black half-sweep pairs on grid l with chunk target t.
template <typename T>
cmg_status time_sweeps(cmg_handle* h, int l, int t, int reps, float* ms) {
  Lev& v = h->lv[l];
  const int k = sizeof(T) == 8 ? 0 : 1;
  const int saved = v.spl_target[k];
  v.spl_target[k] = t;
  const LevelView<T> L = view<T>(h, l);
  Vec3<T> x = Work<T>::x(v), f = Work<T>::f(v);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  cudaError_t e = cudaSuccess;
  for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = launch_rbgs_half<T>(L, x, cview(f), w & 1, h->stream);
  if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    e = launch_rbgs_half<T>(L, x, cview(f), 0, h->stream);
    if (e == cudaSuccess) e = launch_rbgs_half<T>(L, x, cview(f), 1, h->stream);
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  (void)cudaEventDestroy(e0);
  (void)cudaEventDestroy(e1);
  v.spl_target[k] = saved;
  if (e != cudaSuccess) return cuda_fail(h, e, "autotune timing");
  return CMG_OK;
}

// Time `reps` first post-smoothing steps on FP32 grid l (chunk target t):
// the prolongation-fused colour-0 half-sweep + the colour-1 half-sweep, or
// (unfused) the prolongation pass + both plain half-sweeps.
cmg_status time_prolong(cmg_handle* h, int l, int t, int reps, bool unfused, float* ms) {
  Lev& v = h->lv[l];
  Lev& c = h->lv[l + 1];
  const int saved = v.spl_target[1];
  v.spl_target[1] = t;
  const LevelView<float> L = view<float>(h, l);
  Vec3<float> x = Work<float>::x(v), f = Work<float>::f(v), e = Work<float>::x(c);
  CK(zero_vec<float>(h, l + 1, e));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  cudaError_t err = cudaSuccess;
  for (int r = -1; r < reps && err == cudaSuccess; ++r) {   // r = -1: warm-up
    if (r == 0) err = cudaEventRecord(e0, h->stream);
    if (err != cudaSuccess) break;
    if (unfused) {
      err = launch_prolong_add<float>(v.n, h->prob.N, cview(e), x, h->stream, v.ctl);
      if (err == cudaSuccess) err = launch_rbgs_half<float>(L, x, cview(f), 0, h->stream);
    } else {
      err = launch_rbgs_prolong<float>(L, x, cview(f), cview(e), c.n, h->stream);
    }
    if (err == cudaSuccess) err = launch_rbgs_half<float>(L, x, cview(f), 1, h->stream);
  }
  if (err == cudaSuccess) err = cudaEventRecord(e1, h->stream);
  if (err == cudaSuccess) err = cudaEventSynchronize(e1);
  if (err == cudaSuccess) err = cudaEventElapsedTime(ms, e0, e1);
  (void)cudaEventDestroy(e0);
  (void)cudaEventDestroy(e1);
  v.spl_target[1] = saved;
  if (err != cudaSuccess) return cuda_fail(h, err, "autotune timing");
  return CMG_OK;
}

template <typename T>
cmg_status autotune_levels(cmg_handle* h, int* chosen) {
  const int k = sizeof(T) == 8 ? 0 : 1;
  for (int l = 0; l + 1 < h->L; ++l) {
    Lev& v = h->lv[l];
    if (h->galerkin() && l > 0) {
      // Galerkin grids have no face arrays and never run the timed sweeps
      v.spl_target[k] = 0;
      if (chosen) chosen[l] = 0;
      continue;
    }
    CK(zero_vec<T>(h, l, Work<T>::x(v)));
    CK(zero_vec<T>(h, l, Work<T>::f(v)));
    const int reps = v.n >= 255 ? 8 : 16;
    // direct-load sweeps with 1, 2, 4 chunks per lane; FP32 also the staged
    // sweep with 1 or 2 (kTuneStaged) and the two-sample layout (kTuneWide).
    // Three rounds over all candidates in turn; each candidate is judged by
    // its median round (one timing per candidate was at the mercy of clock
    // ramps and L2 state).
    int cand[6] = {1, 2, 4, 0, 0, 0}, nc = 3;
    if (sizeof(T) == 4 && staged_supported(h->prob.N, 1)) {
      cand[nc++] = kTuneStaged | 1;
      cand[nc++] = kTuneStaged | 2;
    }
    if (sizeof(T) == 4 && wide_supported(h->prob.N)) cand[nc++] = kTuneWide | 1;
    constexpr int kRounds = 3;
    float t_ms[kRounds][6] = {};
    for (int r = 0; r < kRounds; ++r)
      for (int ci = 0; ci < nc; ++ci) {
        const cmg_status s = time_sweeps<T>(h, l, cand[ci], reps, &t_ms[r][ci]);
        if (s != CMG_OK) return s;
      }
    float best = 1e30f;
    int best_t = 0;
    for (int ci = 0; ci < nc; ++ci) {
      float a = t_ms[0][ci], b = t_ms[1][ci], c = t_ms[2][ci];
      const float med = std::max(std::min(a, b), std::min(std::max(a, b), c));
      if (med < best) {
        best = med;
        best_t = cand[ci];
      }
    }
    // FP32: the prolongation fused into the first post-smoothing half-sweep
    // or as its own pass (on large grids the fused sweep's extra coarse
    // loads can cost more than the pass)
    if (sizeof(T) == 4 && !h->galerkin()) {
      float tf[kRounds] = {}, tu[kRounds] = {};
      for (int r = 0; r < kRounds; ++r) {
        cmg_status s = time_prolong(h, l, best_t, reps, false, &tf[r]);
        if (s == CMG_OK) s = time_prolong(h, l, best_t, reps, true, &tu[r]);
        if (s != CMG_OK) return s;
      }
      const auto med = [](const float* a) {
        return std::max(std::min(a[0], a[1]), std::min(std::max(a[0], a[1]), a[2]));
      };
      if (med(tu) < med(tf)) best_t |= kTuneUnfused;
    }
    v.spl_target[k] = best_t;
    if (chosen) chosen[l] = best_t;
  }
  return CMG_OK;
}

}  // namespace

extern "C" {

cmg_status cmg_autotune(cmg_handle* h, int precision, int* chosen) {
  if (!h) return CMG_ERR_INVALID_ARG;
  h->ir_opts.n1 = -1;   // captured graphs bake the launch shapes: force a re-capture
  if (precision == CMG_FP64) {
    CK(ensure_fp64(h));
    return autotune_levels<double>(h, chosen);
  }
  if (precision == CMG_FP32) return autotune_levels<float>(h, chosen);
  return fail(h, CMG_ERR_INVALID_ARG, "unknown precision");
}

cmg_status cmg_sample_map(int N, int elem_bytes, long long items, int target, int* lanes_per_node, int* vec_width,
                          int* chunks_per_lane) {
  if (N < 1 || (elem_bytes != 4 && elem_bytes != 8) || items < 0 || !lanes_per_node || !vec_width || !chunks_per_lane)
    return CMG_ERR_INVALID_ARG;
  const SampleMap m = choose_map(N, elem_bytes, (long)items, target);
  *lanes_per_node = m.lpn;
  *vec_width = m.V;
  *chunks_per_lane = m.spl;
  return m.spl > kMaxSPL ? CMG_ERR_UNSUPPORTED : CMG_OK;
}

cmg_status cmg_set_tuning(cmg_handle* h, int precision, const int* spl_targets) {
  if (!h) return CMG_ERR_INVALID_ARG;
  if (precision != CMG_FP64 && precision != CMG_FP32) return fail(h, CMG_ERR_INVALID_ARG, "unknown precision");
  const int k = precision == CMG_FP64 ? 0 : 1;
  for (int l = 0; l < h->L; ++l) {
    const int t = spl_targets ? spl_targets[l] : 0;
    const int c = t & ~(kTuneStaged | kTuneWide | kTuneUnfused | kTuneFused | kTuneTma);
    const bool staged = t & kTuneStaged, wide = t & kTuneWide, unfused = t & kTuneUnfused, fused = t & kTuneFused;
    const bool tma = t & kTuneTma;
    if ((c != 0 && c != 1 && c != 2 && c != 4) || ((staged || wide || unfused || fused || tma) && k == 0) ||
        (staged && c != 1 && c != 2) || (wide && (staged || c != 1)) || (fused && (staged || wide || c == 0)) ||
        (tma && (staged || wide || fused || c == 0)))
      return fail(h, CMG_ERR_INVALID_ARG,
                  "target must be 0, 1, 2 or 4 (FP32: or CMG_TUNE_STAGED | 1 or 2, or CMG_TUNE_WIDE | 1, or "
                  "CMG_TUNE_FUSED | 1, 2 or 4, or CMG_TUNE_TMA | 1, 2 or 4; any of them | CMG_TUNE_UNFUSED)");
  }
  for (int l = 0; l < h->L; ++l) h->lv[l].spl_target[k] = spl_targets ? spl_targets[l] : 0;
  h->ir_opts.n1 = -1;   // captured graphs bake the launch shapes: force a re-capture
  return CMG_OK;
}

}  // extern "C"

// ============================================================================
// Outer solvers
namespace {

// Row weight of the state block in the paper's scaling of the system (its
// state rows are N times the symmetric ones used here).
inline double paper_wy(const cmg_handle* h) { return (double)h->prob.N; }

// ||W (f - S x)||_2 into *rho (host), residual r = f - S x (unweighted) left
// in level-0 r64.
cmg_status true_residual(cmg_handle* h, Vec3c<double> f, Vec3c<double> x, double* rho) {
  Lev& v = h->lv[0];
  Vec3<double> r = Work<double>::r(v);
  CK(launch_residual<double>(view<double>(h, 0), x, f, r, h->stream));
  CK(sumsq3(h, 0, r.y, r.u, r.p, h->dsc, paper_wy(h) * paper_wy(h)));
  CK(fetch(h, h->dsc, 1));
  *rho = std::sqrt(h->hsc[0]);
  return CMG_OK;
}

// One preconditioner application z = M^{-1} W^{-1} v (zero initial guess),
// FP64 in/out: one cycle on the right side whose state block is divided
// by wy (undoing the paper's row scaling of the Krylov vector).
cmg_status precondition(cmg_handle* h, const cmg_cycle& o, Vec3c<double> v, Vec3<double> z, double wy) {
  Lev& l0 = h->lv[0];
  const size_t ny = l0.nodes * h->prob.N, nu = l0.nodes;
  if (o.precision == CMG_FP64) {
    double* fy = l0.f64[0];
    CK((launch_scale_cast<double, double>(1.0 / wy, v.y, fy, ny, h->stream)));
    const bool zg = zero_guess_ok(h, o, 0);
    if (!zg) CK(zero_vec<double>(h, 0, z));
    CK(cycle<double>(h, o, 0, z, Vec3c<double>{fy, v.u, v.p}, zg));
    return CMG_OK;
  }
  // FP32 cycle on the right side (Krylov vectors have unit norm, no scaling
  // is needed for the FP32 range), result converted into FP64.
  const double vscale = 1.0;
  Vec3<float> f32 = Work<float>::f(l0), x32 = Work<float>::x(l0);
  CK((launch_scale_cast<double, float>(vscale / wy, v.y, f32.y, ny, h->stream)));
  CK((launch_scale_cast<double, float>(vscale, v.u, f32.u, nu, h->stream)));
  CK((launch_scale_cast<double, float>(vscale, v.p, f32.p, ny, h->stream)));
  const bool zg = zero_guess_ok(h, o, 0);
  if (!zg) CK(zero_vec<float>(h, 0, x32));
  CK(cycle<float>(h, o, 0, x32, cview(f32), zg));
  CK((launch_scale_cast<float, double>(1.0 / vscale, x32.y, z.y, ny, h->stream)));
  CK((launch_scale_cast<float, double>(1.0 / vscale, x32.u, z.u, nu, h->stream)));
  CK((launch_scale_cast<float, double>(1.0 / vscale, x32.p, z.p, ny, h->stream)));
  return CMG_OK;
}

// End of one refinement iteration inside the graph: residual norm from the
// partials (fixed-order sum), scales for the next iteration, iteration
// count, and the loop condition of the enclosing while node.
// state = [sc, inv_sc, rho, it, maxit, tol_abs].
// FP32 refinement with residual replacement.  Between anchors the cycle's
// right side r^ = sc r is updated recursively in FP32 (r^ <- r^ - S e) and
// the corrections are summed in FP32 (d += e); an anchor folds x += d / sc,
// recomputes the true residual in FP64 and rescales r^ to norm 1.  The FP32
// recursion drifts from the true residual by about eps32 times the size of
// the terms of S e per step, relative to the residual it started from; it
// forms A e from neighbour differences (launch_recur), which keeps those
// terms small for the smooth corrections a cycle returns.  An anchor is taken
// once the recursive norm has dropped below drop = 1e-3 times the last true
// one, after 8 cycles, at maxit, or when the recursive norm reaches the
// tolerance (the stopping test is always made on a true residual).  The
// environment variables CMG_ANCHOR_DROP and CMG_ANCHOR_MAX, read when a
// handle is created, override the two limits.
__device__ double block_total(const double* __restrict__ partial, int count) {
  __shared__ double sh[32];
  double v = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) v += partial[i];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  return t;   // valid in thread 0
}

// After the cycle and the recursive update: the recursive norm, whether the
// anchor runs this iteration, whether the loop continues (if it does not
// anchor).  cond is set only when `graph` (a conditional node exists).
__global__ void ir_recur_control_kernel(const double* __restrict__ partial, int count, double* __restrict__ s,
                                        cudaGraphConditionalHandle cond, int graph) {
  pdl_enter();
  const double t = block_total(partial, count);
  if (threadIdx.x != 0) return;
  const double rho = sqrt(t) * s[kInvSc];
  const double it = s[kIt] + 1.0, since = s[kSince] + 1.0;
  s[kRho] = rho;
  s[kIt] = it;
  s[kSince] = since;
  const bool anchor = !isfinite(rho) || rho <= s[kTolAbs] || rho <= s[kDrop] * s[kRhoAnchor] ||
                      it >= s[kMaxit] || since >= s[kAmax];
  s[kSc] = (isfinite(rho) && rho > 0.0) ? 1.0 / rho : 1.0 / s[kRhoAnchor];
  s[kAnchor] = anchor ? 1.0 : 0.0;
  s[kGo] = anchor ? 0.0 : 1.0;
  if (graph) cudaGraphSetConditional(cond, anchor ? 0u : 1u);
}

// After the anchor's FP64 pass (scale s[kSc]): the true norm, the new scale,
// the stopping test.  Does nothing when no anchor ran.
__global__ void ir_anchor_control_kernel(const double* __restrict__ partial, int count, double* __restrict__ s,
                                         cudaGraphConditionalHandle cond, int graph) {
  pdl_enter();
  if (s[kAnchor] == 0.0) return;
  const double t = block_total(partial, count);
  if (threadIdx.x != 0) return;
  const double sc = s[kSc];
  const double rho = sqrt(t) / sc;
  s[kInvSc] = 1.0 / sc;   // the right side now holds r * sc
  s[kSc] = 1.0 / rho;
  s[kRho] = rho;
  s[kRhoAnchor] = rho;
  s[kSince] = 0.0;
  const bool go = isfinite(rho) && rho > s[kTolAbs] && s[kIt] < s[kMaxit];
  s[kGo] = go ? 1.0 : 0.0;
  if (graph) cudaGraphSetConditional(cond, go ? 1u : 0u);
}

// Host image of the state before the first iteration: right side r^ = sc r
// with true norm rho.
void ir_state_init(const cmg_handle* h, double* hs, double rho, double sc, int maxit, double tol_abs) {
  for (int i = 0; i < kIrStateSize; ++i) hs[i] = 0.0;
  hs[kDrop] = h->anchor_drop;
  hs[kAmax] = (double)h->anchor_max;
  hs[kSc] = rho > 0.0 ? 1.0 / rho : 0.0;
  hs[kInvSc] = 1.0 / sc;
  hs[kRho] = rho;
  hs[kMaxit] = (double)maxit;
  hs[kTolAbs] = tol_abs;
  hs[kRhoAnchor] = rho;
  hs[kGo] = 1.0;
}

// The anchor kernels (each does nothing unless the anchor flag is set).
cmg_status ir_iteration_anchor(cmg_handle* h, Vec3c<double> f, Vec3<double> x, cudaGraphConditionalHandle cond,
                               int graph) {
  Lev& l0 = h->lv[0];
  const size_t ny = l0.nodes * h->prob.N, nu = l0.nodes;
  Vec3<float> f32 = Work<float>::f(l0);
  Vec3<float> d32{l0.d32[0], l0.d32[1], l0.d32[2]};
  double* st = h->ir_state;
  CK(launch_fold(st + kInvSc, st + kAnchor, d32, x, ny, nu, h->stream));
  const int cnt = launch_residual_cast(view<double>(h, 0), cview(x), f, f32, 0.0, st + kSc, paper_wy(h), h->part,
                                       h->part_cap, h->stream, st + kAnchor);
  if (cnt < 0) return fail(h, CMG_ERR_CUDA, "refinement pass launch failed");
  CK(launch_k(ir_anchor_control_kernel, dim3(1), dim3(256), 0, h->stream, (const double*)h->part, cnt, st, cond,
              graph));
  count_launches(1);
  return CMG_OK;
}

// One refinement iteration on the handle's stream (eager) or into a capture:
// cycle, recursive update, control, then the gated anchor.
cmg_status ir_iteration(cmg_handle* h, const cmg_cycle& o, Vec3c<double> f, Vec3<double> x,
                        cudaGraphConditionalHandle cond, int graph, bool anchor_kernels) {
  Lev& l0 = h->lv[0];
  Vec3<float> f32 = Work<float>::f(l0), x32 = Work<float>::x(l0);
  Vec3<float> d32{l0.d32[0], l0.d32[1], l0.d32[2]};
  double* st = h->ir_state;
  // the correction equation starts from zero
  const bool zg = zero_guess_ok(h, o, 0);
  if (!zg) CK(launch_zero3(x32, l0.nodes * h->prob.N, l0.nodes, h->stream));
  CK(cycle<float>(h, o, 0, x32, cview(f32), zg));
  int cnt = launch_recur(view<float>(h, 0), cview(x32), f32, d32, paper_wy(h), h->part, h->part_cap, h->stream);
  if (cnt < 0) return fail(h, CMG_ERR_CUDA, "recursive residual launch failed");
  CK(launch_k(ir_recur_control_kernel, dim3(1), dim3(256), 0, h->stream, (const double*)h->part, cnt, st, cond,
              graph));
  count_launches(1);
  if (!anchor_kernels) return CMG_OK;
  return ir_iteration_anchor(h, f, x, cond, graph);
}

bool same_cycle(const cmg_cycle& a, const cmg_cycle& b) {
  return a.smoother == b.smoother && a.theta == b.theta && a.n1 == b.n1 && a.n2 == b.n2 && a.gamma == b.gamma &&
         a.precision == b.precision && a.tail_n == b.tail_n && a.freeze_u == b.freeze_u && a.ctl32 == b.ctl32;
}

// Sets a loop condition from the state before the first iteration:
// go = rho > tol_abs and maxit > 0 (state = [sc, inv_sc, rho, it, maxit, tol_abs]).
__global__ void ir_start_kernel(const double* __restrict__ state, cudaGraphConditionalHandle cond) {
  const double rho = state[2];
  cudaGraphSetConditional(cond, (isfinite(rho) && rho > state[5] && state[3] < state[4]) ? 1u : 0u);
}

// Adds to graph g: [start kernel] -> [while(cond) { one refinement iteration
// (ir_iteration) }] for one instance.  Kernels are captured on the
// instance's capture stream with all its launches redirected there.
cmg_status add_ir_loop(cmg_handle* h, const cmg_cycle& o, Vec3c<double> f, Vec3<double> x, cudaGraph_t g) {
  if (!h->cap) CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  cudaGraphConditionalHandle cond;
  CK(cudaGraphConditionalHandleCreate(&cond, g, 0, cudaGraphCondAssignDefault));
  // start kernel node
  cudaGraphNode_t start;
  {
    cudaKernelNodeParams kp = {};
    const double* st = h->ir_state;
    void* args[2] = {(void*)&st, (void*)&cond};
    kp.func = (void*)ir_start_kernel;
    kp.gridDim = dim3(1, 1, 1);
    kp.blockDim = dim3(1, 1, 1);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    kp.extra = nullptr;
    CK(cudaGraphAddKernelNode(&start, g, nullptr, 0, &kp));
  }
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, &start, nullptr, 1, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  const cudaStream_t user = h->stream;
  const int prof = h->prof_kinds;
  h->stream = h->cap;
  h->prof_kinds = 0;
  cudaError_t e = cudaStreamBeginCaptureToGraph(h->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  cmg_status ist = CMG_OK;
  const long long k0 = cmg_kernel_launches();
  if (e == cudaSuccess) {
    ist = ir_iteration(h, o, f, x, cond, 1, true);
    cudaGraph_t captured = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(h->cap, &captured);
    if (e == cudaSuccess) e = e2;
  }
  h->stream = user;
  h->prof_kinds = prof;
  if (ist != CMG_OK) {
    h->ir_body_kernels = cmg_kernel_launches() - k0;
    count_launches((int)-h->ir_body_kernels);
    return ist;
  }
  // kernels captured into the body run once per iteration; the launch
  // counter is advanced by replays (see count_replay), not by the capture
  h->ir_body_kernels = cmg_kernel_launches() - k0;
  count_launches((int)-h->ir_body_kernels);
  if (e != cudaSuccess) return cuda_fail(h, e, "capture of the refinement loop");
  return CMG_OK;
}

// Kernels executed by one replay of an instance's loop: start kernel plus
// the body per iteration.
void count_replay(const cmg_handle* h, int iterations) {
  count_launches((int)(1 + h->ir_body_kernels * iterations));
}

// The single-instance refinement graph, rebuilt when the iterate / right-side
// pointers or the cycle options change.
cmg_status build_ir_graph(cmg_handle* h, const cmg_cycle& o, Vec3c<double> f, Vec3<double> x) {
  const void* key[6] = {f.y, f.u, f.p, x.y, x.u, x.p};
  if (h->ir_exec && same_cycle(h->ir_opts, o) && std::equal(key, key + 6, h->ir_key) && h->ir_gscale == h->gscale)
    return CMG_OK;
  if (h->ir_exec) {
    CK(cudaGraphExecDestroy(h->ir_exec));
    h->ir_exec = nullptr;
  }
  if (h->ir_graph) {
    CK(cudaGraphDestroy(h->ir_graph));
    h->ir_graph = nullptr;
  }
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  h->ir_graph = g;
  const cmg_status s = add_ir_loop(h, o, f, x, g);
  if (s != CMG_OK) return s;
  cudaGraphExec_t ex = nullptr;
  CK(cudaGraphInstantiate(&ex, g, 0));
  h->ir_exec = ex;
  h->ir_opts = o;
  h->ir_gscale = h->gscale;
  std::copy(key, key + 6, h->ir_key);
  return CMG_OK;
}

cmg_status solve_cycle(cmg_handle* h, const cmg_cycle& o, double tol, int maxit, Vec3c<double> f, Vec3<double> x,
                       double fnorm, cmg_stats* st) {
  Lev& l0 = h->lv[0];
  const size_t ny = l0.nodes * h->prob.N, nu = l0.nodes;
  double rho = 0;
  cmg_status s = CMG_OK;
  int it = 0;
  if (o.precision == CMG_FP64) {
    s = true_residual(h, f, cview(x), &rho);
    if (s != CMG_OK) return s;
    st->relres0 = rho / fnorm;
    while (std::isfinite(rho) && rho > tol * fnorm && it < maxit) {
      CK(cycle<double>(h, o, 0, x, f));
      ++it;
      s = true_residual(h, f, cview(x), &rho);
      if (s != CMG_OK) return s;
    }
  } else {
    // FP64 iterative refinement around FP32 cycles.  One fused pass forms
    // r = f - S x in FP64 and writes r * sc in FP32 (the next cycle's right
    // side) with the norm partials; the cycle solves S e = r * sc from zero
    // and x += e / sc.  sc = 1 / (previous residual norm) keeps the FP32
    // right side O(1) whatever the residual level.
    Vec3<float> f32 = Work<float>::f(l0), x32 = Work<float>::x(l0);
    auto outer = [&](double sc, double* out) -> cmg_status {
      const int cnt = launch_residual_cast(view<double>(h, 0), cview(x), f, f32, sc, nullptr, paper_wy(h), h->part,
                                           h->part_cap, h->stream);
      if (cnt < 0) return fail(h, CMG_ERR_CUDA, "refinement pass launch failed");
      CK(launch_finish_sum(h->part, cnt, h->dsc, h->stream));
      CK(fetch(h, h->dsc, 1));
      *out = std::sqrt(h->hsc[0]) / sc;
      return CMG_OK;
    };
    double sc = 1.0 / fnorm;
    s = outer(sc, &rho);
    if (s != CMG_OK) return s;
    st->relres0 = rho / fnorm;
    const bool use_graph = h->graphs && h->prof_kinds == 0 && std::isfinite(rho) && rho > tol * fnorm && maxit > 0;
    if (std::isfinite(rho) && rho > tol * fnorm && maxit > 0) {
      Vec3<float> d32{l0.d32[0], l0.d32[1], l0.d32[2]};
      CK(zero_vec<float>(h, 0, d32));
      ir_state_init(h, h->hsc, rho, sc, maxit, tol * fnorm);
      CK(cudaMemcpyAsync(h->ir_state, h->hsc, kIrStateSize * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    }
    if (use_graph) {
      // The loop runs on the device; the host reads the result once.
      s = build_ir_graph(h, o, f, x);
      if (s != CMG_OK) return s;
      CK(cudaGraphLaunch(h->ir_exec, h->stream));
      CK(fetch(h, h->ir_state, kIrStateSize));
      rho = h->hsc[kRho];
      it = (int)h->hsc[kIt];
      count_replay(h, it);
    } else if (std::isfinite(rho) && rho > tol * fnorm && maxit > 0) {
      // the same kernels launched one by one; the host reads the device's
      // decisions after each step and skips the anchor kernels when none is due
      cudaGraphConditionalHandle none = 0;
      while (true) {
        s = ir_iteration(h, o, f, x, none, 0, false);
        if (s != CMG_OK) return s;
        CK(fetch(h, h->ir_state, kIrStateSize));
        if (h->hsc[kAnchor] != 0.0) {
          s = ir_iteration_anchor(h, f, x, none, 0);
          if (s != CMG_OK) return s;
          CK(fetch(h, h->ir_state, kIrStateSize));
        }
        if (h->hsc[kGo] == 0.0) break;
      }
      rho = h->hsc[kRho];
      it = (int)h->hsc[kIt];
    }
  }
  st->iters = it;
  st->cycles = it;
  st->relres = rho / fnorm;
  if (!std::isfinite(rho)) return fail(h, CMG_ERR_NONFINITE, "residual norm is not finite");
  if (rho > tol * fnorm) return fail(h, CMG_ERR_NOT_CONVERGED, "maximum iterations reached");
  return CMG_OK;
}

// Flat [y | pad | u | pad | p | pad] Krylov vector: every segment starts on a
// 256-byte boundary (the node kernels use 16-byte vector loads); the pads
// are zeroed once at allocation and stay zero under every vector operation.
inline size_t pad32(size_t v) { return (v + 31) & ~(size_t)31; }
Vec3<double> flat3(double* base, size_t ny, size_t nu) {
  return {base, base + pad32(ny), base + pad32(ny) + pad32(nu)};
}

cmg_status solve_fgmres(cmg_handle* h, const cmg_cycle& o, double tol, int maxit, int restart, Vec3c<double> f,
                        Vec3<double> x, double fnorm, cmg_stats* st) {
  Lev& l0 = h->lv[0];
  const size_t ny = l0.nodes * h->prob.N, nu = l0.nodes, nt = 2 * pad32(ny) + pad32(nu);
  const size_t pad = nt;
  if (restart > h->gm_cap || h->nt != nt) {
    if (h->gm) {
      CK(cudaStreamSynchronize(h->stream));
      CK(cudaFree(h->gm));
      h->gm = nullptr;
      h->gm_cap = 0;
    }
    void* q = nullptr;
    CK(cudaMalloc(&q, (size_t)(2 * restart + 2) * pad * sizeof(double)));
    h->gm = static_cast<double*>(q);
    CK(cudaMemsetAsync(q, 0, (size_t)(2 * restart + 2) * pad * sizeof(double), h->stream));
    h->gm_cap = restart;
    h->nt = nt;
    h->nt_pad = pad;
  }
  double* V = h->gm;                                   // restart+1 vectors
  double* Z = h->gm + (size_t)(restart + 1) * pad;     // restart vectors
  double* X = h->gm + (size_t)(2 * restart + 1) * pad; // flat iterate
  const Vec3<double> Xv = flat3(X, ny, nu);
  CK(cudaMemcpyAsync(Xv.y, x.y, ny * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpyAsync(Xv.u, x.u, nu * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpyAsync(Xv.p, x.p, ny * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));

  double* d_h1 = h->dsc + 64;
  double* d_h2 = h->dsc + 192;
  double* d_nrm = h->dsc + 320;
  double* d_y = h->dsc + 384;
  std::vector<double> H((size_t)(restart + 1) * restart), cs(restart), sn(restart), g(restart + 1), yk(restart);
  auto Hat = [&](int i, int k) -> double& { return H[(size_t)i * restart + k]; };

  auto residual_to_v0 = [&](double* beta) -> cmg_status {
    Vec3<double> r0 = flat3(V, ny, nu);
    CK(launch_residual<double>(view<double>(h, 0), cview(Xv), f, r0, h->stream, paper_wy(h)));
    CK(launch_sumsq(V, nt, h->red, 0, 1.0, h->stream));
    CK(launch_finish_sum(h->red, kRedBlocks, d_nrm, h->stream));
    CK(fetch(h, d_nrm, 1));
    *beta = std::sqrt(h->hsc[0]);
    return CMG_OK;
  };

  double beta = 0;
  cmg_status s = residual_to_v0(&beta);
  if (s != CMG_OK) return s;
  st->relres0 = beta / fnorm;
  double relres = st->relres0;
  int total = 0;
  bool breakdown = false;
  while (std::isfinite(relres) && relres > tol && total < maxit && !breakdown) {
    CK(launch_scale_by(V, d_nrm, V, nt, h->stream));    // v0 = r0 / ||r0||
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int kd = 0;
    for (int k = 0; k < restart; ++k) {
      double* vk = V + (size_t)k * pad;
      double* zk = Z + (size_t)k * pad;
      double* w = V + (size_t)(k + 1) * pad;
      s = precondition(h, o, cview(flat3(vk, ny, nu)), flat3(zk, ny, nu), paper_wy(h));
      if (s != CMG_OK) return s;
      ++st->cycles;
      CK(launch_residual<double>(view<double>(h, 0), cview(flat3(zk, ny, nu)), Vec3c<double>{nullptr, nullptr, nullptr},
                                 flat3(w, ny, nu), h->stream, paper_wy(h)));   // w = W S z_k
      // classical Gram-Schmidt, twice
      CK(launch_mdot(V, pad, k + 1, w, nt, h->red, d_h1, h->stream));
      CK(launch_maxpy(V, pad, k + 1, d_h1, -1.0, w, nt, h->stream));
      CK(launch_mdot(V, pad, k + 1, w, nt, h->red, d_h2, h->stream));
      CK(launch_maxpy(V, pad, k + 1, d_h2, -1.0, w, nt, h->stream));
      CK(launch_sumsq(w, nt, h->red, 0, 1.0, h->stream));
      CK(launch_finish_sum(h->red, kRedBlocks, d_nrm, h->stream));
      CK(cudaMemcpyAsync(h->hsc, d_h1, 256 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaMemcpyAsync(h->hsc + 256, d_h2, 256 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaMemcpyAsync(h->hsc + 512, d_nrm, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      for (int i = 0; i <= k; ++i) Hat(i, k) = h->hsc[i] + h->hsc[256 + i];
      const double hn = std::sqrt(h->hsc[512]);
      Hat(k + 1, k) = hn;
      if (!std::isfinite(hn)) return fail(h, CMG_ERR_NONFINITE, "Arnoldi norm is not finite");
      if (hn > 0) CK(launch_scale_by(w, d_nrm, w, nt, h->stream));
      else breakdown = true;
      for (int i = 0; i < k; ++i) {
        const double t = cs[i] * Hat(i, k) + sn[i] * Hat(i + 1, k);
        Hat(i + 1, k) = -sn[i] * Hat(i, k) + cs[i] * Hat(i + 1, k);
        Hat(i, k) = t;
      }
      const double rr = std::hypot(Hat(k, k), Hat(k + 1, k));
      cs[k] = Hat(k, k) / rr;
      sn[k] = Hat(k + 1, k) / rr;
      Hat(k, k) = rr;
      Hat(k + 1, k) = 0.0;
      g[k + 1] = -sn[k] * g[k];
      g[k] = cs[k] * g[k];
      ++total;
      kd = k + 1;
      relres = std::fabs(g[k + 1]) / fnorm;
      if (relres <= tol || total >= maxit || breakdown) break;
    }
    for (int i = kd - 1; i >= 0; --i) {
      double t = g[i];
      for (int j = i + 1; j < kd; ++j) t -= Hat(i, j) * yk[j];
      yk[i] = t / Hat(i, i);
    }
    std::memcpy(h->hsc, yk.data(), kd * sizeof(double));
    CK(cudaMemcpyAsync(d_y, h->hsc, kd * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(launch_maxpy(Z, pad, kd, d_y, 1.0, X, nt, h->stream));
    s = residual_to_v0(&beta);
    if (s != CMG_OK) return s;
    relres = beta / fnorm;
  }
  CK(cudaMemcpyAsync(x.y, Xv.y, ny * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpyAsync(x.u, Xv.u, nu * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpyAsync(x.p, Xv.p, ny * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  st->iters = total;
  st->relres = relres;
  if (!std::isfinite(relres)) return fail(h, CMG_ERR_NONFINITE, "residual norm is not finite");
  if (relres > tol) return fail(h, CMG_ERR_NOT_CONVERGED, "maximum iterations reached");
  return CMG_OK;
}

}  // namespace

extern "C" cmg_status cmg_solve(cmg_handle* h, const cmg_cycle* opts, int method, double tol, int maxit, int restart,
                                const double* fy, const double* fu, const double* fp, double* y, double* u, double* p,
                                cmg_stats* stats) {
  if (!h) return CMG_ERR_INVALID_ARG;
  cmg_status s = check_cycle(h, opts);
  if (s != CMG_OK) return s;
  if (!vec_ok(fy, fu, fp) || !vec_ok(y, u, p)) return fail(h, CMG_ERR_INVALID_ARG, "null pointer");
  if (!(tol > 0.0) || maxit < 0) return fail(h, CMG_ERR_INVALID_ARG, "tol must be > 0 and maxit >= 0");
  if (method != CMG_METHOD_CYCLE && method != CMG_METHOD_FGMRES) return fail(h, CMG_ERR_INVALID_ARG, "unknown method");
  if (method == CMG_METHOD_FGMRES && (restart < 1 || restart > kMaxRestart))
    return fail(h, CMG_ERR_INVALID_ARG, "restart must be in [1, 60]");
  cmg_stats local{};
  cmg_stats* st = stats ? stats : &local;
  *st = cmg_stats{};
  CK(sumsq3(h, 0, fy, fu, fp, h->dsc, paper_wy(h) * paper_wy(h)));
  CK(fetch(h, h->dsc, 1));
  const double fnorm = std::sqrt(h->hsc[0]);   // ||W f||
  if (!std::isfinite(fnorm)) return fail(h, CMG_ERR_NONFINITE, "right-hand side is not finite");
  const Vec3c<double> f{fy, fu, fp};
  const Vec3<double> x{y, u, p};
  if (fnorm == 0.0) {
    CK(zero_vec<double>(h, 0, x));
    CK(cudaStreamSynchronize(h->stream));
    return CMG_OK;
  }
  CK(opts->precision == CMG_FP64 ? ensure_fp64(h) : ensure_galerkin32(h));
  if (method == CMG_METHOD_CYCLE) return solve_cycle(h, *opts, tol, maxit, f, x, fnorm, st);
  return solve_fgmres(h, *opts, tol, maxit, restart, f, x, fnorm, st);
}

// L1 + box constrained problem: globalised semismooth Newton (Sec. 4,
// Algorithm 2).  In the symmetric scaling E[p_paper] = sum_j p_j; each Newton
// system is the linear-quadratic system with the control row as the paper
// writes it (G = h^2, coupling d / nu restricted to the active sets: per-node
// factor dw = chi / nu on d, injected to coarse grids) and right side
// (0, -h^2 F, 0), solved by cmg_solve.  (Multiplying that row by nu gives
// the same iterates but a right side nu times smaller, whose relative
// residual stalls at the rounding floor.)
extern "C" cmg_status cmg_ssn_solve(cmg_handle* h, const cmg_cycle* opts, int method, double beta, double a,
                                    double b, double tol, double inner_tol, int maxit, const double* yd, double* y,
                                    double* u, double* p, cmg_ssn_stats* stats) {
  if (!h) return CMG_ERR_INVALID_ARG;
  cmg_status s = check_cycle(h, opts);
  if (s != CMG_OK) return s;
  if (!yd || !vec_ok(y, u, p) || (reinterpret_cast<uintptr_t>(yd) & 15))
    return fail(h, CMG_ERR_INVALID_ARG, "null or misaligned vector");
  if (!(a < 0.0 && b > 0.0 && beta >= 0.0 && tol > 0.0 && inner_tol > 0.0 && maxit >= 0) || !std::isfinite(a) ||
      !std::isfinite(b) || !std::isfinite(beta))
    return fail(h, CMG_ERR_INVALID_ARG, "need a < 0 < b, beta >= 0, tol > 0, inner_tol > 0, maxit >= 0");
  if (opts->freeze_u) return fail(h, CMG_ERR_INVALID_ARG, "the Newton systems need the control update");
  if (h->galerkin()) return fail(h, CMG_ERR_UNSUPPORTED, "semismooth Newton: rediscretised coarse grids only");
  if (method != CMG_METHOD_CYCLE && method != CMG_METHOD_FGMRES) return fail(h, CMG_ERR_INVALID_ARG, "unknown method");
  cmg_ssn_stats local{};
  cmg_ssn_stats* st = stats ? stats : &local;
  *st = cmg_ssn_stats{};
  Lev& l0 = h->lv[0];
  const int N = h->prob.N;
  const size_t ny = l0.nodes * N, nu = l0.nodes;
  const double nuc = h->prob.nu, hh = l0.h;
  // work vectors, each segment on a 256-byte boundary
  const size_t sy = pad32(ny), su = pad32(nu);
  if (!h->ssn) {
    void* q = nullptr;
    CK(cudaMalloc(&q, (4 * sy + 6 * su) * sizeof(double) + su * sizeof(float)));
    h->allocs.push_back(q);
    h->ssn = static_cast<double*>(q);
  }
  double* fy = h->ssn;
  double* fp = fy + sy;
  double* dy = fp + sy;
  double* dp = dy + sy;
  double* fu = dp + sy;
  double* du = fu + su;
  double* Tu = du + su;
  double* Tdp = Tu + su;
  double* F = Tdp + su;
  double* spare = F + su;
  float* chi = reinterpret_cast<float*>(spare + su);
  (void)spare;
  const long nodes = (long)nu;
  auto merit = [&](const double* uu, const double* duu, const double* tu, const double* tdp, double g, double* Fout,
                   float* chio, double* out) -> cmg_status {
    const int cnt = launch_ssn_map(nodes, uu, duu, tu, tdp, g, nuc, beta, a, b, Fout, chio, h->part, h->part_cap,
                                   h->stream);
    if (cnt < 0) return fail(h, CMG_ERR_CUDA, "optimality map launch failed");
    CK(launch_finish_sum(h->part, cnt, h->dsc, h->stream));
    CK(fetch(h, h->dsc, 1));
    *out = hh * std::sqrt(h->hsc[0]);   // phi = sqrt(F' M F), M = h^2 I
    return CMG_OK;
  };
  auto inner = [&](double* xy, double* xu, double* xp) -> cmg_status {
    cmg_stats is{};
    const cmg_status r = cmg_solve(h, opts, method, inner_tol, 200, 30, fy, fu, fp, xy, xu, xp, &is);
    st->inner_total += is.iters;
    return r == CMG_ERR_NOT_CONVERGED ? CMG_OK : r;   // at the rounding floor the last iterate is kept
  };
  cmg_status res = CMG_OK;
  // (1) y0, p0 for u0: the Newton system's form with no control coupling
  //     (dw = 0) and right side (c y_d, h^2 u0, 0) leaves u = u0 and solves
  //     the 2N PDEs of Algorithm 2's first line
  h->gscale = 1.0 / nuc;
  h->dw_on = true;
  const double hh2 = hh * hh;
  for (int l = 0; l < h->L && res == CMG_OK; ++l)
    if (launch_fill32((long)h->lv[l].nodes, 0.f, h->lv[l].dw, h->stream) != cudaSuccess) res = CMG_ERR_CUDA;
  if (res == CMG_OK && refresh_dw(h) != cudaSuccess) res = CMG_ERR_CUDA;
  if (res == CMG_OK) {
    CK(launch_spread(nodes, N, l0.c, yd, fy, h->stream));
    CK(launch_scale64(nodes, hh2, u, fu, h->stream));
    CK(cudaMemsetAsync(fp, 0, ny * sizeof(double), h->stream));
    CK(cudaMemsetAsync(y, 0, ny * sizeof(double), h->stream));
    CK(cudaMemsetAsync(p, 0, ny * sizeof(double), h->stream));
    res = inner(y, u, p);
  }
  double phi = 0.0;
  if (res == CMG_OK) {
    CK(launch_sum_samples(nodes, N, p, Tu, h->stream));
    res = merit(u, nullptr, Tu, nullptr, 0.0, F, chi, &phi);
    st->merit0 = phi;
  }
  const double sigma_ls = 1e-4, rho_ls = 0.5;
  while (res == CMG_OK && phi > tol && st->newton < maxit) {
    // (2) active sets -> dw = chi / nu on every grid; right side (0, -h^2 F, 0)
    CK(launch_scale32(nodes, (float)(1.0 / nuc), chi, l0.dw, h->stream));
    if (refresh_dw(h) != cudaSuccess) { res = fail(h, CMG_ERR_CUDA, "active-set update failed"); break; }
    CK(cudaMemsetAsync(fy, 0, ny * sizeof(double), h->stream));
    CK(launch_scale64(nodes, -hh2, F, fu, h->stream));
    CK(cudaMemsetAsync(dy, 0, ny * sizeof(double), h->stream));
    CK(cudaMemsetAsync(du, 0, nu * sizeof(double), h->stream));
    CK(cudaMemsetAsync(dp, 0, ny * sizeof(double), h->stream));
    res = inner(dy, du, dp);
    if (res != CMG_OK) break;
    // (3) backtracking line search on phi; T(u + g du) = Tu + g T(du) is linear
    CK(launch_sum_samples(nodes, N, dp, Tdp, h->stream));
    double g = 1.0, trial = 0.0;
    for (int k = 0; k < 40; ++k) {
      res = merit(u, du, Tu, Tdp, g, nullptr, nullptr, &trial);
      if (res != CMG_OK || trial - phi <= -sigma_ls * phi) break;
      g *= rho_ls;
    }
    if (res != CMG_OK) break;
    // (4) x += g dx; active sets and phi at the new iterate
    CK(launch_axpy64((long)ny, g, dy, y, h->stream));
    CK(launch_axpy64(nodes, g, du, u, h->stream));
    CK(launch_axpy64((long)ny, g, dp, p, h->stream));
    CK(launch_axpy64(nodes, g, Tdp, Tu, h->stream));
    res = merit(u, nullptr, Tu, nullptr, 0.0, F, chi, &phi);
    ++st->newton;
  }
  st->merit = phi;
  // back to the linear-quadratic operators (G = nu h^2, dw = 1)
  h->gscale = 1.0;
  h->dw_on = false;
  for (int l = 0; l < h->L; ++l) (void)launch_fill32((long)h->lv[l].nodes, 1.f, h->lv[l].dw, h->stream);
  const cudaError_t er = refresh_dw(h);
  if (res != CMG_OK) return res;
  if (er != cudaSuccess) return cuda_fail(h, er, "restoring the operators");
  if (!std::isfinite(phi)) return fail(h, CMG_ERR_NONFINITE, "merit function is not finite");
  if (phi > tol) return fail(h, CMG_ERR_NOT_CONVERGED, "maximum Newton iterations reached");
  return CMG_OK;
}

// ============================================================================
// Batched solves: many independent instances in one graph launch.
struct cmg_batch {
  std::vector<cmg_handle*> inst;
  cudaStream_t stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> key;
  cmg_cycle opts{};
  std::string err;
  // batched persistent form (cmg_batch.cu): device tables, persistent grid
  // per depth, and the refinement loop as one graph with a while node
  int mode = 0;                      // form of the last FP32 solve: CMG_BATCH_PERSISTENT or CMG_BATCH_BRANCHES
  int force = 0;                     // cmg_batch_set_form: CMG_BATCH_PERSISTENT, else the branches
  long long wait_limit = 0;          // polls per barrier wait (0 = the default)
  std::vector<void*> pallocs;
  BatchTables T{};
  int* act = nullptr;                // [count] (T.act points here)
  int* any = nullptr;                // device: some instance still iterating
  int* hany = nullptr;               // pinned host copy
  std::vector<int> grid_down, grid_up;
  std::vector<int> leg_phases;       // per depth: 1 = one launch per phase, 0 = the persistent kernel
  int leg_force = -1;                // CMG_BATCH_LEG_* override (-1 = by the depth's work)
  int Nmax = 0, cm = 0;
  BatchCoarse* coarse = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraph_t pgraph = nullptr;
  cudaGraphExec_t pexec = nullptr;
  std::vector<const void*> pkey;
  cmg_cycle popts{};
  long long body_kernels = 0;
  bool graph_failed = false;         // the loop's capture was refused: it runs eagerly
  std::string graph_error;
};

namespace {

cmg_status bfail(cmg_batch* b, cmg_status st, const std::string& msg) {
  if (b) b->err = msg;
  return st;
}

#define BCK(call)                                                                                \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) {                                                                     \
      (void)cudaGetLastError();                                                                  \
      return bfail(b, e_ == cudaErrorMemoryAllocation ? CMG_ERR_OOM : CMG_ERR_CUDA,              \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                          \
    }                                                                                            \
  } while (0)

}  // namespace

// ---- batched persistent form: host side ------------------------------------

namespace {

// Items (warps of nodes) from which a grid depth runs one launch per phase
// instead of the persistent kernel: enough warps to fill every SM several
// times, so launch latency is small beside the work.
constexpr long kBatchPhaseItems = 152L * 32 * 4;

// Sample map of the batched kernels: FP32 maps (elem4 = 1) take 16-byte
// vectors where N allows, FP64 maps 8-byte ones; rule kBatchMapPhase gives
// 16 samples per lane, kBatchMapCoop four.
void batch_map(int N, int elem4, int rule, int& lpn, int& V, int& spl) {
  if (elem4) V = N % 4 == 0 ? 4 : (N % 2 == 0 ? 2 : 1);
  else V = N % 2 == 0 ? 2 : 1;
  spl = (rule == kBatchMapPhase && elem4 ? 16 : 4) / V;
  const int E = V * spl;   // samples per lane
  const int need = (N + E - 1) / E;
  lpn = 1;
  while (lpn < need) lpn <<= 1;
}

// The persistent form covers FP32 V-cycles with red-black smoothing (n1, n2
// >= 1, the control updated), rediscretised (averaged) coarse grids with one
// coarsest size for all instances, distributed or local control, and N <= 128.
bool batch_persistent_ok(const cmg_batch* b, const cmg_cycle& o, std::string* why) {
  auto no = [&](const char* m) {
    if (why) *why = m;
    return false;
  };
  if (o.precision != CMG_FP32 || o.smoother != CMG_SMOOTH_RBGS || o.gamma != 1 || o.n1 < 1 || o.n2 < 1 ||
      o.freeze_u)
    return no("cycle options outside the persistent form (FP32 red-black V-cycle, n1, n2 >= 1)");
  const int m = b->inst[0]->coarse.m;
  for (const cmg_handle* h : b->inst) {
    if (h->prob.N > 128) return no("a sample count above 128");
    if (h->prob.coarse_coeff != CMG_COARSE_AVERAGED) return no("coarse grids other than averaged");
    if (h->coarse.m != m || !h->coarse32.Ainv32) return no("coarsest grids of different sizes");
    if (h->L < 2) return no("an instance with a single grid");
  }
  return true;
}

template <typename T>
cudaError_t palloc(cmg_batch* b, T** p, size_t count) {
  void* q = nullptr;
  const cudaError_t e = cudaMalloc(&q, (count ? count : 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  b->pallocs.push_back(q);
  *p = static_cast<T*>(q);
  return cudaSuccess;
}

void batch_free_tables(cmg_batch* b) {
  if (b->pexec) (void)cudaGraphExecDestroy(b->pexec);
  if (b->pgraph) (void)cudaGraphDestroy(b->pgraph);
  b->pexec = nullptr;
  b->pgraph = nullptr;
  for (void* q : b->pallocs) (void)cudaFree(q);
  b->pallocs.clear();
  if (b->hany) (void)cudaFreeHost(b->hany);
  b->hany = nullptr;
  b->T = BatchTables{};
}

// Per-instance control of the refinement, the decisions of the single-
// instance loop (ir_recur_control_kernel, ir_anchor_control_kernel) from the
// per-item partial sums; CTA b serves instance b.
__global__ void batch_recur_control_kernel(BatchTables T) {
  const int b = blockIdx.x;
  if (*T.err || !T.act[b]) return;
  const int* pre = batch_prefix(T, 0, kBkAll32, 0);
  const double t = block_total(T.partial + pre[b], pre[b + 1] - pre[b]);
  if (threadIdx.x != 0) return;
  double* s = T.inst[b].state;
  const double rho = sqrt(t) * s[kInvSc];
  const double it = s[kIt] + 1.0, since = s[kSince] + 1.0;
  s[kRho] = rho;
  s[kIt] = it;
  s[kSince] = since;
  const bool anchor = !isfinite(rho) || rho <= s[kTolAbs] || rho <= s[kDrop] * s[kRhoAnchor] ||
                      it >= s[kMaxit] || since >= s[kAmax];
  s[kSc] = (isfinite(rho) && rho > 0.0) ? 1.0 / rho : 1.0 / s[kRhoAnchor];
  s[kAnchor] = anchor ? 1.0 : 0.0;
  s[kGo] = anchor ? 0.0 : 1.0;
}

__global__ void batch_anchor_control_kernel(BatchTables T) {
  const int b = blockIdx.x;
  if (*T.err || !T.act[b]) return;
  double* s = T.inst[b].state;
  if (s[kAnchor] == 0.0) return;
  const int* pre = batch_prefix(T, 0, kBkAll64, 0);
  const double t = block_total(T.partial + pre[b], pre[b + 1] - pre[b]);
  if (threadIdx.x != 0) return;
  const double sc = s[kSc];
  const double rho = sqrt(t) / sc;
  s[kInvSc] = 1.0 / sc;
  s[kSc] = 1.0 / rho;
  s[kRho] = rho;
  s[kRhoAnchor] = rho;
  s[kSince] = 0.0;
  s[kGo] = (isfinite(rho) && rho > s[kTolAbs] && s[kIt] < s[kMaxit]) ? 1.0 : 0.0;
}

// Iterating flags for the next iteration and the loop condition (some
// instance still iterating and no barrier wait ran out).
__global__ void batch_next_kernel(BatchTables T, int* act, int* any, cudaGraphConditionalHandle cond, int graph) {
  const int err = *T.err;
  int mine = 0;
  for (int i = threadIdx.x; i < T.count; i += blockDim.x) {
    const int a = (!err && T.inst[i].state[kGo] != 0.0) ? 1 : 0;
    act[i] = a;
    mine |= a;
  }
  const int go = __syncthreads_or(mine);
  if (threadIdx.x == 0) {
    *any = go;
    if (graph) cudaGraphSetConditional(cond, go ? 1u : 0u);
  }
}

}  // namespace

cudaError_t cmg::launch_batch_recur_control(const BatchTables& T, cudaStream_t s) {
  batch_recur_control_kernel<<<T.count, 256, 0, s>>>(T);
  count_launches(1);
  return cudaGetLastError();
}
cudaError_t cmg::launch_batch_anchor_control(const BatchTables& T, cudaStream_t s) {
  batch_anchor_control_kernel<<<T.count, 256, 0, s>>>(T);
  count_launches(1);
  return cudaGetLastError();
}

namespace {

// Device tables of the batch for the current vectors and options.
cmg_status batch_build_tables(cmg_batch* b, const cmg_cycle& o, const double* const* fy, const double* const* fu,
                              const double* const* fp, double* const* y, double* const* u, double* const* p) {
  batch_free_tables(b);
  const int count = (int)b->inst.size();
  int D = 0;
  for (const cmg_handle* h : b->inst) D = std::max(D, h->L);
  std::vector<BatchLevel> lev((size_t)count * kMaxLevels);
  std::vector<BatchInst> inst(count);
  std::vector<BatchCoarse> co(count);
  std::vector<int> pre((size_t)D * kBkKinds * kBkClasses * (count + 1), 0);
  int cls_mask[kMaxLevels] = {};
  auto items = [](long nodes, int per) { return (int)((nodes + per - 1) / per); };
  // the form of each depth's legs, from its work in warps of nodes under
  // the persistent kernels' map: grids with much work get one launch per
  // phase and map class (the registers of one variant, every SM's warps
  // resident, 16 samples per lane); the rest run in the persistent
  // kernels (one launch per leg, barriers instead of launches)
  b->leg_phases.assign(D, 0);
  int maps[kMaxLevels];
  for (int d = 0; d < kMaxLevels; ++d) maps[d] = kBatchMapCoop;
  for (int d = 0; d < D; ++d) {
    long work = 0;
    for (const cmg_handle* h : b->inst)
      if (d < h->L - 1) {
        int lpn, V, spl;
        batch_map(h->prob.N, 1, kBatchMapCoop, lpn, V, spl);
        work += items((long)h->lv[d].n * h->lv[d].n, 32 / lpn);
      }
    b->leg_phases[d] = b->leg_force >= 0 ? b->leg_force : (work >= kBatchPhaseItems ? 1 : 0);
    maps[d] = b->leg_phases[d] ? kBatchMapPhase : kBatchMapCoop;
  }
  b->Nmax = 0;
  b->cm = b->inst[0]->coarse.m;
  for (int i = 0; i < count; ++i) {
    cmg_handle* h = b->inst[i];
    const int N = h->prob.N;
    b->Nmax = std::max(b->Nmax, N);
    int V = 1, lpn64, V64, spl64;
    batch_map(N, 0, kBatchMapCoop, lpn64, V64, spl64);
    for (int l = 0; l < h->L; ++l) {
      BatchLevel& B = lev[(size_t)i * kMaxLevels + l];
      B.L = view<float>(h, l, 0, o.ctl32);
      B.x = Work<float>::x(h->lv[l]);
      B.f = Work<float>::f(h->lv[l]);
      B.r = Work<float>::r(h->lv[l]);
      batch_map(N, 1, maps[l], B.lpn, B.V, B.spl);
      V = B.V;
      B.nc = l + 1 < h->L ? h->lv[l + 1].n : 0;
    }
    BatchInst& I = inst[i];
    I.L64 = view<double>(h, 0);
    I.f64 = Vec3c<double>{fy[i], fu[i], fp[i]};
    I.x64 = Vec3<double>{y[i], u[i], p[i]};
    Lev& l0 = h->lv[0];
    I.d32 = Vec3<float>{l0.d32[0], l0.d32[1], l0.d32[2]};
    I.state = h->ir_state;
    I.wy2 = (float)(paper_wy(h) * paper_wy(h));
    I.lpn64 = lpn64;
    I.V64 = V64;
    I.spl64 = spl64;
    I.levels = h->L;
    const CoarseData cd = coarse_for<float>(h);
    const Lev& cl = h->lv[h->L - 1];
    co[i] = BatchCoarse{cd.m, N, cd.n, cd.ctl, cd.Ainv32, cd.Minv, cl.c, cl.d, cl.e, cd.dw,
                        cview(Work<float>::f(h->lv[h->L - 1])), Work<float>::x(h->lv[h->L - 1])};
    const int npw64 = 32 / lpn64;
    const int cls = V == 4 ? 1 : (V == 2 ? 2 : 3);
    for (int d = 0; d < D; ++d) {
      int cnt[kBkKinds] = {0, 0, 0, 0, 0};
      if (d < h->L - 1) {
        const int n = h->lv[d].n, nc = h->lv[d + 1].n;
        const int npw = 32 / lev[(size_t)i * kMaxLevels + d].lpn;
        cnt[kBkColour0] = items(colour_count(n, 0), npw);
        cnt[kBkColour1] = items(colour_count(n, 1), npw);
        cnt[kBkCoarse] = items((long)nc * nc, npw);
        cnt[kBkAll32] = items((long)n * n, npw);
        cls_mask[d] |= 1 << (cls - 1);
      }
      if (d == 0) cnt[kBkAll64] = items((long)h->lv[0].n * h->lv[0].n, npw64);
      for (int k = 0; k < kBkKinds; ++k)
        for (int c : {0, cls}) pre[(((size_t)d * kBkKinds + k) * kBkClasses + c) * (count + 1) + i + 1] = cnt[k];
    }
  }
  long max_all = 0;
  std::vector<long> max_depth(D, 0);
  for (int d = 0; d < D; ++d)
    for (int k = 0; k < kBkKinds; ++k)
      for (int c = 0; c < kBkClasses; ++c) {
        int* row = &pre[(((size_t)d * kBkKinds + k) * kBkClasses + c) * (count + 1)];
        for (int i = 0; i < count; ++i) row[i + 1] += row[i];
        if (c != 0) continue;
        if (k <= kBkAll32) max_depth[d] = std::max<long>(max_depth[d], row[count]);
        if (d == 0 && k >= kBkAll32) max_all = std::max<long>(max_all, row[count]);
      }
  // per row, the instance of every 8th item (the first item of each CTA of
  // a one-item-per-warp launch)
  std::vector<int> first;
  int first_off[kMaxLevels][kBkKinds][kBkClasses] = {};
  for (int d = 0; d < D; ++d)
    for (int k = 0; k < kBkKinds; ++k)
      for (int c = 0; c < kBkClasses; ++c) {
        const int* row = &pre[(((size_t)d * kBkKinds + k) * kBkClasses + c) * (count + 1)];
        first_off[d][k][c] = (int)first.size();
        int i = 0;
        for (int it = 0; it < row[count]; it += 8) {
          while (row[i + 1] <= it) ++i;
          first.push_back(i);
        }
      }
  if (first.empty()) first.push_back(0);
  // one allocation per table
  BatchLevel* dlev;
  BatchInst* dinst;
  int *dpre, *dact, *derr, *dany, *dfirst;
  unsigned* dbar;
  double* dpart;
  BCK(palloc(b, &dlev, lev.size()));
  BCK(palloc(b, &dinst, inst.size()));
  BCK(palloc(b, &b->coarse, co.size()));
  BCK(palloc(b, &dpre, pre.size()));
  BCK(palloc(b, &dfirst, first.size()));
  BCK(palloc(b, &dact, (size_t)count));
  BCK(palloc(b, &derr, 1));
  BCK(palloc(b, &dany, 1));
  BCK(palloc(b, &dbar, 2));
  BCK(palloc(b, &dpart, (size_t)std::max<long>(max_all, 1)));
  BCK(cudaMallocHost(&b->hany, sizeof(int)));
  BCK(cudaMemcpyAsync(dlev, lev.data(), lev.size() * sizeof(BatchLevel), cudaMemcpyHostToDevice, b->stream));
  BCK(cudaMemcpyAsync(dinst, inst.data(), inst.size() * sizeof(BatchInst), cudaMemcpyHostToDevice, b->stream));
  BCK(cudaMemcpyAsync(b->coarse, co.data(), co.size() * sizeof(BatchCoarse), cudaMemcpyHostToDevice, b->stream));
  BCK(cudaMemcpyAsync(dpre, pre.data(), pre.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
  BCK(cudaMemcpyAsync(dfirst, first.data(), first.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  BatchTables& T = b->T;
  T.count = count;
  T.depths = D;
  T.lev = dlev;
  T.inst = dinst;
  T.pre = dpre;
  T.first = dfirst;
  T.act = dact;
  T.bar = dbar;
  T.err = derr;
  T.limit = b->wait_limit > 0 ? b->wait_limit : (1LL << 26);
  T.partial = dpart;
  T.n1 = o.n1;
  T.n2 = o.n2;
  for (int d = 0; d < kMaxLevels; ++d) {
    T.cls_mask[d] = cls_mask[d];
    T.maps[d] = maps[d];
    for (int k = 0; k < kBkKinds; ++k)
      for (int c = 0; c < kBkClasses; ++c) {
        T.items[d][k][c] = d < D ? pre[(((size_t)d * kBkKinds + k) * kBkClasses + c) * (count + 1) + count] : 0;
        T.first_off[d][k][c] = first_off[d][k][c];
      }
  }
  b->act = dact;
  b->any = dany;
  b->grid_down.assign(D, 0);
  b->grid_up.assign(D, 0);
  const int cap_d = batch_grid(0, 0), cap_u = batch_grid(1, 0);
  if (cap_d < 1 || cap_u < 1) return bfail(b, CMG_ERR_UNSUPPORTED, "no co-resident grid for the persistent kernels");
  for (int d = 0; d < D; ++d) {
    const long want = std::max<long>(1, (max_depth[d] + 63) / 64);   // a chunk of 8 items per warp, 8 warps
    // persistent legs (the per-phase launches size each class's grid to its
    // items, one warp per item)
    b->grid_down[d] = (int)std::min<long>(want, cap_d);
    b->grid_up[d] = (int)std::min<long>(want, cap_u);
  }
  return CMG_OK;
}

// One iteration of the batched refinement loop on stream s (eager, or into
// a capture): V-cycle (down-legs, coarsest solves, up-legs), recursion and
// its control, the gated anchor and its control, the next flags.
cmg_status batch_body(cmg_batch* b, cudaStream_t s, cudaGraphConditionalHandle cond, int graph) {
  const BatchTables& T = b->T;
  const int D = T.depths;
  for (int d = 0; d + 1 < D; ++d)
    BCK(b->leg_phases[d] ? launch_batch_down_phases(T, d, s)
                         : launch_batch_down(T, d, b->grid_down[d], s));
  BCK(launch_batch_coarse(b->coarse, T.count, b->Nmax, b->cm, T.act, T.err, s));
  for (int d = D - 2; d >= 0; --d)
    BCK(b->leg_phases[d] ? launch_batch_up_phases(T, d, s)
                         : launch_batch_up(T, d, b->grid_up[d], s));
  BCK(launch_batch_recur(T, s));
  BCK(launch_batch_recur_control(T, s));
  BCK(launch_batch_anchor(T, s));
  BCK(launch_batch_anchor_control(T, s));
  BCK(launch_k(batch_next_kernel, dim3(1), dim3(256), 0, s, T, b->act, b->any, cond, graph));
  count_launches(1);
  return CMG_OK;
}

// The batched loop as one graph: [next flags] -> while (some instance
// iterating) { batch_body }.
cmg_status batch_build_graph(cmg_batch* b) {
  if (!b->cap) BCK(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  BCK(cudaGraphCreate(&g, 0));
  b->pgraph = g;
  cudaGraphConditionalHandle cond;
  BCK(cudaGraphConditionalHandleCreate(&cond, g, 0, cudaGraphCondAssignDefault));
  cudaGraphNode_t start;
  {
    cudaKernelNodeParams kp = {};
    BatchTables T = b->T;
    int* act = b->act;
    int* any = b->any;
    int graph = 1;
    void* args[5] = {(void*)&T, (void*)&act, (void*)&any, (void*)&cond, (void*)&graph};
    kp.func = (void*)batch_next_kernel;
    kp.gridDim = dim3(1, 1, 1);
    kp.blockDim = dim3(256, 1, 1);
    kp.kernelParams = args;
    BCK(cudaGraphAddKernelNode(&start, g, nullptr, 0, &kp));
  }
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  BCK(cudaGraphAddNode(&node, g, &start, nullptr, 1, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  BCK(cudaStreamBeginCaptureToGraph(b->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  const long long k0 = cmg_kernel_launches();
  const cmg_status st = batch_body(b, b->cap, cond, 1);
  cudaGraph_t captured = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(b->cap, &captured);
  b->body_kernels = cmg_kernel_launches() - k0;
  count_launches((int)-b->body_kernels);
  if (st != CMG_OK) return st;
  BCK(e2);
  cudaGraphExec_t ex = nullptr;
  BCK(cudaGraphInstantiate(&ex, g, 0));
  b->pexec = ex;
  return CMG_OK;
}

bool batch_graphs_enabled(const cmg_batch* b) {
  for (const cmg_handle* h : b->inst)
    if (!h->graphs || h->prof_kinds) return false;
  return true;
}

}  // namespace

extern "C" cmg_status cmg_batch_create(const cmg_problem* probs, const double* const* xi_host, int count,
                                       void* stream, cmg_batch** out) {
  if (!out) return CMG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!probs || !xi_host || count < 1 || count > 4096) return CMG_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i)
    if (probs[i].coarse_coeff == CMG_COARSE_GALERKIN) return CMG_ERR_UNSUPPORTED;   // the batch kernels are 5-point
  cmg_batch* b = new (std::nothrow) cmg_batch();
  if (!b) return CMG_ERR_OOM;
  b->stream = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < count; ++i) {
    cmg_handle* h = nullptr;
    const cmg_status st = cmg_create(&probs[i], xi_host[i], stream, &h);
    if (st != CMG_OK) {
      cmg_batch_destroy(b);
      return st;
    }
    b->inst.push_back(h);
  }
  *out = b;
  return CMG_OK;
}

extern "C" void cmg_batch_destroy(cmg_batch* b) {
  if (!b) return;
  batch_free_tables(b);
  if (b->cap) (void)cudaStreamDestroy(b->cap);
  if (b->exec) (void)cudaGraphExecDestroy(b->exec);
  if (b->graph) (void)cudaGraphDestroy(b->graph);
  for (cmg_handle* h : b->inst) cmg_destroy(h);
  delete b;
}

extern "C" const char* cmg_batch_last_error(const cmg_batch* b) { return b ? b->err.c_str() : "null batch"; }

extern "C" cmg_handle* cmg_batch_instance(cmg_batch* b, int i) {
  return (b && i >= 0 && i < (int)b->inst.size()) ? b->inst[i] : nullptr;
}

extern "C" cmg_status cmg_batch_solve(cmg_batch* b, const cmg_cycle* opts, double tol, int maxit,
                                      const double* const* fy, const double* const* fu, const double* const* fp,
                                      double* const* y, double* const* u, double* const* p, cmg_stats* stats) {
  if (!b) return CMG_ERR_INVALID_ARG;
  if (!opts || !fy || !fu || !fp || !y || !u || !p || !stats) return bfail(b, CMG_ERR_INVALID_ARG, "null argument");
  const int count = (int)b->inst.size();
  for (int i = 0; i < count; ++i) {
    if (check_cycle(b->inst[i], opts) != CMG_OK) return bfail(b, CMG_ERR_INVALID_ARG, b->inst[i]->err);
    if (!vec_ok(fy[i], fu[i], fp[i]) || !vec_ok(y[i], u[i], p[i]))
      return bfail(b, CMG_ERR_INVALID_ARG, "null vector pointer for instance " + std::to_string(i));
  }
  if (!(tol > 0.0) || maxit < 0) return bfail(b, CMG_ERR_INVALID_ARG, "tol must be > 0 and maxit >= 0");
  if (opts->precision != CMG_FP32) {
    // FP64 cycles: instance by instance (the batched graph is the FP32 form)
    cmg_status worst = CMG_OK;
    for (int i = 0; i < count; ++i) {
      const cmg_status st = cmg_solve(b->inst[i], opts, CMG_METHOD_CYCLE, tol, maxit, 1, fy[i], fu[i], fp[i], y[i],
                                      u[i], p[i], &stats[i]);
      if (st != CMG_OK && worst == CMG_OK) worst = st;
    }
    return worst;
  }
  // 1. ||W f|| of every instance, one synchronisation
  for (int i = 0; i < count; ++i) {
    cmg_handle* h = b->inst[i];
    BCK(sumsq3(h, 0, fy[i], fu[i], fp[i], h->dsc, paper_wy(h) * paper_wy(h)));
    BCK(cudaMemcpyAsync(h->hsc, h->dsc, sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  }
  BCK(cudaStreamSynchronize(b->stream));
  std::vector<double> fnorm(count);
  for (int i = 0; i < count; ++i) {
    fnorm[i] = std::sqrt(b->inst[i]->hsc[0]);
    if (!std::isfinite(fnorm[i])) return bfail(b, CMG_ERR_NONFINITE, "right side " + std::to_string(i));
  }
  // 2. first refinement pass of every instance, one synchronisation
  for (int i = 0; i < count; ++i) {
    cmg_handle* h = b->inst[i];
    stats[i] = cmg_stats{};
    if (fnorm[i] == 0.0) {
      BCK(zero_vec<double>(h, 0, Vec3<double>{y[i], u[i], p[i]}));
      // x = 0 solves it: a state that stops before the first iteration
      ir_state_init(h, h->hsc, 0.0, 1.0, maxit, 0.0);
      h->hsc[kGo] = 0.0;
      BCK(cudaMemcpyAsync(h->ir_state, h->hsc, kIrStateSize * sizeof(double), cudaMemcpyHostToDevice, b->stream));
      BCK(cudaStreamSynchronize(b->stream));
      continue;
    }
    Vec3<float> f32 = Work<float>::f(h->lv[0]);
    const int cnt = launch_residual_cast(view<double>(h, 0), Vec3c<double>{y[i], u[i], p[i]},
                                         Vec3c<double>{fy[i], fu[i], fp[i]}, f32, 1.0 / fnorm[i], nullptr,
                                         paper_wy(h), h->part, h->part_cap, b->stream);
    if (cnt < 0) return bfail(b, CMG_ERR_CUDA, "refinement pass launch failed");
    BCK(launch_finish_sum(h->part, cnt, h->dsc, b->stream));
    BCK(cudaMemcpyAsync(h->hsc, h->dsc, sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  }
  BCK(cudaStreamSynchronize(b->stream));
  for (int i = 0; i < count; ++i) {
    cmg_handle* h = b->inst[i];
    if (fnorm[i] == 0.0) continue;
    double* hs = h->hsc;
    const double rho = fnorm[i] > 0.0 ? std::sqrt(hs[0]) * fnorm[i] : 0.0;
    stats[i].relres0 = fnorm[i] > 0.0 ? rho / fnorm[i] : 0.0;
    ir_state_init(h, hs, rho, fnorm[i] > 0.0 ? 1.0 / fnorm[i] : 1.0, maxit, tol * fnorm[i]);
    BCK(cudaMemcpyAsync(h->ir_state, hs, kIrStateSize * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    Lev& l0 = h->lv[0];
    const size_t ny = l0.nodes * h->prob.N;
    BCK(cudaMemsetAsync(l0.d32[0], 0, ny * sizeof(float), b->stream));
    BCK(cudaMemsetAsync(l0.d32[1], 0, l0.nodes * sizeof(float), b->stream));
    BCK(cudaMemsetAsync(l0.d32[2], 0, ny * sizeof(float), b->stream));
  }
  // 3a. the batched persistent form: one launch per grid depth and leg for all
  // instances, the loop as one graph (or eagerly, one synchronisation per
  // iteration, while a profiling window is open or graphs are off)
  std::string why;
  // CMG_BATCH_AUTO takes the branches: on the 96-instance workload (n up to
  // 255, N in [16, 128]) they solve in 429-447 ms against 548 ms persistent
  const bool persistent = b->force == CMG_BATCH_PERSISTENT;
  if (persistent) {
    if (!batch_persistent_ok(b, *opts, &why)) return bfail(b, CMG_ERR_UNSUPPORTED, "persistent form: " + why);
    std::vector<const void*> key;
    for (int i = 0; i < count; ++i) {
      const void* k[6] = {fy[i], fu[i], fp[i], y[i], u[i], p[i]};
      key.insert(key.end(), k, k + 6);
    }
    if (!b->T.count || key != b->pkey || !same_cycle(b->popts, *opts)) {
      b->pkey.clear();
      const cmg_status st = batch_build_tables(b, *opts, fy, fu, fp, y, u, p);
      if (st != CMG_OK) return st;
      b->pkey = key;
      b->popts = *opts;
    }
    BCK(cudaMemsetAsync(b->T.err, 0, sizeof(int), b->stream));
    BCK(cudaMemsetAsync(b->T.bar, 0, 2 * sizeof(unsigned), b->stream));
    b->mode = CMG_BATCH_PERSISTENT;
    long long iters = 0;
    if (batch_graphs_enabled(b) && !b->pexec && !b->graph_failed) {
      // a capture this driver refuses (the cooperative launches inside a
      // conditional body) leaves the loop eager, not the solve failed
      if (batch_build_graph(b) != CMG_OK) {
        if (b->pgraph) (void)cudaGraphDestroy(b->pgraph);
        b->pgraph = nullptr;
        (void)cudaGetLastError();
        b->graph_failed = true;
        b->graph_error = b->err;
      }
    }
    if (b->pexec) {
      BCK(cudaGraphLaunch(b->pexec, b->stream));
      count_launches(1);
    } else {
      cudaGraphConditionalHandle none{};
      BCK(launch_k(batch_next_kernel, dim3(1), dim3(256), 0, b->stream, b->T, b->act, b->any, none, 0));
      count_launches(1);
      for (;;) {
        BCK(cudaMemcpyAsync(b->hany, b->any, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
        BCK(cudaStreamSynchronize(b->stream));
        if (!*b->hany || iters > (long long)maxit + 1) break;
        const cmg_status st = batch_body(b, b->stream, none, 0);
        if (st != CMG_OK) return st;
        ++iters;
      }
    }
    int herr = 0;
    BCK(cudaMemcpyAsync(&herr, b->T.err, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    for (int i = 0; i < count; ++i) {
      cmg_handle* h = b->inst[i];
      BCK(cudaMemcpyAsync(h->hsc, h->ir_state, kIrStateSize * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    }
    BCK(cudaStreamSynchronize(b->stream));
    long long most = 0;
    cmg_status worst = CMG_OK;
    for (int i = 0; i < count; ++i) {
      const double* hs = b->inst[i]->hsc;
      most = std::max<long long>(most, (long long)hs[kIt]);
      stats[i].iters = (int)hs[kIt];
      stats[i].cycles = (int)hs[kIt];
      stats[i].relres = fnorm[i] > 0.0 ? hs[kRho] / fnorm[i] : 0.0;
      if (!std::isfinite(hs[kRho])) worst = CMG_ERR_NONFINITE;
      else if (fnorm[i] > 0.0 && stats[i].relres > tol && worst == CMG_OK) worst = CMG_ERR_NOT_CONVERGED;
    }
    if (b->pexec) count_launches((int)(1 + b->body_kernels * most));
    if (herr) return bfail(b, CMG_ERR_TIMEOUT, "a grid-wide barrier wait of the batched kernels ran out");
    if (worst != CMG_OK) b->err = "some instances did not reach the tolerance";
    return worst;
  }
  b->mode = CMG_BATCH_BRANCHES;
  // 3b. the graph: one independent branch (start kernel + while loop) per instance
  std::vector<const void*> key;
  for (int i = 0; i < count; ++i) {
    const void* k[6] = {fy[i], fu[i], fp[i], y[i], u[i], p[i]};
    key.insert(key.end(), k, k + 6);
  }
  if (!b->exec || key != b->key || !same_cycle(b->opts, *opts)) {
    if (b->exec) BCK(cudaGraphExecDestroy(b->exec));
    if (b->graph) BCK(cudaGraphDestroy(b->graph));
    b->exec = nullptr;
    b->graph = nullptr;
    cudaGraph_t g = nullptr;
    BCK(cudaGraphCreate(&g, 0));
    b->graph = g;
    for (int i = 0; i < count; ++i) {
      const cmg_status st = add_ir_loop(b->inst[i], *opts, Vec3c<double>{fy[i], fu[i], fp[i]},
                                        Vec3<double>{y[i], u[i], p[i]}, g);
      if (st != CMG_OK) return bfail(b, st, b->inst[i]->err);
    }
    cudaGraphExec_t ex = nullptr;
    BCK(cudaGraphInstantiate(&ex, g, 0));
    b->exec = ex;
    b->key = key;
    b->opts = *opts;
  }
  BCK(cudaGraphLaunch(b->exec, b->stream));
  for (int i = 0; i < count; ++i) {
    cmg_handle* h = b->inst[i];
    BCK(cudaMemcpyAsync(h->hsc, h->ir_state, kIrStateSize * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  }
  BCK(cudaStreamSynchronize(b->stream));
  cmg_status worst = CMG_OK;
  for (int i = 0; i < count; ++i) {
    const double* hs = b->inst[i]->hsc;
    count_replay(b->inst[i], (int)hs[kIt]);
    stats[i].iters = (int)hs[kIt];
    stats[i].cycles = (int)hs[kIt];
    stats[i].relres = fnorm[i] > 0.0 ? hs[kRho] / fnorm[i] : 0.0;
    if (!std::isfinite(hs[kRho])) worst = CMG_ERR_NONFINITE;
    else if (fnorm[i] > 0.0 && stats[i].relres > tol && worst == CMG_OK) worst = CMG_ERR_NOT_CONVERGED;
  }
  if (worst != CMG_OK) b->err = "some instances did not reach the tolerance";
  return worst;
}

extern "C" cmg_status cmg_batch_set_form(cmg_batch* b, int form) {
  if (!b) return CMG_ERR_INVALID_ARG;
  if (form != CMG_BATCH_AUTO && form != CMG_BATCH_PERSISTENT && form != CMG_BATCH_BRANCHES)
    return bfail(b, CMG_ERR_INVALID_ARG, "unknown batch form");
  b->force = form;
  return CMG_OK;
}

extern "C" int cmg_batch_form(const cmg_batch* b) { return b ? b->mode : -1; }

extern "C" cmg_status cmg_batch_set_legs(cmg_batch* b, int legs) {
  if (!b) return CMG_ERR_INVALID_ARG;
  if (legs != CMG_BATCH_LEGS_BY_WORK && legs != CMG_BATCH_LEGS_PERSISTENT && legs != CMG_BATCH_LEGS_PHASES)
    return bfail(b, CMG_ERR_INVALID_ARG, "unknown leg form");
  b->leg_force = legs;
  b->pkey.clear();   // rebuilt with the new leg forms on the next solve
  return CMG_OK;
}

extern "C" cmg_status cmg_batch_set_wait_limit(cmg_batch* b, long long polls) {
  if (!b) return CMG_ERR_INVALID_ARG;
  if (polls < 0) return bfail(b, CMG_ERR_INVALID_ARG, "polls must be >= 0");
  b->wait_limit = polls;
  b->pkey.clear();   // the tables carry the limit: rebuilt on the next solve
  return CMG_OK;
}

extern "C" cmg_status cmg_batch_autotune(cmg_batch* b, int precision) {
  if (!b) return CMG_ERR_INVALID_ARG;
  for (cmg_handle* h : b->inst) {
    const cmg_status st = cmg_autotune(h, precision, nullptr);
    if (st != CMG_OK) return bfail(b, st, h->err);
  }
  b->opts.n1 = -1;   // force a re-capture of the batch graph
  return CMG_OK;
}
