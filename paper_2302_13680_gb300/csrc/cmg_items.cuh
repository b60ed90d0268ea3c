// Per-node work items of the cycle, shared by the one-kernel-per-step path
// (cmg_stencil.cu) and the cluster-resident coarse-grid cycle (cmg_tail.cu).
//
// An item is one mesh node: its lpn lanes (consecutive lanes of one warp)
// cover the node's N samples in chunks of V contiguous elements.  Items may
// be called with an out-of-range node index (valid == false); every lane of
// the warp must reach the shuffle reductions, so no item returns early.
//
// CG selects loads that bypass L1 (ld.global.cg): required when the data was
// written earlier in the same kernel by another CTA (the cluster kernel).
#pragma once

#include "cmg_common.cuh"

namespace cmg {

template <typename T, int V, bool CG>
__device__ __forceinline__ vec<T, V> ldx(const T* p) {
  if constexpr (!CG) {
    return *reinterpret_cast<const vec<T, V>*>(p);
  } else {
    vec<T, V> r;
    if constexpr (sizeof(T) == 4 && V == 4) {
      const float4 t = __ldcg(reinterpret_cast<const float4*>(p));
      r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
    } else if constexpr (sizeof(T) == 8 && V == 2) {
      const double2 t = __ldcg(reinterpret_cast<const double2*>(p));
      r.v[0] = t.x; r.v[1] = t.y;
    } else {
#pragma unroll
      for (int k = 0; k < V; ++k) r.v[k] = __ldcg(p + k);
    }
    return r;
  }
}
template <typename T, int V, bool CG>
__device__ __forceinline__ vec<T, V> ldx_if(bool ok, const T* p) {
  return ok ? ldx<T, V, CG>(p) : vzero<T, V>();
}
template <typename T, bool CG>
__device__ __forceinline__ T ld1(const T* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}
__device__ __forceinline__ unsigned long long dbits(double v) {
  return static_cast<unsigned long long>(__double_as_longlong(v));
}

template <typename T, int V>
__device__ __forceinline__ void fma_faces(vec<T, V>& acc, const vec<T, V>& kW, const vec<T, V>& vW,
                                          const vec<T, V>& kE, const vec<T, V>& vE, const vec<T, V>& kS,
                                          const vec<T, V>& vS, const vec<T, V>& kN, const vec<T, V>& vN) {
#pragma unroll
  for (int k = 0; k < V; ++k) {
    T a = acc.v[k];
    a = fma(kW.v[k], vW.v[k], a);
    a = fma(kE.v[k], vE.v[k], a);
    a = fma(kS.v[k], vS.v[k], a);
    a = fma(kN.v[k], vN.v[k], a);
    acc.v[k] = a;
  }
}

// 1 / diag(A_j): stored (FP64 path) or from the four faces (FP32 path).
template <typename T, int V, bool CG>
__device__ __forceinline__ vec<T, V> inv_diag(const LevelView<T>& L, size_t off, const vec<T, V>& kW,
                                              const vec<T, V>& kE, const vec<T, V>& kS, const vec<T, V>& kN) {
  vec<T, V> ia;
  if constexpr (sizeof(T) == 8) {
    ia = ldx<T, V, CG>(reinterpret_cast<const T*>(L.inva) + off);
  } else {
#pragma unroll
    for (int k = 0; k < V; ++k) ia.v[k] = __frcp_rn((kW.v[k] + kE.v[k]) + (kS.v[k] + kN.v[k]));
  }
  return ia;
}

// ---------------------------------------------------------------------------
// r = f - S x (or r = S x when f.y == nullptr) at one node; y block times wy.
// DIFF: (A v)_i formed as sum_f k_f (v_i - v_f) (v_f = 0 outside the grid)
// instead of a_i v_i - sum_f k_f v_f: for a smooth v the differences are
// small and nearly exact, so the rounding error scales with the differences
// rather than with |v|.
// ---------------------------------------------------------------------------
template <typename T, int V, int SPL, bool CG, bool DIFF = false>
__device__ __forceinline__ void residual_item(const LevelView<T>& L, const Vec3c<T>& x, const Vec3c<T>& f,
                                              const Vec3<T>& r, long node, int lane, int lpn, T wy) {
  const int n = L.n, N = L.N;
  const size_t ld = (size_t)L.ld;
  const bool valid = node < (long)n * n;
  const T c = (T)L.c, e = (T)L.e;
  const bool apply = f.y == nullptr;
  using A = acc_t<T>;
  T pacc = T(0);   // this lane's part of sum_j p_j
  // local control: the control enters as chi_i u_i and its row exists only
  // where chi_i = 1
  const int iy = valid ? (int)(node / n) : 0, ix = valid ? (int)(node - (long)iy * n) : 0;
  const bool ctl = L.ctl.inside(iy, ix);
  if (valid) {
    const size_t o = (size_t)node * ld;
    const T* kWp = L.kx + ((size_t)iy * (n + 1) + ix) * ld;
    const T* kSp = L.ky + ((size_t)iy * n + ix) * ld;
    const bool hW = ix > 0, hE = ix < n - 1, hS = iy > 0, hN = iy < n - 1;
    const T uu = ctl ? ld1<T, CG>(x.u + node) : T(0);
#pragma unroll
    for (int s = 0; s < SPL; ++s) {
      const int j = (lane + s * lpn) * V;
      if (j < N) {
        const vec<T, V> kW = ldx<T, V, CG>(kWp + j), kE = ldx<T, V, CG>(kWp + ld + j);
        const vec<T, V> kS = ldx<T, V, CG>(kSp + j), kN = ldx<T, V, CG>(kSp + (size_t)n * ld + j);
        const vec<T, V> y = ldx<T, V, CG>(x.y + o + j), p = ldx<T, V, CG>(x.p + o + j);
        const vec<T, V> yW = ldx_if<T, V, CG>(hW, x.y + o - ld + j), yE = ldx_if<T, V, CG>(hE, x.y + o + ld + j);
        const vec<T, V> yS = ldx_if<T, V, CG>(hS, x.y + o - (size_t)n * ld + j);
        const vec<T, V> yN = ldx_if<T, V, CG>(hN, x.y + o + (size_t)n * ld + j);
        const vec<T, V> pW = ldx_if<T, V, CG>(hW, x.p + o - ld + j), pE = ldx_if<T, V, CG>(hE, x.p + o + ld + j);
        const vec<T, V> pS = ldx_if<T, V, CG>(hS, x.p + o - (size_t)n * ld + j);
        const vec<T, V> pN = ldx_if<T, V, CG>(hN, x.p + o + (size_t)n * ld + j);
        vec<T, V> ry, rp;
        if constexpr (DIFF) {
#pragma unroll
          for (int k = 0; k < V; ++k) {
            T ay = kW.v[k] * (y.v[k] - yW.v[k]);
            ay = fma(kE.v[k], y.v[k] - yE.v[k], ay);
            ay = fma(kS.v[k], y.v[k] - yS.v[k], ay);
            ay = fma(kN.v[k], y.v[k] - yN.v[k], ay);
            T ap = kW.v[k] * (p.v[k] - pW.v[k]);
            ap = fma(kE.v[k], p.v[k] - pE.v[k], ap);
            ap = fma(kS.v[k], p.v[k] - pS.v[k], ap);
            ap = fma(kN.v[k], p.v[k] - pN.v[k], ap);
            ry.v[k] = c * y.v[k] + ap;
            rp.v[k] = ay + e * uu;
            pacc += p.v[k];
          }
        } else {
          vec<T, V> offy = vzero<T, V>(), offp = vzero<T, V>();
          fma_faces<T, V>(offy, kW, yW, kE, yE, kS, yS, kN, yN);
          fma_faces<T, V>(offp, kW, pW, kE, pE, kS, pS, kN, pN);
#pragma unroll
          for (int k = 0; k < V; ++k) {
            const T a = (kW.v[k] + kE.v[k]) + (kS.v[k] + kN.v[k]);
            // state rows: c y + A p ; adjoint rows: A y + e u
            ry.v[k] = c * y.v[k] + (a * p.v[k] - offp.v[k]);
            rp.v[k] = (a * y.v[k] - offy.v[k]) + e * uu;
            pacc += p.v[k];
          }
        }
        if (!apply) {
          const vec<T, V> fy = ldx<T, V, CG>(f.y + o + j), fp = ldx<T, V, CG>(f.p + o + j);
#pragma unroll
          for (int k = 0; k < V; ++k) {
            ry.v[k] = fy.v[k] - ry.v[k];
            rp.v[k] = fp.v[k] - rp.v[k];
          }
        }
        if (wy != T(1)) {
#pragma unroll
          for (int k = 0; k < V; ++k) ry.v[k] *= wy;
        }
        stv<T, V>(r.y + o + j, ry);
        stv<T, V>(r.p + o + j, rp);
      }
    }
  }
  const A psum = group_sum((A)pacc, lpn);
  if (valid && lane == 0) {
    if (ctl) {
      const A su = (A)L.G * (A)ld1<T, CG>(x.u + node) + (A)d_of(L, node) * psum;   // control row: G u + d_i sum_j p_j
      r.u[node] = (T)(apply ? su : (A)ld1<T, CG>(f.u + node) - su);
    } else {
      r.u[node] = T(0);
    }
  }
}

// x + (P e) at fine node (fy, fx), samples j .. j+V-1: the value the
// prolongation kernel would leave there (same operations in the same
// order), formed where a half-sweep reads it as a neighbour.
template <typename T, int V, bool CG>
__device__ __forceinline__ vec<T, V> prolonged(const T* xv, const T* ev, int nf, int nc, size_t ld, int fy, int fx,
                                               int j) {
  vec<T, V> v = ldx<T, V, CG>(xv + ((size_t)fy * nf + fx) * ld + j);
  int Jr[2] = {0, 0}, Ir[2] = {0, 0};
  T wy[2] = {T(0), T(0)}, wx[2] = {T(0), T(0)};
  int ny, nx;
  if (fy & 1) { Jr[0] = (fy - 1) >> 1; wy[0] = T(1); ny = 1; }
  else { Jr[0] = (fy >> 1) - 1; Jr[1] = fy >> 1; wy[0] = wy[1] = T(0.5); ny = 2; }
  if (fx & 1) { Ir[0] = (fx - 1) >> 1; wx[0] = T(1); nx = 1; }
  else { Ir[0] = (fx >> 1) - 1; Ir[1] = fx >> 1; wx[0] = wx[1] = T(0.5); nx = 2; }
  for (int a = 0; a < ny; ++a) {
    if (Jr[a] < 0 || Jr[a] >= nc) continue;
    for (int b = 0; b < nx; ++b) {
      if (Ir[b] < 0 || Ir[b] >= nc) continue;
      const T wt = wy[a] * wx[b];
      const vec<T, V> ec = ldx<T, V, CG>(ev + ((size_t)Jr[a] * nc + Ir[b]) * ld + j);
#pragma unroll
      for (int k = 0; k < V; ++k) v.v[k] = fma(wt, ec.v[k], v.v[k]);
    }
  }
  return v;
}

// ---------------------------------------------------------------------------
// Red-black collective GS at the g-th node of `colour`: local right sides
// from the current neighbours, then Eq. (13).  With b_p the rhs of the
// first block row, b_y of the last, b_u of the control row:
//   u = (b_u + d sum_j (c b_y,j / a_j^2 - b_p,j / a_j)) / sigma
//   y_j = (b_y,j - e u) / a_j,   p_j = (b_p,j - c y_j) / a_j
// with 1/sigma stored per node, so u costs one multiply; the sum over
// samples, 1/sigma and u are FP64 (schur_u) and their loads are issued
// together with the node's other loads, ahead of the group sum.
// ---------------------------------------------------------------------------
// PRO: the neighbours are read as x + P e (coarse correction e on the grid
// of nc nodes per side), i.e. the prolongation is fused into this half-sweep.
// ZG: x is zero on entry (the first half-sweep of a cycle from a zero
// guess): the neighbour terms vanish and are neither loaded nor added, so
// x need not be cleared beforehand (a colour-0 sweep writes every colour-0
// value and the colour-1 sweep after it every colour-1 value, reading only
// colour-0 neighbours).  Same values as the plain sweep on a cleared x:
// adding k * 0 leaves a sum unchanged, up to the sign of a zero.
// rbgs_node: the node (iy, ix) (valid = false: no loads or stores, only the
// group's shuffles) reading its neighbours (and a frozen u) from xs and
// writing its new values to x; the half-sweeps pass xs = x, the one-launch
// full sweep (cmg_fused.cu) reads the old iterate from one buffer and writes
// another.
template <typename T, int V, int SPL, bool CG, bool PRO = false, bool ZG = false>
__device__ __forceinline__ void rbgs_node(const LevelView<T>& L, const Vec3c<T>& xs, const Vec3<T>& x,
                                          const Vec3c<T>& f, bool valid, int iy, int ix, int lane, int lpn,
                                          const Vec3c<T> e, int nc) {
  const int n = L.n, N = L.N;
  const size_t ld = (size_t)L.ld;
  const T c = (T)L.c;
  const long node = (long)iy * n + ix;
  const bool ctl = L.ctl.inside(iy, ix);   // taken here so (iy, ix) need not stay live
  const size_t o = (size_t)node * ld;
  vec<T, V> bp[SPL], by[SPL], ia[SPL];
  T tacc = T(0);   // this lane's part of the sum over samples
  double bu = 0.0, isg = 0.0;   // control-row right side (or the frozen u) and 1/sigma, loaded with the rest
  double dwv = 1.0;             // per-node factor on d (semismooth Newton systems only), loaded with them
  if (valid) {
    bu = L.freeze_u ? (double)ld1<T, CG>(xs.u + node) : (double)ld1<T, CG>(f.u + node);
    isg = isigma_of<T>(L, node);
    if (L.dw) dwv = (double)L.dw[node];
    const T* kWp = L.kx + ((size_t)iy * (n + 1) + ix) * ld;
    const T* kSp = L.ky + ((size_t)iy * n + ix) * ld;
    const bool hW = ix > 0, hE = ix < n - 1, hS = iy > 0, hN = iy < n - 1;
#pragma unroll
    for (int s = 0; s < SPL; ++s) {
      const int j = (lane + s * lpn) * V;
      if (j < N) {
        const vec<T, V> kW = ldx<T, V, CG>(kWp + j), kE = ldx<T, V, CG>(kWp + ld + j);
        const vec<T, V> kS = ldx<T, V, CG>(kSp + j), kN = ldx<T, V, CG>(kSp + (size_t)n * ld + j);
        bp[s] = ldx<T, V, CG>(f.y + o + j);   // first block row: c y + A p = f_y
        by[s] = ldx<T, V, CG>(f.p + o + j);   // last block row:  A y + e u = f_p
        if constexpr (PRO) {
          const auto nb = [&](bool h, const T* xv, const T* ev, int fy, int fx) {
            return h ? prolonged<T, V, CG>(xv, ev, n, nc, ld, fy, fx, j) : vzero<T, V>();
          };
          fma_faces<T, V>(bp[s], kW, nb(hW, xs.p, e.p, iy, ix - 1), kE, nb(hE, xs.p, e.p, iy, ix + 1), kS,
                          nb(hS, xs.p, e.p, iy - 1, ix), kN, nb(hN, xs.p, e.p, iy + 1, ix));
          fma_faces<T, V>(by[s], kW, nb(hW, xs.y, e.y, iy, ix - 1), kE, nb(hE, xs.y, e.y, iy, ix + 1), kS,
                          nb(hS, xs.y, e.y, iy - 1, ix), kN, nb(hN, xs.y, e.y, iy + 1, ix));
        } else if constexpr (!ZG) {
          fma_faces<T, V>(bp[s], kW, ldx_if<T, V, CG>(hW, xs.p + o - ld + j), kE,
                          ldx_if<T, V, CG>(hE, xs.p + o + ld + j), kS,
                          ldx_if<T, V, CG>(hS, xs.p + o - (size_t)n * ld + j), kN,
                          ldx_if<T, V, CG>(hN, xs.p + o + (size_t)n * ld + j));
          fma_faces<T, V>(by[s], kW, ldx_if<T, V, CG>(hW, xs.y + o - ld + j), kE,
                          ldx_if<T, V, CG>(hE, xs.y + o + ld + j), kS,
                          ldx_if<T, V, CG>(hS, xs.y + o - (size_t)n * ld + j), kN,
                          ldx_if<T, V, CG>(hN, xs.y + o + (size_t)n * ld + j));
        }
        ia[s] = inv_diag<T, V, CG>(L, o + j, kW, kE, kS, kN);
#pragma unroll
        for (int k = 0; k < V; ++k) {
          const T iak = ia[s].v[k];
          tacc += (c * iak) * (iak * by[s].v[k]) - iak * bp[s].v[k];
        }
      }
    }
  }
  const double su = schur_u<T>(L, tacc, lpn, bu, L.d * dwv, isg);
  if (valid) {
    // frozen control: u_i keeps its value and only the state and adjoint
    // rows are solved (Eq. (14) with u_i given instead of zero); a node
    // without a control basis function (local control) takes Eq. (14) with
    // u_i = 0
    const double uu = L.freeze_u ? bu : (ctl ? su : 0.0);
    if (lane == 0 && !L.freeze_u) x.u[node] = (T)uu;
    const T uT = (T)uu, e = (T)L.e;
#pragma unroll
    for (int s = 0; s < SPL; ++s) {
      const int j = (lane + s * lpn) * V;
      if (j < N) {
        vec<T, V> yn, pn;
#pragma unroll
        for (int k = 0; k < V; ++k) {
          yn.v[k] = ia[s].v[k] * (by[s].v[k] - e * uT);
          pn.v[k] = ia[s].v[k] * (bp[s].v[k] - c * yn.v[k]);
        }
        stv<T, V>(x.y + o + j, yn);
        stv<T, V>(x.p + o + j, pn);
      }
    }
  }
}

template <typename T, int V, int SPL, bool CG, bool PRO = false, bool ZG = false>
__device__ __forceinline__ void rbgs_item(const LevelView<T>& L, const Vec3<T>& x, const Vec3c<T>& f, int colour,
                                          long g, int lane, int lpn, const Vec3c<T> e = Vec3c<T>{nullptr, nullptr,
                                                                                                   nullptr},
                                          int nc = 0) {
  const bool valid = g < colour_count(L.n, colour);
  int iy = 0, ix = 0;
  if (valid) colour_node(g, L.n, colour, iy, ix);
  rbgs_node<T, V, SPL, CG, PRO, ZG>(L, cview(x), x, f, valid, iy, ix, lane, lpn, e, nc);
}

// Damped collective Jacobi, Eq. (11): x_i += theta S~_i^{-1} r_i.
template <typename T, int V, int SPL, bool CG>
__device__ __forceinline__ void jacobi_item(const LevelView<T>& L, const Vec3<T>& x, const Vec3c<T>& r,
                                            double theta, long node, int lane, int lpn) {
  const int n = L.n, N = L.N;
  const size_t ld = (size_t)L.ld;
  const bool valid = node < (long)n * n;
  const T c = (T)L.c;
  const size_t o = (size_t)(valid ? node : 0) * ld;
  vec<T, V> bp[SPL], by[SPL], ia[SPL];
  T tacc = T(0);
  double ru = 0.0, isg = 0.0;   // loaded with the rest, ahead of the group sum
  T xu = T(0);
  const int iy = valid ? (int)(node / n) : 0, ix = valid ? (int)(node - (long)iy * n) : 0;
  double dwv = 1.0;   // per-node factor on d (semismooth Newton systems only)
  if (valid) {
    ru = (double)ld1<T, CG>(r.u + node);
    xu = ld1<T, CG>(x.u + node);
    isg = isigma_of<T>(L, node);
    if (L.dw) dwv = (double)L.dw[node];
    const T* kWp = L.kx + ((size_t)iy * (n + 1) + ix) * ld;
    const T* kSp = L.ky + ((size_t)iy * n + ix) * ld;
#pragma unroll
    for (int s = 0; s < SPL; ++s) {
      const int j = (lane + s * lpn) * V;
      if (j < N) {
        bp[s] = ldx<T, V, CG>(r.y + o + j);
        by[s] = ldx<T, V, CG>(r.p + o + j);
        ia[s] = inv_diag<T, V, CG>(L, o + j, ldx<T, V, CG>(kWp + j), ldx<T, V, CG>(kWp + ld + j),
                                   ldx<T, V, CG>(kSp + j), ldx<T, V, CG>(kSp + (size_t)n * ld + j));
#pragma unroll
        for (int k = 0; k < V; ++k) {
          const T iak = ia[s].v[k];
          tacc += (c * iak) * (iak * by[s].v[k]) - iak * bp[s].v[k];
        }
      }
    }
  }
  const double sdu = schur_u<T>(L, tacc, lpn, ru, L.d * dwv, isg);
  if (valid) {
    const double du = (L.freeze_u || !L.ctl.inside(iy, ix)) ? 0.0 : sdu;
    if (lane == 0) {
      if (sizeof(T) == 4 && L.ctl32) x.u[node] = (T)((float)xu + (float)theta * (float)du);
      else x.u[node] = (T)((double)xu + theta * du);
    }
    const T duT = (T)du, e = (T)L.e, th = (T)theta;
#pragma unroll
    for (int s = 0; s < SPL; ++s) {
      const int j = (lane + s * lpn) * V;
      if (j < N) {
        vec<T, V> yv = ldx<T, V, CG>(x.y + o + j), pv = ldx<T, V, CG>(x.p + o + j);
#pragma unroll
        for (int k = 0; k < V; ++k) {
          const T dy = ia[s].v[k] * (by[s].v[k] - e * duT);
          const T dp = ia[s].v[k] * (bp[s].v[k] - c * dy);
          yv.v[k] += th * dy;
          pv.v[k] += th * dp;
        }
        stv<T, V>(x.y + o + j, yv);
        stv<T, V>(x.p + o + j, pv);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Transfers.  Coarse node (J, I) sits on fine node (2J+1, 2I+1).
// ---------------------------------------------------------------------------

// c = P^T r at one coarse node (weights 1, 1/2, 1/4); if zx.y is set, the
// coarse iterate at that node is also cleared (zero initial guess).  With
// colour0, r is known to vanish at the colour-1 fine points (the four edge
// neighbours of the coinciding point), which are then not read.
template <typename T, int V, int SPL, bool CG>
__device__ __forceinline__ void restrict_item(int nf, int N, const Vec3c<T>& r, const Vec3<T>& cv,
                                              const Vec3<T>& zx, long node, int lane, int lpn, bool colour0 = false) {
  const int nc = (nf - 1) / 2;
  if (node >= (long)nc * nc) return;   // no shuffles below
  const int J = (int)(node / nc), I = (int)(node - (long)J * nc);
  const size_t ld = (size_t)N;
  const long fc = (long)(2 * J + 1) * nf + (2 * I + 1);
  const T w[3] = {T(0.5), T(1), T(0.5)};
#pragma unroll
  for (int s = 0; s < SPL; ++s) {
    const int j = (lane + s * lpn) * V;
    if (j < N) {
      vec<T, V> ay = vzero<T, V>(), ap = vzero<T, V>();
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          if (colour0 && ((dx + dy) & 1)) continue;   // edge points are colour 1: residual zero
          const T wt = w[dy + 1] * w[dx + 1];
          const size_t o = (size_t)(fc + (long)dy * nf + dx) * ld + j;
          const vec<T, V> vy = ldx<T, V, CG>(r.y + o), vp = ldx<T, V, CG>(r.p + o);
#pragma unroll
          for (int k = 0; k < V; ++k) {
            ay.v[k] = fma(wt, vy.v[k], ay.v[k]);
            ap.v[k] = fma(wt, vp.v[k], ap.v[k]);
          }
        }
      stv<T, V>(cv.y + (size_t)node * ld + j, ay);
      stv<T, V>(cv.p + (size_t)node * ld + j, ap);
      if (zx.y) {
        stv<T, V>(zx.y + (size_t)node * ld + j, vzero<T, V>());
        stv<T, V>(zx.p + (size_t)node * ld + j, vzero<T, V>());
      }
    }
  }
  if (lane == 0) {
    T au = T(0);
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (colour0 && ((dx + dy) & 1)) continue;
        au = fma(w[dy + 1] * w[dx + 1], ld1<T, CG>(r.u + fc + (long)dy * nf + dx), au);
      }
    cv.u[node] = au;
    if (zx.y) zx.u[node] = T(0);
  }
}

// x += P e at one fine node: 1 x coinciding coarse node, 1/2 x each of two
// edge neighbours, 1/4 x each of four cell corners (zero outside the grid).
// With local control the control block is corrected only at fine nodes that
// carry a control basis function (ctl).
template <typename T, int V, int SPL, bool CG>
__device__ __forceinline__ void prolong_item(int nf, int N, const Vec3c<T>& e, const Vec3<T>& x, long node,
                                             int lane, int lpn, const CtlBox& ctl = CtlBox{}) {
  const int nc = (nf - 1) / 2;
  if (node >= (long)nf * nf) return;   // no shuffles below
  const int iy = (int)(node / nf), ix = (int)(node - (long)iy * nf);
  int Jr[2] = {0, 0}, Ir[2] = {0, 0};
  T wy[2] = {T(0), T(0)}, wx[2] = {T(0), T(0)};
  int ny, nx;
  if (iy & 1) { Jr[0] = (iy - 1) >> 1; wy[0] = T(1); ny = 1; }
  else { Jr[0] = (iy >> 1) - 1; Jr[1] = iy >> 1; wy[0] = wy[1] = T(0.5); ny = 2; }
  if (ix & 1) { Ir[0] = (ix - 1) >> 1; wx[0] = T(1); nx = 1; }
  else { Ir[0] = (ix >> 1) - 1; Ir[1] = ix >> 1; wx[0] = wx[1] = T(0.5); nx = 2; }
  const size_t ld = (size_t)N;
#pragma unroll
  for (int s = 0; s < SPL; ++s) {
    const int j = (lane + s * lpn) * V;
    if (j < N) {
      vec<T, V> vy = ldx<T, V, CG>(x.y + (size_t)node * ld + j), vp = ldx<T, V, CG>(x.p + (size_t)node * ld + j);
      for (int a = 0; a < ny; ++a) {
        if (Jr[a] < 0 || Jr[a] >= nc) continue;
        for (int b = 0; b < nx; ++b) {
          if (Ir[b] < 0 || Ir[b] >= nc) continue;
          const T wt = wy[a] * wx[b];
          const size_t o = ((size_t)Jr[a] * nc + Ir[b]) * ld + j;
          const vec<T, V> ey = ldx<T, V, CG>(e.y + o), ep = ldx<T, V, CG>(e.p + o);
#pragma unroll
          for (int k = 0; k < V; ++k) {
            vy.v[k] = fma(wt, ey.v[k], vy.v[k]);
            vp.v[k] = fma(wt, ep.v[k], vp.v[k]);
          }
        }
      }
      stv<T, V>(x.y + (size_t)node * ld + j, vy);
      stv<T, V>(x.p + (size_t)node * ld + j, vp);
    }
  }
  if (lane == 0 && ctl.inside(iy, ix)) {
    T vu = ld1<T, CG>(x.u + node);
    for (int a = 0; a < ny; ++a) {
      if (Jr[a] < 0 || Jr[a] >= nc) continue;
      for (int b = 0; b < nx; ++b) {
        if (Ir[b] < 0 || Ir[b] >= nc) continue;
        vu = fma(wy[a] * wx[b], ld1<T, CG>(e.u + (size_t)Jr[a] * nc + Ir[b]), vu);
      }
    }
    x.u[node] = vu;
  }
}

// Dispatch on (V, SPL) chosen from N and the element size (see choose_map).
#define CMG_SPL_SWITCH(SPLV, V_, ...)                                           \
  switch (SPLV) {                                                              \
    case 1: { constexpr int V = V_, SPL = 1; __VA_ARGS__; } break;             \
    case 2: { constexpr int V = V_, SPL = 2; __VA_ARGS__; } break;             \
    case 4: { constexpr int V = V_, SPL = 4; __VA_ARGS__; } break;             \
    case 8: { constexpr int V = V_, SPL = 8; __VA_ARGS__; } break;             \
    default: return cudaErrorInvalidValue;                                     \
  }

// FP32 with V = 2 is the wide layout (kTuneWide): one chunk per lane only.
#define CMG_DISPATCH(T, MAP, ...)                                              \
  do {                                                                         \
    if ((MAP).V == 1) { CMG_SPL_SWITCH((MAP).spl, 1, __VA_ARGS__) }            \
    else if constexpr (sizeof(T) == 8) { CMG_SPL_SWITCH((MAP).spl, 2, __VA_ARGS__) } \
    else if ((MAP).V == 2) {                                                   \
      if ((MAP).spl != 1) return cudaErrorInvalidValue;                        \
      constexpr int V = 2, SPL = 1;                                            \
      __VA_ARGS__;                                                             \
    }                                                                          \
    else { CMG_SPL_SWITCH((MAP).spl, 4, __VA_ARGS__) }                         \
  } while (0)

}  // namespace cmg

namespace cmg {

// Outer-residual item of FP64 iterative refinement: r = f - S x in FP64 at
// one node, written as FP32 scaled by s (the right side of the next FP32
// cycle); returns this lane's part of ||W r s||^2 (state block weighted by
// wy) accumulated in FP32 -- the stopping test needs the norm to ~1e-7
// relative accuracy, not the residual itself.
template <int V, int SPL>
__device__ __forceinline__ float residual_cast_item(const LevelView<double>& L, const Vec3c<double>& x,
                                                    const Vec3c<double>& f, const Vec3<float>& r, long node,
                                                    int lane, int lpn, double s, float wy2) {
  using T = double;
  const int n = L.n, N = L.N;
  const size_t ld = (size_t)L.ld;
  const bool valid = node < (long)n * n;
  const T c = L.c, e = L.e;
  T pacc = 0.0;
  float sq = 0.f;
  const float sf = (float)s;
  const int iy = valid ? (int)(node / n) : 0, ix = valid ? (int)(node - (long)iy * n) : 0;
  const bool ctl = L.ctl.inside(iy, ix);   // local control: chi_i
  if (valid) {
    const size_t o = (size_t)node * ld;
    const T* kWp = L.kx + ((size_t)iy * (n + 1) + ix) * ld;
    const T* kSp = L.ky + ((size_t)iy * n + ix) * ld;
    const bool hW = ix > 0, hE = ix < n - 1, hS = iy > 0, hN = iy < n - 1;
    const T xu = ctl ? x.u[node] : 0.0;
    const unsigned long long xu_bits = dbits(xu);
    const T eu = e * xu;
#pragma unroll
    for (int q = 0; q < SPL; ++q) {
      const int j = (lane + q * lpn) * V;
      if (j < N) {
        const vec<T, V> kW = ldv<T, V>(kWp + j), kE = ldv<T, V>(kWp + ld + j);
        const vec<T, V> kS = ldv<T, V>(kSp + j), kN = ldv<T, V>(kSp + (size_t)n * ld + j);
        const vec<T, V> y = ldv<T, V>(x.y + o + j), p = ldv<T, V>(x.p + o + j);
        const vec<T, V> fy = ldv<T, V>(f.y + o + j), fp = ldv<T, V>(f.p + o + j);
        // diag(A_j) read (finest grid) instead of three FP64 adds: this pass is
        // bound by the FP64 pipe, not by memory
        vec<T, V> av;
        if (L.a64) {
          av = ldv<T, V>(L.a64 + o + j);
        } else {
#pragma unroll
          for (int k = 0; k < V; ++k) av.v[k] = (kW.v[k] + kE.v[k]) + (kS.v[k] + kN.v[k]);
        }
        const vec<T, V> yW = ldv_if<T, V>(hW, x.y + o - ld + j), yE = ldv_if<T, V>(hE, x.y + o + ld + j);
        const vec<T, V> yS = ldv_if<T, V>(hS, x.y + o - (size_t)n * ld + j);
        const vec<T, V> yN = ldv_if<T, V>(hN, x.y + o + (size_t)n * ld + j);
        const vec<T, V> pW = ldv_if<T, V>(hW, x.p + o - ld + j), pE = ldv_if<T, V>(hE, x.p + o + ld + j);
        const vec<T, V> pS = ldv_if<T, V>(hS, x.p + o - (size_t)n * ld + j);
        const vec<T, V> pN = ldv_if<T, V>(hN, x.p + o + (size_t)n * ld + j);
        // Where every iterate value this chunk reads is zero (a zero initial
        // guess), f - S x = f exactly: the FP64 arithmetic is skipped, with
        // the zero test made on the bit patterns (integer pipe; -0 counts
        // as zero) so it costs no FP64 operations.
        unsigned long long nzb = xu_bits;
#pragma unroll
        for (int k = 0; k < V; ++k)
          nzb |= dbits(y.v[k]) | dbits(p.v[k]) | dbits(yW.v[k]) | dbits(yE.v[k]) | dbits(yS.v[k]) |
                 dbits(yN.v[k]) | dbits(pW.v[k]) | dbits(pE.v[k]) | dbits(pS.v[k]) | dbits(pN.v[k]);
        vec<float, V> ry, rp;
        if ((nzb << 1) == 0ull) {
#pragma unroll
          for (int k = 0; k < V; ++k) {
            ry.v[k] = (float)fy.v[k] * sf;
            rp.v[k] = (float)fp.v[k] * sf;
            sq = fmaf(wy2 * ry.v[k], ry.v[k], sq);
            sq = fmaf(rp.v[k], rp.v[k], sq);
          }
        } else {
          vec<T, V> offy = vzero<T, V>(), offp = vzero<T, V>();
          fma_faces<T, V>(offy, kW, yW, kE, yE, kS, yS, kN, yN);
          fma_faces<T, V>(offp, kW, pW, kE, pE, kS, pS, kN, pN);
#pragma unroll
          for (int k = 0; k < V; ++k) {
            const T a = av.v[k];
            const T ryk = fy.v[k] - fma(c, y.v[k], fma(a, p.v[k], -offp.v[k]));   // f_y - c y - A p
            const T rpk = (fp.v[k] - eu) - fma(a, y.v[k], -offy.v[k]);             // f_p - e u - A y
            ry.v[k] = (float)ryk * sf;   // scaled after rounding: FP32 multiplies instead of FP64
            rp.v[k] = (float)rpk * sf;
            sq = fmaf(wy2 * ry.v[k], ry.v[k], sq);
            sq = fmaf(rp.v[k], rp.v[k], sq);
            pacc += p.v[k];
          }
        }
        stv<float, V>(r.y + o + j, ry);
        stv<float, V>(r.p + o + j, rp);
      }
    }
  }
  const double psum = group_sum(pacc, lpn);
  if (valid && lane == 0) {
    const float ru = ctl ? (float)((f.u[node] - (L.G * x.u[node] + d_of(L, node) * psum)) * s) : 0.f;
    r.u[node] = ru;
    sq = fmaf(ru, ru, sq);
  }
  return sq;
}

// One node of the FP32 refinement between anchors (residual replacement):
// the scaled residual r (the cycle's right side) is updated in place,
// r <- r - S e (A e from neighbour differences, see residual_item), the
// running correction d += e, and this lane's part of ||W r||^2 is returned
// (squares in FP32; wy2 weights the state block).  Each lane reads its own r
// entries before writing them, so the update in place is safe.
template <int V, int SPL>
__device__ __forceinline__ float recur_item(const LevelView<float>& L, const Vec3c<float>& e, const Vec3<float>& r,
                                            const Vec3<float>& d, long node, int lane, int lpn, float wy2) {
  residual_item<float, V, SPL, false, true>(L, e, cview(r), r, node, lane, lpn, 1.0f);
  const int N = L.N;
  const size_t ld = (size_t)L.ld;
  float sq = 0.f;
  if (node < (long)L.n * L.n) {
    const size_t o = (size_t)node * ld;
#pragma unroll
    for (int s = 0; s < SPL; ++s) {
      const int j = (lane + s * lpn) * V;
      if (j < N) {
        const vec<float, V> ry = ldv<float, V>(r.y + o + j), rp = ldv<float, V>(r.p + o + j);
        const vec<float, V> ey = ldv<float, V>(e.y + o + j), ep = ldv<float, V>(e.p + o + j);
        vec<float, V> dy = ldv<float, V>(d.y + o + j), dp = ldv<float, V>(d.p + o + j);
#pragma unroll
        for (int k = 0; k < V; ++k) {
          sq = fmaf(wy2 * ry.v[k], ry.v[k], sq);
          sq = fmaf(rp.v[k], rp.v[k], sq);
          dy.v[k] += ey.v[k];
          dp.v[k] += ep.v[k];
        }
        stv<float, V>(d.y + o + j, dy);
        stv<float, V>(d.p + o + j, dp);
      }
    }
    if (lane == 0) {
      const float ru = r.u[node];
      sq = fmaf(ru, ru, sq);
      d.u[node] += e.u[node];
    }
  }
  return sq;
}

}  // namespace cmg
