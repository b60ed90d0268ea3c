// One red-black collective Gauss-Seidel sweep in one launch (FP32): the
// colour-0 half-sweep and the colour-1 half-sweep after it (the GS variant
// named after Eq. (11), Eq. (13) at every node), on tiles of the grid.
//
// Two launches per sweep read every face, f and the other colour's y, p
// once per half-sweep (40 bytes per node-sample and sweep in FP32).  Here a
// CTA takes a tile of W columns x BH rows and walks it row by row: in
// phase p it updates the colour-0 nodes of row p and the colour-1 nodes of
// row p - 2, whose colour-0 neighbours (rows p - 3 .. p - 1) are then final.
// The faces, f and old values a row needs are read by phases two rows
// apart and stay in L1/L2 between them, so the sweep moves each once
// (32 bytes per node-sample: faces 8, f 8, old y, p 8, new y, p 8).
//
// The old iterate is read from one buffer (xa) and the new one written to
// another (xb), so tiles never wait for each other: colour 0 reads only xa
// (the colour-1 values before the sweep), colour 1 reads only the colour-0
// values of xb, and a tile computes the colour-0 nodes one column and one
// row beyond its edges itself (the halo) instead of waiting for its
// neighbours.  A halo node is computed by the same code from the same
// inputs as by the tile that owns it, so both store the same bits; nothing
// else writes colour-0 values and nothing reads colour-1 values of xb
// during the sweep.  The result equals the two half-sweeps bit for bit
// (the same per-node arithmetic and sample map).
//
// Modes: plain (xa is the iterate), zero (the iterate is zero: colour 0 reads
// no neighbours, as rbgs_zero_kernel), prolong (colour 0 reads its
// neighbours as xa + P e, as rbgs_prolong_kernel).
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "cmg_items.cuh"

namespace cmg {

namespace {

constexpr int kFusedMaxWarps = 12;   // 384 threads: up to 168 registers at one CTA per SM
constexpr int kFusedW = 32;          // widest tile in nodes

template <int V, int SPL, int MODE>
__global__ void __launch_bounds__(kFusedMaxWarps * 32, 1)
    rbgs_fused_kernel(LevelView<float> L, Vec3c<float> xa, Vec3<float> xb, Vec3c<float> f, Vec3c<float> e, int nc,
                      int lpn, int W, int BH, int strips, int tiles) {
  pdl_enter();
  const int n = L.n;
  const int npw = 32 / lpn;   // nodes per warp
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int lane = threadIdx.x & (lpn - 1);
  const int slot = (threadIdx.x & 31) / lpn;
  const Vec3c<float> xbc = cview(xb);
  for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int c0 = (t % strips) * W, c1 = min(n, c0 + W);
    const int r0 = (t / strips) * BH, r1 = min(n, r0 + BH);
    const int ca = max(c0 - 1, 0), cb = min(c1, n - 1);   // colour-0 columns, halo included
    for (int p = r0 - 1; p <= r1 + 1; ++p) {
      // colour 0 on row p (rows r0 - 1 and r1 are halo rows)
      int nr = 0, first0 = 0;
      if (p >= 0 && p < n && p <= r1) {
        first0 = ca + ((p + ca) & 1);
        nr = first0 <= cb ? (cb - first0) / 2 + 1 : 0;
      }
      // colour 1 on row q = p - 2
      const int q = p - 2;
      int nb = 0, first1 = 0;
      if (q >= r0 && q < r1) {
        first1 = c0 + (((q + c0) & 1) ^ 1);
        nb = first1 < c1 ? (c1 - 1 - first1) / 2 + 1 : 0;
      }
      const int wr = (nr + npw - 1) / npw, wb = (nb + npw - 1) / npw;
      // warp-uniform tasks: a warp takes npw nodes of one colour
      for (int k = warp; k < wr + wb; k += nwarps) {
        const bool red = k < wr;
        const int i = (red ? k : k - wr) * npw + slot;
        const bool valid = i < (red ? nr : nb);
        const int iy = valid ? (red ? p : q) : 0, ix = valid ? (red ? first0 : first1) + 2 * i : 0;
        if constexpr (MODE == kFusedPlain) {
          // one call site for both colours (the registers of one node update)
          rbgs_node<float, V, SPL, false>(L, red ? xa : xbc, xb, f, valid, iy, ix, lane, lpn, e, nc);
        } else if (red) {
          if constexpr (MODE == kFusedZero)
            rbgs_node<float, V, SPL, false, false, true>(L, xa, xb, f, valid, iy, ix, lane, lpn, e, nc);
          else
            rbgs_node<float, V, SPL, false, true>(L, xa, xb, f, valid, iy, ix, lane, lpn, e, nc);
        } else {
          rbgs_node<float, V, SPL, false>(L, xbc, xb, f, valid, iy, ix, lane, lpn, e, nc);
        }
      }
      __syncthreads();   // this phase's colour-0 values before the next phase's colour-1 nodes read them
    }
  }
}

template <int MODE>
cudaError_t launch_mode(const FusedPlan& P, const LevelView<float>& L, Vec3c<float> xa, Vec3<float> xb,
                        Vec3c<float> f, Vec3c<float> e, int nc, cudaStream_t st) {
  const dim3 grid(P.grid), block(P.threads);
  switch (P.spl) {
    case 1:
      return launch_k(rbgs_fused_kernel<4, 1, MODE>, grid, block, 0, st, L, xa, xb, f, e, nc, P.lpn, P.W, P.BH,
                      P.strips, P.tiles);
    case 2:
      return launch_k(rbgs_fused_kernel<4, 2, MODE>, grid, block, 0, st, L, xa, xb, f, e, nc, P.lpn, P.W, P.BH,
                      P.strips, P.tiles);
    case 4:
      return launch_k(rbgs_fused_kernel<4, 4, MODE>, grid, block, 0, st, L, xa, xb, f, e, nc, P.lpn, P.W, P.BH,
                      P.strips, P.tiles);
    default:
      return cudaErrorNotSupported;
  }
}

template <int MODE>
int resident_ctas(int spl, int threads) {
  int per = 0;
  cudaError_t e = cudaErrorNotSupported;
  if (spl == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, rbgs_fused_kernel<4, 1, MODE>, threads, 0);
  if (spl == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, rbgs_fused_kernel<4, 2, MODE>, threads, 0);
  if (spl == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, rbgs_fused_kernel<4, 4, MODE>, threads, 0);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return per;
}

}  // namespace

// The launch shape of the one-launch sweep on an n x n grid of N samples:
// the half-sweeps' sample map (both colours must have the same one, V = 4,
// 1, 2 or 4 chunks per lane), tiles of up to kFusedW columns, and a band
// height that minimises the phases the busiest CTA walks (waves x (BH + 3)).
namespace {
FusedPlan make_plan(int n, int N, int spl_target) {
  FusedPlan P;
  if (spl_target & (kTuneStaged | kTuneWide)) return P;
  const SampleMap m0 = choose_map(N, 4, colour_count(n, 0), spl_target);
  const SampleMap m1 = choose_map(N, 4, colour_count(n, 1), spl_target);
  if (m0.lpn != m1.lpn || m0.V != m1.V || m0.spl != m1.spl || m0.V != 4 || m0.spl > 4 || n < 3) return P;
  const int npw = 32 / m0.lpn;
  // the widest tile whose phase (at most (W + 3) / 2 colour-0 nodes, halo
  // included, and (W + 1) / 2 colour-1 nodes) takes one task per warp
  const auto warps_for = [npw](int w) { return ((w + 3) / 2 + npw - 1) / npw + ((w + 1) / 2 + npw - 1) / npw; };
  int W = std::min(kFusedW, n);
  while (W > 2 && warps_for(W) > kFusedMaxWarps) --W;
  const int warps = warps_for(W);
  if (warps > kFusedMaxWarps) return P;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess) {
    (void)cudaGetLastError();
    return P;
  }
  const int per = resident_ctas<kFusedPlain>(m0.spl, warps * 32);
  if (per < 1) return P;
  const long slots = (long)sms * per;
  const int strips = (n + W - 1) / W;
  long best = -1;
  int bands_best = 1;
  for (int bands = 1; bands <= n; ++bands) {
    const int BH = (n + bands - 1) / bands;
    if ((long)(bands - 1) * BH >= n) continue;   // a band would be empty
    const long tiles = (long)strips * bands;
    const long cost = ((tiles + slots - 1) / slots) * (BH + 3);
    if (best < 0 || cost < best) {
      best = cost;
      bands_best = bands;
    }
  }
  P.ok = true;
  P.lpn = m0.lpn;
  P.spl = m0.spl;
  P.W = W;
  P.BH = (n + bands_best - 1) / bands_best;
  P.strips = strips;
  P.tiles = strips * ((n + P.BH - 1) / P.BH);
  P.threads = warps * 32;
  P.grid = (int)std::min<long>(P.tiles, slots);
  return P;
}

std::mutex g_plan_mu;
std::map<std::tuple<int, int, int, int>, FusedPlan> g_plans;   // (device, n, N, target)
}  // namespace

FusedPlan fused_plan(int n, int N, int spl_target) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return FusedPlan{};
  }
  const auto key = std::make_tuple(dev, n, N, spl_target);
  {
    std::lock_guard<std::mutex> g(g_plan_mu);
    const auto it = g_plans.find(key);
    if (it != g_plans.end()) return it->second;
  }
  const FusedPlan P = make_plan(n, N, spl_target);
  std::lock_guard<std::mutex> g(g_plan_mu);
  g_plans[key] = P;
  return P;
}

cudaError_t launch_rbgs_fused(const LevelView<float>& L, Vec3c<float> xa, Vec3<float> xb, Vec3c<float> f,
                              int mode, Vec3c<float> e, int nc, cudaStream_t st) {
  if (L.freeze_u || xa.y == xb.y) return cudaErrorNotSupported;
  const FusedPlan P = fused_plan(L.n, L.N, L.spl_target);
  if (!P.ok) return cudaErrorNotSupported;
  cudaError_t err;
  if (mode == kFusedZero) err = launch_mode<kFusedZero>(P, L, xa, xb, f, e, nc, st);
  else if (mode == kFusedProlong) err = launch_mode<kFusedProlong>(P, L, xa, xb, f, e, nc, st);
  else err = launch_mode<kFusedPlain>(P, L, xa, xb, f, e, nc, st);
  count_launches(1);
  return err != cudaSuccess ? err : cudaGetLastError();
}

}  // namespace cmg
