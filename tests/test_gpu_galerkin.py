"""GPU parity of the Galerkin coarse operators (Sec. 3: S_l = P^T S_{l-1} P)
against the sparse-matrix oracle (oracle/galerkin.py), through the C ABI.

The oracle assembles S_0 from the block definition, forms the coarse
matrices by sparse products, smooths with dense node-block solves and
solves the coarsest grid with a sparse direct solver; the GPU builds 9-point
stencils by a triple-product kernel and runs Eq. (13) with the Galerkin
diagonal entries.  Both smoothers: damped collective Jacobi, and collective
Gauss-Seidel (red-black on the 5-point finest grid, four colours on the
9-point grids).  FP64 bars: operators within 1e-12 relative (max-norm per
block), the coarsest direct solve within 1e-11; one Jacobi sweep within 1e-10 (the oracle's
dense block solve and Eq. (13) round differently, amplified by the local
condition); cycle iterates within 1e-9; solutions converged to 1e-12 within 1e-7
of the sparse direct solution (the control block's sensitivity sets that floor)
and, for the repeated cycle, within 1e-9 of the oracle's converged iterate.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

import inputs
import oracle.cmg_oracle as O
import oracle.galerkin as G

pytestmark = pytest.mark.gpu

# (n, N, K, nu, amp, seed, coarsest): several grids and tiles, ragged sample
# counts, all three coarsest grids (m = 1, 9, 49) and a sample count above
# one CTA's 128-thread reduction
CASES = [
    (15, 5, 3, 1e-3, 0.8, 7, 3),
    (31, 8, 4, 1e-4, 0.5, 1, 3),
    (15, 6, 3, 1e-3, 0.8, 8, 1),
    (31, 3, 2, 1e-5, 1.0, 9, 7),
    (7, 130, 4, 1e-4, 1.0, 11, 3),
]
IDS = [f"n{c[0]}_N{c[1]}_c{c[6]}" for c in CASES]


@pytest.fixture(scope="module")
def P():
    from paper_2302_13680_gb300 import build

    build.build()
    import paper_2302_13680_gb300 as P

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return P


@pytest.fixture(scope="module", params=CASES, ids=IDS)
def case(request, P):
    n, N, K, nu, amp, seed, coarsest = request.param
    xi = inputs.draw_xi(seed, N, K)
    H = P.Hierarchy(n, N, xi, nu, amp, coarsest_n=coarsest, coarse="galerkin")
    levels = O.make_hierarchy(n, N, nu, O.sine_mode_field(xi, amp), coarsest_n=coarsest)
    S = G.hierarchy(levels)
    yield H, levels, S
    H.close()


def dev(z, n, N):
    y, u, p = O.unpack(z, n, N)
    return (torch.tensor(y.reshape(n * n, N), device="cuda"), torch.tensor(u.reshape(n * n), device="cuda"),
            torch.tensor(p.reshape(n * n, N), device="cuda"))


def host(v):
    return np.concatenate([t.double().cpu().numpy().ravel() for t in v])


def assert_blocks(got, ref, n, N, tol, what):
    for name, g, r in zip("yup", O.unpack(got, n, N), O.unpack(ref, n, N)):
        scale = max(np.abs(r).max(), 1e-300)
        e = float(np.abs(g - r).max() / scale)
        assert e <= tol, f"{what} block {name}: rel err {e:.3e} > {tol:.1e}"


def opts(smoother="jacobi", gamma=1):
    """Jacobi (theta = 1/2), or Gauss-Seidel: red-black on the finest grid, four colours below."""
    import paper_2302_13680_gb300 as P

    sm = P.SMOOTH_JACOBI if smoother == "jacobi" else P.SMOOTH_RBGS
    return P.CycleOptions(smoother=sm, theta=0.5, precision=P.FP64, gamma=gamma)


def jacobi():
    return opts("jacobi")


SMOOTHERS = ["jacobi", "gs"]


def test_residual_every_level(case):
    H, levels, S = case
    N = levels[0].N
    rng = np.random.default_rng(21)
    for l, lv in enumerate(levels):
        dim = S[l].shape[0]
        z, f = rng.standard_normal(dim), rng.standard_normal(dim)
        r = H.zeros(l)
        H.residual(l, dev(z, lv.n, N), dev(f, lv.n, N), r)
        assert_blocks(host(r), f - S[l] @ z, lv.n, N, 1e-12, f"residual level {l}")
        H.residual(l, dev(z, lv.n, N), None, r)
        assert_blocks(host(r), S[l] @ z, lv.n, N, 1e-12, f"apply level {l}")


@pytest.mark.parametrize("smoother", SMOOTHERS)
def test_one_sweep_every_grid(case, smoother):
    H, levels, S = case
    ns = [lv.n for lv in levels]
    N = levels[0].N
    fine = levels[0]
    rng = np.random.default_rng(22)
    for l, lv in enumerate(levels[:-1]):
        m = lv.n * lv.n
        z = rng.standard_normal(S[l].shape[0])
        # right side of the size a cycle sees: the blocks scaled like the operator's rows
        f = rng.standard_normal(S[l].shape[0])
        f[: m * N] *= fine.c
        f[m * N: m * N + m] *= fine.G
        f[m * N + m:] *= fine.h ** 2
        x = dev(z, lv.n, N)
        H.smooth(l, opts(smoother), 1, x, dev(f, lv.n, N))
        ref = G.smooth(S, ns, N, l, z, f, smoother, 0.5)
        assert_blocks(host(x), ref, lv.n, N, 1e-10, f"{smoother} level {l}")


def test_coarse_solve(case):
    H, levels, S = case
    N = levels[0].N
    lv = levels[-1]
    f = np.random.default_rng(23).standard_normal(S[-1].shape[0])
    x = H.zeros(len(levels) - 1)
    H.coarse_solve(dev(f, lv.n, N), x)
    # block elimination (Gauss-Jordan inverses, Schur system with the mass products) against a
    # sparse LU: 1.1e-12 measured on the 7 x 7 coarsest grid, so the bar is 1e-11
    assert_blocks(host(x), spla.spsolve(S[-1].tocsc(), f), lv.n, N, 1e-11, "coarse solve")


@pytest.mark.parametrize("smoother", SMOOTHERS)
@pytest.mark.parametrize("gamma", [1, 2])
def test_cycle_iterates(case, gamma, smoother):
    H, levels, S = case
    N, n = levels[0].N, levels[0].n
    ns = [lv.n for lv in levels]
    rng = np.random.default_rng(24)
    z = rng.standard_normal(S[0].shape[0])
    f = O.pack(O.fine_rhs(levels[0], inputs.target_sinsin(n)))
    x = dev(z, n, N)
    for k in range(2):
        H.cycle(opts(smoother, gamma), x, dev(f, n, N))
        z = G.cycle(S, ns, N, 0, z, f, n1=2, n2=2, theta=0.5, gamma=gamma, smoother=smoother)
        assert_blocks(host(x), z, n, N, 1e-9, f"cycle {k}")


@pytest.mark.parametrize("smoother", SMOOTHERS)
@pytest.mark.parametrize("method", ["cycle", "fgmres"])
def test_converged_solution(case, method, smoother):
    H, levels, S = case
    import paper_2302_13680_gb300 as P

    N, n = levels[0].N, levels[0].n
    f = O.pack(O.fine_rhs(levels[0], inputs.target_sinsin(n)))
    x = H.zeros(0)
    m = P.METHOD_CYCLE if method == "cycle" else P.METHOD_FGMRES
    # to 1e-12.  Any two iterates at that residual may differ by up to ~1e-8 in the control block
    # (u = sum_j p_j / nu amplifies the residual by ~1e4 here: the sparse direct solution, residual
    # 1e-13 .. 5e-12, lies within 1.1e-8 of the oracle's converged iterate), so against the direct
    # solution the bar is 1e-7.  The repeated cycle follows the oracle's own stationary iteration,
    # whose converged iterate shares that error: against it the bar is 1e-9.
    st, _ = H.solve(opts(smoother), dev(f, n, N), x, method=m, tol=1e-12, maxit=100, restart=30)
    assert st.relres <= 1e-12
    ref = spla.spsolve(S[0].tocsc(), f)
    assert_blocks(host(x), ref, n, N, 1e-7, f"{method} solution")
    if method == "cycle":
        # the same stationary iteration as the oracle's: the same number of cycles, the same iterate
        _, it, _ = G.solve_stationary(S, [lv.n for lv in levels], N, f, tol=1e-12, maxit=100, smoother=smoother)
        assert abs(st.iters - it) <= 1
        z, _, _ = G.solve_stationary(S, [lv.n for lv in levels], N, f, tol=0.0, maxit=st.iters, smoother=smoother)
        assert_blocks(host(x), z, n, N, 1e-9, "cycle solution vs the oracle's iterate after as many cycles")


def test_unsupported_combinations_are_refused(P):
    """A frozen control (the 9-point sweeps update u in every colour) and the
    FP32 control row (the Galerkin control row sums in FP64) are refused."""
    xi = inputs.draw_xi(7, 4, 3)
    H = P.Hierarchy(15, 4, xi, 1e-3, 0.8, coarse="galerkin")
    try:
        f = H.zeros(0)
        for o in (P.CycleOptions(smoother=P.SMOOTH_RBGS, precision=P.FP32, ctl32=1),
                  P.CycleOptions(smoother=P.SMOOTH_JACOBI, precision=P.FP32, freeze_u=1),
                  P.CycleOptions(smoother=P.SMOOTH_JACOBI, precision=P.FP64, freeze_u=1)):
            with pytest.raises(P.CMGError) as ei:
                H.solve(o, f, H.zeros(0))
            assert ei.value.status == 7
    finally:
        H.close()
    with pytest.raises(P.CMGError):
        P.Hierarchy(15, 4, xi, 1e-3, 0.8, coarse="galerkin", control_box=(0.25, 0.75, 0.25, 0.75))


def test_fp64_autotune_skips_galerkin_grids(P):
    """The FP64 autotuner times red-black sweeps; Galerkin grids below the
    finest run the Jacobi path only and are left at the size heuristic."""
    xi = inputs.draw_xi(7, 5, 3)
    H = P.Hierarchy(15, 5, xi, 1e-3, 0.8, coarse="galerkin")
    try:
        chosen = H.autotune(P.FP64)
        assert chosen[0] in (1, 2, 4) and all(t == 0 for t in chosen[1:])
        levels = O.make_hierarchy(15, 5, 1e-3, O.sine_mode_field(xi, 0.8))
        S = G.hierarchy(levels)
        f = O.pack(O.fine_rhs(levels[0], inputs.target_sinsin(15)))
        x = H.zeros(0)
        st, _ = H.solve(jacobi(), dev(f, 15, 5), x, tol=1e-12, maxit=100)
        assert_blocks(host(x), spla.spsolve(S[0].tocsc(), f), 15, 5, 1e-7, "solution after autotune")
    finally:
        H.close()


# ---- FP32 cycles on the Galerkin grids ----------------------------------
# The per-sample arithmetic runs in FP32 on FP32 copies of the FP64 Galerkin
# planes; the control row's sums over samples, Eq. (13)'s Schur scalar and
# the coarsest elimination stay FP64.  Inputs are FP32-representable, the
# oracle FP64; errors relative to each block's largest entry.  Measured
# maxima over these cases: apply 1.6e-7 (FP32 planes, 9-term sums), one
# sweep 3.7e-7, the coarsest solve 5.7e-8 (FP64 elimination, FP32 results),
# one V-cycle from a random iterate 2.0e-5 (the cycle shrinks the iterate's
# rough part, so the rounding of the input is large against the output);
# the bars leave a factor of 5 or more.  FP64 refinement around FP32 cycles
# to 1e-11 lands where FP64 cycles do (1.5e-8 from the sparse direct
# solution at worst, the control block's sensitivity): bar 1e-7.
RES32, SWEEP32, COARSE32, CYCLE32 = 1e-6, 2e-6, 3e-7, 1e-4


def f32(z):
    return np.asarray(z, dtype=np.float32).astype(np.float64)


def dev32(z, n, N):
    return tuple(t.float() for t in dev(z, n, N))


def opts32(smoother="jacobi", gamma=1):
    import paper_2302_13680_gb300 as P

    o = opts(smoother, gamma)
    o.precision = P.FP32
    return o


def test_fp32_residual_every_level(case):
    H, levels, S = case
    N = levels[0].N
    rng = np.random.default_rng(31)
    for l, lv in enumerate(levels):
        dim = S[l].shape[0]
        z, f = f32(rng.standard_normal(dim)), f32(rng.standard_normal(dim))
        r = H.zeros(l, torch.float32)
        H.residual(l, dev32(z, lv.n, N), dev32(f, lv.n, N), r)
        assert_blocks(host(r), f - S[l] @ z, lv.n, N, RES32, f"FP32 residual level {l}")
        H.residual(l, dev32(z, lv.n, N), None, r)
        assert_blocks(host(r), S[l] @ z, lv.n, N, RES32, f"FP32 apply level {l}")


@pytest.mark.parametrize("smoother", SMOOTHERS)
def test_fp32_one_sweep_every_grid(case, smoother):
    H, levels, S = case
    ns = [lv.n for lv in levels]
    N = levels[0].N
    fine = levels[0]
    rng = np.random.default_rng(32)
    for l, lv in enumerate(levels[:-1]):
        m = lv.n * lv.n
        z = f32(rng.standard_normal(S[l].shape[0]))
        f = rng.standard_normal(S[l].shape[0])
        f[: m * N] *= fine.c
        f[m * N: m * N + m] *= fine.G
        f[m * N + m:] *= fine.h ** 2
        f = f32(f)
        x = dev32(z, lv.n, N)
        H.smooth(l, opts32(smoother), 1, x, dev32(f, lv.n, N))
        ref = G.smooth(S, ns, N, l, z, f, smoother, 0.5)
        assert_blocks(host(x), ref, lv.n, N, SWEEP32, f"FP32 {smoother} level {l}")


def test_fp32_coarse_solve(case):
    H, levels, S = case
    N = levels[0].N
    lv = levels[-1]
    f = f32(np.random.default_rng(33).standard_normal(S[-1].shape[0]))
    x = H.zeros(len(levels) - 1, torch.float32)
    H.coarse_solve(dev32(f, lv.n, N), x)
    assert_blocks(host(x), spla.spsolve(S[-1].tocsc(), f), lv.n, N, COARSE32, "FP32 coarse solve")


@pytest.mark.parametrize("smoother", SMOOTHERS)
@pytest.mark.parametrize("gamma", [1, 2])
def test_fp32_cycle_iterate(case, gamma, smoother):
    H, levels, S = case
    N, n = levels[0].N, levels[0].n
    ns = [lv.n for lv in levels]
    rng = np.random.default_rng(34)
    z = f32(rng.standard_normal(S[0].shape[0]))
    f = f32(O.pack(O.fine_rhs(levels[0], inputs.target_sinsin(n))))
    x = dev32(z, n, N)
    H.cycle(opts32(smoother, gamma), x, dev32(f, n, N))
    ref = G.cycle(S, ns, N, 0, z, f, n1=2, n2=2, theta=0.5, gamma=gamma, smoother=smoother)
    assert_blocks(host(x), ref, n, N, CYCLE32, "FP32 cycle")


@pytest.mark.parametrize("smoother", SMOOTHERS)
@pytest.mark.parametrize("method", ["cycle", "fgmres"])
def test_fp32_refined_solution(case, method, smoother):
    """FP64 refinement around FP32 cycles (stationary, or FGMRES with the
    FP32 cycle as preconditioner) to 1e-11: the sparse direct solution, in
    as many cycles (within one) as FP64 cycles take."""
    H, levels, S = case
    import paper_2302_13680_gb300 as P

    N, n = levels[0].N, levels[0].n
    f = O.pack(O.fine_rhs(levels[0], inputs.target_sinsin(n)))
    x = H.zeros(0)
    m = P.METHOD_CYCLE if method == "cycle" else P.METHOD_FGMRES
    st, _ = H.solve(opts32(smoother), dev(f, n, N), x, method=m, tol=1e-11, maxit=200, restart=30)
    assert st.relres <= 1e-11
    st64, _ = H.solve(opts(smoother), dev(f, n, N), H.zeros(0), method=m, tol=1e-11, maxit=200, restart=30)
    assert abs(st.cycles - st64.cycles) <= 1
    assert_blocks(host(x), spla.spsolve(S[0].tocsc(), f), n, N, 1e-7, f"FP32-refined {method} solution")


def test_fp32_autotune_skips_galerkin_grids(P):
    """The FP32 autotuner times red-black half-sweeps of the 5-point grids:
    the Galerkin grids are left at the size heuristic, and FP32-refined
    solves after it converge."""
    xi = inputs.draw_xi(7, 8, 3)
    H = P.Hierarchy(31, 8, xi, 1e-4, 0.8, coarse="galerkin")
    try:
        chosen = H.autotune(P.FP32)
        assert chosen[0] != 0 and all(t == 0 for t in chosen[1:])
        levels = O.make_hierarchy(31, 8, 1e-4, O.sine_mode_field(xi, 0.8))
        S = G.hierarchy(levels)
        f = O.pack(O.fine_rhs(levels[0], inputs.target_sinsin(31)))
        x = H.zeros(0)
        st, _ = H.solve(opts32("gs"), dev(f, 31, 8), x, tol=1e-11, maxit=200)
        assert st.relres <= 1e-11
        assert_blocks(host(x), spla.spsolve(S[0].tocsc(), f), 31, 8, 1e-7, "FP32 solution after autotune")
    finally:
        H.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_residual_large_grid(P, dtype):
    """The residual on a 9-point grid above the one-launch size (n = 127 below
    n = 255: the three-launch form with the per-node sums of p) and on the
    grids below it, in FP64 and FP32, against the sparse Galerkin product;
    and one sweep of either smoother on the n = 127 grid against the
    oracle's."""
    n, N = 255, 4
    xi = inputs.draw_xi(13, N, 3)
    H = P.Hierarchy(n, N, xi, 1e-4, 0.8, coarse="galerkin")
    try:
        levels = O.make_hierarchy(n, N, 1e-4, O.sine_mode_field(xi, 0.8))
        S = G.hierarchy(levels)
        rng = np.random.default_rng(35)
        tol = 1e-12 if dtype == torch.float64 else RES32
        for l in (1, 2):
            lv = levels[l]
            dim = S[l].shape[0]
            z, f = f32(rng.standard_normal(dim)), f32(rng.standard_normal(dim))
            cast = (lambda v: v) if dtype == torch.float64 else (lambda v: tuple(t.float() for t in v))
            r = H.zeros(l, dtype)
            H.residual(l, cast(dev(z, lv.n, N)), cast(dev(f, lv.n, N)), r)
            assert_blocks(host(r), f - S[l] @ z, lv.n, N, tol, f"residual level {l} (n = {lv.n})")
        # one sweep of either smoother on the n = 127 grid: in FP32 its 4,096
        # nodes per colour (16,129 in all) take the two-nodes-per-warp forms of
        # the colour and Jacobi kernels
        fine, lv = levels[0], levels[1]
        m = lv.n * lv.n
        z = f32(rng.standard_normal(S[1].shape[0]))
        fr = rng.standard_normal(S[1].shape[0])
        fr[: m * N] *= fine.c
        fr[m * N: m * N + m] *= fine.G
        fr[m * N + m:] *= fine.h ** 2
        fr = f32(fr)
        for sm in SMOOTHERS:
            x = cast(dev(z, lv.n, N))
            H.smooth(1, opts(sm) if dtype == torch.float64 else opts32(sm), 1, x, cast(dev(fr, lv.n, N)))
            ref = G.smooth(S, [v.n for v in levels], N, 1, z, fr, sm, 0.5)
            assert_blocks(host(x), ref, lv.n, N, 1e-10 if dtype == torch.float64 else SWEEP32, f"{sm} sweep, n = 127")
    finally:
        H.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_gs_above_256_samples(P, dtype):
    """N = 260, above the 256 samples the four-colour sweep keeps in
    registers: the sweep then parks each node's local right sides in its own
    y, p slots between its two passes, with the per-node sums of p kept in a
    scratch array.  One sweep on the 9-point grid, and one V-cycle, against
    the oracle (FP64 bars as above; FP32 as SWEEP32 and CYCLE32)."""
    n, N = 15, 260
    xi = inputs.draw_xi(12, N, 4)
    H = P.Hierarchy(n, N, xi, 1e-3, 0.8, coarse="galerkin")
    try:
        levels = O.make_hierarchy(n, N, 1e-3, O.sine_mode_field(xi, 0.8))
        S = G.hierarchy(levels)
        ns = [lv.n for lv in levels]
        fine, lv = levels[0], levels[1]
        m = lv.n * lv.n
        rng = np.random.default_rng(36)
        z = f32(rng.standard_normal(S[1].shape[0]))
        f = rng.standard_normal(S[1].shape[0])
        f[: m * N] *= fine.c
        f[m * N: m * N + m] *= fine.G
        f[m * N + m:] *= fine.h ** 2
        f = f32(f)
        cast = (lambda v: v) if dtype == torch.float64 else (lambda v: tuple(t.float() for t in v))
        o = opts("gs") if dtype == torch.float64 else opts32("gs")
        x = cast(dev(z, lv.n, N))
        H.smooth(1, o, 1, x, cast(dev(f, lv.n, N)))
        tol = 1e-10 if dtype == torch.float64 else SWEEP32
        assert_blocks(host(x), G.smooth(S, ns, N, 1, z, f, "gs", 0.5), lv.n, N, tol, "gs sweep, N = 260")
        z0 = f32(rng.standard_normal(S[0].shape[0]))
        f0 = f32(O.pack(O.fine_rhs(fine, inputs.target_sinsin(n))))
        x = cast(dev(z0, n, N))
        H.cycle(o, x, cast(dev(f0, n, N)))
        ref = G.cycle(S, ns, N, 0, z0, f0, n1=2, n2=2, theta=0.5, gamma=1, smoother="gs")
        tol = 1e-9 if dtype == torch.float64 else CYCLE32
        assert_blocks(host(x), ref, n, N, tol, "gs cycle, N = 260")
    finally:
        H.close()
