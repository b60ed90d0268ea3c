"""GPU parity: every kernel of libcmg against the CPU oracle, through the C ABI.

FP64 bar (the solver's own acceptance rule): single kernels, sweeps and
cycle iterates within 1e-12 relative (max-norm per block, scaled by the
block's max magnitude); converged solutions within 1e-9 relative.  The
FP32 kernels are held to 2e-5 relative against the FP64 oracle on
FP32-representable inputs: each output is a short sum (<= 10 terms) of
products of O(1)-conditioned values, so its rounding error is a few units
of 2^-24 ~ 6e-8 times the largest term; sweeps and the control Schur
quotient amplify it by at most the local condition, which stays below
~100 on these grids.
"""
import numpy as np
import pytest
import torch

import inputs
import oracle.cmg_oracle as O

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5


@pytest.fixture(scope="module")
def cmg():
    from paper_2302_13680_gb300 import build

    build.build()
    import paper_2302_13680_gb300 as P

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return P


def relerr(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = max(np.abs(ref).max(), 1e-300)
    return float(np.abs(got - ref).max() / scale)


def to_dev(v, dtype=torch.float64):
    y, u, p = v
    n = u.shape[0]
    return (torch.tensor(np.asarray(y).reshape(n * n, -1), dtype=dtype, device="cuda").contiguous(),
            torch.tensor(np.asarray(u).reshape(n * n), dtype=dtype, device="cuda").contiguous(),
            torch.tensor(np.asarray(p).reshape(n * n, -1), dtype=dtype, device="cuda").contiguous())


def to_host(v, n):
    y, u, p = (t.double().cpu().numpy() for t in v)
    return y.reshape(n, n, -1), u.reshape(n, n), p.reshape(n, n, -1)


def assert_close(got, ref, tol, what=""):
    for name, g, r in zip("yup", got, ref):
        e = relerr(g, r)
        assert e <= tol, f"{what} block {name}: rel err {e:.3e} > {tol:.1e}"


def rand_level_vec(n, N, seed, dtype=np.float64):
    rng = np.random.default_rng(seed)
    v = (rng.standard_normal((n, n, N)), rng.standard_normal((n, n)), rng.standard_normal((n, n, N)))
    return tuple(np.asarray(b, dtype=dtype).astype(np.float64) for b in v)


# (n, N, K, nu, amp, seed, coarsest, coarse rule, control region): the small
# configuration, ragged sample counts (scalar and 2-wide vector paths,
# partial lane groups), all three coarsest grids, a sample count that spans
# several chunks per lane, both coarse-coefficient rules, and local control
# (the paper's region (0.25, 0.75)^2, and an off-centre box) including a
# coarsest 7 x 7 grid with nodes outside the region.
LOCAL = (0.25, 0.75, 0.25, 0.75)
CASES = [
    (31, 8, 4, 1e-4, 0.5, 1, 3, "averaged", None),
    (31, 8, 4, 1e-4, 0.5, 1, 3, "nodal", None),
    (15, 5, 3, 1e-3, 0.8, 7, 3, "averaged", None),
    (15, 6, 3, 1e-3, 0.8, 8, 1, "averaged", None),
    (31, 3, 2, 1e-5, 1.0, 9, 7, "nodal", None),
    (15, 1, 2, 1e-2, 0.6, 10, 3, "averaged", None),
    (63, 64, 16, 1e-6, 1.0, 2, 3, "averaged", None),
    (15, 130, 4, 1e-4, 1.0, 11, 3, "averaged", None),
    (31, 8, 4, 1e-4, 0.5, 1, 3, "averaged", LOCAL),
    (15, 5, 3, 1e-3, 0.8, 7, 3, "averaged", LOCAL),
    (15, 6, 3, 1e-3, 0.8, 8, 1, "averaged", (0.3, 0.7, 0.1, 0.6)),
    (31, 3, 2, 1e-5, 1.0, 9, 7, "nodal", LOCAL),
    (63, 64, 16, 1e-6, 1.0, 2, 3, "averaged", LOCAL),
]
IDS = [f"n{c[0]}_N{c[1]}_c{c[6]}_{c[7][:3]}" + ("" if c[8] is None else "_local") for c in CASES]


@pytest.fixture(scope="module", params=CASES, ids=IDS)
def case(request, cmg):
    n, N, K, nu, amp, seed, coarsest, coarse, box = request.param
    xi = inputs.draw_xi(seed, N, K)
    H = cmg.Hierarchy(n, N, xi, nu, amp, coarsest_n=coarsest, coarse=coarse, control_box=box)
    levels = O.make_hierarchy(n, N, nu, O.sine_mode_field(xi, amp), coarsest_n=coarsest, coarse=coarse,
                              control_box=box)
    yield H, levels
    H.close()


def test_hierarchy_shape(case):
    H, levels = case
    assert H.level_n == [lv.n for lv in levels]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_residual_every_level(case, prec):
    H, levels = case
    dt, tol = (torch.float64, TOL64) if prec == "f64" else (torch.float32, TOL32)
    npdt = np.float64 if prec == "f64" else np.float32
    for l, lv in enumerate(levels):
        x = rand_level_vec(lv.n, lv.N, 100 + l, npdt)
        f = rand_level_vec(lv.n, lv.N, 200 + l, npdt)
        r = H.zeros(l, dt)
        H.residual(l, to_dev(x, dt), to_dev(f, dt), r)
        assert_close(to_host(r, lv.n), O.residual(lv, x, f), tol, f"residual level {l}")
        # operator apply (f = NULL)
        H.residual(l, to_dev(x, dt), None, r)
        assert_close(to_host(r, lv.n), O.apply_S(lv, *x), tol, f"apply level {l}")


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("smoother", ["rbgs", "jacobi"])
def test_one_sweep(case, prec, smoother):
    H, levels = case
    dt, tol = (torch.float64, TOL64) if prec == "f64" else (torch.float32, TOL32)
    npdt = np.float64 if prec == "f64" else np.float32
    import paper_2302_13680_gb300 as P

    opts = P.CycleOptions(smoother=P.SMOOTH_RBGS if smoother == "rbgs" else P.SMOOTH_JACOBI, theta=0.5)
    for l in (0, len(levels) - 2):
        if l < 0:
            continue
        lv = levels[l]
        # f of the size a cycle sees, x a random iterate
        x = rand_level_vec(lv.n, lv.N, 300 + l, npdt)
        f = rand_level_vec(lv.n, lv.N, 400 + l, npdt)
        f = tuple(b * s for b, s in zip(f, (lv.c, lv.G, lv.h ** 2)))
        f = tuple(np.asarray(b, dtype=npdt).astype(np.float64) for b in f)
        xd = to_dev(x, dt)
        H.smooth(l, opts, 1, xd, to_dev(f, dt))
        if smoother == "rbgs":
            ref = O.rbgs_sweep(lv, x, f)
        else:
            ref = O.jacobi_sweep(lv, x, f, 0.5)
        assert_close(to_host(xd, lv.n), ref, tol, f"{smoother} level {l}")


def test_red_half_sweep_leaves_black_nodes(case):
    H, levels = case
    lv = levels[0]
    import paper_2302_13680_gb300 as P

    x = rand_level_vec(lv.n, lv.N, 7)
    f = rand_level_vec(lv.n, lv.N, 8)
    xd = to_dev(x)
    H.smooth(0, P.CycleOptions(), 2, xd, to_dev(f))
    ref = O.rbgs_sweep(lv, O.rbgs_sweep(lv, x, f), f)
    assert_close(to_host(xd, lv.n), ref, TOL64, "two sweeps")


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_transfers(case, prec):
    H, levels = case
    dt, tol = (torch.float64, 1e-14) if prec == "f64" else (torch.float32, 1e-6)
    npdt = np.float64 if prec == "f64" else np.float32
    for l in range(len(levels) - 1):
        nf, nc = levels[l].n, levels[l + 1].n
        N = levels[l].N
        r = rand_level_vec(nf, N, 500 + l, npdt)
        c = H.zeros(l + 1, dt)
        H.restrict(l, to_dev(r, dt), c)
        assert_close(to_host(c, nc), O.restrict(nf, r), tol, f"restrict {l}")
        e = rand_level_vec(nc, N, 600 + l, npdt)
        x = rand_level_vec(nf, N, 700 + l, npdt)
        xd = to_dev(x, dt)
        H.prolong_add(l, to_dev(e, dt), xd)
        pe = O.prolong(nf, e, levels[l].chi)
        assert_close(to_host(xd, nf), tuple(a + b for a, b in zip(x, pe)), tol, f"prolong {l}")


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_coarse_solve(case, prec):
    H, levels = case
    dt, tol = (torch.float64, TOL64) if prec == "f64" else (torch.float32, TOL32)
    npdt = np.float64 if prec == "f64" else np.float32
    lv = levels[-1]
    f = rand_level_vec(lv.n, lv.N, 800, npdt)
    x = H.zeros(len(levels) - 1, dt)
    H.coarse_solve(to_dev(f, dt), x)
    assert_close(to_host(x, lv.n), O.coarse_solve(lv, f), tol, "coarse")


@pytest.mark.parametrize("tail_n", [0, 31])
@pytest.mark.parametrize("gamma", [1, 2])
@pytest.mark.parametrize("smoother", ["rbgs", "jacobi"])
def test_cycle_iterates(case, gamma, smoother, tail_n):
    """Cycle k of the GPU from the oracle's iterate k-1 matches the oracle's cycle k,
    with the coarse grids run one launch per step (tail_n = 0) or as one
    cluster launch (tail_n = 31).

    Red-black iterates are held to 1e-12.  Damped Jacobi forms the explicit
    residual f - S x before each update; its rounding is relative to |f| +
    |S x| while the update scales with |r|, which after the first sweeps is
    up to ~5x smaller, so its iterates are held to 5e-12."""
    H, levels = case
    import paper_2302_13680_gb300 as P

    lv = levels[0]
    yd = inputs.target_modes(lv.n, 3)
    f = O.fine_rhs(lv, yd)
    oopts = O.CycleOptions(smoother=smoother, gamma=gamma)
    gopts = P.CycleOptions(smoother=P.SMOOTH_RBGS if smoother == "rbgs" else P.SMOOTH_JACOBI, gamma=gamma,
                           tail_n=tail_n)
    x = O.zeros_like_level(lv)
    fd = to_dev(f)
    for k in range(3):
        xd = to_dev(x)
        H.cycle(gopts, xd, fd)
        x = O.cycle(levels, 0, x, f, oopts)
        assert_close(to_host(xd, lv.n), x, TOL64 if smoother == "rbgs" else 5 * TOL64, f"cycle {k}")


@pytest.mark.parametrize("method", ["cycle", "fgmres"])
def test_converged_solution(case, method):
    H, levels = case
    import paper_2302_13680_gb300 as P

    lv = levels[0]
    yd = inputs.target_sinsin(lv.n)
    f = O.fine_rhs(lv, yd)
    opts = O.CycleOptions()
    if method == "cycle":
        ref = O.solve_stationary(levels, f, opts, tol=1e-11, maxit=60)
        m = P.METHOD_CYCLE
    else:
        ref = O.fgmres(levels, f, opts, tol=1e-11)
        m = P.METHOD_FGMRES
    fd = to_dev(f)
    xd = H.zeros(0)
    st, _ = H.solve(P.CycleOptions(), fd, xd, method=m, tol=1e-11, maxit=60, restart=30)
    assert st.relres <= 1e-11
    assert ref.relres <= 1e-11
    assert abs(st.iters - ref.iters) <= 1
    assert_close(to_host(xd, lv.n), ref.x, 1e-9, "solution")


@pytest.mark.parametrize("ctl32", [0, 1])
@pytest.mark.parametrize("method", ["cycle", "fgmres"])
def test_mixed_precision_solve(case, method, ctl32):
    """FP32 cycles (Eq. (13)'s per-node Schur scalar in FP64, or, with
    ctl32, in FP32 too) inside FP64 refinement / FGMRES reach the FP64
    residual tolerance 1e-11, and the converged solution is then within
    the FP64 bar of 1e-9 of the oracle's, block by block."""
    H, levels = case
    import paper_2302_13680_gb300 as P

    lv = levels[0]
    f = O.fine_rhs(lv, inputs.target_sinsin(lv.n))
    ref = O.fgmres(levels, f, O.CycleOptions(), tol=1e-12)
    fd = to_dev(f)
    xd = H.zeros(0)
    m = P.METHOD_CYCLE if method == "cycle" else P.METHOD_FGMRES
    st, _ = H.solve(P.CycleOptions(precision=P.FP32, ctl32=ctl32), fd, xd, method=m, tol=1e-11, maxit=80,
                    restart=30)
    assert st.relres <= 1e-11
    assert_close(to_host(xd, lv.n), ref.x, 1e-9, f"mixed {method} ctl32={ctl32}")


@pytest.mark.parametrize("tail_n", [0, 31])
def test_frozen_control_cycle_iterates(case, tail_n):
    """Cycles with the control held fixed (Eq. (14) local solves with u_i
    given, zero control correction on coarse grids) against the oracle."""
    H, levels = case
    import paper_2302_13680_gb300 as P

    lv = levels[0]
    f = O.fine_rhs(lv, inputs.target_modes(lv.n, 4))
    rng = np.random.default_rng(12)
    x = (np.zeros((lv.n, lv.n, lv.N)), rng.standard_normal((lv.n, lv.n)), np.zeros((lv.n, lv.n, lv.N)))
    fd = to_dev(f)
    for k in range(2):
        xd = to_dev(x)
        H.cycle(P.CycleOptions(freeze_u=1, tail_n=tail_n), xd, fd)
        x = O.cycle(levels, 0, x, f, O.CycleOptions(freeze_u=True))
        assert_close(to_host(xd, lv.n), x, TOL64, f"frozen cycle {k}")


@pytest.mark.parametrize("spl", [1, 2])
@pytest.mark.parametrize("freeze", [0, 1])
def test_staged_half_sweep_matches_direct(case, spl, freeze):
    """The FP32 half-sweep that stages its loads through shared memory
    (CMG_TUNE_STAGED) performs the same operations in the same order as the
    direct-load sweep: two sweeps on every grid agree bit for bit (grids
    whose sample count is not a multiple of 4 fall back to the direct
    sweep)."""
    H, levels = case
    import paper_2302_13680_gb300 as P

    staged = 16
    out = []
    for t in (spl, staged | spl):
        H.set_tuning(P.FP32, [t] * (H.levels - 1) + [0])
        res = []
        for lv in range(H.levels - 1):
            n = H.level_n[lv]
            x = to_dev(rand_level_vec(n, levels[lv].N, 900 + lv, np.float32), torch.float32)
            f = to_dev(rand_level_vec(n, levels[lv].N, 950 + lv, np.float32), torch.float32)
            H.smooth(lv, P.CycleOptions(precision=P.FP32, freeze_u=freeze), 2, x, f)
            res.append(x)
        out.append(res)
    H.set_tuning(P.FP32, None)
    for a, b in zip(*out):
        for ta, tb in zip(a, b):
            assert torch.equal(ta, tb)


def test_wide_layout_matches_oracle(case):
    """FP32 node kernels in the two-samples-per-lane layout (CMG_TUNE_WIDE;
    ignored where N is odd or above 64): residual, one sweep of each
    smoother and a refinement solve against the FP64 oracle, as for the
    default layout."""
    H, levels = case
    import paper_2302_13680_gb300 as P

    wide = 32
    H.set_tuning(P.FP32, [wide | 1] * (H.levels - 1) + [0])
    try:
        for l, lv in enumerate(levels[:-1]):
            x = rand_level_vec(lv.n, lv.N, 700 + l, np.float32)
            f = rand_level_vec(lv.n, lv.N, 750 + l, np.float32)
            r = H.zeros(l, torch.float32)
            H.residual(l, to_dev(x, torch.float32), to_dev(f, torch.float32), r)
            assert_close(to_host(r, lv.n), O.residual(lv, x, f), TOL32, f"wide residual level {l}")
            fs = tuple(np.asarray(b * s, dtype=np.float32).astype(np.float64) for b, s in zip(f, (lv.c, lv.G, lv.h ** 2)))
            for sm in ("rbgs", "jacobi"):
                opts = P.CycleOptions(precision=P.FP32, theta=0.5,
                                      smoother=P.SMOOTH_RBGS if sm == "rbgs" else P.SMOOTH_JACOBI)
                xd = to_dev(x, torch.float32)
                H.smooth(l, opts, 1, xd, to_dev(fs, torch.float32))
                ref = O.rbgs_sweep(lv, x, fs) if sm == "rbgs" else O.jacobi_sweep(lv, x, fs, 0.5)
                assert_close(to_host(xd, lv.n), ref, TOL32, f"wide {sm} level {l}")
        lv = levels[0]
        f = O.fine_rhs(lv, inputs.target_sinsin(lv.n))
        ref = O.fgmres(levels, f, O.CycleOptions(), tol=1e-12)
        xd = H.zeros(0)
        st, _ = H.solve(P.CycleOptions(precision=P.FP32), to_dev(f), xd, method=P.METHOD_CYCLE, tol=1e-10, maxit=60)
        assert st.relres <= 1e-10
        for name, g, r in zip("yup", to_host(xd, lv.n), ref.x):
            assert relerr(g, r) <= 1e-6, name
    finally:
        H.set_tuning(P.FP32, None)


@pytest.mark.parametrize("gamma", [1, 2])
@pytest.mark.parametrize("smoother", ["rbgs", "jacobi"])
def test_fp32_cycle_cluster_matches_per_launch(case, gamma, smoother):
    """FP32 cycles with every grid n <= 31 in one cluster launch against the
    one-launch-per-step path (which computes the post-smoothing residual at
    colour 0 only and fuses the prolongation into the next half-sweep): the
    same algorithm, FP32 rounding in different orders."""
    H, levels = case
    import paper_2302_13680_gb300 as P

    lv = levels[0]
    f = tuple(np.asarray(b, dtype=np.float32).astype(np.float64) for b in O.fine_rhs(lv, inputs.target_modes(lv.n, 5)))
    sm = P.SMOOTH_RBGS if smoother == "rbgs" else P.SMOOTH_JACOBI
    fd = to_dev(f, torch.float32)
    out = []
    for tail_n in (0, 31):
        xd = H.zeros(0, torch.float32)
        for _ in range(2):
            H.cycle(P.CycleOptions(precision=P.FP32, smoother=sm, gamma=gamma, tail_n=tail_n), xd, fd)
        out.append(to_host(xd, lv.n))
    assert_close(out[1], out[0], TOL32, "fp32 cluster vs per-launch")
