"""The one-launch red-black sweep (CMG_TUNE_FUSED, csrc/cmg_fused.cu) against
the two half-sweep launches and against the CPU oracle, through the C ABI.

The fused sweep updates colour 0 and then colour 1 (the Gauss-Seidel
variant after Eq. (11), Eq. (13) per node) over tiles of the grid, reading
the old iterate from one buffer and writing the new one to another, with
the colour-0 halo of every tile recomputed.  Its per-node arithmetic and
sample map are those of the half-sweeps, so every result here must agree
with them bit for bit: pairs of sweeps, odd sweep counts (a pair and a
half-sweep pair), whole cycles (the zero-iterate and prolongation-fused
first sweeps included, with the prolongation fused or as its own pass), on
grids whose tiles are ragged (n not a multiple of the tile width) and at
N = 256 in the shapes of the large workload.  Against the FP64 oracle the
FP32 bar of the other parity tests (2e-5) holds for two sweeps, and FP64
refinement with fused FP32 cycles converges to the oracle's solution
within 1e-9.
"""
import numpy as np
import pytest
import torch

import inputs
import oracle.cmg_oracle as O

pytestmark = pytest.mark.gpu

TOL32 = 2e-5
FUSED, UNFUSED = 128, 64

# (n, N, K, nu, amp, seed, coarsest, coarse rule, control region)
CASES = [
    (31, 8, 4, 1e-4, 0.5, 1, 3, "averaged", None),
    (63, 64, 16, 1e-6, 1.0, 2, 3, "averaged", None),
    (63, 256, 32, 1e-6, 1.0, 3, 3, "averaged", None),
    (127, 32, 8, 1e-5, 1.0, 4, 3, "nodal", None),
    (63, 64, 16, 1e-6, 1.0, 2, 3, "averaged", (0.25, 0.75, 0.25, 0.75)),
    (31, 12, 4, 1e-3, 0.8, 7, 7, "averaged", None),
    (15, 6, 3, 1e-3, 0.8, 8, 1, "averaged", None),   # N % 4 != 0: the half-sweeps run
]
IDS = [f"n{c[0]}_N{c[1]}_c{c[6]}_{c[7][:3]}" + ("" if c[8] is None else "_local") for c in CASES]


@pytest.fixture(scope="module")
def cmg():
    from paper_2302_13680_gb300 import build

    build.build()
    import paper_2302_13680_gb300 as P

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return P


@pytest.fixture(scope="module", params=CASES, ids=IDS)
def case(request, cmg):
    n, N, K, nu, amp, seed, coarsest, coarse, box = request.param
    xi = inputs.draw_xi(seed, N, K)
    H = cmg.Hierarchy(n, N, xi, nu, amp, coarsest_n=coarsest, coarse=coarse, control_box=box)
    levels = O.make_hierarchy(n, N, nu, O.sine_mode_field(xi, amp), coarsest_n=coarsest, coarse=coarse,
                              control_box=box)
    yield H, levels
    H.set_tuning(cmg.FP32, None)
    H.close()


def to_dev(v, dtype=torch.float32):
    y, u, p = v
    n = u.shape[0]
    return (torch.tensor(np.asarray(y).reshape(n * n, -1), dtype=dtype, device="cuda").contiguous(),
            torch.tensor(np.asarray(u).reshape(n * n), dtype=dtype, device="cuda").contiguous(),
            torch.tensor(np.asarray(p).reshape(n * n, -1), dtype=dtype, device="cuda").contiguous())


def to_host(v, n):
    y, u, p = (t.double().cpu().numpy() for t in v)
    return y.reshape(n, n, -1), u.reshape(n, n), p.reshape(n, n, -1)


def rand_vec(n, N, seed):
    rng = np.random.default_rng(seed)
    v = (rng.standard_normal((n, n, N)), rng.standard_normal((n, n)), rng.standard_normal((n, n, N)))
    return tuple(np.asarray(b, dtype=np.float32).astype(np.float64) for b in v)


def relerr(got, ref):
    scale = max(np.abs(ref).max(), 1e-300)
    return float(np.abs(np.asarray(got) - np.asarray(ref)).max() / scale)


def equal(a, b):
    return all(torch.equal(s, t) for s, t in zip(a, b))


def targets(H, t):
    return [t] * (H.levels - 1) + [0]


@pytest.mark.parametrize("spl", [1, 2, 4])
@pytest.mark.parametrize("sweeps", [2, 3, 4])
def test_fused_sweeps_equal_half_sweeps(case, spl, sweeps):
    """Sweeps on every grid from random x and f: fused tuning and half-sweep
    tuning with the same chunk target give the same bits."""
    H, levels = case
    import paper_2302_13680_gb300 as P

    opts = P.CycleOptions(precision=P.FP32)
    for l, lv in enumerate(levels[:-1]):
        x0 = rand_vec(lv.n, lv.N, 300 + l)
        f = to_dev(rand_vec(lv.n, lv.N, 350 + l))
        out = []
        for t in (spl, FUSED | spl):
            H.set_tuning(P.FP32, targets(H, t))
            x = to_dev(x0)
            H.smooth(l, opts, sweeps, x, f)
            out.append(x)
        assert equal(*out), (l, lv.n, spl, sweeps)
    H.set_tuning(P.FP32, None)


@pytest.mark.parametrize("spl", [2, 4])
@pytest.mark.parametrize("unfused", [0, UNFUSED])
@pytest.mark.parametrize("n12", [(2, 2), (1, 1), (3, 2)])
def test_fused_cycle_equals_half_sweep_cycle(case, spl, unfused, n12):
    """Whole FP32 V-cycles (coarse grids from zero: the zero-iterate fused
    sweep; the prolongation fused into the first post-smoothing sweep or
    as its own pass), three in a row: the same bits either way."""
    H, levels = case
    import paper_2302_13680_gb300 as P

    lv = levels[0]
    n1, n2 = n12
    opts = P.CycleOptions(precision=P.FP32, n1=n1, n2=n2)
    f = to_dev(rand_vec(lv.n, lv.N, 401))
    out = []
    for t in (spl | unfused, FUSED | spl | unfused):
        H.set_tuning(P.FP32, targets(H, t))
        x = to_dev(rand_vec(lv.n, lv.N, 400))
        for _ in range(3):
            H.cycle(opts, x, f)
        out.append(x)
    H.set_tuning(P.FP32, None)
    assert equal(*out)


def test_fused_pair_matches_oracle(case):
    """Two fused sweeps on every grid against two of the oracle's red-black
    sweeps (FP64) on FP32-representable inputs."""
    H, levels = case
    import paper_2302_13680_gb300 as P

    H.set_tuning(P.FP32, targets(H, FUSED | 4))
    try:
        for l, lv in enumerate(levels[:-1]):
            x = rand_vec(lv.n, lv.N, 500 + l)
            f = rand_vec(lv.n, lv.N, 550 + l)
            fs = tuple(np.asarray(b * s, dtype=np.float32).astype(np.float64) for b, s in zip(f, (lv.c, lv.G, lv.h ** 2)))
            xd = to_dev(x)
            H.smooth(l, P.CycleOptions(precision=P.FP32), 2, xd, to_dev(fs))
            ref = O.rbgs_sweep(lv, O.rbgs_sweep(lv, x, fs), fs)
            for name, g, r in zip("yup", to_host(xd, lv.n), ref):
                assert relerr(g, r) <= TOL32, (l, name, relerr(g, r))
    finally:
        H.set_tuning(P.FP32, None)


def test_fused_refinement_solve_matches_oracle(case):
    """FP64 refinement around FP32 cycles whose sweeps are fused, to the
    paper's relative residual 1e-11: within 1e-9 of the oracle's converged
    solution."""
    H, levels = case
    import paper_2302_13680_gb300 as P

    lv = levels[0]
    f = O.fine_rhs(lv, inputs.target_sinsin(lv.n))
    ref = O.fgmres(levels, f, O.CycleOptions(), tol=1e-12)
    H.set_tuning(P.FP32, targets(H, FUSED | 4))
    try:
        xd = tuple(torch.zeros_like(t) for t in to_dev(f, torch.float64))
        st, _ = H.solve(P.CycleOptions(precision=P.FP32), to_dev(f, torch.float64), xd, method=P.METHOD_CYCLE,
                        tol=1e-11, maxit=80)
        assert st.relres <= 1e-11
        for name, g, r in zip("yup", to_host(xd, lv.n), ref.x):
            assert relerr(g, r) <= 1e-9, (name, relerr(g, r))
    finally:
        H.set_tuning(P.FP32, None)


def test_autotuned_shapes_with_the_fused_flag_added(case):
    """cmg_autotune leaves the fused flag off; adding it to every grid of the
    tuned shapes that it covers gives the same bits in a cycle."""
    H, levels = case
    import paper_2302_13680_gb300 as P

    chosen = H.autotune(P.FP32)
    assert all((t & ~UNFUSED) in (1, 2, 4, 16 | 1, 16 | 2, 32 | 1) for t in chosen[:-1])
    fused = [t | FUSED if (t & (16 | 32)) == 0 and t else t for t in chosen]
    lv = levels[0]
    f = to_dev(rand_vec(lv.n, lv.N, 601))
    out = []
    for tt in (chosen, fused):
        H.set_tuning(P.FP32, tt)
        x = to_dev(rand_vec(lv.n, lv.N, 600))
        H.cycle(P.CycleOptions(precision=P.FP32), x, f)
        out.append(x)
    H.set_tuning(P.FP32, None)
    assert equal(*out)
