"""The red-black half-sweep with its operands gathered by TMA tensor loads
(CMG_TUNE_TMA, csrc/cmg_tma_sweep.cu) against the direct half-sweep and the
CPU oracle, through the C ABI.

A task is a segment of one colour's nodes in a grid row; one producer
thread per CTA loads boxes that take every other node (the segment's right
sides, the rows above and below, the left/right neighbours, the faces) into
a ring of shared-memory stages, with the neighbours outside the grid as the
loads' zero fill; consumer warps run rbgs_node's arithmetic on them with its
sample map, so every result here must equal the direct half-sweep's bit for
bit: sweeps on every grid with 1, 2 and 4 chunks per lane (ragged last
segments, odd and even rows), whole V- and W-cycles (the zero-iterate and
prolongation sweeps stay direct), local control, a sample count of 256 in
the large workload's shape, and N % 4 != 0 (the flag is ignored).  FP64
refinement with these cycles converges to the oracle's solution within
1e-9, and no bounded wait of the kernel runs out.
"""
import ctypes

import numpy as np
import pytest
import torch

import inputs
import oracle.cmg_oracle as O

pytestmark = pytest.mark.gpu

TMA, UNFUSED = 256, 64

# (n, N, K, nu, amp, seed, coarsest, coarse rule, control region)
CASES = [
    (31, 8, 4, 1e-4, 0.5, 1, 3, "averaged", None),
    (63, 64, 16, 1e-6, 1.0, 2, 3, "averaged", None),
    (63, 256, 32, 1e-6, 1.0, 3, 3, "averaged", None),
    (127, 32, 8, 1e-5, 1.0, 4, 3, "nodal", None),
    (63, 64, 16, 1e-6, 1.0, 2, 3, "averaged", (0.25, 0.75, 0.25, 0.75)),
    (31, 12, 4, 1e-3, 0.8, 7, 7, "averaged", None),
    (15, 6, 3, 1e-3, 0.8, 8, 1, "averaged", None),   # N % 4 != 0: the direct kernel runs
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
@pytest.mark.parametrize("sweeps", [1, 3])
def test_tma_sweeps_equal_direct_sweeps(case, spl, sweeps):
    """Sweeps on every grid from random x and f: the TMA-gathered and the
    direct half-sweeps with the same chunks per lane give the same bits."""
    H, levels = case
    import paper_2302_13680_gb300 as P

    opts = P.CycleOptions(precision=P.FP32)
    for l, lv in enumerate(levels[:-1]):
        x0 = rand_vec(lv.n, lv.N, 300 + l)
        f = to_dev(rand_vec(lv.n, lv.N, 350 + l))
        out = []
        for t in (spl, TMA | spl):
            H.set_tuning(P.FP32, targets(H, t))
            x = to_dev(x0)
            H.smooth(l, opts, sweeps, x, f)
            out.append(x)
        assert equal(*out), (l, lv.n, spl, sweeps)
    H.set_tuning(P.FP32, None)


@pytest.mark.parametrize("spl", [2, 4])
@pytest.mark.parametrize("unfused", [0, UNFUSED])
@pytest.mark.parametrize("gamma", [1, 2])
def test_tma_cycles_equal_direct_cycles(case, spl, unfused, gamma):
    """Whole FP32 cycles, three in a row, V and W: the same bits with the
    TMA-gathered half-sweeps on every grid as with the direct ones."""
    H, levels = case
    import paper_2302_13680_gb300 as P

    lv = levels[0]
    opts = P.CycleOptions(precision=P.FP32, gamma=gamma, n1=2 if gamma == 1 else 1, n2=2 if gamma == 1 else 1)
    f = to_dev(rand_vec(lv.n, lv.N, 401))
    out = []
    for t in (spl | unfused, TMA | spl | unfused):
        H.set_tuning(P.FP32, targets(H, t))
        x = to_dev(rand_vec(lv.n, lv.N, 400))
        for _ in range(3):
            H.cycle(opts, x, f)
        out.append(x)
    H.set_tuning(P.FP32, None)
    assert equal(*out)


def test_tma_sweep_pair_matches_oracle(case):
    """Two TMA-gathered sweeps on every grid against two of the oracle's
    red-black sweeps (FP64) on FP32-representable inputs (the FP32 bar of
    the other parity tests, 2e-5)."""
    H, levels = case
    import paper_2302_13680_gb300 as P

    H.set_tuning(P.FP32, targets(H, TMA | 4))
    try:
        for l, lv in enumerate(levels[:-1]):
            x = rand_vec(lv.n, lv.N, 500 + l)
            f = rand_vec(lv.n, lv.N, 550 + l)
            fs = tuple(np.asarray(b * s, dtype=np.float32).astype(np.float64) for b, s in zip(f, (lv.c, lv.G, lv.h ** 2)))
            xd = to_dev(x)
            H.smooth(l, P.CycleOptions(precision=P.FP32), 2, xd, to_dev(fs))
            ref = O.rbgs_sweep(lv, O.rbgs_sweep(lv, x, fs), fs)
            for name, g, r in zip("yup", to_host(xd, lv.n), ref):
                assert relerr(g, r) <= 2e-5, (l, name, relerr(g, r))
    finally:
        H.set_tuning(P.FP32, None)


def test_tma_refinement_solve_matches_oracle(case):
    """FP64 refinement around FP32 cycles with TMA-gathered half-sweeps, to
    the paper's relative residual 1e-11: within 1e-9 of the oracle's
    converged solution."""
    H, levels = case
    import paper_2302_13680_gb300 as P

    lv = levels[0]
    f = O.fine_rhs(lv, inputs.target_sinsin(lv.n))
    ref = O.fgmres(levels, f, O.CycleOptions(), tol=1e-12)
    H.set_tuning(P.FP32, targets(H, TMA | 4))
    try:
        xd = tuple(torch.zeros_like(t) for t in to_dev(f, torch.float64))
        st, _ = H.solve(P.CycleOptions(precision=P.FP32), to_dev(f, torch.float64), xd, method=P.METHOD_CYCLE,
                        tol=1e-11, maxit=80)
        assert st.relres <= 1e-11
        for name, g, r in zip("yup", to_host(xd, lv.n), ref.x):
            assert relerr(g, r) <= 1e-9, (name, relerr(g, r))
    finally:
        H.set_tuning(P.FP32, None)


def test_tma_rejected_where_not_allowed(cmg):
    """FP64 targets take no flag; the flag needs 1, 2 or 4 chunks and no
    other layout flag."""
    xi = inputs.draw_xi(1, 8, 4)
    H = cmg.Hierarchy(15, 8, xi, 1e-3, 0.8)
    try:
        for prec, t in ((cmg.FP64, TMA | 1), (cmg.FP32, TMA), (cmg.FP32, TMA | 16 | 1), (cmg.FP32, TMA | 32 | 1),
                        (cmg.FP32, TMA | 128 | 1)):
            with pytest.raises(cmg.CMGError):
                H.set_tuning(prec, [t] * (H.levels - 1) + [0])
        H.set_tuning(cmg.FP32, [TMA | UNFUSED | 2] * (H.levels - 1) + [0])
    finally:
        H.close()


def test_no_tma_wait_ran_out(cmg):
    """Every bounded wait of the TMA-gathered sweeps above completed."""
    lib = cmg.load_library()
    count = ctypes.c_uint(123)
    assert lib.cmg_sweep_wait_timeouts(ctypes.byref(count)) == 0
    assert count.value == 0
    assert lib.cmg_sweep_wait_timeouts(None) == 1
