"""Error paths of the C ABI on the GPU: each returns a status, leaves the
handle usable, and never faults the device (the failures are made on the
host side of the call: bad arguments, a non-finite right side, too few
iterations)."""
import numpy as np
import pytest
import torch

import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_2302_13680_gb300 import build

    build.build()
    import paper_2302_13680_gb300 as P

    pr = inputs.make_problem(**inputs.CONFIGS["n31_N8"])
    h = P.Hierarchy(pr.n, pr.N, pr.xi, pr.nu, pr.amp)
    yield h, P, pr
    h.close()


def rhs(h, pr):
    yd = torch.tensor(pr.yd.reshape(-1), dtype=torch.float64, device="cuda")
    return h.rhs(yd)


def test_not_converged_then_usable(H):
    h, P, pr = H
    f = rhs(h, pr)
    x = h.zeros(0)
    st, status = h.solve(P.CycleOptions(), f, x, maxit=1, raise_on_fail=False)
    assert status == 4 and st.iters == 1
    st, status = h.solve(P.CycleOptions(), f, x, maxit=50)
    assert status == 0 and st.relres <= 1e-10


def test_nonfinite_rhs_reported(H):
    h, P, pr = H
    f = rhs(h, pr)
    f[0][5, 3] = float("nan")
    x = h.zeros(0)
    st, status = h.solve(P.CycleOptions(), f, x, raise_on_fail=False)
    assert status == 5
    f = rhs(h, pr)
    st, status = h.solve(P.CycleOptions(), f, x, maxit=50)
    assert status == 0


def test_invalid_arguments(H):
    h, P, pr = H
    f = rhs(h, pr)
    x = h.zeros(0)
    r = h.zeros(0)
    with pytest.raises(P.CMGError) as e:
        h.residual(h.levels, x, f, r)
    assert e.value.status == 1
    for bad in (lambda: h.solve(P.CycleOptions(gamma=3), f, x),
                lambda: h.solve(P.CycleOptions(smoother=P.SMOOTH_JACOBI, theta=0.0), f, x),
                lambda: h.solve(P.CycleOptions(), f, x, method=P.METHOD_FGMRES, restart=0),
                lambda: h.cycle(P.CycleOptions(precision=P.FP32), x, f)):     # FP64 vectors, FP32 cycle
        with pytest.raises(P.CMGError) as e:
            bad()
        assert e.value.status == 1
    with pytest.raises(TypeError):
        h.residual(0, tuple(t.float() for t in x), f, r)       # mixed dtypes
    st, status = h.solve(P.CycleOptions(), f, x, maxit=50)
    assert status == 0


def test_zero_rhs_gives_zero(H):
    h, P, pr = H
    f = h.zeros(0)
    x = tuple(torch.ones_like(t) for t in h.zeros(0))
    st, status = h.solve(P.CycleOptions(), f, x)
    assert status == 0
    assert all(float(t.abs().max()) == 0.0 for t in x)


def test_set_samples_recomputes_coefficients(H):
    """New field draws through the device entry point give the same operator
    as a fresh hierarchy built from them."""
    h, P, pr = H
    xi2 = inputs.draw_xi(99, pr.N, pr.K)
    h2 = P.Hierarchy(pr.n, pr.N, xi2, pr.nu, pr.amp)
    rng = np.random.default_rng(1)
    x = tuple(torch.tensor(rng.standard_normal(t.shape), device="cuda") for t in h.zeros(0))
    r1, r2 = h.zeros(0), h2.zeros(0)
    h.set_samples(torch.tensor(xi2, device="cuda"))
    h.residual(0, x, None, r1)
    h2.residual(0, x, None, r2)
    torch.cuda.synchronize()
    for a, b in zip(r1, r2):
        assert torch.equal(a, b)
    h.set_samples(torch.tensor(pr.xi, device="cuda"))
    h2.close()


def test_graph_refinement_matches_eager_and_respects_maxit(H):
    """The FP32 refinement loop runs as a captured graph with a device-side
    while node; with a profiling window open it runs eagerly instead.  Both
    enqueue the same kernels in the same order, so iterates and counts agree."""
    h, P, pr = H
    f = rhs(h, pr)
    opts = P.CycleOptions(precision=P.FP32)
    xg = h.zeros(0)
    st_g, status = h.solve(opts, f, xg)
    assert status == 0 and st_g.relres <= 1e-10
    xe = h.zeros(0)
    h.profile_begin(1, 0)
    st_e, status = h.solve(opts, f, xe)
    h.profile_end()
    assert status == 0
    assert st_e.iters == st_g.iters
    for a, b in zip(xg, xe):
        assert torch.equal(a, b)
    # second graph solve from the same buffers reuses the captured graph
    for t in xg:
        t.zero_()
    st_2, status = h.solve(opts, f, xg)
    assert status == 0 and st_2.iters == st_g.iters
    for a, b in zip(xg, xe):
        assert torch.equal(a, b)
    # the device loop stops at maxit
    for t in xg:
        t.zero_()
    st_1, status = h.solve(opts, f, xg, maxit=2, raise_on_fail=False)
    assert status == 4 and st_1.iters == 2


def test_graphs_disabled_by_environment(H, monkeypatch):
    """CMG_GRAPHS=0 at creation runs the same refinement loop eagerly:
    same iterate, same cycle count, one host round trip per cycle."""
    h, P, pr = H
    f = rhs(h, pr)
    opts = P.CycleOptions(precision=P.FP32)
    xg = h.zeros(0)
    st_g, _ = h.solve(opts, f, xg)
    monkeypatch.setenv("CMG_GRAPHS", "0")
    h2 = P.Hierarchy(pr.n, pr.N, pr.xi, pr.nu, pr.amp)
    try:
        xe = h2.zeros(0)
        from paper_2302_13680_gb300.cmg import kernel_launches
        k0 = kernel_launches()
        st_e, status = h2.solve(opts, h2.rhs(torch.tensor(pr.yd.reshape(-1), dtype=torch.float64, device="cuda")), xe)
        assert status == 0 and st_e.iters == st_g.iters
        assert kernel_launches() > k0
        for a, b in zip(xg, xe):
            assert torch.equal(a, b)
    finally:
        h2.close()


def test_autotune_keeps_results_and_validates(H, tmp_path):
    h, P, pr = H
    from paper_2302_13680_gb300 import tuning

    f = rhs(h, pr)
    opts = P.CycleOptions(precision=P.FP32)
    x0 = h.zeros(0)
    st0, _ = h.solve(opts, f, x0)
    chosen = tuning.apply_or_tune(h, P.FP32, str(tmp_path / "tune.json"))
    assert len(chosen) == h.levels and chosen[-1] == 0
    # 16: staged sweep, 32: wide layout, 64: prolongation in its own pass
    assert all((t & ~64) in (1, 2, 4, 16 | 1, 16 | 2, 32 | 1) for t in chosen[:-1])
    again = tuning.apply_or_tune(h, P.FP32, str(tmp_path / "tune.json"))   # from the cache
    assert again == chosen
    x1 = h.zeros(0)
    st1, _ = h.solve(opts, f, x1)
    assert st1.iters == st0.iters
    for a, b in zip(x0, x1):
        assert float((a - b).abs().max() / b.abs().max()) <= 1e-12
    with pytest.raises(P.CMGError):
        h.set_tuning(P.FP32, [3] * h.levels)
    h.set_tuning(P.FP32, None)


def test_set_tuning_validates_targets(H):
    h, P, pr = H
    L = h.levels
    for prec, targets in ((P.FP32, [16 | 4]),        # staged sweep takes 1 or 2 chunks per lane
                          (P.FP64, [16 | 1]),        # FP32 only
                          (P.FP32, [3]),
                          (P.FP32, [32 | 2]),        # wide layout: one chunk per lane
                          (P.FP32, [32 | 16 | 1]),   # not with the staged sweep
                          (P.FP64, [32 | 1])):       # FP32 only
        with pytest.raises(P.CMGError) as e:
            h.set_tuning(prec, targets + [0] * (L - 1))
        assert e.value.status == 1
    h.set_tuning(P.FP32, [16 | 2] + [0] * (L - 1))
    h.set_tuning(P.FP32, [32 | 1] * (L - 1) + [0])
    h.set_tuning(P.FP32, None)


def test_misaligned_vector_is_refused(H):
    """Node kernels move 16-byte vectors; a pointer off a 16-byte boundary
    is refused with an argument error instead of reaching the device."""
    h, P, pr = H
    import ctypes
    from paper_2302_13680_gb300.cmg import load_library

    lib = load_library()
    m = h.level_n[0] ** 2
    buf = torch.zeros(m * h.N + 4, dtype=torch.float64, device="cuda")
    u = torch.zeros(m, dtype=torch.float64, device="cuda")
    p = torch.zeros(m * h.N, dtype=torch.float64, device="cuda")
    out = ctypes.c_double()
    ptr = lambda t, off=0: ctypes.c_void_p(t.data_ptr() + off)
    st = lib.cmg_norm(h._h, 0, ptr(buf, 8), ptr(u), ptr(p), ctypes.byref(out))
    assert st == 1
    st = lib.cmg_norm(h._h, 0, ptr(buf), ptr(u), ptr(p), ctypes.byref(out))
    assert st == 0


def test_refinement_reports_a_true_residual(H):
    """FP32 refinement updates its residual recursively in FP32 between FP64
    anchors; the solve must still stop on, and report, a true FP64 residual
    of the returned iterate in the paper's row scaling (state rows times N)."""
    h, P, pr = H
    f = rhs(h, pr)
    for graphs in ("1", "0"):
        import os
        os.environ["CMG_GRAPHS"] = graphs
        h2 = P.Hierarchy(pr.n, pr.N, pr.xi, pr.nu, pr.amp)
        try:
            x = h2.zeros(0)
            st, status = h2.solve(P.CycleOptions(precision=P.FP32), f, x, tol=1e-10)
            assert status == 0
            r = h2.zeros(0)
            h2.residual(0, x, f, r)
            w = float(pr.N)
            num = torch.sqrt((w * r[0]).square().sum() + r[1].square().sum() + r[2].square().sum())
            den = torch.sqrt((w * f[0]).square().sum() + f[1].square().sum() + f[2].square().sum())
            true_rel = float(num / den)
            assert true_rel <= 1e-10
            assert abs(true_rel - st.relres) <= 1e-3 * st.relres
        finally:
            os.environ.pop("CMG_GRAPHS", None)
            h2.close()


def test_new_samples_rebuild_fp64_and_fp32_operators(H):
    """After cmg_set_samples the FP32 operators are rebuilt at once and the
    FP64 coarse operators on first FP64 use: both precisions then agree bit
    for bit with a handle created with the new samples."""
    h, P, pr = H
    spec = dict(inputs.CONFIGS["n31_N8"])
    spec["seed"] = 11
    pr2 = inputs.make_problem(**spec)
    fresh = P.Hierarchy(pr2.n, pr2.N, pr2.xi, pr2.nu, pr2.amp)
    try:
        h.set_samples(torch.tensor(pr2.xi, device="cuda"))
        yd = torch.tensor(pr2.yd.reshape(-1), dtype=torch.float64, device="cuda")
        for hh in (h, fresh):
            hh.f = hh.rhs(yd)
        outs = []
        for hh in (h, fresh):
            x32 = hh.zeros(0, torch.float32)
            hh.cycle(P.CycleOptions(precision=P.FP32), x32, tuple(t.float() for t in hh.f))
            x64 = hh.zeros(0)
            hh.cycle(P.CycleOptions(), x64, hh.f)
            xs = hh.zeros(0)
            st, status = hh.solve(P.CycleOptions(precision=P.FP32), hh.f, xs)
            assert status == 0
            outs.append((x32, x64, xs))
        for a, b in zip(*outs):
            for ta, tb in zip(a, b):
                assert torch.equal(ta, tb)
    finally:
        h.set_samples(torch.tensor(pr.xi, device="cuda"))
        fresh.close()


@pytest.mark.parametrize("precision,method,gamma", [("FP32", "METHOD_CYCLE", 1), ("FP32", "METHOD_CYCLE", 2),
                                                    ("FP32", "METHOD_FGMRES", 1), ("FP64", "METHOD_FGMRES", 1),
                                                    ("FP64", "METHOD_CYCLE", 2)])
def test_solve_does_not_read_stale_work_buffers(H, precision, method, gamma):
    """Corrections and coarse iterates start from zero without their memory
    being cleared (the first colour-0 half-sweep does not read them): a solve
    on a handle whose work buffers hold another solve's values must return
    bit for bit what a fresh handle returns."""
    h, P, pr = H
    f = rhs(h, pr)
    g = tuple(t.clone() for t in f)
    g[0].mul_(-3.0).add_(1e-3)
    opts = P.CycleOptions(precision=getattr(P, precision), gamma=gamma)
    m = getattr(P, method)
    h1 = P.Hierarchy(pr.n, pr.N, pr.xi, pr.nu, pr.amp)
    h2 = P.Hierarchy(pr.n, pr.N, pr.xi, pr.nu, pr.amp)
    try:
        x0 = h1.zeros(0)
        h1.solve(opts, g, x0, method=m, tol=1e-10)   # leaves its corrections in the work buffers
        x1, x2 = h1.zeros(0), h2.zeros(0)
        s1, _ = h1.solve(opts, f, x1, method=m, tol=1e-10)
        s2, _ = h2.solve(opts, f, x2, method=m, tol=1e-10)
        assert s1.iters == s2.iters
        for a, b in zip(x1, x2):
            assert torch.equal(a, b)
    finally:
        h1.close()
        h2.close()


@pytest.mark.parametrize("drop,amax", [("0.5", "1"), ("1e-2", "5"), ("1e-6", "1000")])
def test_refinement_anchor_policy_overrides(H, drop, amax):
    """CMG_ANCHOR_DROP / CMG_ANCHOR_MAX change only when the FP64 anchors are
    taken: from an anchor every cycle to anchors only at the tolerance, the
    solve stops on a true residual below the tolerance."""
    import os

    h, P, pr = H
    f = rhs(h, pr)
    os.environ["CMG_ANCHOR_DROP"], os.environ["CMG_ANCHOR_MAX"] = drop, amax
    try:
        h2 = P.Hierarchy(pr.n, pr.N, pr.xi, pr.nu, pr.amp)
    finally:
        os.environ.pop("CMG_ANCHOR_DROP", None)
        os.environ.pop("CMG_ANCHOR_MAX", None)
    try:
        x = h2.zeros(0)
        st, status = h2.solve(P.CycleOptions(precision=P.FP32), f, x, tol=1e-10, maxit=60)
        assert status == 0
        r = h2.zeros(0)
        h2.residual(0, x, f, r)
        w = float(pr.N)
        num = torch.sqrt((w * r[0]).square().sum() + r[1].square().sum() + r[2].square().sum())
        den = torch.sqrt((w * f[0]).square().sum() + f[1].square().sum() + f[2].square().sum())
        assert float(num / den) <= 1e-10
        assert abs(float(num / den) - st.relres) <= 1e-3 * st.relres
    finally:
        h2.close()
