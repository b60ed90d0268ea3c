"""Batched solves against single-instance solves and the CPU oracle, in both
forms: the persistent form (instances in lockstep by grid depth, one
persistent launch per depth and leg over a work list of (instance, warp of
nodes) items with grid-wide barriers, or one launch per phase and map
class) and the graph of per-instance branches.  Every instance runs
Algorithm 1's V-cycle with Eq. (13) per node inside FP64 refinement, so its
converged solution is held to the FP64 bar (1e-9) against the oracle's."""
import os

import numpy as np
import pytest
import torch

import inputs
import oracle.cmg_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2302_13680_gb300 import build

    build.build()
    import paper_2302_13680_gb300 as P

    return P


@pytest.fixture(scope="module")
def small(P):
    # sample counts of every map class (N % 4 == 0, N % 2 == 0, odd), three grid sizes
    probs = inputs.batch_problems(seed=40, count=7, sizes=(15, 31, 63), n_range=(5, 70))
    probs.append(inputs.make_problem(n=15, N=6, K=3, nu=1e-3, amp=0.5, seed=3))   # zero right side below
    data = rhs_list(probs)
    yield probs, data


def rhs_list(probs, zero_last=True):
    out = []
    for k, pr in enumerate(probs):
        levels = O.make_hierarchy(pr.n, pr.N, pr.nu, O.sine_mode_field(pr.xi, pr.amp))
        f = O.fine_rhs(levels[0], pr.yd)
        if zero_last and k == len(probs) - 1:
            f = tuple(np.zeros_like(b) for b in f)
        out.append((levels, f))
    return out


def dev(v):
    y, u, p = v
    n = u.shape[0]
    return (torch.tensor(y.reshape(n * n, -1), device="cuda"), torch.tensor(u.reshape(-1), device="cuda"),
            torch.tensor(p.reshape(n * n, -1), device="cuda"))


def host(x, n):
    return (x[0].cpu().numpy().reshape(n, n, -1), x[1].cpu().numpy().reshape(n, n),
            x[2].cpu().numpy().reshape(n, n, -1))


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


FORMS = {"persistent-by-work": (1, -1), "persistent-kernels": (1, 0), "phase-launches": (1, 1), "branches": (2, -1),
         "auto": (0, -1)}


@pytest.mark.parametrize("form", list(FORMS))
def test_batch_matches_single_solves_and_oracle(P, small, form):
    probs, data = small
    B = P.Batch(probs)
    try:
        kind, legs = FORMS[form]
        B.set_form(kind)
        if kind == P.BATCH_PERSISTENT:
            B.set_legs(legs)
        fs = [dev(f) for _, f in data]
        xs = B.zeros()
        opts = P.CycleOptions(precision=P.FP32)
        stats, status = B.solve(opts, fs, xs, tol=1e-10, maxit=80)
        assert status == 0
        assert B.form() == (kind if kind != P.BATCH_AUTO else P.BATCH_BRANCHES)
        for k, ((levels, f), st, x) in enumerate(zip(data, stats, xs)):
            pr = probs[k]
            if k == len(probs) - 1:
                assert st.iters == 0 and all(float(t.abs().max()) == 0.0 for t in x)
                continue
            assert st.relres <= 1e-10
            # the same instance solved alone: the same iterations (within one:
            # the batched kernels sum over samples in another order) and the
            # same solution to the accuracy the tolerance gives
            H = P.Hierarchy(pr.n, pr.N, pr.xi, pr.nu, pr.amp)
            xa = H.zeros(0)
            sa, _ = H.solve(opts, fs[k], xa, tol=1e-10, maxit=80)
            assert abs(sa.iters - st.iters) <= 1, (k, sa.iters, st.iters)
            for a, b in zip(x, xa):
                err = float((a - b).abs().max() / b.abs().max())
                assert err <= (1e-9 if kind == P.BATCH_PERSISTENT else 1e-12), (k, pr.n, pr.N, err)
            H.close()
            # and the oracle's converged solution
            ref = O.fgmres(levels, f, O.CycleOptions(), tol=1e-12)
            for g, r in zip(host(x, pr.n), ref.x):
                assert rel(g, r) <= 1e-9, (k, rel(g, r))
        # second call reuses the captured graph
        xs2 = B.zeros()
        stats2, status = B.solve(opts, fs, xs2, tol=1e-10, maxit=80)
        assert status == 0 and [s.iters for s in stats2] == [s.iters for s in stats]
        for a, b in zip(xs, xs2):
            for s, t in zip(a, b):
                assert torch.equal(s, t)
        # per-instance maxit on the device
        xs3 = B.zeros()
        stats3, status = B.solve(opts, fs, xs3, tol=1e-10, maxit=2, raise_on_fail=False)
        assert status == 4
        assert all(s.iters == 2 for s in stats3[:-1]) and stats3[-1].iters == 0
    finally:
        B.close()


def test_persistent_form_eager_equals_graph(P, small, monkeypatch):
    """With graphs off the persistent form runs the same kernels eagerly
    (one synchronisation per iteration): bit-identical results."""
    probs, data = small
    fs = [dev(f) for _, f in data]
    opts = P.CycleOptions(precision=P.FP32)
    out = []
    for graphs in ("1", "0"):
        monkeypatch.setenv("CMG_GRAPHS", graphs)
        B = P.Batch(probs)
        B.set_form(P.BATCH_PERSISTENT)
        xs = B.zeros()
        stats, status = B.solve(opts, fs, xs, tol=1e-10, maxit=80)
        assert status == 0 and B.form() == P.BATCH_PERSISTENT
        out.append((xs, [s.iters for s in stats]))
        B.close()
    assert out[0][1] == out[1][1]
    for a, b in zip(out[0][0], out[1][0]):
        for s, t in zip(a, b):
            assert torch.equal(s, t)


def test_barrier_wait_limit_ends_the_solve_and_the_batch_stays_usable(P, small):
    """A grid-wide barrier wait limited to one poll runs out (the other CTAs
    are still in their phase): the solve returns CMG_ERR_TIMEOUT; with the
    default limit the same batch then solves normally."""
    probs, data = small
    B = P.Batch(probs)
    try:
        B.set_form(P.BATCH_PERSISTENT)
        B.set_legs(P.BATCH_LEGS_PERSISTENT)
        fs = [dev(f) for _, f in data]
        opts = P.CycleOptions(precision=P.FP32)
        B.set_wait_limit(1)
        xs = B.zeros()
        _, status = B.solve(opts, fs, xs, tol=1e-10, maxit=80, raise_on_fail=False)
        assert status == 6   # CMG_ERR_TIMEOUT
        B.set_wait_limit(0)
        xs = B.zeros()
        stats, status = B.solve(opts, fs, xs, tol=1e-10, maxit=80)
        assert status == 0
        assert all(s.relres <= 1e-10 for s in stats[:-1])
    finally:
        B.close()


def test_persistent_form_with_n255_instances(P):
    """Instances as in the batched workload (n in {63, 127, 255}, N in
    [16, 128], random nu and 8-mode targets), including n = 255 ones, against
    the oracle's converged solutions."""
    probs = [inputs.make_problem(n=255, N=20, K=16, nu=3e-5, amp=1.0, seed=71, target="modes", target_seed=171),
             inputs.make_problem(n=127, N=37, K=16, nu=2e-4, amp=1.0, seed=72, target="modes", target_seed=172),
             inputs.make_problem(n=255, N=18, K=16, nu=1e-6, amp=1.0, seed=73, target="modes", target_seed=173),
             inputs.make_problem(n=63, N=50, K=16, nu=8e-4, amp=1.0, seed=74, target="modes", target_seed=174)]
    data = rhs_list(probs, zero_last=False)
    B = P.Batch(probs)
    try:
        B.set_form(P.BATCH_PERSISTENT)
        fs = [dev(f) for _, f in data]
        xs = B.zeros()
        stats, status = B.solve(P.CycleOptions(precision=P.FP32), fs, xs, tol=1e-10, maxit=80)
        assert status == 0 and B.form() == P.BATCH_PERSISTENT
        for (levels, f), st, x, pr in zip(data, stats, xs, probs):
            assert st.relres <= 1e-10
            ref = O.solve_stationary(levels, f, O.CycleOptions(), tol=1e-10, maxit=60)
            for g, r in zip(host(x, pr.n), ref.x):
                assert rel(g, r) <= 1e-9, (pr.n, pr.N, rel(g, r))
    finally:
        B.close()
