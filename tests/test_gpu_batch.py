"""Batched solves (one graph launch, per-instance device-side loops) against
single-instance solves and the CPU oracle."""
import numpy as np
import pytest
import torch

import inputs
import oracle.cmg_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    from paper_2302_13680_gb300 import build

    build.build()
    import paper_2302_13680_gb300 as P

    probs = inputs.batch_problems(seed=40, count=7, sizes=(15, 31, 63), n_range=(5, 70))
    probs.append(inputs.make_problem(n=15, N=6, K=3, nu=1e-3, amp=0.5, seed=3))   # zero right side below
    B = P.Batch(probs)
    yield B, probs, P
    B.close()


def rhs_list(probs):
    out = []
    for k, pr in enumerate(probs):
        levels = O.make_hierarchy(pr.n, pr.N, pr.nu, O.sine_mode_field(pr.xi, pr.amp))
        f = O.fine_rhs(levels[0], pr.yd)
        if k == len(probs) - 1:
            f = tuple(np.zeros_like(b) for b in f)
        out.append((levels, f))
    return out


def dev(v):
    y, u, p = v
    n = u.shape[0]
    return (torch.tensor(y.reshape(n * n, -1), device="cuda"), torch.tensor(u.reshape(-1), device="cuda"),
            torch.tensor(p.reshape(n * n, -1), device="cuda"))


def test_batch_matches_single_solves_and_oracle(batch):
    B, probs, P = batch
    data = rhs_list(probs)
    fs = [dev(f) for _, f in data]
    xs = B.zeros()
    opts = P.CycleOptions(precision=P.FP32)
    stats, status = B.solve(opts, fs, xs, tol=1e-10, maxit=80)
    assert status == 0
    for k, ((levels, f), st, x) in enumerate(zip(data, stats, xs)):
        pr = probs[k]
        if k == len(probs) - 1:
            assert st.iters == 0 and all(float(t.abs().max()) == 0.0 for t in x)
            continue
        assert st.relres <= 1e-10
        # the same instance solved alone (single-instance graph): the same
        # iterations and the same iterate up to rounding
        H = P.Hierarchy(pr.n, pr.N, pr.xi, pr.nu, pr.amp)
        xa = H.zeros(0)
        sa, _ = H.solve(opts, fs[k], xa, tol=1e-10, maxit=80)
        assert sa.iters == st.iters
        for a, b in zip(x, xa):
            err = float((a - b).abs().max() / b.abs().max())
            assert err <= 1e-12, (k, pr.n, pr.N, err)
        H.close()
        # and the oracle's converged solution
        ref = O.fgmres(levels, f, O.CycleOptions(), tol=1e-12)
        n = pr.n
        got = (x[0].cpu().numpy().reshape(n, n, -1), x[1].cpu().numpy().reshape(n, n),
               x[2].cpu().numpy().reshape(n, n, -1))
        for g, r in zip(got, ref.x):
            assert np.abs(g - r).max() <= 1e-6 * np.abs(r).max()
    # second call reuses the captured graph
    xs2 = B.zeros()
    stats2, status = B.solve(opts, fs, xs2, tol=1e-10, maxit=80)
    assert status == 0 and [s.iters for s in stats2] == [s.iters for s in stats]
    # per-instance maxit inside the graph
    xs3 = B.zeros()
    stats3, status = B.solve(opts, fs, xs3, tol=1e-10, maxit=2, raise_on_fail=False)
    assert status == 4
    assert all(s.iters == 2 for s in stats3[:-1]) and stats3[-1].iters == 0
