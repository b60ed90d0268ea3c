"""Semismooth Newton for the L1 + box problem (Sec. 4, Algorithm 2) on the
GPU against the oracle's Algorithm 2: the same Newton steps, the same
control, the merit below the tolerance; afterwards the handle solves the
linear-quadratic problem exactly as before."""
import numpy as np
import pytest
import torch

import inputs
import oracle.cmg_oracle as O

pytestmark = pytest.mark.gpu

# (n, N, K, nu, amp, seed, beta, a, b, target scale): a solution with zero,
# interior and bound-active controls, and a ragged sample count
CASES = [
    (15, 4, 3, 1e-3, 0.6, 3, 1e-3, -1.0, 1.0, 0.03),
    (31, 5, 4, 1e-3, 0.5, 4, 5e-4, -0.5, 0.8, 0.02),
]


@pytest.fixture(scope="module")
def P():
    from paper_2302_13680_gb300 import build

    build.build()
    import paper_2302_13680_gb300 as P

    return P


@pytest.mark.parametrize("case", CASES, ids=[f"n{c[0]}_N{c[1]}" for c in CASES])
@pytest.mark.parametrize("form", ["fp64-cycle", "fp64-fgmres", "fp32-ir"])
def test_semismooth_newton_matches_oracle(P, case, form):
    n, N, K, nu, amp, seed, beta, a, b, scale = case
    xi = inputs.draw_xi(seed, N, K)
    levels = O.make_hierarchy(n, N, nu, O.sine_mode_field(xi, amp))
    yd = inputs.target_modes(n, seed) * scale
    ref = O.semismooth_newton(levels, yd, beta, a, b)
    assert ref.merit[-1] < 1e-9
    H = P.Hierarchy(n, N, xi, nu, amp)
    try:
        prec = P.FP32 if form == "fp32-ir" else P.FP64
        method = P.METHOD_FGMRES if form == "fp64-fgmres" else P.METHOD_CYCLE
        # a linear-quadratic solve first: its captured refinement loop must not
        # be reused for the Newton systems (their control row differs)
        f = H.rhs(torch.tensor(inputs.target_sinsin(n).reshape(-1), device="cuda"))
        H.solve(P.CycleOptions(precision=prec), f, H.zeros(0), tol=1e-10)
        u = torch.zeros(n * n, dtype=torch.float64, device="cuda")
        ydd = torch.tensor(yd.reshape(-1), dtype=torch.float64, device="cuda")
        st, status, y, p = H.ssn_solve(P.CycleOptions(precision=prec), ydd, u, beta, a, b, method=method)
        assert status == 0 and st.merit <= 1e-9
        assert abs(st.newton - ref.newton) <= (1 if form == "fp32-ir" else 0)
        got = u.cpu().numpy().reshape(n, n)
        scale_u = np.abs(ref.u).max()
        assert np.abs(got - ref.u).max() <= 1e-7 * scale_u
        # the zero / bound pattern is the same (each up to the rounding of the
        # decoupled control rows)
        tiny = 1e-12 * scale_u
        assert np.array_equal(np.abs(got) <= tiny, np.abs(ref.u) <= tiny)
        at_bound = lambda v: (np.abs(v - a) <= tiny) | (np.abs(v - b) <= tiny)
        assert np.array_equal(at_bound(got), at_bound(ref.u))
        # states: y_j = A_j^-1 M u, p_j = A_j^-1 (M/N)(y_d - y_j) for the returned control
        yr, pr = O.pde_states(levels, got, yd)
        assert np.abs(y.cpu().numpy() - yr.reshape(n * n, N)).max() <= 1e-6 * np.abs(yr).max()
        assert np.abs(p.cpu().numpy() - pr.reshape(n * n, N)).max() <= 1e-6 * np.abs(pr).max()
    finally:
        H.close()


def test_operators_restored_after_semismooth_newton(P):
    n, N, K, nu, amp, seed, beta, a, b, scale = CASES[0]
    xi = inputs.draw_xi(seed, N, K)
    H = P.Hierarchy(n, N, xi, nu, amp)
    try:
        f = H.rhs(torch.tensor(inputs.target_sinsin(n).reshape(-1), device="cuda"))
        outs = []
        for k in range(2):
            if k == 1:
                u = torch.zeros(n * n, dtype=torch.float64, device="cuda")
                yd = torch.tensor((inputs.target_modes(n, 3) * scale).reshape(-1), device="cuda")
                H.ssn_solve(P.CycleOptions(), yd, u, beta, a, b)
            for prec in (P.FP64, P.FP32):
                x = H.zeros(0)
                H.solve(P.CycleOptions(precision=prec), f, x, tol=1e-10)
                outs.append([t.clone() for t in x])
        for before, after in zip(outs[:2], outs[2:]):
            for s, t in zip(before, after):
                assert torch.equal(s, t)
    finally:
        H.close()


def test_semismooth_newton_rejects_bad_arguments(P):
    n, N, K, nu, amp, seed = 15, 2, 2, 1e-3, 0.5, 1
    H = P.Hierarchy(n, N, inputs.draw_xi(seed, N, K), nu, amp)
    try:
        u = torch.zeros(n * n, dtype=torch.float64, device="cuda")
        yd = torch.zeros(n * n, dtype=torch.float64, device="cuda")
        for beta, a, b in ((1e-3, 0.5, 1.0), (1e-3, -1.0, -0.5), (-1.0, -1.0, 1.0)):
            st, status, _, _ = H.ssn_solve(P.CycleOptions(), yd, u, beta, a, b, raise_on_fail=False)
            assert status == 1
        st, status, _, _ = H.ssn_solve(P.CycleOptions(freeze_u=1), yd, u, 1e-3, -1.0, 1.0, raise_on_fail=False)
        assert status == 1
    finally:
        H.close()
