"""Neumann boundary control on (0,1) x {0} (Sec. 2's control operator as a
Neumann condition; the boundary-control test case of Sec. 3.2) on the GPU,
through the C ABI (cmg_bnd_*), against the sparse-matrix oracle
(oracle/boundary.py): residual and operator on every grid, one damped
collective Jacobi sweep (Eq. (11), Eq. (13) on Gamma, Eq. (14) elsewhere) on
every grid, the transfers, the coarsest solve, V- and W-cycle iterates and
the converged solution.  FP64 bar: 1e-12 for single kernels and sweeps
(relative max-norm per block), cycles within 1e-11, converged solutions
within 1e-9 of the oracle's."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

import inputs
import oracle.boundary as Bd
import oracle.cmg_oracle as O

pytestmark = pytest.mark.gpu

# (n, N, K, nu, amp, seed, coarsest): ragged sample counts, both coarsest
# sizes (7: the paper's three grids at n = 31), nu from 1e-2 to 1e-6
CASES = [(15, 4, 3, 1e-3, 0.8, 7, 3), (31, 5, 4, 1e-4, 1.0, 8, 3), (15, 3, 2, 1e-2, 0.5, 9, 7),
         (31, 27, 4, 1e-6, 1.0, 10, 7)]
IDS = [f"n{c[0]}_N{c[1]}_c{c[6]}" for c in CASES]


@pytest.fixture(scope="module", params=CASES, ids=IDS)
def case(request):
    from paper_2302_13680_gb300 import build

    build.build()
    import paper_2302_13680_gb300 as P

    n, N, K, nu, amp, seed, coarsest = request.param
    xi = inputs.draw_xi(seed, N, K)
    H = P.BoundaryHierarchy(n, N, xi, nu, amp, coarsest_n=coarsest)
    ns, S = Bd.hierarchy(n, N, nu, O.sine_mode_field(xi, amp), coarsest_n=coarsest)
    yield H, ns, S, N
    H.close()


def split(z, n, N):
    m = (n + 1) * n
    return z[: m * N].reshape(m, N), z[m * N: m * N + n], z[m * N + n:].reshape(m, N)


def to_dev(z, n, N):
    return tuple(torch.tensor(np.ascontiguousarray(b), dtype=torch.float64, device="cuda") for b in split(z, n, N))


def to_host(v):
    return np.concatenate([t.cpu().numpy().ravel() for t in v])


def check(got, ref, n, N, tol, what):
    for name, g, r in zip("yup", split(got, n, N), split(ref, n, N)):
        e = float(np.abs(g - r).max() / max(np.abs(r).max(), 1e-300))
        assert e <= tol, f"{what} block {name}: rel err {e:.3e} > {tol:.1e}"


def rand(S, seed):
    return np.random.default_rng(seed).standard_normal(S.shape[0])


def test_grids(case):
    H, ns, S, N = case
    assert H.level_n == ns


def test_residual_and_operator_every_grid(case):
    H, ns, S, N = case
    for l, (n, Sl) in enumerate(zip(ns, S)):
        z, f = rand(Sl, 10 + l), rand(Sl, 20 + l)
        r = H.zeros(l)
        H.residual(l, to_dev(z, n, N), to_dev(f, n, N), r)
        check(to_host(r), f - Sl @ z, n, N, 1e-12, f"residual grid {l}")
        H.residual(l, to_dev(z, n, N), None, r)
        check(to_host(r), Sl @ z, n, N, 1e-12, f"operator grid {l}")


@pytest.mark.parametrize("theta", [0.5, 1.0])
def test_jacobi_sweep_every_grid(case, theta):
    H, ns, S, N = case
    for l, (n, Sl) in enumerate(zip(ns, S)):
        z, f = rand(Sl, 30 + l), rand(Sl, 40 + l)
        x = to_dev(z, n, N)
        H.smooth(l, theta, 1, x, to_dev(f, n, N))
        check(to_host(x), Bd.jacobi_sweep(Sl, n, N, z, f, theta), n, N, 1e-12, f"sweep grid {l}")


def test_transfers(case):
    H, ns, S, N = case
    for l in range(len(ns) - 1):
        n, nc = ns[l], ns[l + 1]
        Pm = Bd.prolongation_matrix(n, N)
        r = rand(S[l], 50 + l)
        c = H.zeros(l + 1)
        H.restrict(l, to_dev(r, n, N), c)
        check(to_host(c), Pm.T @ r, nc, N, 1e-13, f"restriction {l}")
        e, z = rand(S[l + 1], 60 + l), rand(S[l], 70 + l)
        x = to_dev(z, n, N)
        H.prolong_add(l, to_dev(e, nc, N), x)
        check(to_host(x), z + Pm @ e, n, N, 1e-13, f"prolongation {l}")


def test_coarsest_solve(case):
    H, ns, S, N = case
    n = ns[-1]
    f = rand(S[-1], 80)
    x = H.zeros(len(ns) - 1)
    H.coarse_solve(to_dev(f, n, N), x)
    check(to_host(x), spla.spsolve(S[-1].tocsc(), f), n, N, 1e-11, "coarsest solve")


@pytest.mark.parametrize("gamma", [1, 2])
def test_cycle_iterates(case, gamma):
    H, ns, S, N = case
    n = ns[0]
    f = rand(S[0], 90)
    z = np.zeros_like(f)
    x = H.zeros(0)
    fd = to_dev(f, n, N)
    for k in range(2):
        H.cycle(x, fd, theta=0.5, n1=2, n2=2, gamma=gamma)
        z = Bd.cycle(S, ns, N, 0, z, f, n1=2, n2=2, theta=0.5, gamma=gamma)
        check(to_host(x), z, n, N, 1e-11, f"cycle {k}")


def test_converged_solution(case):
    """Cycles to the paper's relative residual 1e-10: the same cycle count
    as the oracle within one, and its converged solution within 1e-9."""
    H, ns, S, N = case
    n = ns[0]
    yd = Bd.node_values(n, lambda X, Y: np.exp(Y * Y) * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y) + X)
    f = Bd.rhs(n, N, yd)
    fd = H.rhs(torch.tensor(yd, device="cuda"))
    check(to_host(fd), f, n, N, 1e-15, "right side")
    x = H.zeros(0)
    st, status = H.solve(fd, x, theta=0.5, tol=1e-10, maxit=100)
    z, it, hist = Bd.solve_stationary(S, ns, N, f, tol=1e-10, maxit=100)
    assert status == 0 and st.relres <= 1e-10 and hist[-1] <= 1e-10
    assert abs(st.iters - it) <= 1, (st.iters, it)
    check(to_host(x), z, n, N, 1e-9, "converged solution")
