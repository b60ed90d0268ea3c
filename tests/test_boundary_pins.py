"""Pins of the Neumann-boundary-control oracle (oracle/boundary.py): the
control acts on Gamma = (0,1) x {0} (Sec. 2 control operator, Sec. 3.2 test
case); the smoother takes Eq. (13) on Gamma and Eq. (14) elsewhere (Sec. 3.1).
CPU only."""
import numpy as np
import scipy.sparse.linalg as spla

import inputs
import oracle.boundary as Bd
import oracle.cmg_oracle as O


def field(N, amp=0.5, seed=1, K=3):
    return O.sine_mode_field(inputs.draw_xi(seed, N, K), amp)


def tridiag(m, lo, mid, hi):
    return np.diag(np.full(m - 1, lo), -1) + np.diag(np.full(m, mid)) + np.diag(np.full(m - 1, hi), 1)


def test_grid_size_is_the_papers():
    """31 interior columns and rows y = 0 .. 31 h: N_h = 992 for h = 1/32."""
    assert Bd.mass(31).size == 992


def test_constant_coefficient_stiffness_closed_form():
    """kappa = 1: A = K_N (x) I + D (x) K with K = tridiag(-1, 2, -1) (x,
    Dirichlet both ends), K_N the y-stiffness with a Neumann first row
    (1, -1) and a Dirichlet last row, D = diag(1/2, 1, ..., 1) (the half
    cells of row 0)."""
    n, N = 7, 2
    kx, ky = Bd.faces(n, N, field(N, amp=0.0))
    A = Bd.stiffness_matrix(n, kx, ky, 0).toarray()
    K = tridiag(n, -1.0, 2.0, -1.0)
    KN = tridiag(n + 1, -1.0, 2.0, -1.0)
    KN[0, 0] = 1.0
    D = np.eye(n + 1)
    D[0, 0] = 0.5
    assert np.abs(A - (np.kron(KN, np.eye(n)) + np.kron(D, K))).max() <= 1e-14


def test_system_is_symmetric_and_masses_are_lumped():
    n, N = 7, 3
    kx, ky = Bd.faces(n, N, field(N))
    S = Bd.system_matrix(n, N, 1e-3, kx, ky)
    assert abs(S - S.T).max() <= 1e-15 * abs(S).max()
    h = 1.0 / (n + 1)
    w = Bd.mass(n)
    assert np.isclose(w.sum(), (n + 0.5) * n * h * h)   # n + 1/2 rows of n cells


def test_full_space_solution_equals_the_reduced_minimiser():
    """The saddle-point system's control equals the minimiser of the reduced
    cost from its normal equations (no saddle-point system formed), with a
    target and a forcing."""
    n, N, nu = 7, 3, 1e-3
    kx, ky = Bd.faces(n, N, field(N))
    S = Bd.system_matrix(n, N, nu, kx, ky)
    yd = Bd.node_values(n, lambda x, y: np.sin(np.pi * x) * np.cos(0.5 * np.pi * y))
    f = Bd.node_values(n, lambda x, y: 1.0 + x * y)
    z = spla.spsolve(S.tocsc(), Bd.rhs(n, N, yd, f))
    m = (n + 1) * n
    u = z[m * N: m * N + n]
    ref = Bd.reduced_control(n, N, nu, kx, ky, yd, f)
    assert np.abs(u - ref).max() <= 1e-9 * np.abs(ref).max()


def test_y_prolongation_reproduces_linear_profiles():
    """Linear interpolation in y with the Dirichlet top: exact on 1 - y."""
    n = 15
    nc = (n - 1) // 2
    h, hc = 1.0 / (n + 1), 2.0 / (n + 1)
    fine = Bd.prolongation_y(n) @ (1.0 - np.arange(nc + 1) * hc)
    assert np.abs(fine - (1.0 - np.arange(n + 1) * h)).max() <= 1e-15


def test_node_blocks_follow_eq13_on_gamma_and_eq14_elsewhere():
    """The dense node blocks the smoother solves are Eq. (12)'s arrow system
    on Gamma (c = h^2/(2N), G = nu h, d = e = -h) and, off Gamma, the same
    without the control row and column, whose solution is Eq. (14)."""
    n, N, nu = 7, 3, 1e-3
    h = 1.0 / (n + 1)
    kx, ky = Bd.faces(n, N, field(N))
    S = Bd.system_matrix(n, N, nu, kx, ky)
    gam, inner = Bd.node_groups(n, N)
    rng = np.random.default_rng(3)
    # Gamma node 2
    B = S[gam[2]][:, gam[2]].toarray()
    a = np.diag(B[:N, N + 1:])
    c, G, d, e = h * h / (2 * N), nu * h, -h, -h
    b = rng.standard_normal(2 * N + 1)
    by, bu, bp = b[:N], b[N], b[N + 1:]
    sigma = G + d * np.sum(c * e / a ** 2)
    u = (bu - d * np.sum(by / a - c * bp / a ** 2)) / sigma
    y = (bp - e * u) / a
    p = (by - c * y) / a
    assert np.abs(np.linalg.solve(B, b) - np.concatenate([y, [u], p])).max() <= 1e-9 * np.abs(u)
    # an interior node (row 3)
    k = 3 * n + 4 - n
    B = S[inner[k]][:, inner[k]].toarray()
    a = np.diag(B[:N, N:])
    c = h * h / N
    b = rng.standard_normal(2 * N)
    by, bp = b[:N], b[N:]
    y = bp / a
    p = (by - c * y) / a
    assert np.abs(np.linalg.solve(B, b) - np.concatenate([y, p])).max() <= 1e-12 * np.abs(p).max()


def test_vcycle_converges_h_robustly_to_the_direct_solution():
    N, nu = 4, 1e-4
    its = []
    for n in (15, 31):
        ns, S = Bd.hierarchy(n, N, nu, field(N))
        yd = Bd.node_values(n, lambda x, y: np.sin(np.pi * x) * np.sin(np.pi * y))
        f = Bd.rhs(n, N, yd)
        z, it, hist = Bd.solve_stationary(S, ns, N, f, tol=1e-10, maxit=80)
        assert hist[-1] <= 1e-10
        ref = spla.spsolve(S[0].tocsc(), f)
        assert np.abs(z - ref).max() <= 1e-6 * np.abs(ref).max()
        its.append(it)
    assert max(its) <= 1.3 * min(its) + 2      # the cycle count does not grow with 1/h


def test_fgmres_converges_to_the_direct_solution_in_fewer_iterations():
    """FGMRES with the V-cycle as right preconditioner reaches the direct
    solution; its residual estimate equals the true weighted residual; it
    needs fewer iterations than the stationary cycle (the paper's Table 3
    pattern)."""
    n, N, nu = 15, 4, 1e-4
    ns, S = Bd.hierarchy(n, N, nu, field(N))
    f = Bd.rhs(n, N, Bd.node_values(n, lambda x, y: np.sin(np.pi * x) * np.sin(np.pi * y)))
    z, it, hist = Bd.fgmres(S, ns, N, f, tol=1e-10)
    true = Bd.paper_norm(f - S[0] @ z, n, N) / Bd.paper_norm(f, n, N)
    assert hist[-1] <= 1e-10 and true <= 2e-10
    ref = spla.spsolve(S[0].tocsc(), f)
    assert np.abs(z - ref).max() <= 1e-6 * np.abs(ref).max()
    _, it_stat, _ = Bd.solve_stationary(S, ns, N, f, tol=1e-10, maxit=80)
    assert it < it_stat


def test_galerkin_coarse_structure_the_gpu_path_relies_on():
    """On every coarse grid of the boundary hierarchy: the control rows couple
    only to row-0 adjoints; the control-control block is a constant 3-point
    stencil along Gamma; the mass (state-state block of a sample) is one
    constant 9-point stencil on rows >= 1 and another on row 0, where the
    centre and side weights are halved and there is no south neighbour."""
    N = 2
    ns, S = Bd.hierarchy(31, N, 1e-4, field(N))
    for l in range(1, len(ns)):
        n = ns[l]
        m = (n + 1) * n
        A = S[l].toarray()
        D = A[m * N: m * N + n, m * N + n:]                     # control rows x adjoint columns
        cols = np.nonzero(D)[1] // N
        assert np.all(cols < n)                                # row-0 nodes only
        U = A[m * N: m * N + n, m * N: m * N + n]
        assert np.allclose(U, np.diag(np.diag(U)) + np.diag(np.diag(U, 1), 1) + np.diag(np.diag(U, -1), -1))
        if n > 1:
            assert np.allclose(np.diag(U), U[0, 0]) and np.allclose(np.diag(U, 1), U[0, 1])
        Y = A[: m * N: N, : m * N: N]                          # sample 0's state-state block

        def stencil(r, ix):
            i = r * n + ix
            return {(k // n - r, k % n - ix): v for k, v in enumerate(Y[i]) if v != 0.0}

        if n >= 3:
            ref = stencil(1, 1)                                # an interior row's stencil
            for r in range(1, n):                              # rows away from the top boundary
                for ix in range(1, n - 1):
                    st = stencil(r, ix)
                    assert st.keys() == ref.keys() and all(np.isclose(st[k], ref[k]) for k in ref)
            top = stencil(0, 1)
            assert all(dy >= 0 for dy, _ in top)               # no south neighbour on Gamma
            assert np.isclose(top[(0, 0)], ref[(0, 0)] / 2) and np.isclose(top[(0, 1)], ref[(0, 1)] / 2)
            assert np.isclose(top[(1, 0)], ref[(1, 0)]) and np.isclose(top[(1, 1)], ref[(1, 1)])
