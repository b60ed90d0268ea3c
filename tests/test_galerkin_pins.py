"""Pins of the Galerkin-coarse-operator oracle (oracle/galerkin.py) against
closed forms, invariants and the level-structured oracle (CPU only).

Sec. 3 defines the coarse matrices as S_l = R S_{l+1} P with R = P^T and
the bilinear P; Sec. 3.2 smooths with damped collective Jacobi."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import inputs
import oracle.cmg_oracle as O
import oracle.galerkin as G


def hier(n, N, nu=1e-4, amp=0.5, seed=1, K=3):
    xi = inputs.draw_xi(seed, N, K)
    return O.make_hierarchy(n, N, nu, O.sine_mode_field(xi, amp))


def tridiag(m, lo, mid, hi):
    return sp.diags([np.full(m - 1, lo), np.full(m, mid), np.full(m - 1, hi)], [-1, 0, 1]).toarray()


def test_system_matrix_equals_the_operator_column_by_column():
    """The sparse assembly from the block definition equals S assembled
    column by column from the level-structured operator apply_S."""
    lv = hier(7, 3)[0]
    S = G.system_matrix(lv).toarray()
    assert np.array_equal(S, O.dense_S(lv))


def test_prolongation_matrix_is_the_bilinear_prolongation():
    rng = np.random.default_rng(3)
    N = 2
    e = (rng.standard_normal((3, 3, N)), rng.standard_normal((3, 3)), rng.standard_normal((3, 3, N)))
    P = G.prolongation_matrix(7, N)
    assert np.abs(P @ O.pack(e) - O.pack(O.prolong(7, e))).max() <= 1e-15
    # and P^T is the restriction (transpose of the bilinear stencil, weights 1, 1/2, 1/4)
    r = (rng.standard_normal((7, 7, N)), rng.standard_normal((7, 7)), rng.standard_normal((7, 7, N)))
    assert np.abs(P.T @ O.pack(r) - O.pack(O.restrict(7, r))).max() <= 1e-14


def test_constant_coefficient_coarse_blocks_closed_form():
    """kappa = 1 (field amplitude 0): on the 7 -> 3 step the Galerkin blocks
    are tensor products of the two 1D Galerkin products of linear
    interpolation, P1^T P1 = tridiag(1/4, 3/2, 1/4) and
    P1^T K P1 = tridiag(-1/2, 1, -1/2) for K = tridiag(-1, 2, -1):
        A_c = T (x) L + L (x) T,   mass M_c = T (x) T  (fine mass = I),
    and the blocks of S_c are c M_c per sample, G M_c, d M_c 1^T, e M_c 1,
    blkdiag(A_c)."""
    N = 3
    levels = hier(7, N, amp=0.0)
    S1 = G.hierarchy(levels[:2])[1].toarray()
    fine = levels[0]
    m = 9
    T = tridiag(3, 0.25, 1.5, 0.25)
    L = tridiag(3, -0.5, 1.0, -0.5)
    A_c = np.kron(T, L) + np.kron(L, T)
    M_c = np.kron(T, T)
    Y = slice(0, m * N)
    U = slice(m * N, m * N + m)
    Pp = slice(m * N + m, m * N + m + m * N)
    for j in range(N):
        sj = slice(j, m * N, N)
        assert np.abs(S1[Y][:, Pp][sj, sj] - A_c).max() <= 1e-14        # state rows, adjoint columns
        assert np.abs(S1[Pp][:, Y][sj, sj] - A_c).max() <= 1e-14        # adjoint rows, state columns
        assert np.abs(S1[Y][:, Y][sj, sj] - fine.c * M_c).max() <= 1e-14 * abs(fine.c)
        assert np.abs(S1[Pp][:, U][sj, :] - fine.e * M_c).max() <= 1e-14 * abs(fine.e)
        assert np.abs(S1[U][:, Pp][:, sj] - fine.d * M_c).max() <= 1e-14 * abs(fine.d)
    assert np.abs(S1[U][:, U] - fine.G * M_c).max() <= 1e-14 * abs(fine.G)
    # no coupling between different samples
    for j in range(N):
        for k in range(N):
            if j != k:
                assert not np.any(S1[Y][:, Pp][j::N, k::N])


def test_coarse_operators_are_symmetric_nine_point():
    """Symmetric at every level (S_0 is, and P^T S P keeps it); every block
    row couples a node to at most its 3 x 3 neighbourhood."""
    N = 2
    levels = hier(15, N)
    S = G.hierarchy(levels)
    for l, (Sl, lv) in enumerate(zip(S, levels)):
        assert abs(Sl - Sl.T).max() <= 1e-15 * abs(Sl).max()
        n, m = lv.n, lv.n * lv.n
        coo = Sl.tocoo()

        def node_of(idx):
            idx = np.asarray(idx)
            return np.where(idx < m * N, idx // N, np.where(idx < m * N + m, idx - m * N, (idx - m * N - m) // N))

        a, b = node_of(coo.row), node_of(coo.col)
        assert np.abs(a // n - b // n).max() <= 1 and np.abs(a % n - b % n).max() <= 1


def test_node_block_is_the_arrow_system_of_eq12():
    """At a Galerkin grid the (2N+1) x (2N+1) block of node i has the arrow
    form of Eq. (12) with the diagonal entries of the Galerkin blocks:
    c_i = c M_ii, G_i = G M_ii, d_i = d M_ii, e_i = e M_ii, a_ij = (A_j)_ii,
    so Eq. (13) (the level-structured oracle's local_solve) solves it."""
    N = 3
    levels = hier(15, N)
    S = G.hierarchy(levels)
    fine = levels[0]
    rng = np.random.default_rng(5)
    for l in (1, 2):
        n = levels[l].n
        M_ii = None
        for i in (0, n + 1, n * n - 1):
            idx = G.node_indices(n, N, i)
            B = S[l][idx][:, idx].toarray()
            a = np.diag(B[:N, N + 1:])
            mii = B[N, N] / fine.G
            if M_ii is None:
                M_ii = mii
            assert abs(mii - M_ii) <= 1e-12 * M_ii           # constant per grid
            arrow = np.zeros_like(B)
            arrow[:N, :N] = fine.c * M_ii * np.eye(N)
            arrow[:N, N + 1:] = np.diag(a)
            arrow[N, N] = fine.G * M_ii
            arrow[N, N + 1:] = fine.d * M_ii
            arrow[N + 1:, :N] = np.diag(a)
            arrow[N + 1:, N] = fine.e * M_ii
            assert np.abs(B - arrow).max() <= 1e-13 * np.abs(B).max()
            rhs = rng.standard_normal(2 * N + 1)
            z = np.linalg.solve(B, rhs)
            # Eq. (13) written out: u from the Schur complement, then y, p
            c_, G_, d_, e_ = fine.c * M_ii, fine.G * M_ii, fine.d * M_ii, fine.e * M_ii
            b_y, b_u, b_p = rhs[:N], rhs[N], rhs[N + 1:]
            sigma = G_ + d_ * np.sum(c_ * e_ / a ** 2)
            u = (b_u - d_ * np.sum(b_y / a - c_ * b_p / a ** 2)) / sigma
            y = (b_p - e_ * u) / a
            p = (b_y - c_ * y) / a
            assert np.abs(np.concatenate([y, [u], p]) - z).max() <= 1e-10 * np.abs(z).max()
        # the mass diagonal is a square of 1D diagonals: (P1^T P1)_II = 1/4 + 1 + 1/4 = 3/2 on grid 1;
        # (P1^T tridiag(1/4, 3/2, 1/4) P1)_II = (1/4 + 1 + 1/4) 3/2 + 4 (1/2)(1/4)(1) = 11/4 on grid 2
        assert abs(M_ii - {1: 1.5 ** 2, 2: 2.75 ** 2}[l]) <= 1e-12 * M_ii


def test_galerkin_correction_annihilates_the_restricted_residual():
    """With S_c = P^T S P the exact coarse correction leaves a residual that
    restricts to zero, for any iterate and right side."""
    N = 2
    levels = hier(15, N)
    S = G.hierarchy(levels[:2])
    P = G.prolongation_matrix(15, N)
    rng = np.random.default_rng(7)
    z = rng.standard_normal(S[0].shape[0])
    f = rng.standard_normal(S[0].shape[0])
    r = f - S[0] @ z
    ec = spla.spsolve(S[1].tocsc(), P.T @ r)
    r2 = f - S[0] @ (z + P @ ec)
    assert np.linalg.norm(P.T @ r2) <= 1e-10 * np.linalg.norm(P.T @ r)


def test_jacobi_sweep_on_the_finest_grid_matches_eq13_sweep():
    """On the finest grid (no Galerkin product yet) the dense-block Jacobi
    step equals the level-structured oracle's Eq. (13) Jacobi step."""
    N = 3
    lv = hier(7, N)[0]
    rng = np.random.default_rng(9)
    x = (rng.standard_normal((7, 7, N)), rng.standard_normal((7, 7)), rng.standard_normal((7, 7, N)))
    f = tuple(b * s for b, s in zip((rng.standard_normal((7, 7, N)), rng.standard_normal((7, 7)),
                                     rng.standard_normal((7, 7, N))), (lv.c, lv.G, lv.h ** 2)))
    got = G.jacobi_sweep(G.system_matrix(lv), 7, N, O.pack(x), O.pack(f), 0.5)
    ref = O.pack(O.jacobi_sweep(lv, x, f, 0.5))
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("gamma", [1, 2])
def test_galerkin_cycle_converges_to_the_direct_solution(gamma):
    N = 3
    levels = hier(15, N, nu=1e-4)
    S = G.hierarchy(levels)
    f = O.pack(O.fine_rhs(levels[0], inputs.target_sinsin(15)))
    z, it, hist = G.solve_stationary(S, [lv.n for lv in levels], N, f, tol=1e-10, maxit=60, gamma=gamma)
    assert hist[-1] <= 1e-10 and it < 60
    ref = spla.spsolve(S[0].tocsc(), f)
    assert np.abs(z - ref).max() <= 1e-7 * np.abs(ref).max()
    # contraction from the second cycle on (the first raises the residual of the paper's row
    # scaling from x = 0, for every coarse-operator rule), about 0.3 per cycle
    assert all(b < a for a, b in zip(hist[1:], hist[2:]))
    assert (hist[-1] / hist[3]) ** (1.0 / (len(hist) - 4)) < 0.4


def test_four_colour_sweep_is_block_gauss_seidel_in_colour_order():
    """One four-colour sweep on a Galerkin grid equals the textbook block
    Gauss-Seidel step (D + L) z' = f - U z in the node order the colours
    give (L, U: couplings to earlier / later nodes of that order), solved
    as one sparse triangular-block system; and no two nodes of a colour
    are coupled."""
    N = 2
    levels = hier(15, N)
    S = G.hierarchy(levels)
    l, n = 1, levels[1].n
    m = n * n
    cols = G.four_colours(n)
    for c in cols:
        for i in c:
            for k in c:
                if i != k:
                    assert S[l][G.node_indices(n, N, i)][:, G.node_indices(n, N, k)].nnz == 0
    order = np.concatenate(cols)                       # node order of the sweep
    rank = np.empty(m, dtype=int)
    rank[order] = np.arange(m)
    perm = np.concatenate([G.node_indices(n, N, i) for i in order])
    A = S[l].toarray()[np.ix_(perm, perm)]
    blk = np.repeat(rank[order], 2 * N + 1)            # sweep position of every permuted unknown
    lower = blk[:, None] >= blk[None, :]               # block lower triangle, diagonal blocks included
    rng = np.random.default_rng(31)
    z = rng.standard_normal(S[l].shape[0])
    f = rng.standard_normal(S[l].shape[0])
    zp, fp = z[perm], f[perm]
    DL, U = np.where(lower, A, 0.0), np.where(lower, 0.0, A)
    ref = np.empty_like(z)
    ref[perm] = np.linalg.solve(DL, fp - U @ zp)
    got = G.colour_sweep(S[l], n, N, z, f, cols)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


def test_red_black_sweep_on_the_finest_grid_matches_eq13_sweep():
    N = 3
    lv = hier(7, N)[0]
    rng = np.random.default_rng(33)
    x = (rng.standard_normal((7, 7, N)), rng.standard_normal((7, 7)), rng.standard_normal((7, 7, N)))
    f = tuple(b * s for b, s in zip((rng.standard_normal((7, 7, N)), rng.standard_normal((7, 7)),
                                     rng.standard_normal((7, 7, N))), (lv.c, lv.G, lv.h ** 2)))
    got = G.colour_sweep(G.system_matrix(lv), 7, N, O.pack(x), O.pack(f), G.red_black(7))
    ref = O.pack(O.rbgs_sweep(lv, x, f))
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_gauss_seidel_galerkin_cycle_converges_to_the_direct_solution():
    N = 3
    levels = hier(15, N, nu=1e-4)
    S = G.hierarchy(levels)
    f = O.pack(O.fine_rhs(levels[0], inputs.target_sinsin(15)))
    z, it, hist = G.solve_stationary(S, [lv.n for lv in levels], N, f, tol=1e-10, maxit=60, smoother="gs")
    assert hist[-1] <= 1e-10 and it < 20
    ref = spla.spsolve(S[0].tocsc(), f)
    assert np.abs(z - ref).max() <= 1e-7 * np.abs(ref).max()


def test_local_control_galerkin_hierarchy():
    """Local control (u only at the control nodes): a region covering the
    square gives the distributed system; the finest matrix equals the level
    oracle's local-control system on the unknowns that exist; the Galerkin
    V-cycle with Eq. (13) / Eq. (14) node blocks reaches the direct solution."""
    N, n = 3, 15
    field_ = O.sine_mode_field(inputs.draw_xi(1, N, 3), 0.5)
    full = O.make_hierarchy(n, N, 1e-4, field_, control_box=(0.0, 1.0, 0.0, 1.0))
    assert abs(G.system_matrix_local(full[0]) - G.system_matrix(O.make_hierarchy(n, N, 1e-4, field_)[0])).max() == 0
    lv = O.make_hierarchy(n, N, 1e-4, field_, control_box=(0.25, 0.75, 0.25, 0.75))
    S, ctls = G.hierarchy_local(lv)
    m = n * n
    keep = np.concatenate([np.arange(m * N), m * N + ctls[0], m * N + m + np.arange(m * N)])
    assert np.array_equal(S[0].toarray(), O.dense_S(lv[0])[np.ix_(keep, keep)])
    f = O.pack(O.fine_rhs(lv[0], inputs.target_sinsin(n)))[keep]
    z, it, hist = G.solve_stationary_local(S, ctls, [l.n for l in lv], N, f, tol=1e-10)
    assert hist[-1] <= 1e-10 and it < 40
    ref = spla.spsolve(S[0].tocsc(), f)
    assert np.abs(z - ref).max() <= 1e-7 * np.abs(ref).max()


def test_fgmres_with_the_local_galerkin_cycle():
    """FGMRES right-preconditioned by the local-control Galerkin V-cycle
    reaches the direct solution in fewer iterations than the stationary
    cycle, its estimate matching the true weighted residual."""
    N, n = 3, 15
    lv = O.make_hierarchy(n, N, 1e-4, O.sine_mode_field(inputs.draw_xi(1, N, 3), 0.5),
                          control_box=(0.25, 0.75, 0.25, 0.75))
    S, ctls = G.hierarchy_local(lv)
    ns = [l.n for l in lv]
    m = n * n
    keep = np.concatenate([np.arange(m * N), m * N + ctls[0], m * N + m + np.arange(m * N)])
    f = O.pack(O.fine_rhs(lv[0], inputs.target_sinsin(n)))[keep]
    pre = lambda v: G.cycle_local(S, ctls, ns, N, 0, np.zeros_like(v), v)
    z, it, hist = G.fgmres_packed(S[0], pre, f, N, m, tol=1e-10)
    w = np.concatenate([np.full(m * N, float(N)), np.ones(S[0].shape[0] - m * N)])
    assert hist[-1] <= 1e-10
    assert np.linalg.norm(w * (f - S[0] @ z)) / np.linalg.norm(w * f) <= 2e-10
    ref = spla.spsolve(S[0].tocsc(), f)
    assert np.abs(z - ref).max() <= 1e-7 * np.abs(ref).max()
    _, it_stat, _ = G.solve_stationary_local(S, ctls, ns, N, f, tol=1e-10)
    assert it < it_stat
