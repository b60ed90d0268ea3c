"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test compares an oracle function with a result fixed by the paper or
by the mathematics: dense LU of the assembled systems, closed-form
solutions, the smoother spectrum of Lemma 1 / Corollary 1, the damping
remark after Corollary 1, exactness of the 5-point stencil and of bilinear
interpolation, energy identities, and brute-force block definitions of the
collective smoothers.  None of these route through the oracle's own
formula for the thing being pinned.
"""
import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

import inputs
import oracle.cmg_oracle as O


def const_field(eta):
    """kappa_j(x) = eta_j everywhere (also on the boundary)."""
    eta = np.asarray(eta, dtype=np.float64)

    def k(X, Y):
        return np.broadcast_to(eta, X.shape + (eta.size,)).copy()

    return k


def assemble_A_by_faces(level, j):
    """A_j assembled face by face (finite-volume / FE style), independent of
    the stencil code: each interior face (a, b) with coefficient k adds k to
    (a,a), (b,b) and -k to (a,b), (b,a); each boundary face adds k to the
    diagonal of its single interior node."""
    n = level.n
    A = np.zeros((n * n, n * n))
    idx = lambda iy, ix: iy * n + ix
    for iy in range(n):
        for f in range(n + 1):              # vertical faces between columns f-1 and f
            k = level.kx[iy, f, j]
            nodes = [idx(iy, ix) for ix in (f - 1, f) if 0 <= ix < n]
            for a in nodes:
                A[a, a] += k
            if len(nodes) == 2:
                A[nodes[0], nodes[1]] -= k
                A[nodes[1], nodes[0]] -= k
    for f in range(n + 1):
        for ix in range(n):
            k = level.ky[f, ix, j]
            nodes = [idx(iy, ix) for iy in (f - 1, f) if 0 <= iy < n]
            for a in nodes:
                A[a, a] += k
            if len(nodes) == 2:
                A[nodes[0], nodes[1]] -= k
                A[nodes[1], nodes[0]] -= k
    return A


def assemble_S_blocks(level):
    """The full-space matrix in (y, u, p) order from the block definition of
    Eq. (2): C_j = c I, G = g I, D_j = d I, E_j = e I, A_j from faces."""
    n, N = level.n, level.N
    m = n * n
    dim = (2 * N + 1) * m
    S = np.zeros((dim, dim))
    yi = lambda i, j: i * N + j
    ui = lambda i: m * N + i
    pi = lambda i, j: m * N + m + i * N + j
    for j in range(N):
        A = assemble_A_by_faces(level, j)
        for r in range(m):
            S[yi(r, j), yi(r, j)] = level.c
            S[pi(r, j), ui(r)] = level.e
            S[ui(r), pi(r, j)] = level.d
            for s in range(m):
                if A[r, s] != 0.0:
                    S[yi(r, j), pi(s, j)] = A[r, s]     # A_j^T = A_j in the state rows
                    S[pi(r, j), yi(s, j)] = A[r, s]
    for r in range(m):
        S[ui(r), ui(r)] = level.G
    return S


def node_dofs(i, n, N):
    m = n * n
    return ([i * N + j for j in range(N)] + [m * N + i]
            + [m * N + m + i * N + j for j in range(N)])


def small_level(n=7, N=3, nu=1e-3, seed=11, amp=0.8, K=3):
    xi = inputs.draw_xi(seed, N, K)
    return O.make_level(n, N, nu, O.sine_mode_field(xi, amp))


def rand_vec(level, seed):
    rng = np.random.default_rng(seed)
    n, N = level.n, level.N
    return (rng.standard_normal((n, n, N)), rng.standard_normal((n, n)),
            rng.standard_normal((n, n, N)))


# --------------------------------------------------------------------------
# Field and faces
# --------------------------------------------------------------------------

def test_field_special_values():
    # k = 1 mode is 1 at (1/2, 1/2); k = 2 mode vanishes there and is 1/2 at (1/4, 1/2)
    xi = np.array([[0.3, 0.0], [0.0, 0.9]])
    k = O.sine_mode_field(xi, amp=1.7)
    X = np.array([0.5, 0.25, 0.0, 1.0, 0.3])
    Y = np.array([0.5, 0.5, 0.4, 0.7, 0.0])
    v = k(X, Y)
    assert np.allclose(v[0], [np.exp(1.7 * 0.3), 1.0])
    assert np.allclose(v[1, 1], np.exp(1.7 * 0.9 * 0.5))
    assert np.allclose(v[2:], 1.0)          # kappa = 1 on the boundary


def test_faces_of_constant_field_equal_the_constant():
    eta = [0.5, 2.0, 3.25]
    L = O.make_level(7, 3, 1e-2, const_field(eta))
    assert np.allclose(L.kx, np.broadcast_to(eta, L.kx.shape))
    assert np.allclose(L.ky, np.broadcast_to(eta, L.ky.shape))
    assert np.allclose(L.a, 4 * np.broadcast_to(eta, L.a.shape))


def test_harmonic_face_between_two_values():
    # 1/k_f is the mean of 1/k_a and 1/k_b (series resistances)
    ka, kb = 0.25, 4.0
    assert np.isclose(1.0 / O.harmonic_mean(ka, kb), 0.5 * (1 / ka + 1 / kb))


# --------------------------------------------------------------------------
# Operator
# --------------------------------------------------------------------------

def test_stencil_exact_on_biquadratic():
    # -Laplace of x(1-x)y(1-y) is 2y(1-y) + 2x(1-x); the 5-point stencil is
    # exact for quadratics, and the integrated stencil carries h^2.
    n = 15
    L = O.make_level(n, 1, 1.0, const_field([1.0]))
    x, y = inputs.grid_nodes(n)
    v = (x * (1 - x) * y * (1 - y))[:, :, None]
    Av = O.apply_A(L, v)[:, :, 0]
    assert np.allclose(Av, L.h ** 2 * (2 * y * (1 - y) + 2 * x * (1 - x)), rtol=1e-12, atol=1e-15)


def test_apply_A_matches_face_assembly_and_energy():
    L = small_level()
    rng = np.random.default_rng(3)
    v = rng.standard_normal((L.n, L.n, L.N))
    Av = O.apply_A(L, v)
    for j in range(L.N):
        A = assemble_A_by_faces(L, j)
        assert np.allclose(Av[:, :, j].ravel(), A @ v[:, :, j].ravel(), rtol=1e-13, atol=1e-13)
        # energy identity: v^T A v = sum over faces k_f (jump of v)^2, boundary value 0
        vp = np.pad(v[:, :, j], 1)
        energy = (np.sum(L.kx[:, :, j] * (vp[1:-1, 1:] - vp[1:-1, :-1]) ** 2)
                  + np.sum(L.ky[:, :, j] * (vp[1:, 1:-1] - vp[:-1, 1:-1]) ** 2))
        assert np.isclose(v[:, :, j].ravel() @ Av[:, :, j].ravel(), energy, rtol=1e-12)


def test_apply_S_matches_block_assembly_and_is_symmetric():
    L = small_level(n=3, N=2)
    S_blocks = assemble_S_blocks(L)
    S_apply = O.dense_S(L)
    assert np.allclose(S_apply, S_blocks, rtol=1e-14, atol=1e-16)
    assert np.array_equal(S_blocks, S_blocks.T)
    L7 = small_level(n=7, N=3)
    x, z = rand_vec(L7, 1), rand_vec(L7, 2)
    lhs = O.pack(z) @ O.pack(O.apply_S(L7, *x))
    rhs = O.pack(x) @ O.pack(O.apply_S(L7, *z))
    assert np.isclose(lhs, rhs, rtol=1e-12)


# --------------------------------------------------------------------------
# Local solve, Eq. (13)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("N", [1, 2, 8, 64])
def test_local_solve_matches_dense_node_system(N):
    rng = np.random.default_rng(N)
    a = rng.uniform(0.5, 4.0, N)
    c = rng.uniform(0.1, 1.0, N)
    d = -rng.uniform(0.1, 1.0, N)
    e = -rng.uniform(0.1, 1.0, N)
    G = 0.37
    # S~_i of Eq. (12): rows (first block, control row, last block), columns (y~, u, p~)
    St = np.zeros((2 * N + 1, 2 * N + 1))
    St[:N, :N] = np.diag(c)
    St[:N, N + 1:] = np.diag(a)
    St[N, N] = G
    St[N, N + 1:] = d
    St[N + 1:, :N] = np.diag(a)
    St[N + 1:, N] = e
    b = rng.standard_normal(2 * N + 1)
    ref = np.linalg.solve(St, b)
    y, u, p = O.local_solve(b[:N], b[N], b[N + 1:], a, c, G, d, e)
    assert np.allclose(np.concatenate([y, [u], p]), ref, rtol=1e-11, atol=1e-12)


def test_schur_denominator_positive_and_closed_form():
    # the denominator equals G + (h^6/N) sum_j a_j^-2 > 0 for this problem
    L = small_level()
    sig = L.sigma
    h, N = L.h, L.N
    assert np.all(sig > 0)
    assert np.allclose(sig, L.nu * h ** 2 + h ** 6 / N * np.sum(L.a ** -2.0, axis=-1), rtol=1e-13)


# --------------------------------------------------------------------------
# Smoothers against their block definitions
# --------------------------------------------------------------------------

def _node_order(n, N, order):
    return np.concatenate([node_dofs(i, n, N) for i in order])


def test_jacobi_matches_block_jacobi_definition():
    L = small_level(n=7, N=2)
    S = assemble_S_blocks(L)
    x, f = rand_vec(L, 5), rand_vec(L, 6)
    xv, fv = O.pack(x), O.pack(f)
    r = fv - S @ xv
    corr = np.zeros_like(xv)
    for i in range(L.n ** 2):
        dofs = node_dofs(i, L.n, L.N)
        corr[dofs] = np.linalg.solve(S[np.ix_(dofs, dofs)], r[dofs])
    for theta in (1.0, 0.5):
        ref = xv + theta * corr
        got = O.pack(O.jacobi_sweep(L, x, f, theta))
        assert np.allclose(got, ref, rtol=1e-10, atol=1e-12)


def _block_gs_sweep(S, xv, fv, order, n, N):
    perm = _node_order(n, N, order)
    Sp = S[np.ix_(perm, perm)]
    nb = 2 * N + 1
    M = np.zeros_like(Sp)
    for bi in range(len(order)):
        for bj in range(bi + 1):
            sl_i = slice(bi * nb, (bi + 1) * nb)
            sl_j = slice(bj * nb, (bj + 1) * nb)
            M[sl_i, sl_j] = Sp[sl_i, sl_j]
    U = Sp - M
    xn = np.linalg.solve(M, fv[perm] - U @ xv[perm])
    out = np.empty_like(xv)
    out[perm] = xn
    return out


def test_lexicographic_gs_matches_block_definition():
    L = small_level(n=7, N=2)
    S = assemble_S_blocks(L)
    x, f = rand_vec(L, 7), rand_vec(L, 8)
    ref = _block_gs_sweep(S, O.pack(x), O.pack(f), list(range(L.n ** 2)), L.n, L.N)
    got = O.pack(O.lexgs_sweep(L, x, f))
    assert np.allclose(got, ref, rtol=1e-9, atol=1e-11)


def test_red_black_gs_matches_block_definition():
    L = small_level(n=7, N=3)
    S = assemble_S_blocks(L)
    x, f = rand_vec(L, 9), rand_vec(L, 10)
    n = L.n
    red = [iy * n + ix for iy in range(n) for ix in range(n) if (ix + iy) % 2 == 0]
    black = [iy * n + ix for iy in range(n) for ix in range(n) if (ix + iy) % 2 == 1]
    ref = _block_gs_sweep(S, O.pack(x), O.pack(f), red + black, n, L.N)
    got = O.pack(O.rbgs_sweep(L, x, f))
    assert np.allclose(got, ref, rtol=1e-9, atol=1e-11)


# --------------------------------------------------------------------------
# Lemma 1 / Corollary 1 / damping remark (2D form, tensorised sines)
# --------------------------------------------------------------------------

def _match_spectra(a, b):
    cost = np.abs(a[:, None] - b[None, :])
    r, c = linear_sum_assignment(cost)
    return cost[r, c].max()


@pytest.mark.parametrize("theta", [1.0, 0.5])
def test_jacobi_spectrum_matches_lemma1_corollary1(theta):
    """Constant kappa_j = eta_j: the collective Jacobi iteration matrix is
    -H2 (x) S~^{-1}B with H2 the 2D neighbour matrix (eigenvalues
    2cos(a pi h) + 2cos(b pi h)).  S~^{-1}B has the eigenvalues of Lemma 1
    with off-diagonal/diagonal ratio 1/4 instead of 1/2,
        -1/4 {1 (2N-2 times), 1 - r +- i sqrt((1-r) r)},
    r = E[dt^-2] / (nu + E[dt^-2]), dt_j = diag(A_j)/h^2 = 4 eta_j / h^2,
    plus 0 for the control unknown.  Damping maps delta -> 1 - theta + theta delta."""
    n, N, nu = 7, 3, 1e-2
    eta = np.array([0.7, 1.3, 2.1])
    L = O.make_level(n, N, nu, const_field(eta))
    m = n * n
    dim = (2 * N + 1) * m
    f0 = O.zeros_like_level(L)
    Gm = np.zeros((dim, dim))
    for col in range(dim):
        z = np.zeros(dim)
        z[col] = 1.0
        Gm[:, col] = O.pack(O.jacobi_sweep(L, O.unpack(z, n, N), f0, theta))
    ev = np.linalg.eigvals(Gm)
    h = L.h
    E = np.mean((4 * eta / h ** 2) ** -2.0)
    r = E / (nu + E)
    lam = np.concatenate([[-0.25] * (2 * N - 2),
                          -0.25 * np.array([1 - r + 1j * np.sqrt((1 - r) * r),
                                            1 - r - 1j * np.sqrt((1 - r) * r)]), [0.0]])
    mus = [2 * np.cos(a * np.pi * h) + 2 * np.cos(b * np.pi * h)
           for a in range(1, n + 1) for b in range(1, n + 1)]
    delta = np.array([-mu * l for mu in mus for l in lam])
    pred = 1 - theta + theta * delta
    # defective (Jordan) eigenvalues are only accurate to ~sqrt(eps)
    assert _match_spectra(ev, pred) < 1e-6
    # Corollary 1: rho < 1 and equals max|mu| * max|lambda| for theta = 1
    if theta == 1.0:
        assert np.isclose(np.max(np.abs(ev)), max(abs(np.array(mus))) * 0.25, rtol=1e-6)


# --------------------------------------------------------------------------
# Transfers
# --------------------------------------------------------------------------

def test_prolongation_reproduces_bilinear_functions():
    nf = 15
    nc = 7
    xc, yc = inputs.grid_nodes(nc)
    xf, yf = inputs.grid_nodes(nf)
    # x*y vanishes on x = 0 and y = 0, so interpolation is exact away from x = 1, y = 1
    ec = (xc * yc)[:, :, None]
    ef = O.prolong(nf, (ec, xc * yc, ec))
    inner = np.s_[: nf - 1, : nf - 1]
    assert np.allclose(ef[0][inner][:, :, 0], (xf * yf)[inner], atol=1e-14)
    assert np.allclose(ef[1][inner], (xf * yf)[inner], atol=1e-14)
    g = lambda x, y: (1 - x) * (1 - y)
    ef = O.prolong(nf, (g(xc, yc)[:, :, None], g(xc, yc), g(xc, yc)[:, :, None]))
    inner = np.s_[1:, 1:]
    assert np.allclose(ef[2][inner][:, :, 0], g(xf, yf)[inner], atol=1e-14)


def test_restriction_is_transpose_and_weights_sum_to_four():
    nf, N = 15, 2
    rng = np.random.default_rng(4)
    r = (rng.standard_normal((nf, nf, N)), rng.standard_normal((nf, nf)),
         rng.standard_normal((nf, nf, N)))
    nc = 7
    e = (rng.standard_normal((nc, nc, N)), rng.standard_normal((nc, nc)),
         rng.standard_normal((nc, nc, N)))
    assert np.isclose(O.pack(O.restrict(nf, r)) @ O.pack(e), O.pack(r) @ O.pack(O.prolong(nf, e)), rtol=1e-12)
    ones = (np.ones((nf, nf, 1)), np.ones((nf, nf)), np.ones((nf, nf, 1)))
    rc = O.restrict(nf, ones)
    assert np.allclose(rc[1], 4.0)
    # brute force on one coarse node: weights 1 at the centre, 1/2 on edges, 1/4 at corners
    unit = np.zeros((nf, nf))
    # coarse (J, I) sits on fine (2J+1, 2I+1); fine (iy=4, ix=2) is the centre
    # of the cell spanned by fine rows 3, 5 and columns 1, 3
    unit[4, 2] = 1.0
    rc = O.restrict(nf, (np.zeros((nf, nf, 1)), unit, np.zeros((nf, nf, 1))))[1]
    expect = np.zeros((nc, nc))
    for J in (1, 2):
        for I in (0, 1):
            expect[J, I] = 0.25
    assert np.allclose(rc, expect)


# --------------------------------------------------------------------------
# Direct solves and full solvers against dense LU
# --------------------------------------------------------------------------

@pytest.mark.parametrize("N", [1, 2, 4])
def test_coarse_solve_matches_dense_lu(N):
    L = small_level(n=3, N=N, seed=20 + N)
    f = rand_vec(L, 21)
    ref = np.linalg.solve(assemble_S_blocks(L), O.pack(f))
    got = O.pack(O.coarse_solve(L, f))
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-14 * np.abs(ref).max())


@pytest.mark.parametrize("n,N", [(7, 1), (7, 2), (15, 2), (7, 4)])
@pytest.mark.parametrize("method", ["rbgs-V", "rbgs-W", "jacobi-V", "lexgs-V", "fgmres"])
def test_solvers_converge_to_dense_lu(n, N, method):
    xi = inputs.draw_xi(30 + n + N, N, 3)
    levels = O.make_hierarchy(n, N, 1e-3, O.sine_mode_field(xi, 0.7))
    yd = inputs.target_modes(n, 5)
    f = O.fine_rhs(levels[0], yd)
    S = O.dense_S(levels[0])
    ref = np.linalg.solve(S, O.pack(f))
    if method == "fgmres":
        res = O.fgmres(levels, f, O.CycleOptions(), tol=1e-12)
    else:
        sm, cyc = method.split("-")
        opts = O.CycleOptions(smoother=sm, gamma=1 if cyc == "V" else 2)
        res = O.solve_stationary(levels, f, opts, tol=1e-12, maxit=200)
    assert res.relres <= 1e-12
    got = O.pack(res.x)
    assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)


# --------------------------------------------------------------------------
# Closed form, N = 1 reduction, sample permutation
# --------------------------------------------------------------------------

def test_closed_form_constant_field():
    """kappa_j = eta_j, y_d = sin(pi x) sin(pi y): y_j = alpha_j s, u = beta s,
    p_j = gamma_j s with lambda = 8 sin^2(pi h / 2) the eigenvalue of the
    integrated 5-point stencil on s, and
      beta  = (h^2/N) sum_j (eta_j lambda)^-1 / (nu + (h^4/N) sum_j (eta_j lambda)^-2)
      alpha_j = h^2 beta / (eta_j lambda),  gamma_j = (h^2/N)(1 - alpha_j)/(eta_j lambda)."""
    n, N, nu = 15, 3, 1e-4
    eta = np.array([0.6, 1.0, 2.5])
    levels = O.make_hierarchy(n, N, nu, const_field(eta))
    s = inputs.target_sinsin(n)
    f = O.fine_rhs(levels[0], s)
    res = O.fgmres(levels, f, O.CycleOptions(), tol=1e-13)
    h = 1.0 / (n + 1)
    lam = 8 * np.sin(np.pi * h / 2) ** 2
    el = eta * lam
    beta = (h ** 2 / N) * np.sum(1 / el) / (nu + (h ** 4 / N) * np.sum(el ** -2.0))
    alpha = h ** 2 * beta / el
    gamma = (h ** 2 / N) * (1 - alpha) / el
    y, u, p = res.x
    assert np.allclose(u, beta * s, rtol=1e-9, atol=1e-12 * abs(beta))
    assert np.allclose(y, s[:, :, None] * alpha, rtol=1e-9, atol=1e-12)
    assert np.allclose(p, s[:, :, None] * gamma, rtol=1e-8, atol=1e-12 * np.abs(gamma).max())


def test_deterministic_reduction_N1_and_duplicated_samples():
    """N = 1 is the deterministic problem (remark after Theorem 1): with
    u = p / nu eliminated, (M y + A p, A y - M p / nu) = (M y_d, 0).
    N identical samples give the same y and u, and p_j = p(N=1) / N."""
    n = 15
    xi1 = inputs.draw_xi(40, 1, 3)
    lev1 = O.make_hierarchy(n, 1, 1e-3, O.sine_mode_field(xi1, 0.9))
    yd = inputs.target_modes(n, 6)
    f1 = O.fine_rhs(lev1[0], yd)
    r1 = O.fgmres(lev1, f1, O.CycleOptions(), tol=1e-13)
    A = assemble_A_by_faces(lev1[0], 0)
    h2 = lev1[0].h ** 2
    m = n * n
    K = np.block([[h2 * np.eye(m), A], [A, -h2 / 1e-3 * np.eye(m)]])
    sol = np.linalg.solve(K, np.concatenate([h2 * yd.ravel(), np.zeros(m)]))
    assert np.allclose(r1.x[0][:, :, 0].ravel(), sol[:m], rtol=1e-8, atol=1e-10)
    assert np.allclose(r1.x[2][:, :, 0].ravel(), sol[m:], rtol=1e-8, atol=1e-14)
    assert np.allclose(r1.x[1].ravel(), sol[m:] / 1e-3, rtol=1e-8, atol=1e-10)
    Nd = 4
    xid = np.repeat(xi1, Nd, axis=0)
    levd = O.make_hierarchy(n, Nd, 1e-3, O.sine_mode_field(xid, 0.9))
    rd = O.fgmres(levd, O.fine_rhs(levd[0], yd), O.CycleOptions(), tol=1e-13)
    for j in range(Nd):
        assert np.allclose(rd.x[0][:, :, j], r1.x[0][:, :, 0], rtol=1e-8, atol=1e-10)
        assert np.allclose(rd.x[2][:, :, j], r1.x[2][:, :, 0] / Nd, rtol=1e-8, atol=1e-14)
    assert np.allclose(rd.x[1], r1.x[1], rtol=1e-8, atol=1e-10)


def test_sample_permutation():
    n, N = 15, 5
    xi = inputs.draw_xi(50, N, 3)
    perm = np.array([3, 0, 4, 1, 2])
    yd = inputs.target_modes(n, 7)
    opts = O.CycleOptions()
    la = O.make_hierarchy(n, N, 1e-4, O.sine_mode_field(xi, 1.0))
    lb = O.make_hierarchy(n, N, 1e-4, O.sine_mode_field(xi[perm], 1.0))
    ra = O.solve_stationary(la, O.fine_rhs(la[0], yd), opts, tol=1e-12)
    rb = O.solve_stationary(lb, O.fine_rhs(lb[0], yd), opts, tol=1e-12)
    assert np.allclose(rb.x[0], ra.x[0][:, :, perm], rtol=1e-12, atol=1e-14)
    assert np.allclose(rb.x[2], ra.x[2][:, :, perm], rtol=1e-12, atol=1e-16)
    assert np.allclose(rb.x[1], ra.x[1], rtol=1e-12, atol=1e-14)


# --------------------------------------------------------------------------
# Robustness (h- and N-independent contraction, Sec. 3.2)
# --------------------------------------------------------------------------

def test_cycle_counts_are_h_and_N_robust():
    counts = {}
    for n, N in [(15, 8), (31, 8), (63, 8), (31, 2), (31, 16)]:
        xi = inputs.draw_xi(60, N, 4)
        levels = O.make_hierarchy(n, N, 1e-4, O.sine_mode_field(xi, 0.5))
        f = O.fine_rhs(levels[0], inputs.target_sinsin(n))
        res = O.solve_stationary(levels, f, O.CycleOptions(), tol=1e-10, maxit=60)
        assert res.relres <= 1e-10
        counts[(n, N)] = res.iters
    vals = list(counts.values())
    assert max(vals) - min(vals) <= 3, counts
    assert max(vals) <= 16, counts


def test_paper_system_is_row_and_column_scaling_of_symmetric_form():
    """The paper's full-space system (Sec. 2): rows M y_j + A_j^T p_j = M y_d,
    nu M u - sum_j zeta_j M p_j = 0, A_j y_j - M u = M f, with zeta_j = 1/N.
    In the variables (y, u, N p) it equals W S with W = diag(N I, 1, 1), so
    its relative residual is the W-weighted one (paper_norm)."""
    L = small_level(n=3, N=3)
    n, N, h = L.n, L.N, L.h
    m = n * n
    M = h * h * np.eye(m)
    dim = (2 * N + 1) * m
    Sp = np.zeros((dim, dim))
    for j in range(N):
        A = assemble_A_by_faces(L, j)
        ys = slice(j * m, (j + 1) * m)
        ps = slice(N * m + m + j * m, N * m + m + (j + 1) * m)
        us = slice(N * m, N * m + m)
        Sp[ys, ys] = M
        Sp[ys, ps] = A.T
        Sp[us, ps] = -(1.0 / N) * M
        Sp[ps, ys] = A
        Sp[ps, us] = -M
    Sp[N * m:N * m + m, N * m:N * m + m] = L.nu * M
    # sample-major ordering of the paper -> node-major ordering used here
    perm = np.empty(dim, dtype=int)
    for i in range(m):
        for j in range(N):
            perm[i * N + j] = j * m + i
            perm[N * m + m + i * N + j] = N * m + m + j * m + i
    perm[N * m:N * m + m] = np.arange(N * m, N * m + m)
    Sp = Sp[np.ix_(perm, perm)]
    S = assemble_S_blocks(L)
    W = np.diag(np.concatenate([np.full(m * N, float(N)), np.ones(m), np.ones(m * N)]))
    D = np.diag(np.concatenate([np.ones(m * N), np.ones(m), np.full(m * N, 1.0 / N)]))
    assert np.allclose(W @ S @ D, Sp, rtol=1e-13, atol=1e-16)
    r = rand_vec(L, 12)
    assert np.isclose(O.paper_norm(r, N), np.linalg.norm(W @ O.pack(r)), rtol=1e-14)


# --------------------------------------------------------------------------
# Averaged coarse coefficients
# --------------------------------------------------------------------------

def test_averaged_coarsening_constant_and_layered_media():
    """A coarse face of length 2h_f spans two fine faces: in a medium layered
    across the face direction they conduct in series (1/k_c is the mean of
    1/k), in a medium layered along it in parallel (k_c is the weighted mean
    over the three fine lines).  Constant media are reproduced exactly."""
    nf, N = 15, 2
    eta = np.array([0.7, 2.0])
    fine = O.make_level(nf, N, 1e-3, const_field(eta))
    c = O.averaged_coarse_level(fine)
    assert np.allclose(c.kx, eta) and np.allclose(c.ky, eta)
    # kappa depends on x only: vertical faces in series, horizontal faces parallel
    kx_only = lambda X, Y: np.stack([1.0 + 3.0 * (X > 0.4) + X, 2.0 + np.sin(5 * X)], axis=-1)
    fine = O.make_level(nf, N, 1e-3, kx_only)
    c = O.averaged_coarse_level(fine)
    nc = c.n
    for J in range(nc):
        for I in range(nc + 1):
            a, b = fine.kx[2 * J + 1, 2 * I], fine.kx[2 * J + 1, 2 * I + 1]
            assert np.allclose(1.0 / c.kx[J, I], 0.5 * (1.0 / a + 1.0 / b))
    for J in range(nc + 1):
        for I in range(nc):
            cols = fine.ky[2 * J, 2 * I:2 * I + 3]           # equal along y for kappa(x)
            assert np.allclose(c.ky[J, I], 0.25 * cols[0] + 0.5 * cols[1] + 0.25 * cols[2])
    # kappa depends on y only: the roles swap
    ky_only = lambda X, Y: kx_only(Y, X)
    fine = O.make_level(nf, N, 1e-3, ky_only)
    c = O.averaged_coarse_level(fine)
    for J in range(nc + 1):
        for I in range(nc):
            a, b = fine.ky[2 * J, 2 * I + 1], fine.ky[2 * J + 1, 2 * I + 1]
            assert np.allclose(1.0 / c.ky[J, I], 0.5 * (1.0 / a + 1.0 / b))


def test_averaged_coarsening_improves_contraction_on_rough_fields():
    """With a rough field (16 modes, amp 1) and small nu, sampling kappa on
    each coarse grid aliases the field; averaging the fine faces keeps the
    V-cycle contraction near the smooth-field rate (Sec. 3.2 robustness)."""
    n, N = 31, 8
    xi = inputs.draw_xi(2, N, 16)
    rates = {}
    for mode in ("nodal", "averaged"):
        levels = O.make_hierarchy(n, N, 1e-6, O.sine_mode_field(xi, 1.0), coarse=mode)
        f = O.fine_rhs(levels[0], inputs.target_sinsin(n))
        res = O.solve_stationary(levels, f, O.CycleOptions(), tol=1e-10, maxit=60)
        h = res.history
        rates[mode] = float(np.median([h[i + 1] / h[i] for i in range(2, len(h) - 1)]))
        assert res.relres <= 1e-10
    assert rates["averaged"] < 0.8 * rates["nodal"], rates
    assert rates["averaged"] < 0.35, rates


def test_frozen_control_cycles_solve_the_pdes_for_that_control():
    """With u fixed the system decouples into, per sample, A_j y_j = f_p,j - e u
    (state) and A_j p_j = f_y,j - c y_j (adjoint); frozen-control cycles
    (Eq. (14) smoothing with u_i given) converge to those dense solutions and
    leave u untouched."""
    n, N = 15, 3
    xi = inputs.draw_xi(70, N, 3)
    levels = O.make_hierarchy(n, N, 1e-4, O.sine_mode_field(xi, 0.9))
    lv = levels[0]
    f = O.fine_rhs(lv, inputs.target_modes(n, 8))
    u0 = np.sin(np.pi * inputs.grid_nodes(n)[0]) * 3.0
    x = (np.zeros((n, n, N)), u0.copy(), np.zeros((n, n, N)))
    opts = O.CycleOptions(freeze_u=True)
    for _ in range(25):
        x = O.cycle(levels, 0, x, f, opts)
    assert np.array_equal(x[1], u0)
    for j in range(N):
        A = assemble_A_by_faces(lv, j)
        yj = np.linalg.solve(A, (f[2][:, :, j] - lv.e * u0).ravel())
        pj = np.linalg.solve(A, (f[0][:, :, j] - lv.c * yj.reshape(n, n)).ravel())
        assert np.allclose(x[0][:, :, j].ravel(), yj, rtol=1e-9, atol=1e-12)
        assert np.allclose(x[2][:, :, j].ravel(), pj, rtol=1e-9, atol=1e-14)


def test_residual_vanishes_on_the_last_swept_colour():
    """After a collective red-black sweep (colour 0, then colour 1) every
    colour-1 node satisfies its own 2N+1 equations given neighbours that did
    not change afterwards, so f - S x is zero there in all three blocks (up
    to rounding) and not at colour 0; the GPU cycle computes and restricts
    only the colour-0 residual on this basis.  With the control frozen the
    control row is not solved and keeps its residual."""
    lv = small_level(n=7, N=3)
    rng = np.random.default_rng(5)
    n, N = lv.n, lv.N
    f = (rng.standard_normal((n, n, N)), rng.standard_normal((n, n)), rng.standard_normal((n, n, N)))
    x = (rng.standard_normal((n, n, N)), rng.standard_normal((n, n)), rng.standard_normal((n, n, N)))
    x = O.rbgs_sweep(lv, x, f)
    r = O.residual(lv, x, f)
    c1 = O.colour_mask(n, 1)
    c0 = O.colour_mask(n, 0)
    scale = max(np.abs(b).max() for b in f)
    for blk in r:
        assert np.abs(blk[c1]).max() <= 1e-12 * scale
    assert max(np.abs(blk[c0]).max() for blk in r) > 1e-3 * scale
    xf = O.rbgs_sweep(lv, x, f, freeze_u=True)
    rf = O.residual(lv, xf, f)
    assert np.abs(rf[0][c1]).max() <= 1e-12 * scale and np.abs(rf[2][c1]).max() <= 1e-12 * scale
    assert np.abs(rf[1][c1]).max() > 1e-6 * scale


# --------------------------------------------------------------------------
# Local control (the control acts on a subregion; Eq. (14) at the other nodes)
# --------------------------------------------------------------------------

LOCAL_BOX = (0.25, 0.75, 0.25, 0.75)   # the control region D_0 = (0.25, 0.75)^2 of Sec. 3.2


def local_kkt_solution(level, f):
    """Dense solution of the local-control optimality system assembled from
    its definition: the distributed system of assemble_S_blocks with the
    control unknowns (rows and columns) of the nodes outside the control
    region deleted; u = 0 there."""
    S = assemble_S_blocks(level)
    n, N = level.n, level.N
    m = n * n
    chi = level.chi.reshape(m)
    drop = [m * N + i for i in range(m) if chi[i] == 0.0]
    keep = np.setdiff1d(np.arange(S.shape[0]), drop)
    z = np.zeros(S.shape[0])
    z[keep] = np.linalg.solve(S[np.ix_(keep, keep)], O.pack(f)[keep])
    return z


def test_control_indicator_of_the_local_region():
    # n = 7, h = 1/8: nodes at 1/8 .. 7/8; the closed region [1/4, 3/4] holds columns 2/8 .. 6/8
    chi = O.control_indicator(7, LOCAL_BOX)
    expected = np.zeros((7, 7))
    expected[1:6, 1:6] = 1.0
    assert np.array_equal(chi, expected)
    assert np.array_equal(O.control_indicator(3, LOCAL_BOX), np.ones((3, 3)))     # 1/4, 1/2, 3/4
    assert np.array_equal(O.control_indicator(5, (0.0, 1.0, 0.0, 1.0)), np.ones((5, 5)))


@pytest.mark.parametrize("n,N", [(7, 2), (15, 2)])
@pytest.mark.parametrize("method", ["rbgs-V", "rbgs-W", "jacobi-V", "lexgs-V", "fgmres"])
def test_local_control_solvers_converge_to_dense_kkt(n, N, method):
    xi = inputs.draw_xi(40 + n + N, N, 3)
    levels = O.make_hierarchy(n, N, 1e-3, O.sine_mode_field(xi, 0.7), control_box=LOCAL_BOX)
    assert 0.0 < levels[0].chi.mean() < 1.0
    yd = inputs.target_modes(n, 6)
    f = O.fine_rhs(levels[0], yd)
    ref = local_kkt_solution(levels[0], f)
    if method == "fgmres":
        res = O.fgmres(levels, f, O.CycleOptions(), tol=1e-12)
    else:
        sm, cyc = method.split("-")
        opts = O.CycleOptions(smoother=sm, gamma=1 if cyc == "V" else 2)
        res = O.solve_stationary(levels, f, opts, tol=1e-12, maxit=300)
    assert res.relres <= 1e-12
    got = O.pack(res.x)
    assert np.linalg.norm(got - ref) <= 1e-9 * np.linalg.norm(ref)
    # no control outside the region, and some inside
    u = res.x[1]
    assert np.all(u[levels[0].chi == 0.0] == 0.0)
    assert np.abs(u[levels[0].chi == 1.0]).max() > 0.0


def test_local_control_on_the_whole_square_is_the_distributed_problem():
    xi = inputs.draw_xi(7, 3, 3)
    field = O.sine_mode_field(xi, 0.6)
    a = O.make_hierarchy(15, 3, 1e-4, field)
    b = O.make_hierarchy(15, 3, 1e-4, field, control_box=(0.0, 1.0, 0.0, 1.0))
    assert all(np.all(lev.chi == 1.0) for lev in b)
    f = O.fine_rhs(a[0], inputs.target_modes(15, 2))
    xa = xb = O.zeros_like_level(a[0])
    for _ in range(2):
        xa = O.cycle(a, 0, xa, f, O.CycleOptions())
        xb = O.cycle(b, 0, xb, f, O.CycleOptions())
    for u, v in zip(xa, xb):
        assert np.array_equal(u, v)


# --------------------------------------------------------------------------
# Two-level analysis in 1D (Sec. 3.1, Lemma 2, Theorem 1, Fig. 1)
# --------------------------------------------------------------------------

def two_level_1d(Nh, N, nu, eta, theta, n1, n2):
    """The 1D model of Sec. 3.1 in the node-collected ordering z: S = I (x) Bt
    + H (x) B with Bt = [[I/N, D], [D, -1 1^T / (nu N^2)]], B = [[0, -D/2],
    [-D/2, 0]], d_j = 2 eta_j / (h^2 N); collective Jacobi G = I - (I (x)
    Bt^-1) S, damped G_theta = (1 - theta) I + theta G; full weighting with
    rows (1/4, 1/2, 1/4) and linear interpolation 2 R^T (the reading whose
    action on the Fourier modes is the one the paper states); Galerkin coarse
    matrix S_c = R S P.  Returns T = G^n2 (I - P S_c^-1 R S) G^n1."""
    h = 1.0 / (Nh + 1)
    D = np.diag(2.0 * eta / (h * h * N))
    I_N, one = np.eye(N), np.ones((N, 1))
    Bt = np.block([[I_N / N, D], [D, -(one @ one.T) / (nu * N * N)]])
    B = np.block([[np.zeros((N, N)), -D / 2], [-D / 2, np.zeros((N, N))]])
    H = np.diag(np.ones(Nh - 1), 1) + np.diag(np.ones(Nh - 1), -1)
    S = np.kron(np.eye(Nh), Bt) + np.kron(H, B)
    G = np.eye(S.shape[0]) - np.kron(np.eye(Nh), np.linalg.inv(Bt)) @ S
    G = (1 - theta) * np.eye(S.shape[0]) + theta * G
    Nc = (Nh - 1) // 2
    Rt = np.zeros((Nc, Nh))
    for I in range(Nc):
        Rt[I, 2 * I: 2 * I + 3] = (0.25, 0.5, 0.25)
    R = np.kron(Rt, np.eye(2 * N))
    P = np.kron(2 * Rt.T, np.eye(2 * N))
    Sc = R @ S @ P
    CGC = np.eye(S.shape[0]) - P @ np.linalg.solve(Sc, R @ S)
    return np.linalg.matrix_power(G, n2) @ CGC @ np.linalg.matrix_power(G, n1)


def theorem1_spectrum(Nh, N, nu, eta, theta, n1, n2):
    """Theorem 1 with Lemma 1's sigma(C):
        kappa_ji = (c_j^4 (1 - d_ji) d^_jt,i^n + s_j^4 (1 - d_jt,i) d^_ji^n)
                   / (c_j^4 (1 - d_ji) + s_j^4 (1 - d_jt,i)),
    d_ji = -mu_j lambda_i, mu_j = 2 cos(j pi h), jt = Nh + 1 - j, c_j, s_j =
    cos, sin(j pi h / 2), n = n1 + n2, j = 1 .. (Nh+1)/2 - 1, i = 1 .. 2N,
    and zeros.  Damping (the remark after Corollary 2: G_theta = (1 - theta) I
    + theta G): the powers take d^ = 1 - theta + theta d, the weights keep the
    undamped d, and the modes j = (Nh+1)/2 (mu = 0, annihilated by R) add
    (1 - theta)^n, 2N times."""
    h = 1.0 / (Nh + 1)
    dt = 2.0 * eta / (h * h)
    E = np.mean(dt ** -2.0)
    r = E / (nu + E)
    lam = np.concatenate([[-0.5] * (2 * N - 2),
                          -0.5 * np.array([1 - r + 1j * np.sqrt((1 - r) * r), 1 - r - 1j * np.sqrt((1 - r) * r)])])
    n = n1 + n2
    out = []
    for j in range(1, (Nh + 1) // 2):
        jt = Nh + 1 - j
        mu, mut = 2 * np.cos(j * np.pi * h), 2 * np.cos(jt * np.pi * h)
        c2, s2 = np.cos(j * np.pi * h / 2) ** 2, np.sin(j * np.pi * h / 2) ** 2
        for li in lam:
            d, dtl = -mu * li, -mut * li
            dh, dth = 1 - theta + theta * d, 1 - theta + theta * dtl
            num = c2 * c2 * (1 - d) * dth ** n + s2 * s2 * (1 - dtl) * dh ** n
            out.append(num / (c2 * c2 * (1 - d) + s2 * s2 * (1 - dtl)))
    out += [(1 - theta) ** n] * (2 * N)
    return np.array(out)


@pytest.mark.parametrize("theta,n1,n2", [(1.0, 1, 1), (1.0, 2, 2), (0.5, 1, 1), (0.5, 2, 2)])
def test_two_level_spectrum_matches_theorem1(theta, n1, n2):
    """Fig. 1's setting (N_h = 31, N = 10, nu = 1e-2, n1 = n2 = 1) and V(2,2),
    undamped and with theta = 0.5: the eigenvalues of the assembled
    two-level operator are Theorem 1's kappa_ji, the damped correction and
    zeros (2N N_h in all); the spectral radius agrees to rounding."""
    Nh, N, nu = 31, 10, 1e-2
    eta = inputs.draw_xi(12, N, 1)[:, 0] * 0.3 + 1.5        # positive samples of eta
    assert np.all(eta > 0)
    ev = np.linalg.eigvals(two_level_1d(Nh, N, nu, eta, theta, n1, n2))
    pred = theorem1_spectrum(Nh, N, nu, eta, theta, n1, n2)
    pred = np.concatenate([pred, np.zeros(ev.size - pred.size)])
    assert ev.size == 2 * N * Nh
    # defective (Jordan) eigenvalues of the smoother are only accurate to ~sqrt(eps) in eig
    assert _match_spectra(ev, pred) < 1e-6
    assert np.isclose(np.abs(ev).max(), np.abs(pred).max(), rtol=1e-8, atol=1e-12)
    assert np.abs(ev).max() < 1.0


# --------------------------------------------------------------------------
# L1 + box problem: semismooth Newton (Sec. 4, Alg. 2)
# --------------------------------------------------------------------------

def test_newton_system_with_active_sets_matches_dense_lu():
    """The control row's coupling restricted to a node set (d_i = d chi_i) on
    every grid: the cycle and FGMRES converge to the dense solution of the
    system assembled from the blocks with that row coupling."""
    xi = inputs.draw_xi(21, 3, 3)
    levels = O.make_hierarchy(15, 3, 1e-3, O.sine_mode_field(xi, 0.7))
    rng = np.random.default_rng(5)
    chi = (rng.random((15, 15)) > 0.4).astype(np.float64)
    O.set_active(levels, chi)
    L = levels[0]
    S = assemble_S_blocks(L)
    m, N = 15 * 15, 3
    for r in range(m):                      # control row i couples to p_i,j with d chi_i
        for j in range(N):
            S[m * N + r, m * N + m + r * N + j] = L.d * chi.reshape(m)[r]
    f = (np.zeros((15, 15, N)), rng.standard_normal((15, 15)) * L.h ** 2, np.zeros((15, 15, N)))
    ref = np.linalg.solve(S, O.pack(f))
    for method in ("cycle", "fgmres"):
        if method == "cycle":
            res = O.solve_stationary(levels, f, O.CycleOptions(), tol=1e-12, maxit=200)
        else:
            res = O.fgmres(levels, f, O.CycleOptions(), tol=1e-12)
        assert res.relres <= 1e-12
        assert np.linalg.norm(O.pack(res.x) - ref) <= 1e-9 * np.linalg.norm(ref)


def prox_gradient_l1_box(level, yd, beta, a, b, iters=400):
    """Independent solve of the discrete L1 + box problem
        min_u 1/(2N) sum_j |y_j - y_d|^2 + nu/2 |u|^2 + beta |u|_1,  a <= u <= b,
        y_j = h^2 A_j^-1 u   (the objective of Sec. 4 with lumped mass h^2 I, divided by h^2)
    by proximal gradient: u <- clip(shrink(u - t grad, t beta), a, b), with
    dense A_j from the face assembly and step t = 1 / (largest eigenvalue of
    the Hessian)."""
    n, N, nu, h = level.n, level.N, level.nu, level.h
    m = n * n
    K = [h * h * np.linalg.inv(assemble_A_by_faces(level, j)) for j in range(N)]
    Hs = nu * np.eye(m) + sum(Kj @ Kj for Kj in K) / N
    t = 1.0 / np.linalg.eigvalsh(Hs).max()
    yv = yd.reshape(m)
    u = np.zeros(m)
    for _ in range(iters):
        g = nu * u + sum(Kj @ (Kj @ u - yv) for Kj in K) / N
        v = u - t * g
        u = np.clip(np.sign(v) * np.maximum(np.abs(v) - t * beta, 0.0), a, b)
    return u.reshape(n, n)


@pytest.mark.parametrize("inner", ["cycle", "fgmres"])
def test_semismooth_newton_matches_proximal_gradient(inner):
    """Algorithm 2 (multigrid inner solves, line search on phi) reaches
    phi < 1e-9 and the same control as an independent proximal-gradient solve
    of the discrete convex problem, with zero, interior and bound values all
    present; F vanishes at that control."""
    n, N, nu, beta, a, b = 15, 4, 1e-3, 1e-3, -1.0, 1.0
    xi = inputs.draw_xi(3, N, 3)
    levels = O.make_hierarchy(n, N, nu, O.sine_mode_field(xi, 0.6))
    yd = inputs.target_modes(n, 3) * 0.03
    res = O.semismooth_newton(levels, yd, beta, a, b, inner=inner)
    assert res.merit[-1] < 1e-9
    ref = prox_gradient_l1_box(levels[0], yd, beta, a, b)
    assert np.abs(res.u - ref).max() <= 1e-8 * np.abs(ref).max()
    u = res.u
    assert np.any(u == 0.0) and np.any(np.abs(u) == 1.0) and np.any((u != 0.0) & (np.abs(u) < 1.0))
    # F(u_ref) = 0 with T u from the per-sample PDE solves
    _, p = O.pde_states(levels, ref, yd)
    assert np.abs(O.ssn_F(ref, O.expected_adjoint(p), nu, beta, a, b)).max() <= 1e-8


def test_row_wavefront_order_equals_the_red_black_sweep():
    """An implementation identity for a one-pass sweep: updating the red
    nodes of row r and then the black nodes of row r - 1, for r = 0 .. n,
    gives the red-black sweep (all red, then all black) bit for bit -- a
    black node of row r - 1 couples only to red nodes of rows r - 2 .. r,
    all of them final by then, and nodes of one colour never couple."""
    import inputs

    n, N = 15, 4
    lv = O.make_hierarchy(n, N, 1e-4, O.sine_mode_field(inputs.draw_xi(3, N, 3), 0.7),
                          control_box=(0.2, 0.7, 0.3, 0.9))[0]
    rng = np.random.default_rng(41)
    x = (rng.standard_normal((n, n, N)), rng.standard_normal((n, n)), rng.standard_normal((n, n, N)))
    f = tuple(rng.standard_normal(b.shape) * s for b, s in zip(x, (lv.c, lv.G, lv.h ** 2)))
    ref = O.rbgs_sweep(lv, x, f)
    cur = tuple(np.array(b, copy=True) for b in x)

    def update_row(colour, r):
        # a half-sweep computes every node of the colour from the current
        # values; keep row r of it (same-colour nodes do not interact)
        nxt = O.rbgs_half_sweep(lv, cur, f, colour)
        for b, nb in zip(cur, nxt):
            b[r] = nb[r]

    for r in range(n + 1):
        if r < n:
            update_row(0, r)
        if r >= 1:
            update_row(1, r - 1)
    for a, b in zip(cur, ref):
        assert np.array_equal(a, b)
