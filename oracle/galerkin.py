"""Galerkin coarse operators for the collective multigrid: plain sparse-matrix oracle.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this module; it
shares no code with the CUDA library.

Sec. 3 (after the collective smoothing iteration, Eq. (11)) defines the
coarse matrices recursively from the finest one, S_l = R S_{l+1} P with
R = P^T, and its experiments (Sec. 3.2) smooth with the damped collective
Jacobi iteration, theta = 0.5, n1 = n2 = 2.  This module computes exactly
that, from the definitions and nothing else:

* the finest system matrix S assembled as a sparse matrix from the block
  definition of the full-space optimality system (Eq. (2) with this
  problem's blocks; ordering (y, u, p), y and p node-major with the
  sample index fastest, as ``cmg_oracle.pack``);
* the block prolongation P (the bilinear interpolation of every block) as
  a sparse matrix, and S_c = P^T S P by sparse products, level by level;
* collective Jacobi, Eq. (11): x += theta sum_i P_i S_ii^{-1} R_i (f - S x),
  with S_ii the (2N+1) x (2N+1) block of S on node i's unknowns, solved
  densely (no use of its arrow structure); and the Gauss-Seidel variant the
  paper names after Eq. (11): node groups in turn, each node's block row
  solved with the current values of the others (red-black on the 5-point
  finest grid, four colours (iy mod 2, ix mod 2) on the 9-point grids);
* Algorithm 1 with that smoother, the residual f - S x by a sparse
  product, the transfers by P and P^T, and a sparse direct solve on the
  coarsest grid.

Distributed control only (chi = 1, dw = 1 on every grid).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import cmg_oracle as O


def stiffness_matrix(level: O.Level, j: int) -> sp.csr_matrix:
    """A_j of the grid (the stiffness block of Eq. (2)): row i holds the sum of node i's four face
    coefficients on the diagonal and minus the face coefficient towards
    each interior neighbour (a neighbour on the boundary is a zero
    Dirichlet value and has no column)."""
    n = level.n
    rows, cols, vals = [], [], []
    for iy in range(n):
        for ix in range(n):
            i = iy * n + ix
            kW, kE = level.kx[iy, ix, j], level.kx[iy, ix + 1, j]
            kS, kN = level.ky[iy, ix, j], level.ky[iy + 1, ix, j]
            rows.append(i)
            cols.append(i)
            vals.append(kW + kE + kS + kN)
            for (ny, nx), k in (((iy, ix - 1), kW), ((iy, ix + 1), kE), ((iy - 1, ix), kS), ((iy + 1, ix), kN)):
                if 0 <= ny < n and 0 <= nx < n:
                    rows.append(i)
                    cols.append(ny * n + nx)
                    vals.append(-k)
    m = n * n
    return sp.csr_matrix((vals, (rows, cols)), shape=(m, m))


def system_matrix(level: O.Level) -> sp.csr_matrix:
    """The full-space system (Sec. 2, Eq. (2)) in the symmetric form on this grid:

        [ c I_m (x) I_N      0          blkdiag(A_j) ]   y
        [ 0                  G I_m      d (I_m (x) 1_N^T) ]   u
        [ blkdiag(A_j)       e (I_m (x) 1_N)   0      ]   p

    with y, p ordered [node][sample] (I_m (x) B puts B on every node)."""
    if level.chi is not None or level.dw is not None:
        raise ValueError("Galerkin hierarchy: distributed control only")
    n, N = level.n, level.N
    m = n * n
    # blkdiag over samples of A_j in the node-major, sample-fastest ordering:
    # entry (i N + j, k N + j) = (A_j)_{ik}
    rows, cols, vals = [], [], []
    for j in range(N):
        A = stiffness_matrix(level, j).tocoo()
        rows.append(A.row * N + j)
        cols.append(A.col * N + j)
        vals.append(A.data)
    Ablk = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(m * N, m * N))
    Im = sp.identity(m, format="csr")
    ones_col = sp.csr_matrix(np.ones((N, 1)))
    Y = level.c * sp.identity(m * N, format="csr")
    U = level.G * Im
    D = level.d * sp.kron(Im, ones_col.T, format="csr")      # u-row, p columns: d sum_j p_ij
    E = level.e * sp.kron(Im, ones_col, format="csr")        # p-rows, u column: e u_i
    return sp.bmat([[Y, None, Ablk], [None, U, D], [Ablk, E, None]], format="csr")


def prolongation_matrix(nf: int, N: int) -> sp.csr_matrix:
    """Block prolongation (Algorithm 1's P) of a full-space vector from the (nf-1)/2 grid to
    the nf grid: the bilinear interpolation P2 = P1 (x) P1 (row index
    iy nf + ix, the 1D operator along y outside) on every sample of y and
    p and on u."""
    P1 = sp.csr_matrix(O.prolongation_1d(nf))
    P2 = sp.kron(P1, P1, format="csr")
    PN = sp.kron(P2, sp.identity(N, format="csr"), format="csr")
    return sp.block_diag([PN, P2, PN], format="csr")


def hierarchy(levels) -> list[sp.csr_matrix]:
    """S_0 from the finest grid's definition, S_{l+1} = P^T S_l P (Sec. 3; the
    grids of ``levels`` fix only the sizes below the finest)."""
    N = levels[0].N
    S = [system_matrix(levels[0])]
    for l in range(1, len(levels)):
        P = prolongation_matrix(levels[l - 1].n, N)
        S.append((P.T @ S[-1] @ P).tocsr())
    return S


def node_indices(n: int, N: int, i: int) -> np.ndarray:
    """Positions of node i's 2N+1 unknowns (y_i, u_i, p_i) in a packed vector."""
    m = n * n
    return np.concatenate([i * N + np.arange(N), [m * N + i], m * N + m + i * N + np.arange(N)])


_BLOCKS: dict = {}


def node_blocks(S: sp.csr_matrix, n: int, N: int):
    """The positions [n^2, 2N+1] of every node's unknowns and the dense
    diagonal blocks S_ii [n^2, 2N+1, 2N+1] (the node systems of Eq. (12);
    extracted once per matrix)."""
    hit = _BLOCKS.get(id(S))
    if hit is None or hit[0] is not S:
        idx = np.stack([node_indices(n, N, i) for i in range(n * n)])
        B = np.stack([S[row][:, row].toarray() for row in idx])
        hit = (S, idx, B)
        _BLOCKS[id(S)] = hit
    return hit[1], hit[2]


def jacobi_sweep(S: sp.csr_matrix, n: int, N: int, z: np.ndarray, f: np.ndarray, theta: float) -> np.ndarray:
    """One collective Jacobi step (Eq. (11)) on packed vectors: every node's
    block solved densely (one batched solve; the nodes' unknowns are
    disjoint)."""
    idx, B = node_blocks(S, n, N)
    r = f - S @ z
    out = z.copy()
    out[idx] += theta * np.linalg.solve(B, r[idx][..., None])[..., 0]
    return out


def colour_sweep(S: sp.csr_matrix, n: int, N: int, z: np.ndarray, f: np.ndarray, colours) -> np.ndarray:
    """Collective block Gauss-Seidel (the variant named after Eq. (11)): the
    groups of nodes in `colours` (lists of node indices, no two nodes of a
    group coupled) in turn, each node's unknowns replaced by the solution of
    its block row with the current values of all other unknowns."""
    idx_all, B = node_blocks(S, n, N)
    z = z.copy()
    for nodes in colours:
        idx = idx_all[nodes]
        r = f - S @ z
        z[idx] += np.linalg.solve(B[nodes], r[idx][..., None])[..., 0]
    return z


def four_colours(n: int):
    """Nodes by (iy mod 2, ix mod 2), in the order (0,0), (0,1), (1,0), (1,1):
    a 9-point stencil couples no two nodes of one group."""
    iy, ix = np.divmod(np.arange(n * n), n)
    return [np.flatnonzero((iy % 2 == a) & (ix % 2 == b)) for a in (0, 1) for b in (0, 1)]


def red_black(n: int):
    """Red ((ix + iy) even) then black: the 5-point finest grid's ordering."""
    iy, ix = np.divmod(np.arange(n * n), n)
    return [np.flatnonzero((iy + ix) % 2 == c) for c in (0, 1)]


def smooth(S, ns, N: int, l: int, z, f, smoother: str, theta: float):
    """One sweep on grid l: damped collective Jacobi, or Gauss-Seidel in
    red-black order on the finest (5-point) grid and in four colours on the
    Galerkin (9-point) grids."""
    if smoother == "jacobi":
        return jacobi_sweep(S[l], ns[l], N, z, f, theta)
    return colour_sweep(S[l], ns[l], N, z, f, red_black(ns[l]) if l == 0 else four_colours(ns[l]))


def cycle(S, ns, N: int, l: int, z: np.ndarray, f: np.ndarray, n1: int = 2, n2: int = 2, theta: float = 0.5,
          gamma: int = 1, smoother: str = "jacobi") -> np.ndarray:
    """Algorithm 1 on packed vectors with the Galerkin matrices S[l] on the
    grids ns[l] (finest first); gamma = 2 gives the W-cycle."""
    if l == len(S) - 1:
        return spla.spsolve(S[l].tocsc(), f)
    for _ in range(n1):
        z = smooth(S, ns, N, l, z, f, smoother, theta)
    P = prolongation_matrix(ns[l], N)
    fc = P.T @ (f - S[l] @ z)
    ec = np.zeros(S[l + 1].shape[0])
    for _ in range(gamma):
        ec = cycle(S, ns, N, l + 1, ec, fc, n1, n2, theta, gamma, smoother)
    z = z + P @ ec
    for _ in range(n2):
        z = smooth(S, ns, N, l, z, f, smoother, theta)
    return z


def solve_stationary(S, ns, N: int, f: np.ndarray, tol: float = 1e-10, maxit: int = 100, **kw):
    """Repeated cycles from zero until the relative residual of the paper's
    system, ||W (f - S z)|| / ||W f|| (``cmg_oracle.paper_norm``), is <= tol;
    returns (z, cycles, history of relative residuals, the first entry for
    z = 0)."""
    n = ns[0]
    z = np.zeros_like(f)
    fnorm = O.paper_norm(O.unpack(f, n, N), N)
    hist = [1.0]
    it = 0
    while hist[-1] > tol and it < maxit:
        z = cycle(S, ns, N, 0, z, f, **kw)
        it += 1
        hist.append(O.paper_norm(O.unpack(f - S[0] @ z, n, N), N) / fnorm)
    return z, it, hist


# ---------------------------------------------------------------------------
# Local control (Sec. 3.1 after Eq. (13)): the control exists only at the nodes
# with a control basis function (chi = 1); the Galerkin products then act on
# the unknowns that exist.
# ---------------------------------------------------------------------------

def system_matrix_local(level: O.Level) -> sp.csr_matrix:
    """Eq. (2) with u only at the control nodes (ordering y, u on the control
    nodes in node order, p): the control block and its couplings are the
    distributed ones restricted to those nodes."""
    if level.dw is not None:
        raise ValueError("per-node factors on d are not part of this form")
    n, N = level.n, level.N
    m = n * n
    full = system_matrix(O.Level(level.n, level.N, level.nu, level.h, level.kx, level.ky, level.a, level.c,
                                 level.G, level.d, level.e))
    ctl = np.flatnonzero(level.control().ravel() != 0.0)
    keep = np.concatenate([np.arange(m * N), m * N + ctl, m * N + m + np.arange(m * N)])
    return full[keep][:, keep].tocsr()


def prolongation_matrix_local(nf: int, N: int, ctl_f: np.ndarray, ctl_c: np.ndarray) -> sp.csr_matrix:
    """The block prolongation with the control block restricted to the fine
    and coarse control nodes (flat index arrays)."""
    P1 = sp.csr_matrix(O.prolongation_1d(nf))
    P2 = sp.kron(P1, P1, format="csr")
    PN = sp.kron(P2, sp.identity(N, format="csr"), format="csr")
    return sp.block_diag([PN, P2[ctl_f][:, ctl_c], PN], format="csr")


def hierarchy_local(levels):
    """(S_l, control node indices per grid) with S_{l+1} = P^T S_l P."""
    N = levels[0].N
    ctls = [np.flatnonzero(lv.control().ravel() != 0.0) for lv in levels]
    S = [system_matrix_local(levels[0])]
    for l in range(1, len(levels)):
        P = prolongation_matrix_local(levels[l - 1].n, N, ctls[l - 1], ctls[l])
        S.append((P.T @ S[-1] @ P).tocsr())
    return S, ctls


def _local_groups(n: int, N: int, ctl: np.ndarray):
    m = n * n
    pos = -np.ones(m, dtype=int)
    pos[ctl] = np.arange(ctl.size)
    nu_ = ctl.size
    ar = np.arange(N)
    on = [np.concatenate([i * N + ar, [m * N + pos[i]], m * N + nu_ + i * N + ar]) for i in range(m) if pos[i] >= 0]
    off = [np.concatenate([i * N + ar, m * N + nu_ + i * N + ar]) for i in range(m) if pos[i] < 0]
    return [np.stack(g) for g in (on, off) if g]


_LBLOCKS: dict = {}


def jacobi_sweep_local(S, n: int, N: int, ctl: np.ndarray, z, f, theta: float):
    """Collective Jacobi (Eq. (11)) with dense node blocks: 2N+1 unknowns at
    control nodes (Eq. (13)), 2N elsewhere (Eq. (14))."""
    hit = _LBLOCKS.get(id(S))
    if hit is None or hit[0] is not S:
        hit = (S, [(idx, np.stack([S[row][:, row].toarray() for row in idx])) for idx in _local_groups(n, N, ctl)])
        _LBLOCKS[id(S)] = hit
    r = f - S @ z
    out = z.copy()
    for idx, B in hit[1]:
        out[idx] += theta * np.linalg.solve(B, r[idx][..., None])[..., 0]
    return out


def cycle_local(S, ctls, ns, N: int, l: int, z, f, n1: int = 2, n2: int = 2, theta: float = 0.5):
    """Algorithm 1 (V-cycle) on the local-control Galerkin hierarchy."""
    if l == len(S) - 1:
        return spla.spsolve(S[l].tocsc(), f)
    for _ in range(n1):
        z = jacobi_sweep_local(S[l], ns[l], N, ctls[l], z, f, theta)
    P = prolongation_matrix_local(ns[l], N, ctls[l], ctls[l + 1])
    ec = cycle_local(S, ctls, ns, N, l + 1, np.zeros(S[l + 1].shape[0]), P.T @ (f - S[l] @ z), n1, n2, theta)
    z = z + P @ ec
    for _ in range(n2):
        z = jacobi_sweep_local(S[l], ns[l], N, ctls[l], z, f, theta)
    return z


def solve_stationary_local(S, ctls, ns, N: int, f, tol: float = 1e-10, maxit: int = 100, **kw):
    """Repeated V-cycles until the paper's relative residual (state rows
    weighted by N) is <= tol; returns (z, cycles, history)."""
    m = ns[0] ** 2
    w = np.concatenate([np.full(m * N, float(N)), np.ones(S[0].shape[0] - m * N)])
    z = np.zeros_like(f)
    fn = np.linalg.norm(w * f)
    hist = [1.0]
    while hist[-1] > tol and len(hist) <= maxit:
        z = cycle_local(S, ctls, ns, N, 0, z, f, **kw)
        hist.append(np.linalg.norm(w * (f - S[0] @ z)) / fn)
    return z, len(hist) - 1, hist


def fgmres_packed(S0, precondition, f, N: int, m: int, tol: float = 1e-10, maxit: int = 60):
    """Flexible GMRES without restarts on the paper's row scaling W S z = W f
    (W = N on the m N state rows, 1 elsewhere), right-preconditioned by
    `precondition(v)` (one cycle applied to W^{-1} v); Gram-Schmidt applied
    twice, the small least-squares problem solved afresh at every step.
    Returns (z, iterations, history of relative residuals)."""
    w = np.concatenate([np.full(m * N, float(N)), np.ones(S0.shape[0] - m * N)])
    b = w * f
    beta = np.linalg.norm(b)
    V, Z = [b / beta], []
    H = np.zeros((maxit + 1, maxit))
    hist, y = [1.0], np.zeros(0)
    for k in range(maxit):
        z = precondition(V[k] / w)
        Z.append(z)
        v = w * (S0 @ z)
        for _ in range(2):
            for i in range(k + 1):
                c = V[i] @ v
                H[i, k] += c
                v = v - c * V[i]
        H[k + 1, k] = np.linalg.norm(v)
        V.append(v / H[k + 1, k])
        e1 = np.zeros(k + 2)
        e1[0] = beta
        y, *_ = np.linalg.lstsq(H[: k + 2, : k + 1], e1, rcond=None)
        hist.append(np.linalg.norm(e1 - H[: k + 2, : k + 1] @ y) / beta)
        if hist[-1] <= tol:
            break
    return np.array(Z).T @ y, len(Z), hist
