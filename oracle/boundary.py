"""Neumann boundary control on Gamma = (0,1) x {0}: plain sparse-matrix oracle.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this module; it
shares no code with the CUDA library.

Sec. 2 allows a control operator B acting as a Neumann condition on part of
the boundary; Sec. 3.1 (after Eq. (13)) smooths nodes that carry a control
basis function with Eq. (13) and the others with Eq. (14) (u_i = 0); Sec. 3.2
tests the control on Gamma = (0,1) x {0} of the unit square.  This module
writes that problem out:

* grid: h = 1/(n+1); columns ix = 0..n-1 at x = (ix+1) h (Dirichlet at
  x = 0 and x = 1), rows r = 0..n at y = r h, row 0 on Gamma, Dirichlet at
  y = 1; node index r n + ix, (n+1) n nodes (992 for n = 31, the paper's
  N_h for this case);
* stiffness A_j: the integrated 5-point stencil on the dual cells with
  harmonic-mean face coefficients, as on the square; the cells of row 0 are
  half as high, so their two x-faces carry half the coefficient and they
  have no south face (the flux there is the control);
* lumped masses: h^2 per node, h^2/2 on row 0; on Gamma the 1D lumped mass
  h per row-0 node;
* the optimality system in the symmetric scaling used throughout,
      (M/N) y_j + A_j p_j       = (M/N) y_d      (state rows)
      nu h u - h sum_j p_j|Gamma = 0             (control rows, row-0 nodes)
      A_j y_j - h u|Gamma        = M f           (adjoint rows)
  with u on the n row-0 nodes only;
* transfers: row 0 stays on Gamma on every grid (coarse row R = fine row
  2R, the odd fine rows interpolated, the top one against the Dirichlet
  value), the columns as on the square; the control block is prolongated
  along Gamma; coarse matrices S_c = P^T S P (Sec. 3, Galerkin);
* smoothing: collective Jacobi, Eq. (11), with each node's diagonal block
  solved densely: 2N+1 unknowns on Gamma (Eq. (13)), 2N elsewhere
  (Eq. (14)); Algorithm 1 with a sparse direct solve on the coarsest grid.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import cmg_oracle as O


def faces(n: int, N: int, kappa_fn):
    """Face coefficients (harmonic means of the endpoint values of kappa;
    the field of Sec. 3.2 sampled on this grid, as on the square).

    kx [n+1, n+1, N]: row r, face f between columns f-1 and f (f = 0 and
    f = n touch x = 0 and x = 1).  ky [n+1, n, N]: face between rows r and
    r+1 of column ix (r = n touches y = 1)."""
    h = 1.0 / (n + 1)
    t = np.arange(n + 2, dtype=np.float64) * h
    X, Y = np.meshgrid(t, t, indexing="xy")            # [y index, x index], y = 0 .. 1
    kap = kappa_fn(X, Y)                               # [n+2, n+2, N]
    kx = O.harmonic_mean(kap[:-1, :-1], kap[:-1, 1:])  # rows y = 0 .. n h, faces between x neighbours
    ky = O.harmonic_mean(kap[:-1, 1:-1], kap[1:, 1:-1])  # faces between y = r h and (r+1) h, interior x
    return kx, ky


def stiffness_matrix(n: int, kx, ky, j: int) -> sp.csr_matrix:
    """A_j of the state equation (Sec. 2, Eq. (2)'s stiffness block) with the
    Neumann edge: dual-cell fluxes, row 0's x-faces halved, no south face."""
    rows, cols, vals = [], [], []
    for r in range(n + 1):
        s = 0.5 if r == 0 else 1.0
        for ix in range(n):
            i = r * n + ix
            kW, kE = s * kx[r, ix, j], s * kx[r, ix + 1, j]
            kN = ky[r, ix, j]
            kS = ky[r - 1, ix, j] if r > 0 else 0.0
            rows.append(i)
            cols.append(i)
            vals.append(kW + kE + kS + kN)
            for (rr, cc), k in (((r, ix - 1), kW), ((r, ix + 1), kE), ((r - 1, ix), kS), ((r + 1, ix), kN)):
                if 0 <= rr <= n and 0 <= cc < n and k != 0.0:
                    rows.append(i)
                    cols.append(rr * n + cc)
                    vals.append(-k)
    m = (n + 1) * n
    return sp.csr_matrix((vals, (rows, cols)), shape=(m, m))


def mass(n: int) -> np.ndarray:
    """Lumped mass per node (Sec. 2's M): h^2, h^2/2 on row 0."""
    h = 1.0 / (n + 1)
    w = np.full((n + 1, n), h * h)
    w[0] *= 0.5
    return w.ravel()


def system_matrix(n: int, N: int, nu: float, kx, ky) -> sp.csr_matrix:
    """The full-space optimality system (Sec. 2, Eq. (2)) with B the Neumann
    control on the row-0 nodes; ordering (y [node][sample], u [row-0 node],
    p [node][sample])."""
    h = 1.0 / (n + 1)
    m = (n + 1) * n
    rows, cols, vals = [], [], []
    for j in range(N):
        A = stiffness_matrix(n, kx, ky, j).tocoo()
        rows.append(A.row * N + j)
        cols.append(A.col * N + j)
        vals.append(A.data)
    Ablk = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(m * N, m * N))
    Y = sp.diags(np.repeat(mass(n) / N, N))
    U = nu * h * sp.identity(n)
    # B: row-0 node ix of every sample couples to u_ix with weight h
    Bp = sp.csr_matrix((np.full(n * N, h), (np.arange(n * N), np.repeat(np.arange(n), N))), shape=(m * N, n))
    return sp.bmat([[Y, None, Ablk], [None, U, -Bp.T], [Ablk, -Bp, None]], format="csr")


def rhs(n: int, N: int, yd: np.ndarray, f: np.ndarray | None = None) -> np.ndarray:
    """Right side of Eq. (2): (M y_d / N, 0, M f) with yd, f [(n+1) n] node values."""
    w = mass(n)
    fy = np.repeat(w * yd / N, N)
    fp = np.zeros(w.size * N) if f is None else np.repeat(w * f, N)
    return np.concatenate([fy, np.zeros(n), fp])


def node_values(n: int, fn) -> np.ndarray:
    """fn(x, y) at the nodes, [(n+1) n]."""
    h = 1.0 / (n + 1)
    X, Y = np.meshgrid((np.arange(n) + 1) * h, np.arange(n + 1) * h, indexing="xy")
    return fn(X, Y).ravel()


def prolongation_y(n: int) -> np.ndarray:
    """Rows 0..n from rows 0..nc (nc = (n-1)/2): fine row 2R is coarse row R,
    fine row 2R+1 halfway between R and R+1 (R+1 = nc+1 is y = 1: zero)."""
    nc = (n - 1) // 2
    P = np.zeros((n + 1, nc + 1))
    for R in range(nc + 1):
        P[2 * R, R] = 1.0
        P[2 * R + 1, R] = 0.5
        if R > 0:
            P[2 * R - 1, R] = 0.5
    return P


def prolongation_matrix(n: int, N: int) -> sp.csr_matrix:
    Px = sp.csr_matrix(O.prolongation_1d(n))
    P2 = sp.kron(sp.csr_matrix(prolongation_y(n)), Px, format="csr")
    PN = sp.kron(P2, sp.identity(N, format="csr"), format="csr")
    return sp.block_diag([PN, Px, PN], format="csr")


def hierarchy(n: int, N: int, nu: float, kappa_fn, coarsest_n: int = 3):
    """(grid sizes finest first, S_l): S_0 from the definition, S_{l+1} = P^T S_l P
    (the Galerkin coarse matrices of Sec. 3)."""
    kx, ky = faces(n, N, kappa_fn)
    ns = [n]
    while ns[-1] != coarsest_n:
        ns.append((ns[-1] - 1) // 2)
    S = [system_matrix(n, N, nu, kx, ky)]
    for l in range(1, len(ns)):
        P = prolongation_matrix(ns[l - 1], N)
        S.append((P.T @ S[-1] @ P).tocsr())
    return ns, S


def node_groups(n: int, N: int):
    """Unknown positions per node: [n, 2N+1] for the row-0 nodes (y_i, u_i, p_i)
    and [n n, 2N] for the others (y_i, p_i)."""
    m = (n + 1) * n
    ar = np.arange(N)
    gam = np.stack([np.concatenate([i * N + ar, [m * N + i], m * N + n + i * N + ar]) for i in range(n)])
    inner = np.stack([np.concatenate([i * N + ar, m * N + n + i * N + ar]) for i in range(n, m)])
    return gam, inner


_BLOCKS: dict = {}


def _blocks(S, n: int, N: int):
    hit = _BLOCKS.get(id(S))
    if hit is None or hit[0] is not S:
        gam, inner = node_groups(n, N)
        hit = (S, [(idx, np.stack([S[row][:, row].toarray() for row in idx])) for idx in (gam, inner)])
        _BLOCKS[id(S)] = hit
    return hit[1]


def jacobi_sweep(S, n: int, N: int, z: np.ndarray, f: np.ndarray, theta: float) -> np.ndarray:
    """Collective Jacobi, Eq. (11): every node's block solved densely."""
    r = f - S @ z
    out = z.copy()
    for idx, B in _blocks(S, n, N):
        out[idx] += theta * np.linalg.solve(B, r[idx][..., None])[..., 0]
    return out


def cycle(S, ns, N: int, l: int, z, f, n1: int = 2, n2: int = 2, theta: float = 0.5, gamma: int = 1):
    """Algorithm 1 (gamma = 2: W-cycle) with collective Jacobi and a direct
    solve on the coarsest grid."""
    if l == len(S) - 1:
        return spla.spsolve(S[l].tocsc(), f)
    for _ in range(n1):
        z = jacobi_sweep(S[l], ns[l], N, z, f, theta)
    P = prolongation_matrix(ns[l], N)
    fc = P.T @ (f - S[l] @ z)
    ec = np.zeros(S[l + 1].shape[0])
    for _ in range(gamma):
        ec = cycle(S, ns, N, l + 1, ec, fc, n1, n2, theta, gamma)
    z = z + P @ ec
    for _ in range(n2):
        z = jacobi_sweep(S[l], ns[l], N, z, f, theta)
    return z


def paper_norm(v: np.ndarray, n: int, N: int) -> float:
    """The paper's row scaling: state rows N times the symmetric ones."""
    m = (n + 1) * n
    return float(np.sqrt(N * N * np.sum(v[: m * N] ** 2) + np.sum(v[m * N:] ** 2)))


def solve_stationary(S, ns, N: int, f, tol: float = 1e-10, maxit: int = 100, **kw):
    """Repeated cycles from zero until the relative residual of the paper's
    system (Sec. 3.2) is <= tol; returns (z, cycles, history)."""
    n = ns[0]
    z = np.zeros_like(f)
    fn = paper_norm(f, n, N)
    hist = [1.0]
    it = 0
    while hist[-1] > tol and it < maxit:
        z = cycle(S, ns, N, 0, z, f, **kw)
        it += 1
        hist.append(paper_norm(f - S[0] @ z, n, N) / fn)
    return z, it, hist


def reduced_control(n: int, N: int, nu: float, kx, ky, yd: np.ndarray, f: np.ndarray | None = None) -> np.ndarray:
    """The minimiser u of the reduced problem
        J(u) = 1/(2N) sum_j (y_j - y_d)^T M (y_j - y_d) + nu/2 h u^T u,
        A_j y_j = B u + M f,  (B u)_i = h u_ix on row-0 nodes,
    from its normal equations (dense, small grids): the same optimum by a
    route that never forms the saddle-point system."""
    h = 1.0 / (n + 1)
    m = (n + 1) * n
    w = mass(n)
    B = np.zeros((m, n))
    B[np.arange(n), np.arange(n)] = h
    lhs = nu * h * np.eye(n)
    rhs_ = np.zeros(n)
    mf = np.zeros(m) if f is None else w * f
    for j in range(N):
        Ainv = np.linalg.inv(stiffness_matrix(n, kx, ky, j).toarray())
        T = Ainv @ B                                   # y_j = T u + Ainv M f
        lhs += T.T @ (w[:, None] * T) / N
        rhs_ += T.T @ (w * (yd - Ainv @ mf)) / N
    return np.linalg.solve(lhs, rhs_)


def fgmres(S, ns, N: int, f, tol: float = 1e-10, maxit: int = 60, **kw):
    """Flexible GMRES without restarts, right-preconditioned by one cycle, on
    the paper's row scaling W S z = W f (W = diag(N I, 1, 1) on the state,
    control and adjoint rows; the relative residual it minimises is the one
    the paper reports).  Arnoldi with Gram-Schmidt applied twice; the small
    least-squares problem is solved afresh at every step.  Returns
    (z, iterations, history of relative residuals)."""
    n = ns[0]
    m = (n + 1) * n
    w = np.concatenate([np.full(m * N, float(N)), np.ones(S[0].shape[0] - m * N)])
    b = w * f
    beta = np.linalg.norm(b)
    V = [b / beta]
    Z, H = [], np.zeros((maxit + 1, maxit))
    hist = [1.0]
    y = np.zeros(0)
    for k in range(maxit):
        z = cycle(S, ns, N, 0, np.zeros_like(f), V[k] / w, **kw)
        Z.append(z)
        v = w * (S[0] @ z)
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
    z = np.array(Z).T @ y
    return z, len(Z), hist
