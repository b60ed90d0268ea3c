"""Plain FP64 CPU oracle of the collective multigrid method.

TEST INFRASTRUCTURE ONLY.  This module exists to check the CUDA path: only
the tests, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import it.  It shares no code with the CUDA
library and imports nothing from the product package.

It computes, slowly and in the order the paper states them:

* the discrete linear-quadratic problem under uncertainty (Sec. 2, the
  full-space optimality system), in its symmetric form: the N state
  block rows and the N adjoint block rows carry the quadrature weight
  1/N on the mass block only, i.e.
      (h^2/N) y_j + A_j p_j        = (h^2/N) y_d          (state-row block)
      nu h^2 u   - h^2 sum_j p_j   = 0                     (control row)
      A_j y_j    - h^2 u           = h^2 f                 (adjoint-row block)
  which is the generic block form of Eq. (2) with C_j = M/N, G = nu M,
  D_j = E_j = -M, M = h^2 I (lumped mass), A_j the integrated 5-point
  stiffness of -div(kappa_j grad) with harmonic-mean face coefficients;
* the node-collected reduced systems (Eq. 12) and their O(N) solution by
  a Schur complement on u_i (Eq. 13);
* collective smoothing: damped collective Jacobi (Eq. 11), lexicographic
  and red-black collective Gauss-Seidel (the variants named after Eq. 11);
* transfers: bilinear prolongation P and restriction R = P^T, coarse
  operators rediscretised on each grid (the alternative the paper names
  beside its Galerkin choice, Sec. 3) with face coefficients harmonically
  averaged from the next finer grid;
* the coarsest-grid direct solve and the V/W-cycle of Algorithm 1;
* the V-cycle used stationary and as right preconditioner of flexible
  GMRES, stopped on the relative unpreconditioned residual of the paper's
  own (unsymmetric) system (Sec. 3.2; see paper_norm);
* local control (Sec. 3.1 after Eq. (13), and the local-control
  experiment of Sec. 3.2): the control has a basis function only at the
  nodes of a control region (indicator chi); at the other nodes u_i = 0,
  the control row is absent and the smoother takes Eq. (14) with u_i = 0.

Where the paper is silent the code takes one reading and states it in the
docstring of the function it concerns.

Storage: node arrays are [n, n, ...] indexed [iy, ix]; y and p carry a
trailing sample axis [n, n, N]; u is [n, n].  The lexicographic node index
is i = iy * n + ix (x fastest), so reshape(n*n, N) gives the [node][sample]
layout of the CUDA path.
"""
from __future__ import annotations

from dataclasses import dataclass
import numpy as np


# ---------------------------------------------------------------------------
# Random diffusion field and grid levels
# ---------------------------------------------------------------------------

def sine_mode_field(xi: np.ndarray, amp: float):
    """kappa_j(x, y) = exp(amp * sum_k xi[j,k] sin(k pi x) sin(pi y) / k).

    The sine-mode stand-in for the log-normal field of Eq. (15) (Sec. 3.2):
    a log-Gaussian field whose modes vanish on the boundary, so kappa = 1
    there.  Returns a function of coordinate arrays X, Y (same shape S)
    giving an array of shape S + (N,).
    """
    xi = np.asarray(xi, dtype=np.float64)
    N, K = xi.shape

    def kappa(X, Y):
        g = np.zeros(X.shape + (N,))
        for k in range(1, K + 1):
            mode = np.sin(k * np.pi * X) * np.sin(np.pi * Y) / k
            g += mode[..., None] * xi[:, k - 1]
        return np.exp(amp * g)

    return kappa


def harmonic_mean(ka, kb):
    """Face coefficient between two nodes with nodal values ka, kb."""
    return 2.0 * ka * kb / (ka + kb)


@dataclass
class Level:
    """One grid of the hierarchy with its rediscretised operator.

    n     interior nodes per side, h = 1/(n+1)
    kx    [n, n+1, N]  face coefficients on vertical faces; kx[iy, f] lies
          between interior columns f-1 and f (f = 0 and f = n touch the
          boundary x = 0 and x = 1)
    ky    [n+1, n, N]  the same for horizontal faces
    a     [n, n, N]    diag(A_j) at each node (sum of its four faces)
    c, G, d, e        the scalar diagonal blocks of Eq. (12) on this grid:
          c = h^2/N, G = nu h^2, d = e = -h^2
    chi   [n, n]       1.0 where the node carries a control basis function,
          0.0 where it does not (local control); all ones by default
    dw    [n, n]       per-node factor on d (the control row's coupling to the
          adjoint), all ones by default; the semismooth Newton systems of
          Sec. 4 set it to the indicator of the active sets
    """

    n: int
    N: int
    nu: float
    h: float
    kx: np.ndarray
    ky: np.ndarray
    a: np.ndarray
    c: float
    G: float
    d: float
    e: float
    chi: np.ndarray | None = None
    dw: np.ndarray | None = None

    def control(self) -> np.ndarray:
        return np.ones((self.n, self.n)) if self.chi is None else self.chi

    def dnode(self) -> np.ndarray:
        """d_i per node: d times dw_i."""
        return self.d * (np.ones((self.n, self.n)) if self.dw is None else self.dw)

    @property
    def sigma(self) -> np.ndarray:
        """Schur denominator of Eq. (13): G + d_i^T diag(a)^-1 diag(c) diag(a)^-1 e."""
        return self.G + self.dnode() * np.sum(self.c * self.e / self.a ** 2, axis=-1)


def make_level(n: int, N: int, nu: float, kappa_fn) -> Level:
    """Rediscretise the operator on the n x n interior grid."""
    h = 1.0 / (n + 1)
    t = np.arange(n + 2, dtype=np.float64) * h          # includes boundary coordinates
    X, Y = np.meshgrid(t, t, indexing="xy")             # [n+2, n+2]
    kap = kappa_fn(X, Y)                                # [n+2, n+2, N]
    kx = harmonic_mean(kap[1:-1, :-1], kap[1:-1, 1:])   # [n, n+1, N]
    ky = harmonic_mean(kap[:-1, 1:-1], kap[1:, 1:-1])   # [n+1, n, N]
    a = kx[:, :-1] + kx[:, 1:] + ky[:-1, :] + ky[1:, :]
    return Level(n=n, N=N, nu=nu, h=h, kx=kx, ky=ky, a=a,
                 c=h * h / N, G=nu * h * h, d=-h * h, e=-h * h)


def level_from_faces(n: int, N: int, nu: float, kx, ky) -> Level:
    """The rediscretised operator on an n x n grid with given face coefficients."""
    h = 1.0 / (n + 1)
    a = kx[:, :-1] + kx[:, 1:] + ky[:-1, :] + ky[1:, :]
    return Level(n=n, N=N, nu=nu, h=h, kx=kx, ky=ky, a=a,
                 c=h * h / N, G=nu * h * h, d=-h * h, e=-h * h)


def averaged_coarse_level(fine: Level) -> Level:
    """Coarse grid (n-1)/2 whose face coefficients average the fine ones.

    A coarse face spans two fine faces in series along its direction
    (harmonic mean, the effective coefficient of two layers) and three
    fine lines across it, combined in parallel with the full-weighting
    weights 1/4, 1/2, 1/4 (arithmetic mean).  Coarse node (J, I) sits on
    fine node (2J+1, 2I+1); the coarse vertical face I (between coarse
    columns I-1 and I) spans the fine vertical faces 2I and 2I+1.
    """
    nf, N = fine.n, fine.N
    nc = (nf - 1) // 2
    w = (0.25, 0.5, 0.25)
    kx = np.zeros((nc, nc + 1, N))
    for J in range(nc):
        for t, row in enumerate((2 * J, 2 * J + 1, 2 * J + 2)):
            kx[J] += w[t] * harmonic_mean(fine.kx[row, 0:2 * nc + 1:2], fine.kx[row, 1:2 * nc + 2:2])
    ky = np.zeros((nc + 1, nc, N))
    for I in range(nc):
        for t, col in enumerate((2 * I, 2 * I + 1, 2 * I + 2)):
            ky[:, I] += w[t] * harmonic_mean(fine.ky[0:2 * nc + 1:2, col], fine.ky[1:2 * nc + 2:2, col])
    return level_from_faces(nc, N, fine.nu, kx, ky)


def control_indicator(n: int, box) -> np.ndarray:
    """chi of the n x n grid for the closed control region box = (x0, x1, y0,
    y1): 1 at interior nodes (x, y) = ((ix+1) h, (iy+1) h) with x0 <= x <= x1
    and y0 <= y <= y1 (compared in integer arithmetic on the grid index:
    x0 (n+1) <= ix+1 <= x1 (n+1), within a rounding tolerance)."""
    x0, x1, y0, y1 = box
    t = np.arange(1, n + 1, dtype=np.float64)           # (ix + 1)
    s = float(n + 1)
    eps = 1e-9
    inx = (t >= x0 * s - eps) & (t <= x1 * s + eps)
    iny = (t >= y0 * s - eps) & (t <= y1 * s + eps)
    return (iny[:, None] & inx[None, :]).astype(np.float64)


def make_hierarchy(n: int, N: int, nu: float, kappa_fn, coarsest_n: int = 3, coarse: str = "averaged",
                   control_box=None):
    """Nested grids n_l = 2^l - 1 from n down to coarsest_n (finest first).

    coarse = "averaged": coarse face coefficients from the next finer grid
    (averaged_coarse_level); "nodal": every grid samples the field at its
    own nodes and takes harmonic means of endpoint values (make_level).
    control_box = (x0, x1, y0, y1): local control on that closed region,
    each grid with its own indicator (control_indicator); None = control
    everywhere."""
    if n < coarsest_n or (n + 1) & n or (coarsest_n + 1) & coarsest_n:
        raise ValueError("grid sizes must be 2^l - 1 with n >= coarsest_n")
    if coarse not in ("averaged", "nodal"):
        raise ValueError(coarse)
    levels = [make_level(n, N, nu, kappa_fn)]
    while levels[-1].n != coarsest_n:
        m = (levels[-1].n - 1) // 2
        if coarse == "nodal":
            levels.append(make_level(m, N, nu, kappa_fn))
        else:
            levels.append(averaged_coarse_level(levels[-1]))
    if control_box is not None:
        for lev in levels:
            lev.chi = control_indicator(lev.n, control_box)
    return levels


def fine_rhs(level: Level, yd: np.ndarray, f: np.ndarray | None = None):
    """Right-hand side of the symmetric full-space system: ((h^2/N) y_d, 0, h^2 f)."""
    n, N, h = level.n, level.N, level.h
    fy = np.repeat((h * h / N * yd)[:, :, None], N, axis=2)
    fu = np.zeros((n, n))
    fp = np.zeros((n, n, N)) if f is None else np.repeat((h * h * f)[:, :, None], N, axis=2)
    return fy, fu, fp


# ---------------------------------------------------------------------------
# Operator
# ---------------------------------------------------------------------------

def _pad(v):
    """Zero Dirichlet ghosts around the [n, n, ...] node array."""
    width = [(1, 1), (1, 1)] + [(0, 0)] * (v.ndim - 2)
    return np.pad(v, width)


def offdiag_sum(level: Level, v: np.ndarray) -> np.ndarray:
    """sum over the four faces of node i of k_f * v_neighbour (zero outside)."""
    vp = _pad(v)
    return (level.kx[:, :-1] * vp[1:-1, :-2] + level.kx[:, 1:] * vp[1:-1, 2:]
            + level.ky[:-1, :] * vp[:-2, 1:-1] + level.ky[1:, :] * vp[2:, 1:-1])


def apply_A(level: Level, v: np.ndarray) -> np.ndarray:
    """(A_j v_j)_i = sum_faces k_f (v_i - v_nbr): the integrated 5-point stencil."""
    return level.a * v - offdiag_sum(level, v)


def apply_S(level: Level, y, u, p):
    """S x for the block matrix of Eq. (2) with the blocks of this problem.

    With local control the control enters only through chi u, and the
    control row exists only where chi = 1 (0 elsewhere)."""
    chi = level.control()
    cu = chi * u
    sy = level.c * y + apply_A(level, p)
    su = chi * (level.G * cu + level.dnode() * np.sum(p, axis=-1))
    sp = apply_A(level, y) + level.e * cu[:, :, None]
    return sy, su, sp


def residual(level: Level, x, f):
    """r = f - S x, block by block.  With local control the control row is
    absent at nodes without a control basis function: its residual is 0."""
    sy, su, sp = apply_S(level, *x)
    return f[0] - sy, level.control() * (f[1] - su), f[2] - sp


def norm(v) -> float:
    """Euclidean norm over all (2N+1) n^2 entries of a full-space vector."""
    return float(np.sqrt(sum(np.sum(np.asarray(b) ** 2) for b in v)))


def paper_norm(v, N: int) -> float:
    """Euclidean norm of the vector in the scaling of the paper's system.

    The paper writes the full-space optimality system (Sec. 2) with the
    state rows M y_j + A_j^T p_j = M y_d, i.e. N times the symmetric state
    rows used here (its adjoint is N times ours; the control and adjoint
    rows coincide).  Its relative residual (Sec. 3.2) is therefore
    ||W r|| / ||W f|| with W = diag(N I, 1, 1) on (y, u, p) rows.
    """
    y, u, p = v
    return float(np.sqrt(N * N * np.sum(np.asarray(y) ** 2) + np.sum(np.asarray(u) ** 2)
                         + np.sum(np.asarray(p) ** 2)))


# ---------------------------------------------------------------------------
# Local solve, Eq. (13)
# ---------------------------------------------------------------------------

def local_solve(b_p, b_u, b_y, a, c, G, d, e):
    """Solve the reduced node system S~_i x_i = b_i of Eq. (12) by Eq. (13).

    b_p: rhs of the first block row (diag(c) y~ + diag(a) p~ = b_p)
    b_u: rhs of the control row     (G u + d^T p~ = b_u)
    b_y: rhs of the last block row  (diag(a) y~ + e u = b_y)
    a: diag entries of A_j at the node.  c, d, e are vectors over samples
    (scalars broadcast).  Leading axes of b_p, b_y, a are batch axes; the
    last axis is the sample axis; b_u has the batch axes only.
    Returns (y~, u, p~).
    """
    ainv = 1.0 / a
    num = b_u + np.sum(d * (ainv * c * ainv * b_y - ainv * b_p), axis=-1)
    den = G + np.sum(d * ainv * c * ainv * e, axis=-1)
    u = num / den
    y = ainv * (b_y - e * u[..., None])
    p = ainv * (b_p - c * y)
    return y, u, p


# ---------------------------------------------------------------------------
# Collective smoothers
# ---------------------------------------------------------------------------

def colour_mask(n: int, colour: int) -> np.ndarray:
    """Red = colour 0 = (ix + iy) even; black = colour 1."""
    iy, ix = np.indices((n, n))
    return (ix + iy) % 2 == colour


def local_solve_fixed_u(b_p, u, b_y, a, c, e):
    """Eq. (14) with a given control u_i (the paper sets u_i = 0 at nodes
    without a control dof): y~ = diag(a)^-1 (b_y - e u), p~ = diag(a)^-1 (b_p - c y~)."""
    ainv = 1.0 / a
    y = ainv * (b_y - e * u[..., None])
    p = ainv * (b_p - c * y)
    return y, p


def rbgs_half_sweep(level: Level, x, f, colour: int, freeze_u: bool = False):
    """Collective GS on all nodes of one colour.

    Nodes of one colour couple only to nodes of the other colour, so each
    node's local system uses the current values of its neighbours and
    replaces (y~_i, u_i, p~_i) by S~_i^{-1}(f_i - off-diagonal couplings).
    """
    y, u, p = (np.array(b, copy=True) for b in x)
    fy, fu, fp = f
    m = colour_mask(level.n, colour)
    b_p = (fy + offdiag_sum(level, p))[m]      # first block row: c y + A p = f_y
    b_y = (fp + offdiag_sum(level, y))[m]      # last block row:  A y + e u = f_p
    b_u = fu[m]                                # control row has no neighbour coupling
    if freeze_u:
        yn, pn = local_solve_fixed_u(b_p, u[m], b_y, level.a[m], level.c, level.e)
        y[m], p[m] = yn, pn
        return y, u, p
    yn, un, pn = local_solve(b_p, b_u, b_y, level.a[m], level.c, level.G, level.dnode()[m][:, None], level.e)
    # nodes without a control basis function: Eq. (14) with u_i = 0
    off = level.control()[m] == 0.0
    if np.any(off):
        y0, p0 = local_solve_fixed_u(b_p[off], np.zeros(int(off.sum())), b_y[off], level.a[m][off], level.c,
                                     level.e)
        yn[off], pn[off], un[off] = y0, p0, 0.0
    y[m], u[m], p[m] = yn, un, pn
    return y, u, p


def rbgs_sweep(level: Level, x, f, freeze_u: bool = False):
    """One red-black collective GS sweep: red (ix+iy even) first, then black."""
    x = rbgs_half_sweep(level, x, f, 0, freeze_u)
    return rbgs_half_sweep(level, x, f, 1, freeze_u)


def lexgs_sweep(level: Level, x, f):
    """One lexicographic collective GS sweep, node order i = iy*n + ix.

    Pure-Python node loop: for small grids only.
    """
    y, u, p = (np.array(b, copy=True) for b in x)
    fy, fu, fp = f
    n = level.n
    kx, ky = level.kx, level.ky
    for iy in range(n):
        for ix in range(n):
            off_p = np.zeros(level.N)
            off_y = np.zeros(level.N)
            if ix > 0:
                off_p += kx[iy, ix] * p[iy, ix - 1]
                off_y += kx[iy, ix] * y[iy, ix - 1]
            if ix < n - 1:
                off_p += kx[iy, ix + 1] * p[iy, ix + 1]
                off_y += kx[iy, ix + 1] * y[iy, ix + 1]
            if iy > 0:
                off_p += ky[iy, ix] * p[iy - 1, ix]
                off_y += ky[iy, ix] * y[iy - 1, ix]
            if iy < n - 1:
                off_p += ky[iy + 1, ix] * p[iy + 1, ix]
                off_y += ky[iy + 1, ix] * y[iy + 1, ix]
            if level.control()[iy, ix] == 0.0:   # Eq. (14) with u_i = 0
                yi, pi = local_solve_fixed_u(fy[iy, ix] + off_p, np.float64(0.0), fp[iy, ix] + off_y,
                                             level.a[iy, ix], level.c, level.e)
                ui = 0.0
            else:
                yi, ui, pi = local_solve(fy[iy, ix] + off_p, fu[iy, ix], fp[iy, ix] + off_y,
                                         level.a[iy, ix], level.c, level.G, level.dnode()[iy, ix], level.e)
            y[iy, ix], u[iy, ix], p[iy, ix] = yi, ui, pi
    return y, u, p


def jacobi_sweep(level: Level, x, f, theta: float, freeze_u: bool = False):
    """Damped collective Jacobi, Eq. (11): x <- x + theta sum_i P_i S~_i^{-1} R_i (f - S x)."""
    ry, ru, rp = residual(level, x, f)
    if freeze_u:
        dy, dp = local_solve_fixed_u(ry, np.zeros_like(ru), rp, level.a, level.c, level.e)
        return x[0] + theta * dy, x[1], x[2] + theta * dp
    dy, du, dp = local_solve(ry, ru, rp, level.a, level.c, level.G, level.dnode()[:, :, None], level.e)
    off = level.control() == 0.0
    if np.any(off):   # nodes without a control basis function: Eq. (14) with a zero control update
        y0, p0 = local_solve_fixed_u(ry, np.zeros_like(ru), rp, level.a, level.c, level.e)
        dy = np.where(off[:, :, None], y0, dy)
        dp = np.where(off[:, :, None], p0, dp)
        du = np.where(off, 0.0, du)
    return x[0] + theta * dy, x[1] + theta * du, x[2] + theta * dp


@dataclass
class CycleOptions:
    smoother: str = "rbgs"        # "rbgs" | "lexgs" | "jacobi"
    theta: float = 0.5            # Jacobi damping (the paper's value)
    n1: int = 2                   # pre-smoothing steps
    n2: int = 2                   # post-smoothing steps
    gamma: int = 1                # 1 = V-cycle, 2 = W-cycle
    freeze_u: bool = False        # keep u fixed: solve the state and adjoint rows only


def smooth(level: Level, x, f, steps: int, opts: CycleOptions):
    for _ in range(steps):
        if opts.smoother == "rbgs":
            x = rbgs_sweep(level, x, f, opts.freeze_u)
        elif opts.smoother == "lexgs":
            if opts.freeze_u:
                raise ValueError("frozen control is defined for the red-black and Jacobi smoothers")
            x = lexgs_sweep(level, x, f)
        elif opts.smoother == "jacobi":
            x = jacobi_sweep(level, x, f, opts.theta, opts.freeze_u)
        else:
            raise ValueError(opts.smoother)
    return x


# ---------------------------------------------------------------------------
# Grid transfers
# ---------------------------------------------------------------------------

def prolongation_1d(nf: int) -> np.ndarray:
    """Linear interpolation from (nf-1)/2 coarse to nf fine interior nodes.

    Coarse node I sits on fine node 2I+1; fine nodes 2I and 2I+2 receive
    half of it.  Shape [nf, nc].
    """
    nc = (nf - 1) // 2
    P = np.zeros((nf, nc))
    for I in range(nc):
        P[2 * I + 1, I] = 1.0
        P[2 * I, I] = 0.5
        P[2 * I + 2, I] = 0.5
    return P


def _apply_2d(P1, v, transpose: bool):
    """(P1 (x) P1) v, or its transpose, on a node array [rows, cols, ...]:
    the 2D operator is the tensor product of the 1D one, applied along y
    (first axis) and then along x (second axis)."""
    A = P1.T if transpose else P1
    t = np.tensordot(A, v, axes=(1, 0))                 # along y
    t = np.tensordot(A, t, axes=(1, 1))                 # along x -> [x, y, ...]
    return np.swapaxes(t, 0, 1)


def prolong(nf: int, e, chi_f=None):
    """Bilinear prolongation P e of a coarse full-space vector (all three blocks).

    chi_f: the fine grid's control indicator; the control block of P e is
    kept only where the fine grid has a control basis function."""
    P1 = prolongation_1d(nf)
    out = tuple(_apply_2d(P1, np.asarray(b), transpose=False) for b in e)
    if chi_f is not None:
        out = (out[0], chi_f * out[1], out[2])
    return out


def restrict(nf: int, r):
    """Restriction R = P^T of a fine full-space vector (all three blocks).

    Every block row is in integrated (h^2-scaled) form, so the transpose
    of the bilinear prolongation (weights 1, 1/2, 1/4, i.e. 4x the 1/16
    full-weighting stencil) is the consistent restriction.
    """
    P1 = prolongation_1d(nf)
    return tuple(_apply_2d(P1, np.asarray(b), transpose=True) for b in r)


# ---------------------------------------------------------------------------
# Coarsest-grid direct solve
# ---------------------------------------------------------------------------

def dense_A(level: Level, j: int) -> np.ndarray:
    """A_j assembled column by column from its action (small grids)."""
    n = level.n
    m = n * n
    A = np.zeros((m, m))
    for col in range(m):
        v = np.zeros((n, n, level.N))
        v.reshape(m, level.N)[col, j] = 1.0
        A[:, col] = apply_A(level, v)[:, :, j].reshape(m)
    return A


def coarse_solve_fixed_u(level: Level, f):
    """Coarsest solve of the correction equation with a zero control
    correction: y_j = A_j^{-1} f_p,j, p_j = A_j^{-1} (f_y,j - c y_j), u = 0."""
    n, N = level.n, level.N
    y = np.zeros((n, n, N))
    p = np.zeros((n, n, N))
    for j in range(N):
        A = dense_A(level, j)
        y[:, :, j] = np.linalg.solve(A, f[2][:, :, j].ravel()).reshape(n, n)
        p[:, :, j] = np.linalg.solve(A, (f[0][:, :, j] - level.c * y[:, :, j]).ravel()).reshape(n, n)
    return y, np.zeros((n, n)), p


def coarse_solve(level: Level, f):
    """Exact S^{-1} f by block elimination of the per-sample PDE blocks.

    From the adjoint-row block y_j = A_j^{-1}(f_p,j - e u); from the
    state-row block p_j = A_j^{-1}(f_y,j - c y_j); substituting into the
    control row gives the n^2 x n^2 system
        (G I + d c e sum_j A_j^{-2}) u = f_u - d sum_j (A_j^{-1} f_y,j - c A_j^{-2} f_p,j).
    """
    n, N = level.n, level.N
    m = n * n
    fy, fu, fp = (np.asarray(b).reshape(m, -1) if np.asarray(b).ndim == 3 else np.asarray(b).reshape(m) for b in f)
    c, G, d, e = level.c, level.G, level.d, level.e
    Ainv = [np.linalg.inv(dense_A(level, j)) for j in range(N)]
    dn = level.dnode().reshape(m)          # d_i, row i of the control system
    schur = G * np.eye(m)
    rhs = fu.copy()
    for j in range(N):
        A2 = Ainv[j] @ Ainv[j]
        schur += (dn * c * e)[:, None] * A2
        rhs -= dn * (Ainv[j] @ fy[:, j] - c * (A2 @ fp[:, j]))
    # local control: the control rows and unknowns exist only where chi = 1
    on = level.control().reshape(m) != 0.0
    u = np.zeros(m)
    u[on] = np.linalg.solve(schur[np.ix_(on, on)], rhs[on])
    y = np.zeros((m, N))
    p = np.zeros((m, N))
    for j in range(N):
        y[:, j] = Ainv[j] @ (fp[:, j] - e * u)
        p[:, j] = Ainv[j] @ (fy[:, j] - c * y[:, j])
    return y.reshape(n, n, N), u.reshape(n, n), p.reshape(n, n, N)


def dense_S(level: Level) -> np.ndarray:
    """The full (2N+1) n^2 system matrix in the ordering (y, u, p), each block
    flattened [node][sample] (small grids only)."""
    n, N = level.n, level.N
    m = n * n
    dim = (2 * N + 1) * m
    S = np.zeros((dim, dim))
    for col in range(dim):
        z = np.zeros(dim)
        z[col] = 1.0
        S[:, col] = pack(apply_S(level, *unpack(z, n, N)))
    return S


def pack(x) -> np.ndarray:
    y, u, p = x
    return np.concatenate([np.ravel(y), np.ravel(u), np.ravel(p)])


def unpack(z, n: int, N: int):
    m = n * n
    y = z[: m * N].reshape(n, n, N)
    u = z[m * N: m * N + m].reshape(n, n)
    p = z[m * N + m:].reshape(n, n, N)
    return y, u, p


# ---------------------------------------------------------------------------
# Cycles and outer iterations
# ---------------------------------------------------------------------------

def zeros_like_level(level: Level):
    n, N = level.n, level.N
    return np.zeros((n, n, N)), np.zeros((n, n)), np.zeros((n, n, N))


def cycle(levels, l: int, x, f, opts: CycleOptions):
    """Algorithm 1 (V-cycle; gamma = 2 recursive calls gives the W-cycle)."""
    level = levels[l]
    if l == len(levels) - 1:
        if opts.freeze_u:
            # the correction keeps u: x + (y, 0, p) with the coarsest PDEs solved for it
            ey, _, ep = coarse_solve_fixed_u(level, residual(level, x, f))
            return x[0] + ey, x[1], x[2] + ep
        return coarse_solve(level, f)
    x = smooth(level, x, f, opts.n1, opts)
    r = residual(level, x, f)
    fc = restrict(level.n, r)
    ec = zeros_like_level(levels[l + 1])
    for _ in range(opts.gamma):
        ec = cycle(levels, l + 1, ec, fc, opts)
    e = prolong(level.n, ec, level.chi)
    x = (x[0] + e[0], x[1] + e[1], x[2] + e[2])
    return smooth(level, x, f, opts.n2, opts)


@dataclass
class SolveResult:
    x: tuple
    iters: int
    relres: float
    history: list


def solve_stationary(levels, f, opts: CycleOptions, tol: float = 1e-10, maxit: int = 100, x0=None):
    """Repeat the cycle until the relative residual of the paper's system,
    ||W (f - S x)|| / ||W f|| (see paper_norm), is <= tol."""
    N = levels[0].N
    x = zeros_like_level(levels[0]) if x0 is None else tuple(np.array(b, copy=True) for b in x0)
    fnorm = paper_norm(f, N)
    hist = [paper_norm(residual(levels[0], x, f), N) / fnorm]
    it = 0
    while hist[-1] > tol and it < maxit:
        x = cycle(levels, 0, x, f, opts)
        it += 1
        hist.append(paper_norm(residual(levels[0], x, f), N) / fnorm)
    return SolveResult(x=x, iters=it, relres=hist[-1], history=hist)


def fgmres(levels, f, opts: CycleOptions, tol: float = 1e-10, maxit: int = 100,
           restart: int = 50, x0=None, precondition=True):
    """Right-preconditioned flexible GMRES(restart) with the cycle as preconditioner.

    GMRES runs on the paper's system W S x = W f (W = diag(N I, 1, 1), see
    paper_norm) so that it minimises the residual the paper reports; the
    preconditioner is one cycle applied to W^{-1} v.  Arnoldi with
    classical Gram-Schmidt applied twice (CGS2), Givens rotations for the
    least-squares problem, stopping test on the recurrence estimate of
    ||W (f - S x)|| / ||W f||, true residual recomputed at every restart
    and at exit.
    """
    lev = levels[0]
    n, N = lev.n, lev.N
    m = n * n * N
    wvec = np.concatenate([np.full(m, float(N)), np.ones(n * n), np.ones(m)])
    x = pack(zeros_like_level(lev)) if x0 is None else pack(x0)
    fv = wvec * pack(f)
    fnorm = np.linalg.norm(fv)
    S = lambda z: wvec * pack(apply_S(lev, *unpack(z, n, N)))
    if precondition:
        M = lambda v: pack(cycle(levels, 0, zeros_like_level(lev), unpack(v / wvec, n, N), opts))
    else:
        M = lambda v: v / wvec
    r = fv - S(x)
    beta = np.linalg.norm(r)
    hist = [beta / fnorm]
    total = 0
    while hist[-1] > tol and total < maxit:
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        k_done = 0
        for k in range(restart):
            z = M(V[k])
            Z.append(z)
            w = S(z)
            Vk = np.array(V)
            h1 = Vk @ w
            w = w - Vk.T @ h1
            h2 = Vk @ w
            w = w - Vk.T @ h2
            H[: k + 1, k] = h1 + h2
            H[k + 1, k] = np.linalg.norm(w)
            V.append(w / H[k + 1, k] if H[k + 1, k] != 0 else w)
            for i in range(k):
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            rho = np.hypot(H[k, k], H[k + 1, k])
            cs[k], sn[k] = H[k, k] / rho, H[k + 1, k] / rho
            H[k, k] = rho
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            total += 1
            k_done = k + 1
            hist.append(abs(g[k + 1]) / fnorm)
            if hist[-1] <= tol or total >= maxit:
                break
        yk = np.linalg.solve(np.triu(H[:k_done, :k_done]), g[:k_done])
        x = x + np.array(Z).T @ yk
        r = fv - S(x)
        beta = np.linalg.norm(r)
        hist[-1] = beta / fnorm
    return SolveResult(x=unpack(x, n, N), iters=total, relres=hist[-1], history=hist)


# ---------------------------------------------------------------------------
# L1 + box constrained problem: globalised semismooth Newton (Sec. 4, Alg. 2)
# ---------------------------------------------------------------------------
#
# In the symmetric scaling used here the paper's adjoint is N times ours, so
# E[p_paper] = sum_j zeta_j p_paper,j = sum_j p_j.  The Newton system of
# Sec. 4 is the linear-quadratic system with the control row as the paper
# writes it, M du - M H sum_j zeta_j dp_paper,j = -M F, i.e. G = h^2 (nu h^2
# divided by nu) and the coupling d / nu restricted to the active sets
# (d_i = (d / nu) chi_i, chi = indicator of I+ u I-), right side (0, -M F, 0):
#     (h^2/N) dy_j + A_j dp_j = 0
#     h^2 du - (h^2/nu) chi sum_j dp_j = -h^2 F(u)
#     A_j dy_j - h^2 du = 0.
# (The same system with its control row multiplied by nu gives the same
# iterates, Eq. (13) being invariant to that row's scale, but a right side
# nu times smaller, whose relative residual stalls at the rounding floor.)
# Coarse grids take the active-set indicator at their coinciding fine node.


def expected_adjoint(p) -> np.ndarray:
    """E[p] of the paper's adjoint = sum over samples of ours (T u, Sec. 4)."""
    return np.sum(np.asarray(p), axis=-1)


def ssn_F(u, Tu, nu: float, beta: float, a: float, b: float) -> np.ndarray:
    """The nonlinear optimality map F(u) of Sec. 4 (componentwise)."""
    mx = lambda v: np.maximum(0.0, v)
    mn = lambda v: np.minimum(0.0, v)
    return u - (mx(Tu - beta) + mn(Tu + beta) - mx(Tu - beta - nu * b) - mn(Tu + beta - nu * a)) / nu


def ssn_active(Tu, nu: float, beta: float, a: float, b: float) -> np.ndarray:
    """Indicator of I+ = {0 <= Tu - beta <= nu b} union I- = {nu a <= Tu + beta <= 0}."""
    ip = (Tu - beta >= 0.0) & (Tu - beta <= nu * b)
    im = (Tu + beta <= 0.0) & (Tu + beta >= nu * a)
    return (ip | im).astype(np.float64)


def set_active(levels, chi_fine, scale: float = 1.0):
    """dw on every grid: scale times the active-set indicator, injected to
    coarse grids."""
    w = np.asarray(chi_fine, dtype=np.float64) * scale
    for lev in levels:
        lev.dw = w
        w = w[1::2, 1::2]


def newton_form(levels, on: bool):
    """Switch every grid's control row between the linear-quadratic form
    (G = nu h^2) and the Newton systems' form (G = h^2)."""
    for lev in levels:
        lev.G = lev.h * lev.h * (1.0 if on else lev.nu)


def pde_states(levels, u, yd, f=None):
    """y_j = A_j^-1 M (f + u), p_j = A_j^-1 (M/N)(y_d - y_j) for every sample:
    the frozen-control cycle solves these 2N PDEs for the given u (first line
    of Alg. 2; dense solves on the grids used here)."""
    lev = levels[0]
    n, N, h = lev.n, lev.N, lev.h
    m = n * n
    src = (u if f is None else u + f) * h * h
    y = np.zeros((n, n, N))
    p = np.zeros((n, n, N))
    for j in range(N):
        A = dense_A(lev, j)
        y[:, :, j] = np.linalg.solve(A, src.reshape(m)).reshape(n, n)
        p[:, :, j] = np.linalg.solve(A, (h * h / N * (yd - y[:, :, j])).reshape(m)).reshape(n, n)
    return y, p


@dataclass
class SSNResult:
    u: np.ndarray
    y: np.ndarray
    p: np.ndarray
    newton: int
    inner: list
    merit: list


def semismooth_newton(levels, yd, beta: float, a: float, b: float, tol: float = 1e-9, inner_tol: float = 1e-10,
                      sigma_ls: float = 1e-4, rho_ls: float = 0.5, maxit: int = 50, opts=None,
                      inner: str = "cycle", u0=None) -> SSNResult:
    """Algorithm 2: semismooth Newton on F(u) = 0 with a backtracking line
    search on phi(u) = sqrt(F^T M F); each Newton system is solved by the
    collective multigrid (stationary cycles or FGMRES) to inner_tol."""
    lev = levels[0]
    n, N, nu, h = lev.n, lev.N, lev.nu, lev.h
    opts = opts or CycleOptions()
    u = np.zeros((n, n)) if u0 is None else np.array(u0, dtype=np.float64)
    y, p = pde_states(levels, u, yd)
    phi = lambda F: float(h * np.linalg.norm(F))
    Tu = expected_adjoint(p)
    F = ssn_F(u, Tu, nu, beta, a, b)
    merits = [phi(F)]
    inners = []
    k = 0
    newton_form(levels, True)
    while merits[-1] > tol and k < maxit:
        set_active(levels, ssn_active(Tu, nu, beta, a, b), 1.0 / nu)
        rhs = (np.zeros((n, n, N)), -h * h * F, np.zeros((n, n, N)))
        if inner == "fgmres":
            res = fgmres(levels, rhs, opts, tol=inner_tol)
        else:
            res = solve_stationary(levels, rhs, opts, tol=inner_tol, maxit=200)
        inners.append(res.iters)
        dy, du, dp = res.x
        gamma = 1.0
        Tdp = expected_adjoint(dp)
        while True:
            Fn = ssn_F(u + gamma * du, Tu + gamma * Tdp, nu, beta, a, b)
            if phi(Fn) - merits[-1] <= -sigma_ls * merits[-1] or gamma < 1e-8:
                break
            gamma *= rho_ls
        u, y, p = u + gamma * du, y + gamma * dy, p + gamma * dp
        Tu = Tu + gamma * Tdp
        F = ssn_F(u, Tu, nu, beta, a, b)
        merits.append(phi(F))
        k += 1
    newton_form(levels, False)
    set_active(levels, np.ones((n, n)))
    return SSNResult(u=u, y=y, p=p, newton=k, inner=inners, merit=merits)
