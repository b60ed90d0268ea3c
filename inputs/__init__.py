"""Seeded synthetic inputs shared by the CUDA path, the CPU oracle and the tests.

This module draws random numbers and samples the problem data (target
state, forcing) at grid nodes.  It holds none of the multigrid method's
arithmetic: no diffusion field, no operator, no smoother.  Both sides
receive the same arrays from here and compute everything else on their own.

Workloads follow the model problem of the paper's numerical section
(Sec. 3.2): a random diffusion field driven by independent standard
normal draws xi_{jk} (one row per sample j, one column per field mode k),
a target state y_d on the unit square and a forcing f (zero in all the
configurations used here).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np


def grid_nodes(n: int):
    """Interior node coordinates of the uniform n x n grid on (0,1)^2.

    Returns (x, y), each of shape [n, n] indexed [iy, ix], with
    x[iy, ix] = (ix + 1) h and y[iy, ix] = (iy + 1) h, h = 1 / (n + 1).
    """
    h = 1.0 / (n + 1)
    t = (np.arange(n, dtype=np.float64) + 1.0) * h
    x, y = np.meshgrid(t, t, indexing="xy")
    return x, y


def draw_xi(seed: int, N: int, K: int) -> np.ndarray:
    """Standard normal field coefficients xi[j, k], shape [N, K], float64."""
    return np.random.default_rng(seed).standard_normal((N, K))


def target_sinsin(n: int) -> np.ndarray:
    """y_d = sin(pi x) sin(pi y) sampled at the interior nodes, shape [n, n]."""
    x, y = grid_nodes(n)
    return np.sin(np.pi * x) * np.sin(np.pi * y)


def target_modes(n: int, seed: int, modes: int = 8) -> np.ndarray:
    """Random sum of `modes` sine modes: sum_m c_m sin(a_m pi x) sin(b_m pi y).

    a_m, b_m uniform on {1..4}, c_m standard normal, all drawn from `seed`.
    """
    rng = np.random.default_rng(seed)
    a = rng.integers(1, 5, size=modes)
    b = rng.integers(1, 5, size=modes)
    c = rng.standard_normal(modes)
    x, y = grid_nodes(n)
    out = np.zeros((n, n))
    for m in range(modes):
        out += c[m] * np.sin(a[m] * np.pi * x) * np.sin(b[m] * np.pi * y)
    return out


def random_state(seed: int, n: int, N: int, scale=(1.0, 1.0, 1.0)):
    """A random full-space vector (y [n*n, N], u [n*n], p [n*n, N]) in float64."""
    rng = np.random.default_rng(seed)
    y = rng.standard_normal((n * n, N)) * scale[0]
    u = rng.standard_normal(n * n) * scale[1]
    p = rng.standard_normal((n * n, N)) * scale[2]
    return y, u, p


@dataclass
class ProblemSpec:
    """One synthetic instance: grid size, samples, field modes and draws."""

    n: int
    N: int
    K: int
    nu: float
    amp: float
    seed: int
    xi: np.ndarray = field(repr=False)
    yd: np.ndarray = field(repr=False)          # [n, n]
    f: np.ndarray = field(repr=False)           # [n, n]
    control_box: tuple | None = None            # local control region (x0, x1, y0, y1); None = everywhere


def make_problem(n: int, N: int, K: int, nu: float, amp: float, seed: int,
                 target: str = "sinsin", target_seed: int | None = None, control_box=None) -> ProblemSpec:
    xi = draw_xi(seed, N, K)
    if target == "sinsin":
        yd = target_sinsin(n)
    elif target == "modes":
        yd = target_modes(n, seed if target_seed is None else target_seed)
    else:
        raise ValueError(f"unknown target {target!r}")
    return ProblemSpec(n=n, N=N, K=K, nu=nu, amp=amp, seed=seed, xi=xi, yd=yd,
                       f=np.zeros((n, n)), control_box=control_box)


# The five workloads (sizes, field, regularisation, seeds) used by the
# tests and the benchmark.  Config names describe the workload.
CONFIGS = {
    # plain FP64 V(2,2) red-black collective GS, n=31, N=8, 4 modes, amp 0.5
    "n31_N8": dict(n=31, N=8, K=4, nu=1e-4, amp=0.5, seed=1),
    # FGMRES + V(2,2), n=255, N=64, 16 modes, amp 1.0, nu=1e-6
    "n255_N64": dict(n=255, N=64, K=16, nu=1e-6, amp=1.0, seed=2),
    # large mixed-precision instance, n=1023, N=256, 32 modes, nu=1e-5
    "n1023_N256": dict(n=1023, N=256, K=32, nu=1e-5, amp=1.0, seed=3),
    # a grid whose finest launches still fit a profiler capture (a few GB on the
    # device, five times the L2 per launch) with the large instance's sample map
    "n511_N128": dict(n=511, N=128, K=32, nu=1e-5, amp=1.0, seed=5),
    # the n=255, N=64 instance with the control acting on (0.25, 0.75)^2 only
    "n255_N64_local": dict(n=255, N=64, K=16, nu=1e-6, amp=1.0, seed=2, control_box=(0.25, 0.75, 0.25, 0.75)),
}


def batch_problems(seed: int = 4, count: int = 96, sizes=(63, 127, 255), n_range=(16, 128),
                   nu_log10=(-6.0, -3.0), K: int = 16, amp: float = 1.0) -> list:
    """Independent instances for batched solves: instance i uses seed + i for
    its field draws and its 8-mode target; n uniform on `sizes`, N uniform on
    [n_range], log10(nu) uniform on [nu_log10]."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed + i)
        n = int(rng.choice(sizes))
        N = int(rng.integers(n_range[0], n_range[1] + 1))
        nu = float(10.0 ** rng.uniform(*nu_log10))
        pr = make_problem(n=n, N=N, K=K, nu=nu, amp=amp, seed=seed + i, target="modes",
                          target_seed=10_000 + seed + i)
        out.append(pr)
    return out
