"""What the learned warm start gains over the method without it.

A small instance of the warm-start workload (n = 63, N = 16 samples, 16
field modes of amplitude 1, nu = 1e-5, random 8-mode targets): the network
is trained on the GPU, by the library's own forward, backward and AdamW
kernels, on solves the method itself generates; on held-out seeds each
problem is then solved to the paper's relative residual 1e-10 from a zero
initial guess and from the network's control u0 (with 0 and 1 frozen-control
cycles completing the state and adjoint first).  Multigrid (Algorithm 1)
finishes every solve, so it is the fallback and the judge: the test asserts
that every solve reaches the tolerance whatever the surrogate, that the
trained surrogate beats the untrained one and the zero control, and prints
the surrogate error, the cycles saved and the end-to-end times (inference
included) as measured, whatever their sign (pytest -s)."""
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

n, N, K, NU, AMP = 63, 16, 16, 1e-5, 1.0
TRAIN, TEST, EPOCHS, BATCH = 192, 24, 25, 8


@pytest.fixture(scope="module")
def trained():
    from paper_2302_13680_gb300 import build

    build.build()
    import paper_2302_13680_gb300 as P
    from paper_2302_13680_gb300 import warmstart as W
    from paper_2302_13680_gb300.learned import WarmStartNet

    first = W.make_instance(1000, n, N, K, NU, AMP)
    H = P.Hierarchy(n, N, first.xi, NU, AMP)
    YD, MLK, U, it = W.generate(H, list(range(1000, 1000 + TRAIN)), n, N, K, NU, AMP)
    S = 1 << int(math.ceil(math.log2(n + 1)))
    net = WarmStartNet(S=S, batch=BATCH, seed=0)
    untrained = WarmStartNet(S=S, batch=BATCH, seed=0)
    hist = W.train(net, YD, MLK, U, n, epochs=EPOCHS, batch=BATCH, lr=2e-3)
    untrained.set_scales(*net.in_scale, net.out_scale)
    yield P, W, H, net, untrained, hist
    net.close()
    untrained.close()
    H.close()


def test_training_lowers_the_loss(trained):
    _, _, _, _, _, hist = trained
    assert hist[-1] < 0.5 * hist[0], hist


def test_warm_start_against_zero_start(trained):
    P, W, H, net, untrained, _ = trained
    seeds = list(range(5000, 5000 + TEST))
    rows = W.evaluate(net, H, seeds, n, N, K, NU, AMP, frozen=(1,))
    base = W.evaluate(untrained, H, seeds[:8], n, N, K, NU, AMP, frozen=())
    s = W.summarise(rows)
    err = s["surrogate_rel_err_mean"]
    err_untrained = W.summarise(base)["surrogate_rel_err_mean"]
    print(f"surrogate error {err:.3f} (untrained {err_untrained:.3f}); cycles zero {s['zero']['cycles_mean']:.2f}, "
          f"warm {s['warm_k0']['cycles_mean']:.2f}, warm+1 frozen {s['warm_k1']['cycles_mean']:.2f}; "
          f"ms zero {s['zero']['ms_mean']:.2f}, warm {s['warm_k0']['ms_mean']:.2f}, "
          f"warm+1 frozen {s['warm_k1']['ms_mean']:.2f}")
    # multigrid finishes every solve to the tolerance, from any start
    for r in rows + base:
        for k, v in r.items():
            if isinstance(v, dict):
                assert v["relres"] <= 1e-10, (r["seed"], k, v)
    # the trained network predicts the control: better than the zero control
    # (error 1) and than its untrained self
    assert err < 0.6, err
    assert err < 0.5 * err_untrained, (err, err_untrained)
