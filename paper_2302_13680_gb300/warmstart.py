"""Train and evaluate the learned warm start (data from the solver itself).

  python -m paper_2302_13680_gb300.warmstart --train 4000 --test 512 --out report.json

1. Data: for every seed, the field draws xi (16 modes, amplitude 1) and an
   8-mode target y_d are drawn, the hierarchy's coefficients are rebuilt on
   the GPU (cmg_set_samples) and the mixed-precision solver solves the
   problem to 1e-10; the network input is (y_d, sample mean of log kappa_j),
   the target the optimal control u*.
2. Training: the BF16 U-Net held by libcmg's network handle (cmg_unet_*,
   bound in learned.py) with AdamW on the masked MSE of normalised u, all
   on libcmg's kernels.
3. Evaluation on held-out seeds, each solved to 1e-10 from
   (a) zero,
   (b) (0, u0, 0) with u0 the network's prediction, and
   (c) (y0, u0, p0) where y0, p0 come from k frozen-control cycles (the
       state and adjoint equations solved for the predicted control);
   reported: surrogate error ||u0 - u*|| / ||u*||, cycles, and end-to-end
   time (inference and frozen cycles included).
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

import inputs

from . import FP32, CycleOptions, Hierarchy
from .learned import WarmStartNet


def make_instance(seed: int, n: int, N: int, K: int, nu: float, amp: float):
    return inputs.make_problem(n=n, N=N, K=K, nu=nu, amp=amp, seed=seed, target="modes", target_seed=seed)


def generate(H, seeds, n, N, K, nu, amp, tol=1e-10):
    """Solve every seed's instance; returns stacked (yd, mlk, u) FP64 CUDA tensors."""
    import torch

    YD = torch.empty(len(seeds), n * n, dtype=torch.float64, device="cuda")
    MLK = torch.empty_like(YD)
    U = torch.empty_like(YD)
    x = H.zeros(0)
    opts = CycleOptions(precision=FP32)
    iters = []
    for k, s in enumerate(seeds):
        pr = make_instance(s, n, N, K, nu, amp)
        H.set_samples(torch.tensor(pr.xi, device="cuda"))
        YD[k] = torch.tensor(pr.yd.reshape(-1), device="cuda")
        f = H.rhs(YD[k])
        for t in x:
            t.zero_()
        st, _ = H.solve(opts, f, x, tol=tol, maxit=200)
        iters.append(st.iters)
        U[k] = x[1]
        H.mean_log_kappa(MLK[k])
    return YD, MLK, U, iters


def train(net, YD, MLK, U, n, epochs=6, batch=8, lr=2e-3, log=None):
    import torch

    net.set_scales(1.0 / float(YD.std()), 1.0 / float(MLK.std()), float(U.std()))
    X_all = torch.cat([net.pack_inputs(YD[i:i + 256], MLK[i:i + 256], n) for i in range(0, YD.shape[0], 256)])
    T_all = torch.cat([net.pack_targets(U[i:i + 256], n) for i in range(0, U.shape[0], 256)])
    count = YD.shape[0]
    steps = epochs * (count // batch)
    g = torch.Generator(device="cpu").manual_seed(0)
    step = 0
    hist = []
    for ep in range(epochs):
        perm = torch.randperm(count, generator=g)
        run = 0.0
        for b in range(count // batch):
            idx = perm[b * batch:(b + 1) * batch].cuda()
            X, T = X_all[idx].contiguous(), T_all[idx].contiguous()
            net.forward(X)
            loss = net.loss(T, n)
            net.backward()
            cur = lr * 0.5 * (1.0 + math.cos(math.pi * step / steps))
            net.adamw_step(lr=cur)
            step += 1
            run += float(loss)
        hist.append(run / (count // batch))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4e}")
    net.check_status()
    return hist


def predict(net, yd, mlk, n):
    X = net.pack_inputs(yd[None], mlk[None], n)
    pred = net.forward(X)
    return net.unpack(pred, n)[0]


def evaluate(net, H, seeds, n, N, K, nu, amp, frozen=(1, 2, 3), tol=1e-10):
    import torch

    opts = CycleOptions(precision=FP32)
    rows = []
    x = H.zeros(0)

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, 1e3 * (time.perf_counter() - t0)

    for s in seeds:
        pr = make_instance(s, n, N, K, nu, amp)
        H.set_samples(torch.tensor(pr.xi, device="cuda"))
        yd = torch.tensor(pr.yd.reshape(-1), device="cuda")
        f = H.rhs(yd)
        mlk = H.mean_log_kappa()
        row = {"seed": s}

        def zero_solve():
            for t in x:
                t.zero_()
            return H.solve(opts, f, x, tol=tol, maxit=200)[0]

        st, ms = timed(zero_solve)
        row["zero"] = {"cycles": st.iters, "ms": ms, "relres": st.relres}
        ustar = x[1].clone()
        for kf in (0,) + tuple(frozen):
            def warm_solve():
                u0 = predict(net, yd, mlk, n)
                for t in x:
                    t.zero_()
                x[1].copy_(u0)
                if kf:
                    H.solve(CycleOptions(precision=FP32, freeze_u=1), f, x, tol=1e-300, maxit=kf,
                            raise_on_fail=False)
                return H.solve(opts, f, x, tol=tol, maxit=200)[0], u0

            (st, u0), ms = timed(warm_solve)
            row[f"warm_k{kf}"] = {"cycles": st.iters + kf, "main_cycles": st.iters, "ms": ms, "relres": st.relres}
        row["surrogate_rel_err"] = float(torch.linalg.norm(u0 - ustar) / torch.linalg.norm(ustar))
        rows.append(row)
    return rows


def summarise(rows):
    keys = [k for k in rows[0] if k.startswith("zero") or k.startswith("warm")]
    out = {"instances": len(rows), "surrogate_rel_err_mean": float(np.mean([r["surrogate_rel_err"] for r in rows]))}
    for k in keys:
        out[k] = {"cycles_mean": float(np.mean([r[k]["cycles"] for r in rows])),
                  "ms_mean": float(np.mean([r[k]["ms"] for r in rows]))}
    return out


def main():
    import torch

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=255)
    ap.add_argument("--N", type=int, default=64)
    ap.add_argument("--K", type=int, default=16)
    ap.add_argument("--nu", type=float, default=1e-5)
    ap.add_argument("--amp", type=float, default=1.0)
    ap.add_argument("--train", type=int, default=4000)
    ap.add_argument("--test", type=int, default=512)
    ap.add_argument("--epochs", type=int, default=6)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    log = lambda m: print(m, flush=True)
    first = make_instance(1000, a.n, a.N, a.K, a.nu, a.amp)
    H = Hierarchy(a.n, a.N, first.xi, a.nu, a.amp)
    t0 = time.perf_counter()
    YD, MLK, U, it_tr = generate(H, list(range(1000, 1000 + a.train)), a.n, a.N, a.K, a.nu, a.amp)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    log(f"generated {a.train} solves in {t_gen:.1f} s (mean {np.mean(it_tr):.1f} cycles)")
    S = 1 << int(math.ceil(math.log2(a.n + 1)))
    net = WarmStartNet(S=S, batch=a.batch, seed=0)
    t0 = time.perf_counter()
    hist = train(net, YD, MLK, U, a.n, epochs=a.epochs, batch=a.batch, lr=a.lr, log=log)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    log(f"trained {a.epochs} epochs in {t_train:.1f} s")
    rows = evaluate(net, H, list(range(5000, 5000 + a.test)), a.n, a.N, a.K, a.nu, a.amp)
    summ = summarise(rows)
    report = {"config": vars(a), "generation_s": t_gen, "training_s": t_train, "loss_history": hist,
              "train_cycles_mean": float(np.mean(it_tr)), "summary": summ}
    log(json.dumps(summ))
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(report, fh, indent=1)


if __name__ == "__main__":
    main()
