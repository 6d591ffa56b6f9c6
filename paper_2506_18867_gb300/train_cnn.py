"""Trains the learned preconditioner (bsc_cnn) on Newton systems the method
generates and compares flexible CG with it against plain block-Jacobi PCG.

Systems: inputs.config_learned (n x n patch, membrane / bending stiffness
ratio log-uniform in [1e3, 1e5], noisy wrinkled state).  For every training
system the context assembles the projected Hessian K and the residual
r = -g, and solves K x* = r by PCG to 1e-7.  Training pairs (residual, exact
correction):
  - the Newton pair (r, x*);
  - Krylov pairs (r - K x_k, x* - x_k) for PCG iterates x_k after a random
    number k of iterations: the residuals a Krylov solver actually hands to
    its preconditioner, whose slow (smooth) modes dominate later on;
  - (K x, x) for a random field x smoothed over a random number of passes.
Each pair takes one Adam step on the energy-norm loss.  Held-out systems (seeds not used in training) are solved to 1e-8 by
both methods; iterations and CUDA-event times are reported.

    python -m paper_2506_18867_gb300.train_cnn --n 512 --systems 2000 --heldout 200 --out DIR
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import bsc, inputs


def smooth_field(torch, n, passes, gen, pins):
    """Gaussian noise on the n x n grid smoothed by `passes` [1 2 1] / 4
    filters per axis (zero outside), unit RMS, zero at the pins: (3, n*n)."""
    x = torch.randn((3, n, n), device="cuda", generator=gen, dtype=torch.float32)
    for _ in range(passes):
        y = 0.5 * x
        y[:, 1:, :] += 0.25 * x[:, :-1, :]
        y[:, :-1, :] += 0.25 * x[:, 1:, :]
        x = y
        y = 0.5 * x
        y[:, :, 1:] += 0.25 * x[:, :, :-1]
        y[:, :, :-1] += 0.25 * x[:, :, 1:]
        x = y
    x = x.reshape(3, -1)
    x[:, pins] = 0.0
    return (x / x.pow(2).mean().sqrt()).contiguous()


class Systems:
    """One context for all systems (same grid and pins); material and state per seed."""

    def __init__(self, n):
        import torch
        self.torch = torch
        self.n = n
        base = inputs.config_learned(0, n)
        self.ctx = bsc.context_for_patch(base, precision=bsc.FP32, pcg_rel_tol=1e-8)
        self.K = self.ctx.new_matrix()
        self.pins = torch.as_tensor(base.pinned, device="cuda", dtype=torch.long)

    def load(self, seed):
        pat = inputs.config_learned(seed, self.n)
        self.ctx.set_material(pat.material)
        C, Ch = self.ctx.to_device(pat.C), self.ctx.to_device(pat.Chat)
        self.ctx.assemble_hessian(C, project=True, out=self.K)
        r = -self.ctx.gradient(C, Ch)
        return pat, r


def timed(torch, fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = fn()
    e1.record()
    e1.synchronize()
    return out, e0.elapsed_time(e1)


def param_layout():
    """(weight slice, shape, bias slice) per layer in the C ABI's order."""
    ch_in, ch_out = (32, 32, 32, 32), (32, 32, 32, 16)
    out, o = [], 0
    for ci, co in zip(ch_in, ch_out):
        nw = 9 * ci * co
        out.append((slice(o, o + nw), (3, 3, ci, co), slice(o + nw, o + nw + co)))
        o += nw + co
    return out


def initial_params(seed, scale=0.5):
    rng = np.random.default_rng(seed)
    lay = param_layout()
    p = np.zeros(lay[-1][2].stop, dtype=np.float32)
    for l, (ws, shape, bs) in enumerate(lay[:3]):
        p[ws] = rng.standard_normal(int(np.prod(shape))) * scale * math.sqrt(2.0 / (9 * shape[2]))
    return p


def evaluate(sy, net, seeds, tol=1e-8):
    torch = sy.torch
    rows = []
    for s in seeds:
        pat, r = sy.load(s)
        (x0, it, rr), t_pcg = timed(torch, lambda: sy.ctx.solve(r, K=sy.K, rel_tol=tol))
        (x1, rep), t_fcg = timed(torch, lambda: net.solve(r, sy.K, rel_tol=tol))
        rows.append({"seed": int(s), "ratio": pat.meta["ratio"], "pcg_iters": it, "pcg_ms": t_pcg,
                     "fcg_iters": rep["fcg_iters"], "fcg_fallback_iters": rep["pcg_iters"],
                     "fell_back": rep["fell_back"], "fcg_ms": t_fcg, "fcg_rel_res": rep["rel_res"]})
    return rows


def summarize(rows):
    it_p = np.array([r["pcg_iters"] for r in rows], float)
    it_f = np.array([r["fcg_iters"] + r["fcg_fallback_iters"] for r in rows], float)
    t_p = np.array([r["pcg_ms"] for r in rows])
    t_f = np.array([r["fcg_ms"] for r in rows])
    return {"systems": len(rows), "pcg_iters_mean": float(it_p.mean()), "fcg_iters_mean": float(it_f.mean()),
            "iteration_ratio_pcg_over_fcg": float(it_p.mean() / it_f.mean()),
            "pcg_ms_mean": float(t_p.mean()), "fcg_ms_mean": float(t_f.mean()),
            "time_ratio_pcg_over_fcg": float(t_p.mean() / t_f.mean()),
            "fallbacks": int(sum(r["fell_back"] for r in rows))}


def krylov_pairs(sy, r, xs, it_full, count, gen):
    torch = sy.torch
    pairs = []
    for _ in range(count):
        k = int(torch.randint(1, max(2, it_full), (1,), generator=gen, device="cuda").item())
        xk, _, _ = sy.ctx.solve(r, K=sy.K, rel_tol=1e-30, max_iter=k, allow_unconverged=True)
        rk = r - sy.ctx.spmv(xk, K=sy.K)
        pairs.append((rk.contiguous(), (xs - xk).contiguous()))
    return pairs


def train(n=512, systems=2000, heldout=200, fields=1, lr=1e-3, seed=0, out=None, log_every=100, krylov=3):
    import torch
    sy = Systems(n)
    net = bsc.Cnn(sy.ctx)
    net.set_params(initial_params(seed))
    gen = torch.Generator("cuda").manual_seed(seed)
    heldout_seeds = list(range(1_000_000, 1_000_000 + heldout))
    before = summarize(evaluate(sy, net, heldout_seeds[: min(20, heldout)]))
    losses, t0 = [], time.perf_counter()
    step, total = 0, systems * (1 + krylov + fields)
    for k in range(systems):
        pat, r = sy.load(1 + k + seed * 100000)
        net.prepare(sy.K)
        xs, it_full, _ = sy.ctx.solve(r, K=sy.K, rel_tol=1e-7)
        pairs = [(r, xs)] + krylov_pairs(sy, r, xs, it_full, krylov, gen)
        for _ in range(fields):
            x = smooth_field(torch, n, int(torch.randint(0, 24, (1,), generator=gen, device="cuda").item()), gen,
                             sy.pins)
            pairs.append((sy.ctx.spmv(x, K=sy.K), x))
        for rr_, xx in pairs:
            frac = step / max(1, total - 1)
            net.loss_grad(rr_, xx)
            net.adam_step(lr * (0.02 + 0.49 * (1.0 + math.cos(math.pi * frac))))
            step += 1
        if k % log_every == 0 or k == systems - 1:
            L = net.loss_grad(r, xs)
            losses.append({"system": k, "newton_pair_loss": L, "seconds": time.perf_counter() - t0})
    train_s = time.perf_counter() - t0
    rows = evaluate(sy, net, heldout_seeds)
    report = {"n": n, "systems": systems, "pairs_per_system": 1 + krylov + fields, "adam_steps": step, "lr": lr,
              "train_seconds": train_s, "loss_log": losses, "heldout_before_training": before,
              "heldout": summarize(rows), "heldout_rows": rows}
    params = net.get_params()
    if out:
        os.makedirs(out, exist_ok=True)
        np.savez(os.path.join(out, f"cnn_learned{n}.npz"), params=params, n=n, systems=systems)
        with open(os.path.join(out, f"train_report{n}.json"), "w") as f:
            json.dump(report, f, indent=1)
    net.close()
    sy.ctx.close()
    return report, params


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--systems", type=int, default=2000)
    ap.add_argument("--heldout", type=int, default=200)
    ap.add_argument("--fields", type=int, default=1)
    ap.add_argument("--krylov", type=int, default=3)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    rep, _ = train(a.n, a.systems, a.heldout, a.fields, a.lr, a.seed, a.out, krylov=a.krylov)
    print(json.dumps({k: v for k, v in rep.items() if k != "heldout_rows"}, indent=1))


if __name__ == "__main__":
    main()
