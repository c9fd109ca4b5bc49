"""Training and evaluation of the warm-start network for the local eigensolves.

The network (a2ls_gnn_* in include/a2ls.h) proposes the starting block of the
block Krylov iteration that solves each subdomain's eigenproblem (Eq. 3.1).
Targets are the eigenvectors that a plain setup (random start) selects; the
forward pass, loss, backward pass and Adam all run in the library's kernels.

    python -m paper_2201_02250_gb300.warm_start --train 300 --test 50 --out report.json

generates log-normal diffusion problems (256 x 256 grid, 64 subdomains,
overlap 2, nev 10), trains on the first set and compares, on the held-out set,
setups with and without the warm start: eigen restart cycles, eigensolve time,
the network's subspace loss, and the GMRES iterations to 1e-8.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import a2ls


def sample_from_problem(prob, **opts):
    """Plain setup of `prob` (eigenvectors as target); returns (sample, setup statistics)."""
    P, keep = a2ls.from_scipy(prob.A, prob.part, prob.overlap, prob.nev, **opts)
    stats = setup_stats(P)
    S = a2ls.GnnSample(P)
    P.close()
    del keep
    return S, stats


def setup_stats(P) -> dict:
    t = P.times()
    cyc = P.eig_stats()[:, 0]
    return {"setup_ms": t["setup_total"], "eig_ms": t["eig_coarse"], "cycles_sum": int(cyc.sum()),
            "cycles_mean": float(cyc.mean()), "cycles_max": int(cyc.max())}


def train(net, samples: list, epochs: int, lr: float, seed: int = 0, batch: int = 1, log=None) -> list:
    """Adam over the samples in a seeded shuffled order; one step per `batch` samples.

    Returns the mean training loss of every epoch."""
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        order = rng.permutation(len(samples))
        tot = 0.0
        for k, j in enumerate(order):
            tot += net.loss_grad(samples[j])
            if (k + 1) % batch == 0 or k == len(order) - 1:
                net.adam_step(lr)
        hist.append(tot / len(samples))
        if log:
            log(f"epoch {ep + 1}/{epochs}: loss {hist[-1]:.4f}")
    return hist


def evaluate(net, problems: list, rtol: float = 1e-8, **opts) -> dict:
    """Setups with random and with warm start on each problem; GMRES to rtol with each."""
    import torch
    rows = []
    for prob in problems:
        row = {"name": prob.name}
        for label, extra in (("random", {}), ("warm", {"warm_start": net})):
            P, keep = a2ls.from_scipy(prob.A, prob.part, prob.overlap, prob.nev, **opts, **extra)
            st = setup_stats(P)
            b = torch.as_tensor(prob.b, device="cuda")
            x = torch.zeros_like(b)
            it, rr, ok = P.solve(b, x, rtol)
            st.update({"gmres_iters": it, "relres": rr, "converged": bool(ok)})
            if label == "random":
                S = a2ls.GnnSample(P)
                st["net_loss"] = net.loss_grad(S)  # gradient discarded below
                S.close()
            row[label] = st
            P.close()
            del keep
        rows.append(row)
    net.set_params(net.params())  # drop the gradients accumulated by the evaluation losses
    agg = {}
    for label in ("random", "warm"):
        for key in ("setup_ms", "eig_ms", "cycles_sum", "cycles_mean", "gmres_iters"):
            agg[f"{label}_{key}"] = float(np.mean([r[label][key] for r in rows]))
    agg["net_loss"] = float(np.mean([r["random"]["net_loss"] for r in rows]))
    return {"per_problem": rows, "mean": agg}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--train", type=int, default=300)
    ap.add_argument("--test", type=int, default=50)
    ap.add_argument("--grid", type=int, default=256)
    ap.add_argument("--blocks", type=int, default=8)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--params-out", default=None, help="write the trained parameters (float32 .npy)")
    ap.add_argument("--out", default=None, help="write the JSON report here")
    a = ap.parse_args(argv)
    from workloads import config_c4  # synthetic problem generator of the repository

    def log(msg):
        print(msg, flush=True)

    opts = {"precision": a.precision}
    t0 = time.time()
    samples, base = [], []
    for k in range(a.train):
        S, st = sample_from_problem(config_c4(1000 + k, m=a.grid, blocks=a.blocks), **opts)
        samples.append(S)
        base.append(st)
    t_gen = time.time() - t0
    log(f"{a.train} training setups in {t_gen:.1f} s")
    net = a2ls.WarmStartNet(seed=a.seed)
    t0 = time.time()
    hist = train(net, samples, a.epochs, a.lr, seed=a.seed, batch=a.batch, log=log)
    t_train = time.time() - t0
    for S in samples:
        S.close()
    test = [config_c4(5000 + k, m=a.grid, blocks=a.blocks) for k in range(a.test)]
    ev = evaluate(net, test, **opts)
    report = {"config": {"grid": a.grid, "subdomains": a.blocks ** 2, "overlap": 2, "nev": 10,
                         "train": a.train, "test": a.test, "epochs": a.epochs, "lr": a.lr, "batch": a.batch,
                         "precision": a.precision},
              "train_setup_s": t_gen, "train_s": t_train, "train_loss": hist,
              "gnn_launches": net.launches(), "eval": ev["mean"], "per_problem": ev["per_problem"]}
    log(json.dumps(report["eval"]))
    if a.params_out:
        np.save(a.params_out, net.params())
    if a.out:
        with open(a.out, "w") as f:
            json.dump(report, f, indent=1)
    net.close()


if __name__ == "__main__":
    main()
