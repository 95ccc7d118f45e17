"""Learned regularisation parameter: data from the method's own solves,
training and evaluation with the project's kernels.

The paper sets alpha a priori (Section 5: alpha = delta for PinT-QBVM,
tau*delta for PinT-MQBVM).  Here a small network predicts
t = log10(alpha / alpha_rule) from spectrum features of g_delta:

* labels: for every training instance the batched sweep (one persistent
  launch) solves the PinT-QBVM system for N_ALPHA values
  alpha_rule * 10^t, t in [LOG_LO, LOG_HI], and reports ||y^0 - z0||; the label
  is the t with the smallest error (the data are synthetic, so z0 is known);
* features: 64-bin radial sine spectrum of g_delta, log10 delta, T, log2 N_t
  (Features kernel);
* training: MSE on t with Adam (MLP kernels), full-batch-shuffled minibatches;
* evaluation: reconstruction error of the predicted alpha against the
  a-priori rule, the discrepancy principle and the best alpha of the scan,
  all measured by sweep runs.

torch provides device memory and the shuffling gather only; every arithmetic
step runs in libqbvm.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np

from . import FORM_PQ, FP32_REFINE, MLP, Features, Sweep

N_ALPHA = 32
LOG_LO, LOG_HI = -2.0, 2.0
IN_DIM = 67


@dataclass
class Dataset:
    feats: "object"          # torch float32 [N, 67] (cuda)
    labels: "object"         # torch float32 [N] (cuda)
    delta: np.ndarray
    best_err: np.ndarray     # smallest error of the scan
    rule_err: np.ndarray     # error at the a-priori alpha (t = 0 on the scan)
    morozov_err: np.ndarray  # error at the discrepancy-principle pick
    seconds: float


def _sweep_chunk(torch, grid, z0, gd, delta, n_alpha, lo, hi, alpha_base=None, precision=FP32_REFINE):
    g_dev = torch.as_tensor(gd.reshape(len(gd), -1), dtype=torch.float64).cuda()
    z_dev = torch.as_tensor(z0.reshape(len(z0), -1), dtype=torch.float64).cuda()
    insts = []
    for b in range(len(gd)):
        insts.append(dict(dim=2, m=grid.M, L=grid.L, T=grid.T, nt=grid.nt, form=FORM_PQ, delta=float(delta[b]),
                          alpha_base=0.0 if alpha_base is None else float(alpha_base[b]),
                          g=g_dev[b], z0=z_dev[b]))
    with Sweep(insts, n_alpha=n_alpha, log10_lo=lo, log10_hi=hi, tau_dp=1.1, precision=precision) as sw:
        sw.run()
        al, disc, err, pick = sw.read()
    return g_dev, al, disc, err, pick


def make_dataset(count: int, seed: int, chunk: int = 4096, M: int = 128, nt: int = 128, T: float = 0.1) -> Dataset:
    """Generate `count` instances, label them with the sweep and compute features."""
    import torch
    import bhcp_inputs as bi

    feats = torch.empty((count, IN_DIM), dtype=torch.float32, device="cuda")
    labels = torch.empty(count, dtype=torch.float32, device="cuda")
    deltas, best, rule, moro = [], [], [], []
    fplan = Features(M, T, nt, chunk)
    ts = LOG_LO + (LOG_HI - LOG_LO) * np.arange(N_ALPHA) / (N_ALPHA - 1)
    i_rule = int(np.argmin(np.abs(ts)))
    t0 = time.perf_counter()
    done = 0
    c = 0
    while done < count:
        b = min(chunk, count - done)
        grid, z0, gd, delta = bi.alpha_training_batch(b, seed * 1000003 + c, M=M, nt=nt, T=T)
        g_dev, al, disc, err, pick = _sweep_chunk(torch, grid, z0, gd, delta, N_ALPHA, LOG_LO, LOG_HI)
        fplan.run(g_dev, delta, feats[done:done + b])
        idx = err.argmin(axis=1)
        labels[done:done + b] = torch.as_tensor(ts[idx], dtype=torch.float32)
        deltas.append(delta)
        best.append(err[np.arange(b), idx])
        rule.append(err[:, i_rule])
        moro.append(err[np.arange(b), pick[:, 0]])
        done += b
        c += 1
    torch.cuda.synchronize()
    fplan.close()
    return Dataset(feats, labels, np.concatenate(deltas), np.concatenate(best), np.concatenate(rule),
                   np.concatenate(moro), time.perf_counter() - t0)


def train(data: Dataset, epochs: int = 20, batch: int = 1024, lr: float = 1e-3, seed: int = 0,
          width: int = 128, log_every: int = 0):
    """Train a fresh network on `data`; returns (mlp, history of (epoch, loss))."""
    import torch

    n = data.feats.shape[0]
    mlp = MLP(IN_DIM, width, max_batch=max(batch, 4096), seed=seed)
    f = data.feats.double()
    mean = f.mean(dim=0).float().cpu().numpy()
    sd = f.std(dim=0).float().cpu().numpy()
    sd[sd < 1e-6] = 1.0
    mlp.set_norm(mean, sd)
    gen = torch.Generator().manual_seed(seed)
    hist = []
    for ep in range(epochs):
        perm = torch.randperm(n, generator=gen).cuda()
        xs = data.feats.index_select(0, perm)
        ys = data.labels.index_select(0, perm)
        for s in range(0, n - batch + 1, batch):
            mlp.train_step(xs[s:s + batch], ys[s:s + batch], lr)
        loss = mlp.last_loss()
        hist.append((ep, loss))
        if log_every and ep % log_every == 0:
            print(f"epoch {ep}: loss {loss:.4f}")
    return mlp, hist


def predict(mlp: MLP, feats):
    import torch
    y = torch.empty(feats.shape[0], dtype=torch.float32, device="cuda")
    out = []
    for s in range(0, feats.shape[0], 4096):
        e = min(feats.shape[0], s + 4096)
        mlp.forward(feats[s:e], y[: e - s])
        out.append(y[: e - s].cpu().numpy().copy())
    return np.concatenate(out)


def evaluate(mlp: MLP, count: int, seed: int, chunk: int = 4096, M: int = 128, nt: int = 128, T: float = 0.1):
    """Reconstruction errors on `count` held-out instances: learned alpha, a-priori
    rule, discrepancy principle (32-point scan) and the scan's best; and the
    solves/s of one-alpha runs (learned or a-priori) against the 32-alpha scan."""
    import torch
    import bhcp_inputs as bi

    fplan = Features(M, T, nt, chunk)
    res = {"learned": [], "rule": [], "morozov": [], "best": [], "t_pred": [], "t_best": []}
    times = {"one_alpha_s": 0.0, "scan_s": 0.0}
    ts = LOG_LO + (LOG_HI - LOG_LO) * np.arange(N_ALPHA) / (N_ALPHA - 1)
    done, c = 0, 0
    while done < count:
        b = min(chunk, count - done)
        grid, z0, gd, delta = bi.alpha_training_batch(b, seed * 1000003 + c, M=M, nt=nt, T=T)
        t0 = time.perf_counter()
        g_dev, al, disc, err, pick = _sweep_chunk(torch, grid, z0, gd, delta, N_ALPHA, LOG_LO, LOG_HI)
        times["scan_s"] += time.perf_counter() - t0
        feats = torch.empty((b, IN_DIM), dtype=torch.float32, device="cuda")
        fplan.run(g_dev, delta, feats)
        t_pred = predict(mlp, feats)
        alpha_rule = delta                      # PinT-QBVM, Section 5
        t0 = time.perf_counter()
        # one-alpha y^0 solves: the sweep's FP32 mode sums y^0 in double-float (~1e-13)
        _, _, _, err_l, _ = _sweep_chunk(torch, grid, z0, gd, delta, 1, 0.0, 0.0,
                                         alpha_base=alpha_rule * 10.0 ** t_pred, precision=FP32_REFINE)
        times["one_alpha_s"] += time.perf_counter() - t0
        _, _, _, err_r, _ = _sweep_chunk(torch, grid, z0, gd, delta, 1, 0.0, 0.0, precision=FP32_REFINE)
        res["learned"].append(err_l[:, 0])
        res["rule"].append(err_r[:, 0])
        res["morozov"].append(err[np.arange(b), pick[:, 0]])
        res["best"].append(err.min(axis=1))
        res["t_pred"].append(t_pred)
        res["t_best"].append(ts[err.argmin(axis=1)])
        done += b
        c += 1
    fplan.close()
    out = {k: np.concatenate(v) for k, v in res.items()}
    out["one_alpha_solves_per_s"] = count / times["one_alpha_s"]
    out["scan_solves_per_s"] = count * N_ALPHA / times["scan_s"]
    out["scan_instances_per_s"] = count / times["scan_s"]
    return out


def save_checkpoint(path: str, mlp: MLP, extra: dict | None = None) -> None:
    """Weights, Adam moments and step (and any extra arrays) in one .npz file."""
    p, m, v, step = mlp.get_params()
    np.savez(path, params=p, adam_m=m, adam_v=v, step=np.array(step), norm_mean=mlp._norm[0],
             norm_sd=mlp._norm[1], **(extra or {}))


def load_checkpoint(path: str, width: int = 128, max_batch: int = 4096) -> MLP:
    z = np.load(path)
    mlp = MLP(IN_DIM, width, max_batch=max_batch)
    mlp.set_norm(z["norm_mean"], z["norm_sd"])
    mlp.set_params(z["params"], z["adam_m"], z["adam_v"], int(z["step"]))
    return mlp
