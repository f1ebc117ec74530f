"""Learned refinement tagger: parameters, training loop and data collection.

The network, its inputs and its training step are the af_cnn_* entry points
of libaf.so (BF16 storage, FP32 arithmetic); this module holds the FP32
master parameters and Adam moments as device tensors and orchestrates:

  collect()  runs the adaptive method with the plain criterion and records,
             at every regrid, each leaf's input X and the plain criterion's
             tag for that leaf one coarse step later (the label);
  Tagger.fit()  minibatch Adam on those samples;
  AMRRun.tags_learned()  (amr.py) tags a forest with the network, falling
             back to the plain criterion where the network is not confident.
"""
from __future__ import annotations

import math

import numpy as np

from . import af

F = 32
NLEVEL = 16


class Tagger:
    def __init__(self, ncomp: int, n: int, seed: int = 0, device="cuda"):
        import torch
        if n not in (8, 16):
            raise ValueError("the tagger is compiled for 8 x 8 and 16 x 16 patches")
        self.ncomp, self.n, self.device = ncomp, n, device
        self.S = n + 4
        rng = np.random.default_rng(seed)
        parts = [
            rng.normal(0.0, math.sqrt(2.0 / (ncomp * 9)), F * ncomp * 9),   # W1
            np.zeros(NLEVEL * F),                                           # level embedding
            rng.normal(0.0, math.sqrt(2.0 / (F * 9)), F * F * 9),           # W2
            np.zeros(F),                                                    # b2
            rng.normal(0.0, math.sqrt(1.0 / F), F),                         # w3
            np.zeros(1),                                                    # b3
        ]
        p = np.concatenate(parts).astype(np.float32)
        assert len(p) == af.cnn_param_count(ncomp)
        self.params = torch.from_numpy(p).to(device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.step = 0
        self.nblocks = 152
        self.partial = torch.zeros(af.cnn_partial_floats(ncomp, self.nblocks), dtype=torch.float32, device=device)

    @property
    def nparam(self) -> int:
        return int(self.params.numel())

    def outputs(self, nsample: int):
        import torch
        return (torch.empty(nsample, dtype=torch.float32, device=self.device),
                torch.empty((nsample, F), dtype=torch.float32, device=self.device),
                torch.empty((nsample, F), dtype=torch.int32, device=self.device))

    def forward(self, x, level, out=None, stream=None):
        nsample = int(level.numel())
        logit, m, arg = out if out is not None else self.outputs(nsample)
        af.cnn_forward(self.ncomp, self.n, nsample, x, level, self.params, logit, m, arg, stream)
        return logit, m, arg

    def infer(self, x, level, out=None, stream=None):
        """Inference: logits and pooled maxima without the maxima's positions
        (af_cnn_forward with d_arg NULL; the same logits bit for bit)."""
        nsample = int(level.numel())
        logit, m = out if out is not None else self.outputs(nsample)[:2]
        af.cnn_forward(self.ncomp, self.n, nsample, x, level, self.params, logit, m, None, stream)
        return logit, m

    def gradient(self, x, level, label, weight, weight_sum: float, fwd, stream=None):
        logit, m, arg = fwd
        af.cnn_backward(self.ncomp, self.n, int(level.numel()), x, level, self.params, logit, m, arg, label, weight,
                        weight_sum, self.partial, self.nblocks, self.grad, stream)
        return self.grad

    def train_step(self, x, level, label, weight, weight_sum: float, lr: float, fwd_buf=None, stream=None):
        fwd = self.forward(x, level, fwd_buf, stream)
        self.gradient(x, level, label, weight, weight_sum, fwd, stream)
        self.step += 1
        af.cnn_adam(self.nparam, self.params, self.m, self.v, self.grad, self.step, lr, stream=stream)
        return fwd

    def fit(self, data, epochs: int = 4, batch: int = 4096, lr: float = 2e-3, log=None):
        """Minibatch Adam over a dataset from collect() (already shuffled):
        batches are contiguous slices, so no gather runs in the loop."""
        x, level, label, weight, wsum = data["x"], data["level"], data["label"], data["weight"], data["wsum"]
        P = int(level.numel())
        row = x[0].numel()
        nb = max(1, P // batch)
        fwd_buf = self.outputs(batch)
        for ep in range(epochs):
            for b in range(nb):
                s = b * batch
                e = min(P, s + batch)
                if e - s != batch:
                    continue
                self.train_step(x.view(-1)[s * row:e * row], level[s:e], label[s:e], weight[s:e], float(wsum[b]),
                                lr, fwd_buf)
            if log is not None:
                log(ep, self.evaluate(data))
        return self

    def evaluate(self, data, limit: int = 1 << 18):
        """Loss and accuracy against the labels (first `limit` samples)."""
        import torch
        P = min(int(data["level"].numel()), limit)
        logit, _, _ = self.forward(data["x"][:P], data["level"][:P])
        y = data["label"][:P]
        pred = (logit >= 0).float()
        acc = float((pred == y).float().mean().item())
        pos = y > 0.5
        recall = float((pred[pos] == 1).float().mean().item()) if bool(pos.any()) else float("nan")
        prec = float((y[pred > 0.5] == 1).float().mean().item()) if bool((pred > 0.5).any()) else float("nan")
        bce = torch.nn.functional.binary_cross_entropy_with_logits(logit, y, weight=data["weight"][:P])
        return {"accuracy": acc, "recall": recall, "precision": prec, "loss": float(bce.item())}


def collect(run, coarse_steps: int, tag: tuple, lmin: int, thr: float, horizon: int = 1, regrid: bool = True):
    """Samples from a run of the method with the plain criterion, regridded
    every `horizon` coarse steps: at each regrid, every leaf's input X and, as
    its label, whether the plain criterion tags it for refinement at the end
    of any of the next `horizon` coarse steps (on the same forest).  The run
    is then regridded with the last of those tags, as the method does.
    Returns device tensors (x uint16 BF16 storage, level int32, label float)."""
    import torch
    xs, levels, labels = [], [], []
    comp, kind, rthr, cthr = tag
    for _ in range(max(1, coarse_steps // horizon)):
        x = run.cnn_inputs(thr)
        lv = run.forest.d_level.clone()
        need = np.zeros(run.forest.nleaf, dtype=bool)
        for _ in range(horizon):
            run.coarse_step()
            tags, _ = run.tags(comp, kind, rthr, cthr)
            need |= tags == 1
        xs.append(x)
        levels.append(lv)
        labels.append(torch.from_numpy(need.astype(np.float32)).to(run.device))
        if regrid:
            run.regrid(tags, lmin)
    return {"x": torch.cat(xs), "level": torch.cat(levels), "label": torch.cat(labels)}


def prepare(data, batch: int, seed: int = 0, pos_weight=None):
    """Shuffle once, weight the classes (positives by #neg/#pos unless given)
    and precompute every batch's weight sum on the host."""
    import torch
    P = int(data["level"].numel())
    g = torch.Generator(device="cpu").manual_seed(seed)
    perm = torch.randperm(P, generator=g).to(data["level"].device)
    out = {k: v[perm].contiguous() for k, v in data.items()}
    y = out["label"].cpu().numpy()
    npos = max(1.0, float(y.sum()))
    pw = float(pos_weight) if pos_weight is not None else max(1.0, (len(y) - npos) / npos)
    w = np.where(y > 0.5, pw, 1.0).astype(np.float32)
    out["weight"] = torch.from_numpy(w).to(out["label"].device)
    nb = max(1, P // batch)
    out["wsum"] = [float(w[b * batch:(b + 1) * batch].sum()) for b in range(nb)]
    out["pos_weight"] = pw
    out["positives"] = int(npos)
    return out


# ------------------------------------------------------------ evaluation
def interior_averages(run, comp: int = 0):
    """Host [nleaf, n, n] interior cell averages of one component (current state)."""
    n, nc = run.cfg.n, run.cfg.ncomp
    lay_w = n + 5
    plane = af.plane_stride(n)
    host = run.current().double().cpu().numpy().reshape(run.forest.nleaf, nc, 4, plane)
    lat = host[:, comp, 0, :lay_w * lay_w].reshape(-1, lay_w, lay_w)
    return lat[:, 2:n + 2, 2:n + 2]


def uniform_global(run, comp: int = 0):
    """Interior averages of a run whose leaves all have one level, as one
    global [side*n, side*n] array (row = y)."""
    F = run.forest
    lv = F.level[0]
    assert (F.level == lv).all()
    n = run.cfg.n
    side = F.B << int(lv)
    a = interior_averages(run, comp)
    g = np.zeros((side * n, side * n))
    for k in range(F.nleaf):
        x, y = F.ix[k], F.iy[k]
        g[y * n:(y + 1) * n, x * n:(x + 1) * n] = a[k]
    return g


def l1_vs_uniform(run, ref_global, comp: int = 0) -> float:
    """sum over leaves and cells of |Q - Q_ref| dx_l dy_l, Q_ref the uniform
    finer run's averages over the leaf cell (exact for cell averages)."""
    F = run.forest
    n = run.cfg.n
    a = interior_averages(run, comp)
    fine = ref_global.shape[0]
    total = 0.0
    for k in range(F.nleaf):
        l = int(F.level[k])
        side = F.B << l
        r = fine // (side * n)
        blk = ref_global[F.iy[k] * n * r:(F.iy[k] + 1) * n * r, F.ix[k] * n * r:(F.ix[k] + 1) * n * r]
        ref = blk.reshape(n, r, n, r).mean(axis=(1, 3))
        total += float(np.abs(a[k] - ref).sum()) * (run.dx0 / (1 << l)) * (run.dy0 / (1 << l))
    return total
