"""Oracle of the learned refinement tagger (test infrastructure only: tests,
the smoke check and the benchmark's CPU baseline may use this module; the
product path never does).

The paper tags a patch for refinement from a per-patch criterion (Section 3:
refinement and coarsening criteria applied to each quadrant; Section 4.4 and
4.5.2 use the largest undivided difference of the cell averages).  The
learned tagger replaces that criterion by a small convolutional network that
sees the patch's cell averages with a two-cell halo and predicts the tag the
plain criterion will give one coarse step later.  The paper has no such
network: everything below is the definition this implementation adopts,
written out plainly in FP64 with numpy.

Definitions (F = 32 feature channels, C = components, S = n + 4):
  input     X[p, c, y, x] = (Q_c(i, j) - mean_interior(Q_c)) / (2 h_l thr),
            (i, j) = (x - 2, y - 2) over the patch and its two ghost layers,
            rounded to BF16 (so a central difference of X of size 1 is the
            plain criterion's threshold)
  layer 1   Z1 = conv3x3_valid(X, bf16(W1)) + emb[level]          [F, S-2, S-2]
            A1 = bf16(relu(Z1))
  layer 2   Z2 = conv3x3_valid(A1, bf16(W2)) + b2                 [F, S-4, S-4]
            M[g] = max(0, max_{y,x} Z2[g, y, x])
  layer 3   logit = w3 . M + b3
  loss      sum_p omega_p BCE(logit_p, label_p) / sum_p omega_p
conv3x3_valid(A, W)[g, y, x] = sum_{f, ky, kx} W[g, f, ky, kx] A[f, y + ky, x + kx].
Parameters are one flat FP32 vector: W1 [F, C, 3, 3], emb [16, F],
W2 [F, F, 3, 3], b2 [F], w3 [F], b3 [1].
"""
from __future__ import annotations

import numpy as np

F = 32
NLEVEL = 16


def param_count(ncomp: int) -> int:
    return F * ncomp * 9 + NLEVEL * F + F * F * 9 + F + F + 1


def unpack(params: np.ndarray, ncomp: int):
    p = np.asarray(params, dtype=np.float64)
    o = 0
    out = {}
    for name, shape in (("W1", (F, ncomp, 3, 3)), ("emb", (NLEVEL, F)), ("W2", (F, F, 3, 3)), ("b2", (F,)),
                        ("w3", (F,)), ("b3", (1,))):
        size = int(np.prod(shape))
        out[name] = p[o:o + size].reshape(shape)
        o += size
    assert o == len(p)
    return out


def bf16(a) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64.
    bfloat16 keeps the top 16 bits of an IEEE binary32 number."""
    f = np.asarray(a, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    rounded = ((bits + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(f)
    out = (rounded & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def conv3x3_valid(A: np.ndarray, W: np.ndarray) -> np.ndarray:
    """A [P, Cin, H, W], W [Cout, Cin, 3, 3] -> [P, Cout, H-2, W-2]."""
    P, cin, H, Wd = A.shape
    out = np.zeros((P, W.shape[0], H - 2, Wd - 2))
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("gf,pfyx->pgyx", W[:, :, ky, kx], A[:, :, ky:ky + H - 2, kx:kx + Wd - 2])
    return out


def forward(X: np.ndarray, level: np.ndarray, params: np.ndarray, ncomp: int, exact: bool = False):
    """Returns logit [P], M [P, F], argmax [P, F] (row-major index into the
    (S-4)^2 map of the first maximum, -1 where M = 0) and the intermediates.
    exact=True skips the BF16 roundings (a smooth function, for checking the
    gradient by finite differences)."""
    w = unpack(params, ncomp)
    rnd = (lambda a: np.asarray(a, dtype=np.float64)) if exact else bf16
    X = np.asarray(X, dtype=np.float64)
    Z1 = conv3x3_valid(X, rnd(w["W1"])) + w["emb"][np.asarray(level)][:, :, None, None]
    A1 = rnd(np.maximum(Z1, 0.0))
    Z2 = conv3x3_valid(A1, rnd(w["W2"])) + w["b2"][None, :, None, None]
    flat = Z2.reshape(Z2.shape[0], F, -1)
    arg = flat.argmax(axis=2)                       # first maximum in row-major order
    zmax = np.take_along_axis(flat, arg[..., None], axis=2)[..., 0]
    M = np.maximum(zmax, 0.0)
    arg = np.where(zmax > 0.0, arg, -1)
    logit = M @ w["w3"] + w["b3"][0]
    return logit, M, arg, {"Z1": Z1, "A1": A1, "Z2": Z2}


def loss(logit, label, omega) -> float:
    l, y, om = (np.asarray(a, dtype=np.float64) for a in (logit, label, omega))
    bce = np.maximum(l, 0.0) - l * y + np.log1p(np.exp(-np.abs(l)))
    return float((om * bce).sum() / om.sum())


def backward(X, level, params, ncomp: int, label, omega, exact: bool = False):
    """Gradient of loss() with respect to the flat parameter vector (chain
    rule through the layers above; BF16 rounding is treated as identity,
    the straight-through reading)."""
    w = unpack(params, ncomp)
    X = np.asarray(X, dtype=np.float64)
    level = np.asarray(level)
    logit, M, arg, mid = forward(X, level, params, ncomp, exact)
    P = X.shape[0]
    om = np.asarray(omega, dtype=np.float64)
    dlogit = om * (1.0 / (1.0 + np.exp(-logit)) - np.asarray(label, dtype=np.float64)) / om.sum()
    g = {k: np.zeros_like(v) for k, v in w.items()}
    g["w3"] = M.T @ dlogit
    g["b3"] = np.array([dlogit.sum()])
    dM = dlogit[:, None] * w["w3"][None, :]
    H2 = mid["Z2"].shape[2]
    dZ2 = np.zeros_like(mid["Z2"]).reshape(P, F, -1)
    pp, gg = np.nonzero(arg >= 0)
    dZ2[pp, gg, arg[pp, gg]] = dM[pp, gg]
    dZ2 = dZ2.reshape(mid["Z2"].shape)
    g["b2"] = dZ2.sum(axis=(0, 2, 3))
    A1 = mid["A1"]
    W2b = np.asarray(w["W2"], dtype=np.float64) if exact else bf16(w["W2"])
    dA1 = np.zeros_like(A1)
    for ky in range(3):
        for kx in range(3):
            g["W2"][:, :, ky, kx] = np.einsum("pgyx,pfyx->gf", dZ2, A1[:, :, ky:ky + H2, kx:kx + H2])
            dA1[:, :, ky:ky + H2, kx:kx + H2] += np.einsum("gf,pgyx->pfyx", W2b[:, :, ky, kx], dZ2)
    dZ1 = dA1 * (mid["Z1"] > 0.0)
    for lv in np.unique(level):
        g["emb"][lv] = dZ1[level == lv].sum(axis=(0, 2, 3))
    H1 = dZ1.shape[2]
    for ky in range(3):
        for kx in range(3):
            g["W1"][:, :, ky, kx] = np.einsum("pfyx,pcyx->fc", dZ1, X[:, :, ky:ky + H1, kx:kx + H1])
    return np.concatenate([g[k].reshape(-1) for k in ("W1", "emb", "W2", "b2", "w3", "b3")])


def adam(params, m, v, grad, step: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam step (Kingma & Ba 2015, Algorithm 1), returns new (params, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def inputs(lattice_avg: np.ndarray, n: int, level: np.ndarray, dx0: float, thr: float) -> np.ndarray:
    """X from the cell averages of every leaf with its two ghost layers:
    lattice_avg [P, C, W, W] (lattice index = cell index + 2, W = n + 5;
    the last row and column are not cells), ghosts already exchanged."""
    A = np.asarray(lattice_avg, dtype=np.float64)[:, :, :n + 4, :n + 4]
    mu = A[:, :, 2:n + 2, 2:n + 2].mean(axis=(2, 3))
    h = dx0 / (2.0 ** np.asarray(level, dtype=np.float64))
    scale = 1.0 / (2.0 * h * thr)
    return bf16((A - mu[:, :, None, None]) * scale[:, None, None, None])


def combine_tags(logit, plain_tags, cmin: float):
    """Tags from the network with the plain criterion as fallback: where the
    network's confidence |2 sigmoid(logit) - 1| is below cmin the plain tag
    is kept; else 1 if it predicts refinement, and otherwise the plain tag
    with refinement removed (-1 stays -1, 1 becomes 0)."""
    prob = 1.0 / (1.0 + np.exp(-np.asarray(logit, dtype=np.float64)))
    conf = np.abs(2.0 * prob - 1.0)
    plain = np.asarray(plain_tags, dtype=np.int8)
    net = np.where(prob >= 0.5, 1, np.where(plain == -1, -1, 0)).astype(np.int8)
    return np.where(conf < cmin, plain, net).astype(np.int8), int((conf < cmin).sum())
