"""Parity of the learned tagger's CUDA kernels (af_cnn_*) with the FP64
oracle (oracle/cnn.py), through the C ABI: inputs, forward pass, gradients,
Adam, the fallback rule, and that training on the GPU learns."""
import numpy as np
import pytest

import oracle as O
import synth as S
from oracle import cnn as OC

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def af():
    from paper_2205_07572_gb300 import af as _af, build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return _af


def _nerr(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def _bf16_bits(vals):
    """float64 values that are BF16 numbers -> int16 tensor of their bits."""
    f = np.asarray(vals, dtype=np.float32)
    bits = (f.view(np.uint32) >> 16).astype(np.uint16)
    assert np.array_equal((bits.astype(np.uint32) << 16).view(np.float32), f)
    return torch.from_numpy(bits.view(np.int16)).cuda()


def _bits_to_float(t):
    b = t.cpu().numpy().view(np.uint16).astype(np.uint32) << 16
    return b.view(np.float32).astype(np.float64)


def _problem(C, N, P, seed):
    rng = np.random.default_rng(seed)
    X = OC.bf16(rng.normal(size=(P, C, N + 4, N + 4)) * 2.0)
    level = rng.integers(0, 8, size=P).astype(np.int32)
    params = (rng.normal(size=OC.param_count(C)) * 0.25).astype(np.float32).astype(np.float64)
    label = rng.integers(0, 2, size=P).astype(np.float32)
    omega = rng.uniform(0.5, 3.0, size=P).astype(np.float32)
    return X, level, params, label, omega


@pytest.mark.parametrize("C,N", [(3, 16), (1, 8), (3, 8), (1, 16)])
def test_inference_forward_equals_training_forward_bitwise(af, C, N):
    """af_cnn_forward without the positions (d_arg NULL, inference: b2 added
    after the max-pool) gives the logits and pooled maxima of the forward
    with them bit for bit, on inputs with ties, zero and negative maxima, on
    more patches than resident CTAs (several patches per CTA)."""
    from paper_2205_07572_gb300.tagger import Tagger
    P = 2500
    X, level, params, _, _ = _problem(C, N, P, seed=7 * C + N)
    X[: P // 4] = OC.bf16(np.round(X[: P // 4]))          # many equal values: ties in the max-pool
    X[P // 4: P // 2] = 0.0                               # constant patches: maxima b2 only
    t = Tagger(C, N)
    t.params.copy_(torch.from_numpy(params.astype(np.float32)))
    x, lv = _bf16_bits(X), torch.from_numpy(level).cuda()
    lg, M, arg = t.forward(x, lv)
    lg_i, M_i = t.infer(x, lv)
    torch.cuda.synchronize()
    assert torch.isfinite(lg).all()
    assert torch.equal(lg.view(torch.int32), lg_i.view(torch.int32))
    assert torch.equal(M.view(torch.int32), M_i.view(torch.int32))
    assert (M == 0).any() and (M > 0).any()


@pytest.mark.parametrize("C,N", [(3, 16), (1, 8), (3, 8), (1, 16)])
def test_forward_matches_oracle(af, C, N):
    X, level, params, _, _ = _problem(C, N, 64, seed=C * 10 + N)
    lg_r, M_r, arg_r, _ = OC.forward(X, level, params, C)
    from paper_2205_07572_gb300.tagger import Tagger
    t = Tagger(C, N)
    t.params.copy_(torch.from_numpy(params.astype(np.float32)))
    lg, M, arg = t.forward(_bf16_bits(X), torch.from_numpy(level).cuda())
    torch.cuda.synchronize()
    assert _nerr(lg.cpu().numpy(), lg_r) < 2e-3
    assert _nerr(M.cpu().numpy(), M_r) < 2e-3
    assert (arg.cpu().numpy() == arg_r).mean() > 0.98


@pytest.mark.parametrize("C,N", [(3, 16), (1, 8)])
def test_gradients_match_oracle(af, C, N):
    X, level, params, label, omega = _problem(C, N, 48, seed=7 + C)
    g_r = OC.backward(X, level, params, C, label, omega)
    from paper_2205_07572_gb300.tagger import Tagger
    t = Tagger(C, N)
    t.params.copy_(torch.from_numpy(params.astype(np.float32)))
    x, lv = _bf16_bits(X), torch.from_numpy(level).cuda()
    fwd = t.forward(x, lv)
    g = t.gradient(x, lv, torch.from_numpy(label).cuda(), torch.from_numpy(omega).cuda(), float(omega.sum()), fwd)
    torch.cuda.synchronize()
    g = g.cpu().numpy().astype(np.float64)
    sizes = [32 * C * 9, 16 * 32, 32 * 32 * 9, 32, 32, 1]
    o = 0
    for s in sizes:
        assert _nerr(g[o:o + s], g_r[o:o + s]) < 2e-2, (o, s, _nerr(g[o:o + s], g_r[o:o + s]))
        o += s
    # deterministic: the same call gives the same bits
    g2 = t.gradient(x, lv, torch.from_numpy(label).cuda(), torch.from_numpy(omega).cuda(), float(omega.sum()), fwd)
    assert np.array_equal(g2.cpu().numpy(), g.astype(np.float32))


def test_adam_matches_oracle(af):
    rng = np.random.default_rng(1)
    n = 1000
    p, g1, g2 = rng.normal(size=n), rng.normal(size=n), rng.normal(size=n)
    dp = torch.from_numpy(p.astype(np.float32)).cuda()
    dm, dv = torch.zeros_like(dp), torch.zeros_like(dp)
    pr, mr, vr = p.astype(np.float32).astype(np.float64), np.zeros(n), np.zeros(n)
    for step, g in ((1, g1), (2, g2)):
        gg = g.astype(np.float32)
        af.cnn_adam(n, dp, dm, dv, torch.from_numpy(gg).cuda(), step, 1e-2)
        pr, mr, vr = OC.adam(pr, mr, vr, gg.astype(np.float64), step, 1e-2)
    torch.cuda.synchronize()
    assert np.allclose(dp.cpu().numpy(), pr, rtol=0, atol=1e-5)


def test_tag_combination_matches_oracle(af):
    rng = np.random.default_rng(4)
    logit = rng.normal(size=500).astype(np.float32) * 3
    plain = rng.choice([-1, 0, 1], size=500).astype(np.int8)
    ref, nref = OC.combine_tags(logit, plain, 0.6)
    out = torch.zeros(500, dtype=torch.int8, device="cuda")
    nf = torch.zeros(1, dtype=torch.int32, device="cuda")
    af.cnn_tags(500, torch.from_numpy(logit).cuda(), torch.from_numpy(plain).cuda(), 0.6, out, nf)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref) and int(nf.item()) == nref


@pytest.mark.parametrize("prec", [0, 1])
def test_inputs_match_oracle(af, prec):
    """X of every leaf of an adaptive forest equals the oracle's (cell averages
    with the exchanged two-cell halo, centred and scaled, BF16)."""
    import ctypes
    from paper_2205_07572_gb300.amr import Forest
    n, lmax, nc = 16, 3, 3
    leaves = sorted(S.balanced_forest(1, 1, 3, lambda l, x, y: x == y), key=lambda t: (t[0], t[2], t[1]))
    st = np.nan_to_num(S.forest_state(n, nc, 1, lmax, leaves, [S.ring_wave, S.gaussian(0.3, 0.6, 0.1),
                                                              lambda x, y: np.sin(7 * x)], nq=2))
    st = st.reshape(len(leaves), -1)
    if prec:
        st = st.astype(np.float32).astype(np.float64)
    lv = np.array([l for l, _, _ in leaves], np.int32)
    ix = np.array([x for _, x, _ in leaves], np.int32)
    iy = np.array([y for _, _, y in leaves], np.int32)
    ip = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    allm = (1 << (lmax + 1)) - 1
    filled = np.empty_like(st)
    O.lib().orc_fill_amr(n, nc, len(leaves), ip(lv), ip(ix), ip(iy), 1, lmax, allm, allm, 0, O._dp(st),
                         O._dp(filled))
    lay = S.Layout(n, nc)
    lat = lay.lattice(filled.reshape(len(leaves), nc, 4, -1))[:, :, 0]
    dx0, thr = 1.0 / n, 4.0
    X_r = OC.inputs(lat, n, lv, dx0, thr)
    F = Forest(1, lmax, leaves)
    cfg = af.config(af.ACOUSTICS, af.F32 if prec else af.F64, n, c=1.0)
    d = torch.from_numpy(st).to(torch.float32 if prec else torch.float64).cuda()
    af.fill_ghosts(cfg, F.c, allm, allm, 0, d)
    x = torch.empty((len(leaves), nc, n + 4, n + 4), dtype=torch.int16, device="cuda")
    af.cnn_inputs(cfg, F.c, af.state_pair(d, None, 0), torch.from_numpy(F.nbr).cuda(), dx0, thr, x)
    torch.cuda.synchronize()
    got = _bits_to_float(x).reshape(X_r.shape)
    same = got == X_r
    assert same.mean() > 0.999
    ulp = np.abs(X_r) * 2.0 ** -7
    assert np.all(np.abs(got - X_r) <= ulp + 1e-30)


def test_training_learns_a_threshold_rule(af):
    """Labels from the plain criterion applied to the input itself (largest
    central difference of channel 0 >= 1): GPU training drives the accuracy
    well above the majority rate."""
    from paper_2205_07572_gb300.tagger import Tagger, prepare
    rng = np.random.default_rng(0)
    P, N, C = 16384, 8, 1
    amp = rng.uniform(0.0, 1.2, size=P)
    kx = rng.uniform(0.5, 2.5, size=P)
    yy, xx = np.meshgrid(np.arange(N + 4), np.arange(N + 4), indexing="ij")
    X = amp[:, None, None] * np.sin(kx[:, None, None] * xx[None] + rng.uniform(0, 6, size=P)[:, None, None])
    X = OC.bf16(X[:, None])
    cd = np.abs(X[:, 0, 2:N + 2, 3:N + 3] - X[:, 0, 2:N + 2, 1:N + 1]).max(axis=(1, 2))
    label = (cd >= 1.0).astype(np.float32)
    data = {"x": _bf16_bits(X), "level": torch.zeros(P, dtype=torch.int32, device="cuda"),
            "label": torch.from_numpy(label).cuda()}
    data = prepare(data, 1024)
    t = Tagger(C, N, seed=1)
    before = t.evaluate(data)
    t.fit(data, epochs=12, batch=1024, lr=3e-3)
    after = t.evaluate(data)
    torch.cuda.synchronize()
    base = max(label.mean(), 1 - label.mean())
    assert after["loss"] < before["loss"]
    assert after["accuracy"] > max(0.9, base + 0.1), (before, after, base)
