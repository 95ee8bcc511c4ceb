"""GPU parity of the learned per-patch threshold against the oracle: patch
features and labels, the network's gradient and inference, steps with a
per-patch eps (records byte-identical), and the features that a step writes
in learned mode."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2302_09883_gb300 import Sim, inputs, learned

pytestmark = pytest.mark.gpu


def _nodes(u, P, px, py, wavelet):
    """Node values of patch (px, py) of a periodic state u (F, G1, G0)."""
    E = P + 1 if wavelet == "bl53" else P
    ys = (py * P + np.arange(E)) % u.shape[1]
    xs = (px * P + np.arange(E)) % u.shape[2]
    return u[:, ys][:, :, xs]


def _patchy_state(n, F, seed):
    """Smooth waves plus noise whose amplitude changes from patch to patch
    (10^U(-7, -2)), so that the labels spread over the eps grid."""
    rng = np.random.default_rng(seed)
    x = np.arange(n) / n
    X, Y = np.meshgrid(x, x)
    amp = 10 ** rng.uniform(-7, -2, size=(8, 8))
    A = np.kron(amp, np.ones((n // 8, n // 8)))
    out = []
    for f in range(F):
        base = 1.0 + 0.1 * np.sin(2 * np.pi * ((f + 1) * X + 2 * Y)) if f == 0 else \
            0.05 * np.cos(2 * np.pi * (3 * X - f * Y)) * np.exp(-4 * (X - 0.5) ** 2)
        out.append(base + A * rng.normal(size=X.shape))
    return np.stack(out).astype(np.float32)


@pytest.mark.parametrize("wavelet,P,L,F", [("bl53", 32, 3, 2), ("bl53", 64, 4, 1), ("haar", 32, 3, 2)])
def test_features_and_labels_match_oracle(wavelet, P, L, F):
    import torch
    n, delta = 256, 1e-4
    u = _patchy_state(n, F, seed=11 + P + F)
    feat, lab = learned.features_labels(torch.from_numpy(u).cuda(), P, L, delta, wavelet)
    feat, lab = feat.cpu().numpy(), lab.cpu().numpy()
    npx = n // P
    labs = []
    for pid in range(npx * npx):
        px, py = pid % npx, pid // npx
        v = _nodes(u.astype(np.float64), P, px, py, wavelet)
        fo = O.patch_features(v, wavelet, P, L)
        assert np.max(np.abs(feat[pid] - fo)) <= 1e-5 * max(1.0, np.max(np.abs(fo))), pid
        lo = O.patch_label(v, wavelet, P, L, delta)
        assert abs(lab[pid] - lo) <= 1e-6, (pid, lab[pid], lo)
        labs.append(lo)
    assert len(set(np.round(labs, 3))) > 4  # the labels do spread


def _net(nin, seed, y0=None, scale=0.3):
    m = learned.Mlp(nin, seed=seed)
    if y0 is not None:  # output near y0: scale the last layer down, shift it
        w = m.weights()
        w[-65:-1] *= scale
        w[-1] = y0
        m.set_weights(w)
    return m


def test_mlp_gradient_and_forward_match_fp64_oracle():
    import torch
    rng = np.random.default_rng(2)
    nin, B = 24, 300
    m = _net(nin, seed=3)
    w = m.weights().astype(np.float64)
    X = rng.normal(size=(B, nin)).astype(np.float32)
    t = rng.normal(size=B).astype(np.float32)
    loss_g, g_g = m.grad(torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda())
    loss_o, g_o = O.mlp_loss_grad(w, X.astype(np.float64), t.astype(np.float64), nin, 64)
    assert abs(loss_g - loss_o) <= 1e-5 * loss_o
    assert np.linalg.norm(g_g - g_o) <= 1e-4 * np.linalg.norm(g_o)
    assert np.max(np.abs(g_g - g_o)) <= 1e-4 * np.max(np.abs(g_o))
    y_g = m.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    y_o = O.mlp_forward(w, X.astype(np.float64), nin, 64)
    assert np.max(np.abs(y_g - y_o) / (1 + np.abs(y_o))) <= 1e-5


def test_mlp_training_fits_and_is_deterministic():
    import torch
    rng = np.random.default_rng(4)
    nin, n = 24, 2048
    X = rng.normal(size=(n, nin)).astype(np.float32)
    t = (0.8 * np.tanh(X[:, 0]) - 0.5 * X[:, 1] * X[:, 2] + 0.3 * X[:, 3] - 4.0).astype(np.float32)
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    runs = []
    for _ in range(2):
        m = _net(nin, seed=5)
        loss0, _ = m.grad(Xd, td)
        hist = m.train(Xd, td, epochs=60, batch=128, lr=3e-3, seed=6)
        loss1, _ = m.grad(Xd, td)
        runs.append((loss0, hist, loss1, m.weights()))
    loss0, hist, loss1, w = runs[0]
    assert loss1 < 0.05 * loss0
    assert np.all(np.isfinite(hist))
    assert np.array_equal(w, runs[1][3])  # fixed-order reductions: same bits


def test_fit_standardises_in_the_library_and_folds_into_the_first_layer():
    # wcs_mlp_fit against the same trainer run by hand: inputs standardised
    # in FP64 here, output bias started at the mean target, the fold done
    # here in FP64.  Columns of very different offsets and scales.
    import torch
    rng = np.random.default_rng(8)
    nin, n, NH = 12, 1024, 64
    X = (rng.normal(size=(n, nin)) * 10.0 ** np.arange(-3, 3, 0.5) + np.arange(nin) * 7.0).astype(np.float32)
    t = (np.tanh(X[:, 0] * 1e3) - 0.2 * X[:, 11] / 300 - 4.0).astype(np.float32)
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    m, hist = learned.fit(Xd, td, epochs=6, batch=128, lr=2e-3, seed=2)
    X64 = X.astype(np.float64)
    mu, sd = X64.mean(0), X64.std(0, ddof=1)
    assert np.allclose(m.input_stats[:nin, 0], mu, rtol=1e-12, atol=1e-12 * np.abs(mu).max())
    assert np.allclose(m.input_stats[:nin, 1], sd, rtol=1e-9)
    assert abs(m.input_stats[nin, 0] - t.astype(np.float64).mean()) <= 1e-12 * 5
    h = learned.Mlp(nin, seed=2)
    w = h.weights()
    w[-1] = np.float32(t.astype(np.float64).mean())
    h.set_weights(w)
    Xs = ((X64 - mu) / np.maximum(sd, 1e-3)).astype(np.float32)
    hist_h = h.train(torch.from_numpy(Xs).cuda(), td, epochs=6, batch=128, lr=2e-3, seed=2)
    assert np.allclose(hist, hist_h, rtol=1e-4)
    w = h.weights().astype(np.float64)
    W1, b1 = w[:NH * nin].reshape(NH, nin) / np.maximum(sd, 1e-3)[None, :], w[NH * nin:NH * nin + NH]
    w[:NH * nin], w[NH * nin:NH * nin + NH] = W1.reshape(-1), b1 - W1 @ mu
    y_fit = m.forward(Xd).cpu().numpy()
    y_ref = O.mlp_forward(w, X64, nin, NH)
    assert np.max(np.abs(y_fit - y_ref)) <= 1e-3 * (1 + np.abs(y_ref).max())


@pytest.mark.parametrize("case", ["d2q9_bf16", "haar_f64"])
def test_per_patch_eps_steps_match_oracle_bytewise(case):
    if case == "d2q9_bf16":
        n, P, L, prec, store, wv, f, tau = 256, 64, 4, "f32", "bf16", "bl53", inputs.shear_wave(256, seed=8), 0.6
    else:
        n, P, L, prec, store, wv, f, tau = 128, 32, 3, "f64", "f64", "haar", inputs.gaussian_bump(128), 0.8
    g = Sim("d2q9", wv, n, n, P, L, 1e-4, prec=prec, store=store, tau=tau)
    o = O.OracleSim("d2q9", wv, n, n, P, L, 1e-4, prec=prec, store=store, tau=tau)
    g.init_macro(f)
    o.init_macro(f)
    rng = np.random.default_rng(9)
    eps = 10 ** rng.uniform(-6, -2.5, size=g.npatch)
    learned.set_patch_eps(g, eps)
    o.set_patch_eps(eps)
    for s in (1, 4):
        g.step(s)
        o.step(s)
        g.sync()
        for p in range(g.npatch):
            assert g.record(p) == o.record(p), "patch %d" % p
    assert np.array_equal(g.export_field(-1), o.export_all())
    # smaller per-patch eps keep more: the same run at min(eps, 1e-6) (an
    # arena large enough for nearly uncompressed records) is not smaller
    u = Sim("d2q9", wv, n, n, P, L, 1e-4, prec=prec, store=store, tau=tau, arena_factor=2.0)
    u.init_macro(f)
    learned.set_patch_eps(u, np.minimum(eps, 1e-6))
    u.step(5)
    u.sync()
    assert u.compressed_bytes() >= g.compressed_bytes()


@pytest.mark.parametrize("case", ["d2q9", "euler"])
def test_learned_mode_steps_features_and_eps_match_oracle(case):
    if case == "d2q9":
        sc, n, per, f, kw = "d2q9", 256, (True, True), inputs.shear_wave(256, seed=10), dict(tau=0.6)
    else:
        sc, n, per, f, kw = "euler2d", 256, (False, False), inputs.four_quadrant(256), dict(cfl=-0.15)
    P, L, lo, hi = 64, 4, 1e-7, 1e-2
    g = Sim(sc, "bl53", n, n, P, L, 1e-4, prec="f32", store="bf16", periodic=per, **kw)
    o = O.OracleSim(sc, "bl53", n, n, P, L, 1e-4, prec="f32", store="bf16", periodic=per, **kw)
    g.init_macro(f)
    o.init_macro(f)
    m = _net(6 * L, seed=12, y0=-4.0, scale=0.02)
    w = m.weights().astype(np.float64)
    learned.use_mlp(g, m, lo, hi)
    o.track_features()
    spread = []
    for k in range(4):
        _, eps_used = learned.patch_data(g, L)
        if k == 0:
            assert np.all(eps_used == 1e-4)
        o.set_patch_eps(eps_used)
        g.step(1)
        o.step(1)
        g.sync()
        for p in range(g.npatch):
            assert g.record(p) == o.record(p), "step %d patch %d" % (k, p)
        feat, eps_next = learned.patch_data(g, L)
        fo = o.features()
        e_idx = np.arange(0, 6 * L, 2)
        assert np.max(np.abs(feat[:, e_idx] - fo[:, e_idx])) <= 1e-4
        assert np.max(np.abs(feat[:, e_idx + 1] - fo[:, e_idx + 1])) <= 1e-5
        want = np.clip(10 ** O.mlp_forward(w, feat.astype(np.float64), 6 * L, 64), lo, hi)
        assert np.max(np.abs(eps_next / want - 1)) <= 1e-4
        assert np.all((eps_next > lo) & (eps_next < hi))  # not hidden by the clamp
        spread.append(np.ptp(np.log10(eps_next)))
    assert min(spread) > 1e-3  # the network does vary eps between patches
    learned.use_mlp(g, None)
    g.step(2)
    g.sync()


def test_mlp_input_size_must_match_levels():
    from paper_2302_09883_gb300._lib import WcsError
    g = Sim("d2q9", "bl53", 256, 256, 64, 4, 1e-4, prec="f32", store="bf16", tau=0.6)
    m = _net(18, seed=1)
    with pytest.raises(WcsError):
        learned.use_mlp(g, m)
    g.init_macro(inputs.shear_wave(256, seed=1))
    g.step(1)
    g.sync()
    assert math.isfinite(g.stats()["mass"])
