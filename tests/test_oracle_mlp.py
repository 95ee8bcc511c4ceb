"""Pins of the oracle's learned-threshold pieces (no GPU)."""
import math

import numpy as np
import pytest

import oracle as O


def test_gelu_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    nin, nh, B = 8, 64, 16
    w = rng.normal(scale=0.3, size=O.mlp_nparam(nin, nh))
    X = rng.normal(size=(B, nin))
    t = rng.normal(size=B)
    loss, g = O.mlp_loss_grad(w, X, t, nin, nh)
    idx = rng.choice(len(w), 40, replace=False)
    for i in idx:
        h = 1e-6
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        lp = np.mean((O.mlp_forward(wp, X, nin, nh) - t) ** 2)
        lm = np.mean((O.mlp_forward(wm, X, nin, nh) - t) ** 2)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd))
    assert abs(loss - np.mean((O.mlp_forward(w, X, nin, nh) - t) ** 2)) < 1e-12


def test_mlp_forward_closed_form_single_unit():
    # with only the path input0 -> hidden0 -> hidden0 -> output active the
    # network is GELU(GELU(a x + b) * c + d) * e + f
    nin, nh = 8, 64
    w = np.zeros(O.mlp_nparam(nin, nh))
    a, b, c, d, e, f = 0.7, -0.2, 1.3, 0.1, -0.9, 0.05
    w[0] = a
    w[nh * nin] = b
    w[nh * nin + nh] = c
    w[nh * nin + nh + nh * nh] = d
    w[nh * nin + nh + nh * nh + nh] = e
    w[-1] = f
    gelu = lambda x: 0.5 * x * (1 + math.erf(x / math.sqrt(2)))
    x = np.zeros((1, nin))
    x[0, 0] = 1.7
    want = gelu(gelu(a * 1.7 + b) * c + d) * e + f
    assert abs(O.mlp_forward(w, x, nin, nh)[0] - want) < 1e-14


def test_features_of_a_linear_patch_have_no_detail_energy():
    P, L = 64, 4
    x = np.arange(P + 1) / P
    X, Y = np.meshgrid(x, x)
    u = np.stack([1 + 0.3 * X - 0.2 * Y, 0.5 + 0.1 * X])
    f = O.patch_features(u, "bl53", P, L)
    assert f.shape == (2 * 3 * L,)
    assert np.all(f < -14)  # log10 of (~0 + 1e-30)


def _cls(k, L):
    if k % (1 << L) == 0:
        return 0
    c = 1
    while k % 2 == 0:
        k //= 2
        c += 1
    return c


def _group(kx, ky, L):
    cx, cy = _cls(kx, L), _cls(ky, L)
    l = max(cx, cy)
    if l == 0:
        return None
    S = (1 if cx == l else 0) | (2 if cy == l else 0)
    return (l - 1) * 3 + S - 1


@pytest.mark.parametrize("wavelet", ["bl53", "haar"])
def test_features_of_planted_coefficients(wavelet):
    # one planted detail per group (value +-(g+1)/7), two fields: after the
    # inverse transform, the features must return log10(sum v^2 / count) and
    # log10(max |v|) of exactly the planted values, group by group.
    P, L = 32, 3
    E = P + 1 if wavelet == "bl53" else P
    rng = np.random.default_rng(3)
    nodes = {}
    for ky in range(E):
        for kx in range(E):
            g = _group(kx, ky, L)
            if g is not None:
                nodes.setdefault(g, []).append((ky, kx))
    assert sorted(nodes) == list(range(3 * L))
    c = np.zeros((2, E, E))
    for g, lst in nodes.items():
        ky, kx = lst[rng.integers(len(lst))]
        c[0, ky, kx] = (g + 1) / 7.0
        ky, kx = lst[rng.integers(len(lst))]
        c[1, ky, kx] = -(g + 1) / 7.0 if g % 2 else 0.0
    c[:, 0, 0] = 1.0  # a coarse value, not a feature
    u = np.stack([O.dwt(c[f], wavelet, P, L, inverse=True) for f in range(2)])
    feat = O.patch_features(u, wavelet, P, L)
    for g in range(3 * L):
        v = np.concatenate([c[f][tuple(np.array(nodes[g]).T)] for f in range(2)])
        assert abs(feat[2 * g] - math.log10(np.sum(v * v) / len(v) + 1e-30)) < 1e-9
        assert abs(feat[2 * g + 1] - math.log10(np.max(np.abs(v)) + 1e-30)) < 1e-9


def _brute_err(u, eps, P, L):
    lay = O.layout("bl53", 2, P, L)
    num = den = 0.0
    for f in range(u.shape[0]):
        c = O.dwt(u[f], "bl53", P, L)
        keep = (np.abs(c.reshape(-1)) >= eps) | lay["coarse"]
        t = np.where(keep, c.reshape(-1), 0.0).reshape(c.shape)
        back = O.dwt(t, "bl53", P, L, inverse=True)
        num += np.sum((back - u[f]) ** 2)
        den += np.sum(u[f] ** 2)
    return math.sqrt(num / den)


def test_label_is_largest_safe_eps():
    rng = np.random.default_rng(1)
    P, L = 32, 3
    x = np.arange(P + 1) / P
    X, Y = np.meshgrid(x, x)
    u = np.stack([1 + 0.1 * np.sin(6 * X) * np.cos(5 * Y) + 1e-4 * rng.normal(size=X.shape),
                  0.2 * np.cos(3 * X + Y)])
    delta = 1e-4
    lab = O.patch_label(u, "bl53", P, L, delta)
    assert -7 < lab < -2
    # brute force: the label is admissible, one bisection step above is not,
    # and no grid value above the label's grid cell is admissible
    assert _brute_err(u, 10 ** lab, P, L) <= delta
    assert _brute_err(u, 10 ** (lab + 1 / 128), P, L) > delta
    k = int(math.floor((lab + 7) * 8 + 1e-9))
    for kk in range(k + 1, 41):
        assert _brute_err(u, O.eps_grid(kk), P, L) > delta


def test_label_bounds():
    P, L = 32, 3
    x = np.arange(P + 1) / P
    X, Y = np.meshgrid(x, x)
    smooth = np.stack([1 + 0.3 * X - 0.2 * Y])  # linear: every eps is admissible
    assert O.patch_label(smooth, "bl53", P, L, 1e-6) == -2.0
    rng = np.random.default_rng(5)
    # noise far below the smallest eps: every eps drops all of it, delta is tighter
    rough = np.stack([1 + 1e-9 * rng.normal(size=X.shape)])
    assert O.patch_label(rough, "bl53", P, L, 1e-12) == -7.0


def _group3(k, L):
    c = [_cls(v, L) for v in k]
    l = max(c)
    if l == 0:
        return None
    S = sum(1 << a for a in range(3) if c[a] == l)
    return (l - 1) * 7 + S - 1


def test_features_of_planted_coefficients_3d():
    # 3-D: 7 groups per level (every non-empty set of axes); one planted
    # coefficient per group, read back from the features after the inverse
    # transform
    P, L = 8, 3
    E = P + 1
    rng = np.random.default_rng(4)
    nodes = {}
    for kz in range(E):
        for ky in range(E):
            for kx in range(E):
                g = _group3((kx, ky, kz), L)
                if g is not None:
                    nodes.setdefault(g, []).append((kz, ky, kx))
    assert sorted(nodes) == list(range(7 * L))
    c = np.zeros((E, E, E))
    for g, lst in nodes.items():
        kz, ky, kx = lst[rng.integers(len(lst))]
        c[kz, ky, kx] = (g + 1) / 11.0
    c[0, 0, 0] = 1.0  # a coarse value, not a feature
    u = O.dwt(c, "bl53", P, L, inverse=True)
    feat = O.patch_features(u[None], "bl53", P, L)
    assert feat.shape == (2 * 7 * L,)
    for g in range(7 * L):
        v = c[tuple(np.array(nodes[g]).T)]
        assert abs(feat[2 * g] - math.log10(np.sum(v * v) / len(v) + 1e-30)) < 1e-9
        assert abs(feat[2 * g + 1] - math.log10(np.max(np.abs(v)) + 1e-30)) < 1e-9


def test_fp32_label_is_close_to_fp64_label_3d():
    P, L = 16, 3
    x = np.arange(P + 1) / P
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    rng = np.random.default_rng(6)
    u = np.stack([1 + 0.05 * np.sin(4 * X + 2 * Y) * np.cos(3 * Z) + 1e-5 * rng.normal(size=X.shape),
                  0.02 * np.cos(2 * X - Z)])
    l64 = O.patch_label(u, "bl53", P, L, 1e-4)
    l32 = O.patch_label(u, "bl53", P, L, 1e-4, prec="f32")
    assert -7 < l64 < -2 and abs(l64 - l32) <= 1 / 128 + 1e-9
