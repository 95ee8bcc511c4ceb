"""GPU parity of the learned per-patch threshold on 3-D (D3Q19) patches: the
3-D features and labels against the oracle (FP32 transforms, FP64 sums and
tests), and learned-mode steps: records byte-identical to the oracle fed the
same per-patch eps, features and the network's eps against the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2302_09883_gb300 import Sim3, inputs, learned

pytestmark = pytest.mark.gpu


def _state3(n, seed):
    """19 smooth fields (the equilibria of a Taylor-Green vortex) plus noise
    whose amplitude changes between octants of the grid."""
    rho, ux, uy, uz = inputs.taylor_green_3d(n, u0=0.04)
    feq = np.stack([O.d3q19_equilibrium(1.0, 0.0, 0.0, 0.0)[i] * rho * (1 + 3 * (ux + uy)) for i in range(19)])
    rng = np.random.default_rng(seed)
    amp = 10 ** rng.uniform(-7, -3, size=(2, 2, 2))
    A = np.kron(amp, np.ones((n // 2, n // 2, n // 2)))
    return (feq + A[None] * rng.normal(size=feq.shape)).astype(np.float32)


def _nodes3(u, P, px, py, pz):
    E = P + 1
    idx = [(np.arange(E) + p * P) % u.shape[1 + k] for k, p in enumerate((pz, py, px))]
    return u[:, idx[0]][:, :, idx[1]][:, :, :, idx[2]]


@pytest.mark.parametrize("n,P", [(32, 16), (64, 32)])
def test_features_and_labels3_match_oracle(n, P):
    import torch
    L, delta = 3, 1e-4
    u = _state3(n, seed=n + P)
    feat, lab = learned.features_labels3(torch.from_numpy(u).cuda(), P, L, delta)
    feat, lab = feat.cpu().numpy(), lab.cpu().numpy()
    npx = n // P
    labs = []
    for pid in range(npx ** 3):
        px, py, pz = pid % npx, (pid // npx) % npx, pid // (npx * npx)
        v = _nodes3(u.astype(np.float64), P, px, py, pz)
        fo = O.patch_features(v, "bl53", P, L, prec="f32")
        assert np.max(np.abs(feat[pid] - fo)) <= 2e-6 * max(1.0, np.max(np.abs(fo))), pid
        lo = O.patch_label(v, "bl53", P, L, delta, prec="f32")
        assert abs(lab[pid] - lo) <= 1e-6, (pid, lab[pid], lo)
        labs.append(lo)
    assert len(set(np.round(labs, 3))) > 1


def test_learned_mode3_steps_match_oracle():
    n, P, L, lo, hi = 64, 32, 3, 1e-7, 1e-2
    f = inputs.taylor_green_3d(n, u0=0.04)
    g = Sim3(n, n, n, P, L, 1e-6, store="bf16", tau=0.55, arena_factor=0.5)
    o = O.OracleSim3("bl53", n, n, n, P, L, 1e-6, prec="f32", store="bf16", tau=0.55)
    g.init_macro(f)
    o.init_macro(f)
    m = learned.Mlp(14 * L, seed=21)
    w = m.weights()
    w[-65:-1] *= 0.02
    w[-1] = -6.0
    m.set_weights(w)
    w = w.astype(np.float64)
    learned.use_mlp(g, m, lo, hi)
    o.track_features()
    for k in range(3):
        _, eps_used = learned.patch_data(g, L)
        if k == 0:
            assert np.all(eps_used == 1e-6)
        o.set_patch_eps(eps_used)
        g.step(1)
        o.step(1)
        g.sync()
        for p in range(g.npatch):
            assert g.record(p) == o.record(p), "step %d patch %d" % (k, p)
        feat, eps_next = learned.patch_data(g, L)
        fo = o.features()
        e_idx = np.arange(0, 14 * L, 2)
        assert np.max(np.abs(feat[:, e_idx] - fo[:, e_idx])) <= 1e-4
        assert np.max(np.abs(feat[:, e_idx + 1] - fo[:, e_idx + 1])) <= 1e-5
        want = np.clip(10 ** O.mlp_forward(w, feat.astype(np.float64), 14 * L, 64), lo, hi)
        assert np.max(np.abs(eps_next / want - 1)) <= 1e-4
        assert np.all((eps_next > lo) & (eps_next < hi))
    learned.use_mlp(g, None)
    g.step(1)
    g.sync()
