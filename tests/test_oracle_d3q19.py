"""Pins of the oracle's D3Q19 scheme and of its 3-D compressed-patch run
(no GPU)."""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_2302_09883_gb300 import inputs


def _lattice_from_equilibrium():
    """Weights and velocities read back from the oracle's equilibrium:
    feq(rho=1, u=0) = w_i, and for a small u along axis a,
    (feq_i / w_i - 1) / (3 u) -> c_ia."""
    w = O.d3q19_equilibrium(1.0, 0.0, 0.0, 0.0)
    eps = 1e-7
    c = np.zeros((19, 3))
    for a in range(3):
        u = [0.0, 0.0, 0.0]
        u[a] = eps
        f = O.d3q19_equilibrium(1.0, *u)
        c[:, a] = (f / w - 1.0) / (3 * eps)
    return w, np.rint(c).astype(int), c


def test_lattice_is_d3q19():
    w, c, craw = _lattice_from_equilibrium()
    assert np.allclose(craw, c, atol=1e-5)
    vecs = {tuple(v) for v in c}
    want = {(0, 0, 0)} | {v for v in itertools.product((-1, 0, 1), repeat=3) if 1 <= sum(map(abs, v)) <= 2}
    assert vecs == want and len(vecs) == 19  # no (+-1,+-1,+-1) corners
    n2 = (c * c).sum(1)
    assert np.allclose(w[n2 == 0], 1 / 3) and np.allclose(w[n2 == 1], 1 / 18) and np.allclose(w[n2 == 2], 1 / 36)
    # isotropy up to fourth order
    assert abs(w.sum() - 1) < 1e-15
    M2 = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(M2, np.eye(3) / 3, atol=1e-15)
    M4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(3)
    want4 = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(M4, want4, atol=1e-15)


def test_equilibrium_moments():
    _, c, _ = _lattice_from_equilibrium()
    rho, u = 1.07, np.array([0.031, -0.017, 0.022])
    f = O.d3q19_equilibrium(rho, *u)
    assert abs(f.sum() - rho) < 1e-15
    assert np.allclose(c.T @ f, rho * u, atol=1e-16)
    P = np.einsum("i,ia,ib->ab", f, c, c)
    assert np.allclose(P, rho * (np.eye(3) / 3 + np.outer(u, u)), atol=1e-15)


def test_collision_conserves_and_relaxes():
    _, c, _ = _lattice_from_equilibrium()
    rng = np.random.default_rng(0)
    f = O.d3q19_equilibrium(1.0, 0.02, 0.01, -0.03) + 1e-3 * rng.normal(size=19)
    g = O.d3q19_collide(f, 0.7)
    assert abs(g.sum() - f.sum()) < 1e-15
    assert np.allclose(c.T @ g, c.T @ f, atol=1e-16)
    # tau = 1: the collision lands on the equilibrium of the moments
    h = O.d3q19_collide(f, 1.0)
    rho = f.sum()
    u = (c.T @ f) / rho
    assert np.allclose(h, O.d3q19_equilibrium(rho, *u), atol=1e-16)


def _amp(ux, axis, n):
    s = np.arange(n)
    shape = [1, 1, 1]
    shape[2 - axis] = n
    return 2.0 / ux.size * float(np.sum(ux * np.sin(2 * np.pi * s / n).reshape(shape)))


def _velocity(F, c):
    rho = F.sum(0)
    return [np.tensordot(c[:, a], F, axes=(0, 0)) / rho for a in range(3)]


@pytest.mark.parametrize("axis", [1, 2])
def test_shear_wave_decays_at_the_lattice_viscosity(axis):
    # u_x = U sin(2 pi s / N) along y or z: amplitude ~ exp(-nu k^2 t),
    # nu = (tau - 1/2) / 3; the same along both axes (isotropy)
    _, c, _ = _lattice_from_equilibrium()
    N, tau, t = 32, 0.8, 150
    dims = (4, N, 4) if axis == 1 else (4, 4, N)
    r = O.OracleRef3(*dims, prec="f64", tau=tau)
    r.init_macro(inputs.shear_wave_3d(*dims, u0=1e-3, axis=axis))
    a0 = _amp(_velocity(r.export_all(), c)[0], axis, N)
    r.step(t)
    a1 = _amp(_velocity(r.export_all(), c)[0], axis, N)
    nu, k = (tau - 0.5) / 3, 2 * np.pi / N
    assert abs(a1 / a0 - np.exp(-nu * k * k * t)) < 2e-3


def test_planar_taylor_green_decays():
    # z-independent vortex u = U (sin kx cos ky, -cos kx sin ky, 0): the
    # amplitude decays as exp(-2 nu k^2 t)
    _, c, _ = _lattice_from_equilibrium()
    N, tau, t, U = 64, 0.7, 400, 1e-3
    k = 2 * np.pi / N
    i = np.arange(N) * k
    Y, X = np.meshgrid(i, i, indexing="ij")
    ux = np.broadcast_to(U * np.sin(X) * np.cos(Y), (4, N, N)).copy()
    uy = np.broadcast_to(-U * np.cos(X) * np.sin(Y), (4, N, N)).copy()
    rho = np.ones((4, N, N))
    r = O.OracleRef3(N, N, 4, prec="f64", tau=tau)
    r.init_macro([rho, ux, uy, np.zeros_like(ux)])
    r.step(t)
    v = _velocity(r.export_all(), c)
    ratio = np.sum(v[0] * ux) / np.sum(ux * ux)
    nu = (tau - 0.5) / 3
    assert abs(ratio - np.exp(-2 * nu * k * k * t)) < 1.5e-3
    assert np.max(np.abs(v[2])) < 1e-12


def test_rest_state_is_kept():
    shape = (16, 16, 16)
    f = [np.ones(shape), np.zeros(shape), np.zeros(shape), np.zeros(shape)]
    s = O.OracleSim3("bl53", 16, 16, 16, 8, 2, 1e-3, tau=0.6)
    s.init_macro(f)
    s.step(3)
    F = s.export_all()
    w = O.d3q19_equilibrium(1.0, 0.0, 0.0, 0.0)
    assert np.max(np.abs(F - w[:, None, None, None])) < 1e-15


@pytest.mark.parametrize("wavelet,P,L", [("bl53", 16, 3), ("haar", 8, 3)])
def test_eps_zero_compressed_run_equals_uncompressed(wavelet, P, L):
    n = 32
    f = inputs.taylor_green_3d(n, u0=0.04)
    s = O.OracleSim3(wavelet, n, n, n, P, L, 0.0, tau=0.55)
    r = O.OracleRef3(n, n, n, tau=0.55)
    s.init_macro(f)
    r.init_macro(f)
    s.step(4)
    r.step(4)
    a, b = s.export_all(), r.export_all()
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))
    assert s.stats()["shared_mismatch"] == 0


def test_compressed_mass_is_conserved_fp64():
    n = 32
    f = inputs.taylor_green_3d(n, u0=0.04)
    s = O.OracleSim3("bl53", n, n, n, 16, 3, 1e-3, tau=0.55)
    s.init_macro(f)
    m0 = s.stats()["coef_sums"].sum()
    assert abs(m0 - f[0].sum()) <= 1e-12 * m0  # the coarse blocks carry the mass
    s.step(6)
    st = s.stats()
    assert abs(st["coef_sums"].sum() - m0) <= 1e-12 * m0
    assert st["shared_mismatch"] == 0
    # and the compression does compress
    assert st["compressed_bytes"] < 0.5 * 19 * 8 * n ** 3


def patch_block(state, p, P):
    """The decoded state on patch p's nodes and the layer around them,
    (19, P+3, P+3, P+3), periodic wrap; p = (px, py, pz)."""
    n = state.shape[1:]
    idx = [(p[a] * P + np.arange(-1, P + 2)) % n[2 - a] for a in range(3)]
    return state[:, idx[2]][:, :, idx[1]][:, :, :, idx[0]]


def test_single_patch_step_equals_the_whole_grid_step():
    """d3q19_patch_step (one patch from its decoded surroundings) writes the
    record the whole-grid oracle step writes for that patch: 64^3, P 32,
    L 3, BF16, every patch, after a step of a vortex with a perturbation."""
    n, P, L, eps, tau = 64, 32, 3, 1e-6, 0.55
    s = O.OracleSim3("bl53", n, n, n, P, L, eps, prec="f32", store="bf16", tau=tau)
    f = inputs.taylor_green_3d(n)
    rng = np.random.default_rng(2)
    f[1] = f[1] + 1e-4 * rng.standard_normal(f[1].shape)
    s.init_macro(f)
    s.step(1)
    state = s.export_all()
    s.step(1)
    npp = n // P
    for pid in range(npp ** 3):
        p = (pid % npp, (pid // npp) % npp, pid // (npp * npp))
        rec = O.d3q19_patch_step(patch_block(state, p, P), P, L, eps, tau, store="bf16", pid=pid)
        assert rec == s.record(pid), pid
