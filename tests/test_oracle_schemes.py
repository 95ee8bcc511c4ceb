"""Pins of the oracle's schemes and of the whole compressed step (no GPU)."""
import numpy as np
import pytest

import oracle as O
from paper_2302_09883_gb300 import inputs

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def test_d2q9_equilibrium_moments():
    # Closed form of the second-order equilibrium: zeroth, first and second
    # moments are rho, rho u and rho u u + rho/3 I.
    for rho, ux, uy in [(1.0, 0.0, 0.0), (1.3, 0.05, -0.02), (0.7, -0.1, 0.08)]:
        f = O.d2q9_equilibrium(rho, ux, uy)
        assert abs(f.sum() - rho) < 1e-15
        assert abs((CX * f).sum() - rho * ux) < 1e-15
        assert abs((CY * f).sum() - rho * uy) < 1e-15
        assert abs((CX * CX * f).sum() - (rho * ux * ux + rho / 3)) < 1e-15
        assert abs((CX * CY * f).sum() - rho * ux * uy) < 1e-15
        assert abs((CY * CY * f).sum() - (rho * uy * uy + rho / 3)) < 1e-15


def test_d2q9_collision_conserves_and_relaxes():
    rng = np.random.default_rng(0)
    f = O.d2q9_equilibrium(1.1, 0.03, 0.01) + rng.normal(scale=1e-3, size=9)
    g = O.d2q9_collide(f, tau=1.0)  # tau = 1: post-collision = equilibrium
    rho = f.sum()
    ux, uy = (CX * f).sum() / rho, (CY * f).sum() / rho
    assert np.allclose(g, O.d2q9_equilibrium(rho, ux, uy), atol=1e-15)
    h = O.d2q9_collide(f, tau=0.6)
    assert abs(h.sum() - f.sum()) < 1e-15
    assert abs((CX * h).sum() - (CX * f).sum()) < 1e-15


def test_d2q9_rest_state_is_fixed():
    s = O.OracleSim("d2q9", "bl53", 64, 64, 32, 3, 1e-4, tau=0.7)
    n = 64
    s.init_macro([np.full((n, n), 1.2), np.zeros((n, n)), np.zeros((n, n))])
    f0 = s.export_all()
    s.step(5)
    assert np.abs(s.export_all() - f0).max() < 1e-15  # round-off only


@pytest.mark.parametrize("tau", [0.8, 0.6])
def test_d2q9_shear_wave_decay_closed_form(tau):
    # Viscous decay u(t) = U exp(-nu k^2 t), nu = (tau - 1/2)/3 (textbook
    # lattice Boltzmann), on a 64^2 periodic lattice; compressed eps=0 run.
    n, U = 64, 1e-3
    f = inputs.shear_wave(n, u0=U, noise=0.0)
    s = O.OracleSim("d2q9", "bl53", n, n, 32, 3, 0.0, tau=tau)
    s.init_macro(f)
    T = 200
    s.step(T)
    F = s.export_all()
    rho = F.sum(0)
    ux = (CX[:, None, None] * F).sum(0) / rho
    k = 2 * np.pi / n
    nu = (tau - 0.5) / 3
    amp = 2 * np.mean(ux * np.sin(k * np.arange(n))[:, None])
    assert abs(amp / (U * np.exp(-nu * k * k * T)) - 1) < 2e-3


def test_compressed_eps0_equals_uncompressed_reference():
    # Patches + ghost sync + DWT/iDWT at eps = 0 give the global scheme.
    n = 64
    f = inputs.gaussian_bump(n, sigma=6.0)
    for wavelet in ["haar", "bl53"]:
        s = O.OracleSim("d2q9", wavelet, n, n, 16, 2, 0.0, tau=0.8)
        r = O.OracleRef("d2q9", wavelet, n, n, tau=0.8)
        s.init_macro(f)
        r.init_macro(f)
        s.step(30)
        r.step(30)
        for i in range(9):
            assert np.abs(s.export_field(i) - r.export_field(i)).max() < 1e-14


def test_compressed_mass_is_conserved_fp64():
    # eq. conservation + shared bordering nodes (Sec. 3.1.1): global mass is
    # exactly conserved by the lossy compression; momentum too (BGK).
    n = 128
    f = inputs.gaussian_bump(n)
    for wavelet in ["haar", "bl53"]:
        s = O.OracleSim("d2q9", wavelet, n, n, 32, 3, 1e-4, tau=0.8)
        s.init_macro(f)
        m0 = s.stats()["coef_sums"]
        s.step(40)
        st = s.stats()
        m1 = st["coef_sums"]
        assert abs(m1.sum() - m0.sum()) <= 1e-13 * m0.sum()
        assert abs((CX * m1).sum() - (CX * m0).sum()) <= 1e-13 * m0.sum()
        assert st["shared_mismatch"] == 0
        # the field really was compressed
        assert st["compressed_bytes"] < 9 * n * n * 8 / 5
        # decoded global mass equals the coefficient-domain mass
        direct = sum(s.export_field(i).sum() for i in range(9))
        assert abs(direct - m1.sum()) <= 1e-12 * m1.sum()


def test_fp32_oracle_close_to_fp64():
    n = 128
    f = inputs.shear_wave(n, noise=1e-4)
    a = O.OracleSim("d2q9", "bl53", n, n, 64, 4, 1e-4, prec="f64", tau=0.6)
    b = O.OracleSim("d2q9", "bl53", n, n, 64, 4, 1e-4, prec="f32", store="bf16", tau=0.6)
    a.init_macro(f)
    b.init_macro(f)
    a.step(10)
    b.step(10)
    x, y = a.export_all(), b.export_all()
    assert np.linalg.norm(x - y) / np.linalg.norm(x) < 1e-4
    assert b.stats()["shared_mismatch"] == 0


# ------------------------------------------------------------------ Euler
def _euler_flux(W, nx, ny, gamma=1.4):
    rho, mx, my, E = W
    u, v = mx / rho, my / rho
    p = (gamma - 1) * (E - 0.5 * rho * (u * u + v * v))
    un = u * nx + v * ny
    return np.array([rho * un, mx * un + p * nx, my * un + p * ny, (E + p) * un])


def _cons(rho, u, v, p, gamma=1.4):
    return np.array([rho, rho * u, rho * v, p / (gamma - 1) + 0.5 * rho * (u * u + v * v)])


def test_rusanov_consistency_and_antisymmetry():
    WL = _cons(1.0, 0.3, -0.2, 1.0)
    WR = _cons(0.4, -0.1, 0.5, 0.3)
    for nx, ny in [(1, 0), (-1, 0), (0, 1), (0, -1)]:
        # consistency with the physical flux (eq. flux_def)
        assert np.allclose(O.rusanov(WL, WL, nx, ny), _euler_flux(WL, nx, ny), atol=1e-15)
        # conservation across a face: F(L,R,N) = -F(R,L,-N), bit for bit
        assert np.array_equal(O.rusanov(WL, WR, nx, ny), -O.rusanov(WR, WL, -nx, -ny))


def _exact_riemann(rhoL, uL, pL, rhoR, uR, pR, xi, g=1.4):
    """Textbook exact Riemann solver (Newton on the star pressure)."""
    cL, cR = np.sqrt(g * pL / rhoL), np.sqrt(g * pR / rhoR)

    def fk(p, rho, pk, c):
        if p > pk:
            A, B = 2 / ((g + 1) * rho), (g - 1) / (g + 1) * pk
            return (p - pk) * np.sqrt(A / (p + B))
        return 2 * c / (g - 1) * ((p / pk) ** ((g - 1) / (2 * g)) - 1)

    p = 0.5 * (pL + pR)
    for _ in range(100):
        f = fk(p, rhoL, pL, cL) + fk(p, rhoR, pR, cR) + uR - uL
        dp = 1e-7 * p
        df = (fk(p + dp, rhoL, pL, cL) + fk(p + dp, rhoR, pR, cR) - fk(p - dp, rhoL, pL, cL)
              - fk(p - dp, rhoR, pR, cR)) / (2 * dp)
        p = max(p - f / df, 1e-12)
    us = 0.5 * (uL + uR) + 0.5 * (fk(p, rhoR, pR, cR) - fk(p, rhoL, pL, cL))
    out = np.zeros((len(xi), 3))
    for n, s in enumerate(xi):
        if s < us:
            rho, u, pk, c, sign = rhoL, uL, pL, cL, -1
        else:
            rho, u, pk, c, sign = rhoR, uR, pR, cR, 1
        if p > pk:  # shock
            S = u + sign * c * np.sqrt((g + 1) / (2 * g) * p / pk + (g - 1) / (2 * g))
            rs = rho * (p / pk + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * p / pk + 1)
            out[n] = (rs, us, p) if sign * (s - S) < 0 else (rho, u, pk)
        else:  # rarefaction
            cs = c * (p / pk) ** ((g - 1) / (2 * g))
            head, tail = u + sign * c, us + sign * cs
            if sign * (s - head) > 0:
                out[n] = (rho, u, pk)
            elif sign * (s - tail) < 0:
                out[n] = (rho * (p / pk) ** (1 / g), us, p)
            else:
                uu = 2 / (g + 1) * (-sign * c + (g - 1) / 2 * u + s)
                cc = -sign * (uu - s)
                rr = rho * (cc / c) ** (2 / (g - 1))
                out[n] = (rr, uu, pk * (cc / c) ** (2 * g / (g - 1)))
    return out


def test_euler_sod_converges_to_exact_riemann_solution():
    # First-order Rusanov on the Sod tube along x: L1 error against the
    # exact solution small and shrinking under refinement.
    errs = []
    for n in (128, 256):
        r = O.OracleRef("euler2d", "bl53", n, 16, periodic=(False, True), cfl=0.4)
        f = inputs.sod_x(n)
        f = [a[:16, :] for a in f]
        r.init_macro(f)
        while r.time < 0.15:
            r.step(1)
        t = r.time
        rho = r.export_field(0)[0]
        x = np.arange(n + 1) / n
        ex = _exact_riemann(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, (x - 0.5) / t)
        errs.append(np.mean(np.abs(rho - ex[:, 0])))
        assert np.allclose(r.export_field(0), rho[None, :], atol=0)  # stays 1-D
    assert errs[0] < 0.03 and errs[1] < errs[0] * 0.8


def test_euler_uniform_state_and_contact_advection():
    # A uniform state is fixed.  A density bump with constant velocity and
    # pressure is a contact wave: the Rusanov scheme keeps u and p uniform
    # (the pressure and kinetic terms cancel exactly) and moves the bump at u.
    n = 64
    x = np.arange(n) / n
    X, Y = np.meshgrid(x, x)
    rho = 1.0 + 0.2 * np.exp(-((X - 0.4) ** 2 + (Y - 0.5) ** 2) / 0.005)
    u0 = 0.5
    r = O.OracleRef("euler2d", "bl53", n, n, periodic=(True, True), cfl=0.3)
    r.init_macro([rho, np.full_like(rho, u0), np.zeros_like(rho), np.ones_like(rho)])
    m0 = r.export_field(0)
    c0 = ((m0 - 1) * X).sum() / (m0 - 1).sum()
    r.step(10)
    W = [r.export_field(q) for q in range(4)]
    u = W[1] / W[0]
    p = 0.4 * (W[3] - 0.5 * W[1] * u)
    assert np.abs(u - u0).max() < 1e-13 and np.abs(p - 1).max() < 1e-13
    assert np.abs(W[2]).max() < 1e-13
    assert abs(W[0].sum() - m0.sum()) < 1e-12 * m0.sum()
    c1 = ((W[0] - 1) * X).sum() / (W[0] - 1).sum()
    assert abs((c1 - c0) / (u0 * r.time) - 1) < 0.05
    uu = O.OracleRef("euler2d", "bl53", 32, 32, periodic=(False, False))
    f = [np.full((33, 33), v) for v in (0.9, 0.2, -0.1, 1.3)]
    uu.init_macro(f)
    W0 = [uu.export_field(q) for q in range(4)]
    uu.step(3)
    for q in range(4):
        assert np.abs(uu.export_field(q) - W0[q]).max() < 1e-15


def test_euler_compressed_eps0_matches_reference_and_conserves():
    n = 64
    f = inputs.four_quadrant(n)
    s = O.OracleSim("euler2d", "bl53", n, n, 32, 3, 0.0, periodic=(False, False), cfl=0.4)
    r = O.OracleRef("euler2d", "bl53", n, n, periodic=(False, False), cfl=0.4)
    s.init_macro(f)
    r.init_macro(f)
    s.step(20)
    r.step(20)
    for q in range(4):
        assert np.abs(s.export_field(q) - r.export_field(q)).max() < 1e-12
    # periodic lossy run conserves all four integrals
    p = O.OracleSim("euler2d", "bl53", n, n, 32, 3, 1e-3, periodic=(True, True), cfl=0.4)
    ff = [a[:n, :n] for a in f]
    p.init_macro(ff)
    m0 = p.stats()["coef_sums"]
    p.step(20)
    m1 = p.stats()["coef_sums"]
    assert np.all(np.abs(m1 - m0) <= 1e-12 * np.abs(m0).max())
    assert p.stats()["shared_mismatch"] == 0


def test_euler_fixed_time_step_mode():
    # cfl < 0 selects a fixed step dt/h = -cfl (used to compare runs at equal
    # physical times)
    n = 64
    r = O.OracleRef("euler2d", "bl53", n, n, periodic=(False, False), cfl=-0.1)
    r.init_macro(inputs.four_quadrant(n))
    r.step(7)
    assert abs(r.time - 7 * 0.1 / n) < 1e-15


def test_import_roundtrip_and_single_field():
    # eps 0 keeps every coefficient: importing a state and exporting it again
    # returns it up to the FP64 rounding of one forward and one inverse
    # transform; importing one field leaves the others as they decode.
    rng = np.random.default_rng(5)
    n, P, L = 64, 32, 3
    o = O.OracleSim("d2q9", "bl53", n, n, P, L, 0.0)
    v = 1.0 / 9.0 + 1e-3 * rng.normal(size=(9, n, n))
    o.import_field(-1, v)
    back = o.export_all()
    assert np.max(np.abs(back - v)) <= 1e-14
    assert o.stats()["shared_mismatch"] == 0
    w = v[4] + 1e-2 * rng.normal(size=(n, n))
    o.import_field(4, w)
    back2 = o.export_all()
    assert np.max(np.abs(back2[4] - w)) <= 1e-14
    others = [q for q in range(9) if q != 4]
    assert np.max(np.abs(back2[others] - back[others])) <= 1e-14
    # mass of the imported state from the coarse blocks alone
    mass = o.stats()["coef_sums"].sum()
    assert abs(mass - back2.sum()) <= 1e-12 * abs(mass)
