"""Seeded synthetic inputs (macroscopic initial fields) and workload shapes.

This module holds no arithmetic of the method: it only produces the initial
macroscopic fields (density, velocity, pressure) that both the CUDA library
and the CPU oracle turn into their state.  Arrays are float64, shaped
(ny_nodes, nx_nodes), x fastest.
"""
import numpy as np

# Workloads: the shapes, sizes and parameters of the benchmark cases.
WORKLOADS = {
    # D2Q9 BGK, 128^2 periodic, 16 Haar patches of 32^2, 3 levels, FP64.
    "d2q9_haar_128": dict(scheme="d2q9", wavelet="haar", n=128, P=32, L=3, eps=1e-4, prec="f64",
                          store="f64", rule="const", tau=0.8, steps=100, init="bump"),
    # D2Q9 BGK, 2048^2 periodic, BL5/3 patches of 64 cells, 4 levels, FP32
    # compute, BF16 details with per-band scale, shear wave + noise.
    "d2q9_bl53_2048": dict(scheme="d2q9", wavelet="bl53", n=2048, P=64, L=4, eps=1e-3, prec="f32",
                           store="bf16", rule="const", tau=0.6, steps=2000, init="shear"),
    # 2-D Euler, Rusanov, 4096 cells (4097 nodes) per axis, outflow, BL5/3
    # patches of 64, 4 levels, FP32 compute, int8 details.
    "euler_bl53_4096": dict(scheme="euler2d", wavelet="bl53", n=4096, P=64, L=4, eps=1e-3, prec="f32",
                            store="i8", rule="const", cfl=0.4, gamma=1.4, steps=1500, init="quadrants",
                            periodic=(False, False)),
    # Linear transport (the paper's Sec. 3.1.2): 128 cells (129 nodes) per
    # axis on [-1, 1]^2, 2 x 2 patches of 64 cells, outflow, velocity
    # (0.9, 0.9), CFL 0.45, Gaussian 1 + exp(-30 r^2), run to t = 0.5;
    # FP32 compute, thresholded details stored in FP32 (no quantisation).
    "transport_128": dict(scheme="transport", wavelet="bl53", n=128, P=64, L=4, eps=0.01, prec="f32",
                          store="f32", rule="capped", cfl=0.45, velocity=(0.9, 0.9), length=2.0, t_end=0.5,
                          init="transport", periodic=(False, False)),
    # Shallow water, Godunov flux with exact Riemann solver (the paper's
    # Sec. 3.2.4 cost study): 128 cells (129 nodes) per axis on [0, 1]^2,
    # outflow, h = 2 on the central 0.5 x 0.5 square and 1 elsewhere, at rest,
    # g = 9.81, 38245 steps of dt = 10 s / 38245, 4 levels, c = 5e-4.
    "swe_129": dict(scheme="swe", wavelet="bl53", n=128, P=64, L=4, eps=5e-4, prec="f32", store="f32",
                    rule="capped", gravity=9.81, dt=10.0 / 38245, steps=38245, length=1.0, init="swe_square",
                    periodic=(False, False)),
}


def gaussian_bump(n, amp=0.1, sigma=8.0, center=None):
    """rho = 1 + amp*exp(-r^2/(2 sigma^2)) around the centre node, u = 0."""
    c = (n / 2.0, n / 2.0) if center is None else center
    j, i = np.meshgrid(np.arange(n, dtype=np.float64), np.arange(n, dtype=np.float64), indexing="ij")
    r2 = (i - c[0]) ** 2 + (j - c[1]) ** 2
    rho = 1.0 + amp * np.exp(-r2 / (2.0 * sigma * sigma))
    return [rho, np.zeros_like(rho), np.zeros_like(rho)]


def shear_wave(n, u0=0.05, noise=1e-4, seed=0):
    """rho = 1, u_x = u0 sin(2 pi y / n) + N(0, noise) per node, u_y = 0."""
    y = np.arange(n, dtype=np.float64)[:, None]
    ux = u0 * np.sin(2.0 * np.pi * y / n) * np.ones((1, n))
    if noise > 0:
        ux = ux + np.random.default_rng(seed).normal(0.0, noise, size=(n, n))
    return [np.ones((n, n)), ux, np.zeros((n, n))]


# Four-quadrant Riemann data (rho, u, v, p), quadrants split at x = y = 1/2.
QUADRANTS = {
    "NE": (1.5, 0.0, 0.0, 1.5),
    "NW": (0.5323, 1.206, 0.0, 0.3),
    "SW": (0.138, 1.206, 1.206, 0.029),
    "SE": (0.5323, 0.0, 1.206, 0.3),
}


def transport_gaussian(n, t=0.0, velocity=(0.9, 0.9), lo=-1.0, hi=1.0):
    """f(x, y) = 1 + exp(-30 ((x - a t)^2 + (y - b t)^2)) on the n + 1 nodes
    per axis of [lo, hi]^2: the initial state (t = 0) of the transport
    workload, and its exact solution at time t."""
    x = lo + (hi - lo) * np.arange(n + 1, dtype=np.float64) / n
    X, Y = np.meshgrid(x - velocity[0] * t, x - velocity[1] * t, indexing="xy")
    return [1.0 + np.exp(-30.0 * (X * X + Y * Y))]


def swe_square(n, h_in=2.0, h_out=1.0, half=0.25):
    """Water at rest, h = h_in on the nodes with |x - 1/2| <= half and
    |y - 1/2| <= half, h_out elsewhere; n + 1 nodes per axis on [0, 1]^2.
    Returns (h, u, v)."""
    x = np.arange(n + 1, dtype=np.float64) / n
    X, Y = np.meshgrid(x, x, indexing="xy")
    h = np.where((np.abs(X - 0.5) <= half) & (np.abs(Y - 0.5) <= half), h_in, h_out)
    return [h, np.zeros_like(h), np.zeros_like(h)]


def four_quadrant(n):
    """Nodes x_k = k/n, k = 0..n on [0,1]^2; a node with x >= 1/2 is east."""
    x = np.arange(n + 1, dtype=np.float64) / n
    X, Y = np.meshgrid(x, x, indexing="xy")
    out = [np.zeros_like(X) for _ in range(4)]
    for name, st in QUADRANTS.items():
        east = X >= 0.5 if name in ("NE", "SE") else X < 0.5
        north = Y >= 0.5 if name in ("NE", "NW") else Y < 0.5
        m = east & north
        for q in range(4):
            out[q][m] = st[q]
    return out


def sod_x(n, periodic=False):
    """1-D Sod tube along x, replicated along y (n+1 nodes for outflow)."""
    m = n if periodic else n + 1
    x = np.arange(m, dtype=np.float64) / n
    left = x < 0.5
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    ones = np.ones((m, 1))
    return [ones * rho, np.zeros((m, m)), np.zeros((m, m)), ones * p]


def batch_specs(count=96, seed=0, sides=(256, 512, 1024, 2048)):
    """Independent D2Q9 runs: side, bump amplitude, width and centre."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        side = int(rng.choice(sides))
        out.append(dict(side=side, amp=float(rng.uniform(0.01, 0.1)), sigma=float(rng.uniform(4.0, 32.0)),
                        cx=float(rng.uniform(0, side)), cy=float(rng.uniform(0, side))))
    return out


def initial_fields(w, n=None, seed=0):
    """Initial macroscopic fields of a workload dict (optionally resized)."""
    n = w["n"] if n is None else n
    if w["init"] == "bump":
        return gaussian_bump(n)
    if w["init"] == "shear":
        return shear_wave(n, seed=seed)
    if w["init"] == "quadrants":
        return four_quadrant(n)
    if w["init"] == "transport":
        return transport_gaussian(n, velocity=w.get("velocity", (0.9, 0.9)))
    if w["init"] == "swe_square":
        return swe_square(n)
    raise ValueError(w["init"])


def taylor_green_3d(n, u0=0.04, rho0=1.0):
    """Decaying Taylor-Green vortex on an n^3 periodic node grid (k = 2 pi/n):
    u = u0 (sin kx cos ky cos kz, -cos kx sin ky cos kz, 0), pressure
    rho0 u0^2/16 (cos 2kx + cos 2ky)(cos 2kz + 2), rho = rho0 + 3 p (lattice
    c_s^2 = 1/3).  Arrays (z, y, x)."""
    k = 2.0 * np.pi / n
    i = np.arange(n, dtype=np.float64) * k
    Z, Y, X = np.meshgrid(i, i, i, indexing="ij")
    ux = u0 * np.sin(X) * np.cos(Y) * np.cos(Z)
    uy = -u0 * np.cos(X) * np.sin(Y) * np.cos(Z)
    uz = np.zeros_like(ux)
    p = rho0 * u0 * u0 / 16.0 * (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0)
    return [rho0 + 3.0 * p, ux, uy, uz]


def taylor_green_3d_device(n, u0=0.04, rho0=1.0, device="cuda"):
    """taylor_green_3d generated directly in device memory (float64 torch
    tensors), for grids too large to build on the host."""
    import torch
    k = 2.0 * np.pi / n
    i = torch.arange(n, dtype=torch.float64, device=device) * k
    s, c, c2 = torch.sin(i), torch.cos(i), torch.cos(2 * i)
    ux = u0 * s[None, None, :] * c[None, :, None] * c[:, None, None]
    uy = -u0 * c[None, None, :] * s[None, :, None] * c[:, None, None]
    p = rho0 * u0 * u0 / 16.0 * (c2[None, None, :] + c2[None, :, None]) * (c2[:, None, None] + 2.0)
    return [(rho0 + 3.0 * p).contiguous(), ux.contiguous(), uy.contiguous(), torch.zeros_like(ux)]


def shear_wave_3d(nx, ny, nz, u0=0.01, axis=1, noise=0.0, seed=0):
    """rho = 1, u_x = u0 sin(2 pi s / n_s) with s the coordinate along
    `axis` (1 = y, 2 = z), plus N(0, noise) per node; arrays (z, y, x)."""
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    s, n = (Y, ny) if axis == 1 else (Z, nz)
    ux = u0 * np.sin(2 * np.pi * s / n)
    if noise:
        ux = ux + np.random.default_rng(seed).normal(0.0, noise, ux.shape)
    z = np.zeros(ux.shape)
    return [np.ones(ux.shape), ux.astype(np.float64), z, z.copy()]


def gaussian_bump_device(n, amp, sigma, cx, cy, device="cuda"):
    """gaussian_bump with an arbitrary centre, generated directly in device
    memory (float64 torch tensors) for large batches."""
    import torch
    i = torch.arange(n, dtype=torch.float64, device=device)
    r2 = (i[None, :] - cx) ** 2 + (i[:, None] - cy) ** 2
    rho = 1.0 + amp * torch.exp(-r2 / (2.0 * sigma * sigma))
    z = torch.zeros_like(rho)
    return [rho, z, z.clone()]
