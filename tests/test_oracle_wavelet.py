"""Pins of the oracle's wavelet, threshold and codec against what the paper
and mathematics fix (no GPU)."""
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_matrices():
    rows, mats = [], []
    for line in open(os.path.join(GOLDEN, "bl53_A_j3.txt")):
        line = line.strip()
        if line.startswith("#"):
            if rows:
                mats.append(np.array(rows, float))
                rows = []
            continue
        if line:
            rows.append([float(v) for v in line.split()])
    mats.append(np.array(rows, float))
    return [m for m in mats if m.size]


def test_bl53_matrix_A_matches_paper():
    # Sec. 2.1.2: the printed A for j = 3 (v = A u, v interleaves s and d).
    A8, _ = _read_matrices()
    A = np.array([O.dwt(np.eye(9)[i], "bl53", 8, 1) for i in range(9)]).T
    assert np.array_equal(A * 8, A8)


def test_bl53_matrix_Ainv_matches_paper():
    _, Ainv8 = _read_matrices()
    Ainv = np.array([O.dwt(np.eye(9)[i], "bl53", 8, 1, inverse=True) for i in range(9)]).T
    assert np.array_equal(Ainv * 8, Ainv8)
    A8, _ = _read_matrices()
    assert np.allclose((A8 / 8) @ (Ainv8 / 8), np.eye(9), atol=0)


@pytest.mark.parametrize("P,L", [(8, 3), (64, 4), (128, 6)])
def test_bl53_linear_functions_have_no_details(P, L):
    # Sec. 2.1: the BL5/3 wavelet filters out linear polynomials (1-D and the
    # bilinear tensor case).
    x = np.arange(P + 1) / P
    c1 = O.dwt(3.0 - 2.5 * x, "bl53", P, L)
    coarse = np.arange(P + 1) % (1 << L) == 0
    assert np.abs(c1[~coarse]).max() < 1e-14
    X, Y = np.meshgrid(x, x)
    c2 = O.dwt(1.0 + 2 * X - 3 * Y + 0.5 * X * Y, "bl53", P, L)
    m = np.outer(coarse, coarse)
    assert np.abs(c2[~m]).max() < 1e-14


@pytest.mark.parametrize("j", range(2, 8))
def test_bl53_trapezoid_conservation_one_level(j):
    # eq. conservation: trapezoid sum at j-1 equals half the one at j.  It
    # needs an interior sample at j-1 (j >= 2), hence P/2^L >= 2.
    rng = np.random.default_rng(j)
    n = 1 << j
    u = rng.normal(size=n + 1)
    v = O.dwt(u, "bl53", n, 1)
    s = v[0::2]
    tr = lambda a: 0.5 * (a[0] + a[-1]) + a[1:-1].sum()
    assert abs(tr(s) - 0.5 * tr(u)) <= 1e-15 * (1 + abs(tr(u))) * 4


def test_bl53_trapezoid_conservation_levels_2d():
    rng = np.random.default_rng(7)
    P, L = 64, 4
    u = rng.normal(size=(P + 1, P + 1))
    c = O.dwt(u, "bl53", P, L)
    w = np.ones(P + 1)
    w[0] = w[-1] = 0.5
    mass = w @ u @ w
    cs = c[:: 1 << L, :: 1 << L]
    wc = np.ones(cs.shape[0])
    wc[0] = wc[-1] = 0.5
    assert abs(wc @ cs @ wc * 4.0 ** L - mass) < 1e-12


def test_mass_kept_when_all_details_nullified():
    # Sec. 2.1.2 example text: masses equal "even when all the details are
    # nullified"; corollary of Sec. 3.1.1.
    rng = np.random.default_rng(3)
    P, L = 32, 3
    u = rng.normal(size=(P + 1, P + 1)) + 2.0
    c = O.dwt(u, "bl53", P, L)
    rec = O.encode(c[None], "bl53", P, L, eps=1e300)
    d = O.decode(rec, 1, (P + 1, P + 1), "bl53", P, L)[0]
    back = O.dwt(d, "bl53", P, L, inverse=True)
    w = np.ones(P + 1)
    w[0] = w[-1] = 0.5
    assert abs(w @ back @ w - w @ u @ w) <= 1e-13 * abs(w @ u @ w)
    assert not np.allclose(back, u)  # details really were removed


def test_e2_nonnull_count_is_481():
    # Sec. 2.1.2: 481 non-null coefficients out of 16641; fixes the tensor
    # (rows then columns) decomposition and the hard threshold.
    meta = dict(l.split() for l in open(os.path.join(GOLDEN, "e2_nonnull.txt")) if l[0] != "#")
    L, tau = int(meta["levels"]), float(meta["threshold"])
    x = np.arange(129) / 129.0
    X, Y = np.meshgrid(x, x)
    f = np.exp(X - Y) * np.sin(2 * np.pi * (X + Y)) * np.where(Y - X ** 2 >= 0, 1.0, 2.0)
    c = O.dwt(f, "bl53", 128, L).reshape(-1)
    lay = O.layout("bl53", 2, 128, L)
    co = lay["coarse"]
    count = np.count_nonzero(c[co]) + np.count_nonzero(np.abs(c[~co]) >= tau)
    assert lay["n_all"] == int(meta["total"])
    assert count == int(meta["nonnull"])
    # the same count through the codec
    rec = O.encode(O.dwt(f, "bl53", 128, L)[None], "bl53", 128, L, eps=tau)
    nedge = int.from_bytes(rec[16 + 8:16 + 12], "little")
    nint = int.from_bytes(rec[16 + 12:16 + 16], "little")
    assert np.count_nonzero(c[co]) + nedge + nint == int(meta["nonnull"])


def test_haar_closed_forms():
    # Haar (not in the paper): coarse = 2^L-cell block mean, level-1 detail =
    # b - a; details of constants vanish.
    rng = np.random.default_rng(1)
    P, L = 16, 3
    u = rng.normal(size=P)
    c = O.dwt(u, "haar", P, L)
    assert np.allclose(c[:: 1 << L], u.reshape(-1, 1 << L).mean(1), atol=1e-15)
    u1 = O.dwt(u, "haar", P, 1)
    assert np.allclose(u1[1::2], u[1::2] - u[0::2], atol=1e-15)
    k = O.dwt(np.full(P, 3.25), "haar", P, L)
    assert np.abs(k[np.arange(P) % (1 << L) != 0]).max() == 0.0


@pytest.mark.parametrize("wavelet,P,L", [("haar", 8, 3), ("bl53", 8, 3), ("bl53", 16, 2)])
def test_tensor_equals_kronecker_bruteforce(wavelet, P, L):
    # The N-D transform is the Kronecker product of the 1-D operator (rows
    # then columns, Sec. 2.1.2), checked against the dense matrix on small
    # patches.
    E = P + 1 if wavelet == "bl53" else P
    A1 = np.array([O.dwt(np.eye(E)[i], wavelet, P, L) for i in range(E)]).T
    rng = np.random.default_rng(5)
    u = rng.normal(size=(E, E))
    c = O.dwt(u, wavelet, P, L)
    assert np.allclose(c, A1 @ u @ A1.T, atol=1e-13)
    back = O.dwt(c, wavelet, P, L, inverse=True)
    assert np.allclose(back, u, atol=1e-13)


def test_layout_band_sizes_and_edges():
    for wavelet, P, L in [("bl53", 64, 4), ("haar", 32, 3), ("bl53", 32, 3)]:
        lay = O.layout(wavelet, 2, P, L)
        E = P + 1 if wavelet == "bl53" else P
        n0 = (P >> L) + (1 if wavelet == "bl53" else 0)
        assert lay["n_c"] == n0 * n0 == lay["coarse"].sum()
        assert lay["nb"] == (L + 1) ** 2
        size = lambda c: n0 if c == 0 else P >> c
        counts = np.bincount(lay["band"], minlength=lay["nb"])
        for b in range(lay["nb"]):
            cx, cy = divmod(b, L + 1)
            assert counts[b] == size(cx) * size(cy)
        ky, kx = np.divmod(np.arange(E * E), E)
        expect = (wavelet == "bl53") & ((kx == 0) | (kx == P) | (ky == 0) | (ky == P))
        assert np.array_equal(lay["edge"], expect)
        assert np.array_equal(lay["coarse"], (kx % (1 << L) == 0) & (ky % (1 << L) == 0))


def _bruteforce_survivors(c, wavelet, P, L, eps, rule="const"):
    lay = O.layout(wavelet, 2, P, L)
    flat = c.reshape(-1)
    taus = np.array([eps * O.band_factor(wavelet, 2, P, L, b, rule) for b in range(lay["nb"])])
    keep = np.abs(flat) >= taus[lay["band"]]
    keep[lay["coarse"]] = True
    return lay, flat, keep


@pytest.mark.parametrize("rule", ["const", "accum", "capped"])
def test_threshold_mask_bruteforce(rule):
    # Hard threshold on details only (Sec. 2.2); strict "< tau" is zeroed.
    rng = np.random.default_rng(11)
    P, L = 32, 3
    c = rng.normal(scale=1e-3, size=(P + 1, P + 1))
    eps = 1e-3
    rec = O.encode(c[None], "bl53", P, L, eps, rule=rule)
    d = O.decode(rec, 1, (P + 1, P + 1), "bl53", P, L)[0]
    lay, flat, keep = _bruteforce_survivors(c, "bl53", P, L, eps, rule)
    got = d.reshape(-1)
    assert np.array_equal(got[keep], flat[keep])  # F64 storage is exact
    assert np.all(got[~keep] == 0)


def test_eps_zero_keeps_everything():
    rng = np.random.default_rng(12)
    P, L = 16, 2
    c = rng.normal(size=(3, P + 1, P + 1))
    c[0, 3, 5] = 0.0
    rec = O.encode(c, "bl53", P, L, 0.0)
    d = O.decode(rec, 3, (P + 1, P + 1), "bl53", P, L)
    assert np.array_equal(d, c)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=10000).astype(np.float32),
                        # exact ties: low half 0x8000 with even / odd kept bit
                        np.array([0x3F808000, 0x3F818000, 0xBF808000, 0x00008000], np.uint32).view(np.float32),
                        np.array([0.0, -0.0, 1e-40, 3.4e38], np.float32)])
    ours = O.bf16_bits(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(ours, ref)


def test_quantised_storage_roundtrip():
    # BF16 with a power-of-two band scale equals plain BF16 rounding; int8 is
    # rint(d/s) with s = max|d|/127 (float32).
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    P, L = 16, 2
    c = rng.normal(scale=1e-2, size=(1, P + 1, P + 1)).astype(np.float32).astype(np.float64)
    lay = O.layout("bl53", 2, P, L)
    rec = O.encode(c, "bl53", P, L, 0.0, prec="f32", store="bf16")
    d = O.decode(rec, 1, (P + 1, P + 1), "bl53", P, L, prec="f32", store="bf16")[0].reshape(-1)
    flat = c[0].reshape(-1)
    interior = ~lay["edge"] & ~lay["coarse"]
    want = torch.from_numpy(flat[interior].astype(np.float32)).to(torch.bfloat16).float().numpy()
    assert np.array_equal(d[interior].astype(np.float32), want)
    assert np.array_equal(d[lay["edge"]], flat[lay["edge"]])  # edge lines kept in FP32
    # int8 at a threshold that half an int8 step stays below in every band
    eps = 1e-3
    rec8 = O.encode(c, "bl53", P, L, eps, prec="f32", store="i8")
    d8 = O.decode(rec8, 1, (P + 1, P + 1), "bl53", P, L, prec="f32", store="i8")[0].reshape(-1)
    for b in np.unique(lay["band"][interior]):
        m = interior & (lay["band"] == b) & (np.abs(flat) >= eps)
        v = flat[m].astype(np.float32)
        s = np.float32(np.abs(v).max()) / np.float32(127)
        assert np.float32(0.5) * s <= np.float32(eps)
        q = np.clip(np.rint(v / s), -127, 127).astype(np.float32)
        assert np.array_equal(d8[m].astype(np.float32), q * s)


def test_accumulation_and_capped_factor_reading():
    # Reading of Sec. 2.2 (parity unpinned): finest band gets c, coarser
    # details smaller thresholds; accumulation sums levels, capped takes max.
    P, L = 64, 4
    lay = O.layout("bl53", 2, P, L)
    nb = lay["nb"]
    cls = [(b // (L + 1), b % (L + 1)) for b in range(nb)]
    for b, (cx, cy) in enumerate(cls):
        if b == 0:
            continue
        mx = cx if cx else L
        my = cy if cy else L
        assert O.band_factor("bl53", 2, P, L, b, "const") == 1.0
        assert O.band_factor("bl53", 2, P, L, b, "accum") == 2.0 ** -((mx - 1) + (my - 1))
        assert O.band_factor("bl53", 2, P, L, b, "capped") == 2.0 ** -(max(mx, my) - 1)


def _bandmask(rec, P, L, field=0):
    off = int(np.frombuffer(rec, np.uint32, 1, 16 + 16 * field)[0])
    nc = ((P >> L) + 1) ** 2
    return int(np.frombuffer(rec, np.uint64, 1, off + 4 * nc)[0])


@pytest.mark.parametrize("eps", [1e-4, 1e-3, 1e-2])
def test_int8_kept_details_err_at_most_their_threshold(eps):
    # The threshold of Sec. 2.2 is the method's error control (a dropped
    # detail errs by less than tau).  Int8 storage errs by up to half a step,
    # max|d|/254 per band, whatever tau is; so int8 may hold a field only if
    # that stays within every band's threshold, else the field's interior
    # survivors are BF16 (relative error <= 2^-8).  Bands with one large
    # outlier (a shock) and many small details force the BF16 form.
    rng = np.random.default_rng(11)
    P, L = 32, 3
    lay = O.layout("bl53", 2, P, L)
    interior = ~lay["edge"] & ~lay["coarse"]
    for outlier in (0.0, 0.05, 1.0):
        c = (rng.normal(scale=3e-3, size=(1, P + 1, P + 1))).astype(np.float32).astype(np.float64)
        flat = c[0].reshape(-1)
        k = np.flatnonzero(interior & (lay["band"] == lay["band"][interior][0]))[3]
        flat[k] = outlier if outlier else flat[k]
        c[0] = flat.reshape(P + 1, P + 1)
        for rule in ("const", "accum", "capped"):
            rec = O.encode(c, "bl53", P, L, eps, prec="f32", store="i8", rule=rule)
            d = O.decode(rec, 1, (P + 1, P + 1), "bl53", P, L, prec="f32", store="i8")[0].reshape(-1)
            wide = _bandmask(rec, P, L) & 1
            tau = np.array([np.float32(eps * O.band_factor("bl53", 2, P, L, b, rule)) for b in range(lay["nb"])])
            kept = interior & (np.abs(flat) >= tau[lay["band"]]) & (d != 0)
            err = np.abs(d - flat)
            if wide:
                # BF16 of each value (power-of-two band scales are exact)
                assert np.all(err[kept] <= np.abs(flat[kept]) * 2.0 ** -8)
                # and int8 would have broken the bound in some band
                over = False
                for b in np.unique(lay["band"][kept]):
                    m = kept & (lay["band"] == b)
                    over |= 0.5 * np.float32(np.abs(flat[m]).max().astype(np.float32) / np.float32(127)) > tau[b]
                assert over
            else:
                assert np.all(err[kept] <= tau[lay["band"][kept]])
            if outlier == 1.0 and eps <= 1e-3:
                assert wide  # 1/254 is above every threshold here


def test_int8_four_quadrant_run_stays_finite():
    # Regression of a measured failure: with an int8 step tied only to the
    # band maximum, the FP32 int8 run of the four-quadrant Riemann problem
    # (512^2, P 64, L 4, eps 1e-4, dt/h 0.15) lost positivity near the
    # low-pressure quadrant and went non-finite at step ~425.
    from paper_2302_09883_gb300 import inputs
    n = 512
    o = O.OracleSim("euler2d", "bl53", n, n, 64, 4, 1e-4, prec="f32", store="i8", periodic=(False, False),
                    cfl=-0.15, gamma=1.4)
    o.init_macro(inputs.four_quadrant(n))
    o.step(450)
    W = o.export_all()
    assert np.isfinite(W).all()
    rho = W[0]
    p = 0.4 * (W[3] - 0.5 * (W[1] ** 2 + W[2] ** 2) / rho)
    assert rho.min() > 0.1 and p.min() > 0.0
