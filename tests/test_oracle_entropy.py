"""Pins of the oracle's entropy stage (order-0 byte-wise rANS, entropy.hpp):
exact round trips, the coded length against the cross-entropy of the data
under the normalised table (a property of arithmetic/ANS coding that holds
whatever the implementation), frequency normalisation, and the coded state
of a run."""
import numpy as np
import pytest

import oracle as O
from paper_2302_09883_gb300 import inputs


@pytest.mark.parametrize("kind", ["uniform", "skewed", "constant", "two", "text"])
def test_rans_roundtrip_and_entropy_bound(kind):
    rng = np.random.default_rng(7)
    n = 20000
    if kind == "uniform":
        d = rng.integers(0, 256, n, dtype=np.uint8)
    elif kind == "skewed":
        d = np.minimum(rng.geometric(0.3, n), 255).astype(np.uint8)
    elif kind == "constant":
        d = np.full(n, 17, np.uint8)
    elif kind == "two":
        d = rng.choice(np.array([0, 255], np.uint8), n, p=[0.9, 0.1])
    else:
        d = np.frombuffer(b"the wavelet coefficients of a patch " * 600, np.uint8)[:n]
    data = d.tobytes()
    coded, back = O.rans_roundtrip(data)
    assert back == data
    cnt = np.bincount(d, minlength=256)
    f = O.rans_freqs(cnt)
    assert f.sum() == 4096 and np.all(f[cnt > 0] >= 1) and np.all(f[cnt == 0] == 0)
    # ANS codes within a few bytes of the cross-entropy of the data under
    # the table (sum of log2(M / f_s) bits) plus the 4-byte final state
    bits = float(np.sum(cnt[cnt > 0] * np.log2(4096.0 / f[cnt > 0])))
    assert len(coded) <= bits / 8 + 4 + 8
    assert len(coded) >= bits / 8 - 8


def test_rans_frequencies_track_the_counts():
    cnt = np.zeros(256, np.uint64)
    cnt[[3, 9, 200]] = [1000, 3000, 1]
    f = O.rans_freqs(cnt)
    assert f[200] == 1 and f.sum() == 4096
    assert abs(f[3] / 4096 - 0.25) < 0.01 and abs(f[9] / 4096 - 0.75) < 0.01


def test_entropy_coded_state_of_a_run_decodes_to_its_records():
    n = 256
    o = O.OracleSim("d2q9", "bl53", n, n, 64, 4, 1e-5, prec="f32", store="bf16", tau=0.6)
    o.init_macro(inputs.shear_wave(n, seed=3))
    o.step(3)
    code = o.entropy_code()
    npatch = int(np.frombuffer(code, np.uint32, 1, 0)[0])
    assert npatch == o.npatch and int(np.frombuffer(code, np.uint32, 1, 4)[0]) == 12
    f = np.frombuffer(code, np.uint16, 256, 8).astype(np.uint32)
    assert f.sum() == 4096
    sizes = np.frombuffer(code, np.uint32, 2 * npatch, 8 + 512).reshape(npatch, 2)
    p = 8 + 512 + 8 * npatch
    recs = b""
    for k in range(npatch):
        rec = o.record(k)
        assert sizes[k, 0] == len(rec)
        recs += rec
        p += int(sizes[k, 1])
    assert p == len(code)
    # the whole state is smaller coded than as records
    assert len(code) < len(recs)
