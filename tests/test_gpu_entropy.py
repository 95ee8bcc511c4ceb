"""GPU: the library's entropy stage (order-0 rANS over the records) gives the
oracle's coded state byte for byte, decodes back on the device, and codes
the state into fewer bytes than the records."""
import numpy as np
import pytest

import oracle as O
from paper_2302_09883_gb300 import Sim, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("scheme,store,eps,periodic", [("d2q9", "bf16", 1e-6, (True, True)),
                                                        ("d2q9", "i8", 1e-5, (True, True)),
                                                        ("d2q9", "f32", 1e-3, (True, True)),
                                                        ("euler2d", "i8", 1e-3, (False, False)),
                                                        ("transport", "f32", 1e-2, (False, False))])
def test_entropy_coded_state_matches_oracle(scheme, store, eps, periodic):
    n = 256 if scheme != "transport" else 128
    if scheme == "d2q9":
        f, kw = inputs.shear_wave(n, seed=12), dict(tau=0.6)
    elif scheme == "euler2d":
        f, kw = inputs.four_quadrant(n), dict(cfl=0.4)
    else:
        f, kw = inputs.transport_gaussian(n), dict(cfl=0.45, velocity=(0.9, 0.9), length=2.0)
    g = Sim(scheme, "bl53", n, n, 64, 4, eps, prec="f32", store=store, periodic=periodic, **kw)
    o = O.OracleSim(scheme, "bl53", n, n, 64, 4, eps, prec="f32", store=store, periodic=periodic, **kw)
    g.init_macro(f)
    o.init_macro(f)
    g.step(5)
    o.step(5)
    code = g.entropy_code()
    assert code == o.entropy_code()
    # the coded streams (without the 520-byte table and the per-patch sizes)
    # are shorter than the records
    assert len(code) - (8 + 512 + 8 * g.npatch) < g.stats()["live_bytes"]
    g.close()
