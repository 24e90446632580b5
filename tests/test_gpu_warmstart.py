"""Learned warm start on a small transportation family (10 supplies x 15 demands):
the network trained on solver-generated solutions must lower the mean iteration count
to 1e-4 on held-out LPs, every held-out LP must still be solved, and warm-started
objectives must agree with cold-started ones within the tolerance asked for."""
import numpy as np
import pytest

import lpgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ws():
    from paper_2312_14832_b300 import build
    build.build()
    from paper_2312_14832_b300 import warmstart
    return warmstart


def test_warm_start_reduces_iterations(ws):
    fam = lpgen.transport_family(10, 15, seed=0)
    train = [lpgen.transport_instance(fam, s) for s in range(1, 3001)]
    P = np.array([lp["features"] for lp in train])
    X, Y, W, its, st, _ = ws.solve_family(train, tol=1e-6)
    assert np.all(st == 0)
    model = ws.WarmStart(P.shape[1], train[0]["n"], train[0]["m"], hidden=256, max_batch=256, seed=0)
    fit = model.fit(P, X, Y, W, epochs=40, batch=256, lr=1e-3)
    assert fit["losses"][-1] < 0.5 * fit["losses"][0]
    held = [lpgen.transport_instance(fam, s) for s in range(100001, 100201)]
    Ph = np.array([lp["features"] for lp in held])
    ev = ws.evaluate(model, held, Ph, tols=(1e-4,))
    r = ev["1e-04"]
    assert r["cold_optimal"] == r["warm_optimal"] == len(held)
    assert r["warm_iters_mean"] < r["cold_iters_mean"]
    model.close()
