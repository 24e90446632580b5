"""The warm-start network on the GPU (tcgen05 GEMMs, BF16 operands, FP32 accumulation)
against the CPU oracle of the same network (oracle/mlp.py, float64 with BF16 rounding at
the same points).  Tolerances: forward outputs and every gradient tensor within 2e-3 in
relative Frobenius norm (FP32 accumulation order; rare 1-ulp BF16 rounding differences
of hidden activations), loss within 1e-4 relative."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pk():
    from paper_2312_14832_b300 import build
    build.build()
    import paper_2312_14832_b300 as pk
    return pk


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - np.asarray(b, np.float64)) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("n_in,hidden,n_out,rows", [(100, 256, 300, 200), (37, 128, 129, 128), (5, 384, 1, 3)])
def test_mlp_forward_and_gradients_match_oracle(pk, n_in, hidden, n_out, rows):
    from oracle import mlp as omlp
    rng = np.random.default_rng(n_in + hidden + n_out)
    params = omlp.init_params(n_in, hidden, n_out, seed=3)
    X = rng.standard_normal((rows + 50, n_in)).astype(np.float32)
    T = rng.standard_normal((rows + 50, n_out)).astype(np.float32)
    idx = rng.permutation(rows + 50)[:rows].astype(np.int32)
    with pk.MLP(n_in, hidden, n_out, max_batch=max(rows, 1)) as net:
        net.set_params(params)
        back = net.get_params()
        for a, b in zip(back, params):
            np.testing.assert_array_equal(a, b)
        net.load_data(X, T)
        Y = net.forward(idx)
        loss, grads = net.gradients(idx)
    ref = omlp.forward(params, X[idx])
    assert rel(Y, ref["Y"]) <= 2e-3
    rloss, rgrads = omlp.loss_and_grads(params, X[idx], T[idx])
    assert abs(loss - rloss) <= 1e-4 * rloss
    for g, r in zip(grads, rgrads):
        assert rel(g, r) <= 2e-3


def test_mlp_training_reduces_loss(pk):
    from oracle import mlp as omlp
    rng = np.random.default_rng(0)
    n_in, hidden, n_out = 20, 256, 40
    A = rng.standard_normal((n_in, n_out)) / np.sqrt(n_in)
    X = rng.standard_normal((2048, n_in)).astype(np.float32)
    T = np.tanh(X @ A).astype(np.float32)
    with pk.MLP(n_in, hidden, n_out, max_batch=128) as net:
        net.set_params(omlp.init_params(n_in, hidden, n_out, seed=1))
        net.load_data(X, T)
        losses, ms = net.train(epochs=8, batch=128, lr=2e-3, weight_decay=0.0, seed=0)
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.25 * losses[0]
