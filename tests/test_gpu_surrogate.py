"""GPU parity of the learned surrogate's kernels against the FP64 oracle.

Tolerances (BF16 operands, FP32 accumulation):
* forward: the inputs and the three hidden activations are rounded to BF16
  (relative RMS ~1e-3 each), so the output agrees with the FP64 network to a
  norm-wise relative 1e-2.  Replaying the same four roundings in the oracle's
  arithmetic leaves the FP32 accumulation (2e-5 of max |y|) plus the rare
  activation that lies on a BF16 rounding boundary and rounds the other way:
  one BF16 step there moves all outputs of that point (by at most ~1e-3 of
  max |y|).  With ~1e-7 accumulation differences against 4e-3 steps, a few of
  the 230k activations flip, so >= 95% of the points match to 2e-5.
* gradients: dY and the backpropagated dZ are rounded to BF16 as well; per
  layer the gradient agrees norm-wise to 3e-2 with cosine similarity >= 0.999.
* Adam: the first step from zero moments is -lr g / (|g| + eps) in FP32 for
  the GPU's own gradient g, to 1e-6 lr.
"""

import numpy as np
import pytest

import workloads
from oracle.mlp_oracle import MLPOracle, gelu
from workloads.mlp import BOX_CENTRE, BOX_HALF, init_weights, round_to_bf16

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def srw():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2607_00488_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def solar_lk(srw):
    wl = workloads.solar_set_workload()
    lk = srw.Likelihood(wl, workloads.load_counts(wl["name"]))
    yield lk
    lk.close()


def bf16_params(n_out, seed=5):
    return [(round_to_bf16(W), round_to_bf16(b)) for W, b in init_weights(n_out, seed=seed)]


def emulated_forward(params, theta):
    """The oracle's network with the GPU's four BF16 roundings replayed."""
    net = MLPOracle(params, BOX_CENTRE, BOX_HALF)
    a = round_to_bf16(net.inputs(theta).astype(np.float32)).astype(np.float64)
    for k, (W, b) in enumerate(net.params):
        z = a @ W.T + b
        a = round_to_bf16(gelu(z).astype(np.float32)).astype(np.float64) if k < 3 else z
    return a


@pytest.fixture(scope="module")
def sur(srw, solar_lk):
    params = bf16_params(2048)
    s = srw.Surrogate(solar_lk, params, BOX_CENTRE, BOX_HALF)
    yield s, params
    s.close()


def test_forward_matches_oracle(sur):
    s, params = sur
    theta = workloads.theta_box(300, 41)  # 300 points: two full row tiles and a ragged one
    got = s.forward(theta).astype(np.float64)
    want, _ = MLPOracle(params, BOX_CENTRE, BOX_HALF).forward(theta)
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert rel <= 1e-2, rel
    emu = emulated_forward(params, theta)
    d = (np.abs(got - emu) / np.max(np.abs(emu))).max(axis=1)  # per point
    assert np.mean(d <= 2e-5) >= 0.95, np.sort(d)[-20:]
    assert d.max() <= 2e-3, d.max()


def test_weights_round_trip(sur):
    s, params = sur
    back = s.weights()
    for (W, b), (W2, b2) in zip(params, back):
        assert np.array_equal(W, W2) and np.array_equal(b, b2)


def test_gradients_match_oracle(sur):
    s, params = sur
    rng = np.random.default_rng(42)
    theta = workloads.theta_box(200, 43)
    targets = rng.normal(size=(200, 2048)).astype(np.float32)
    loss, grads = s.gradients(theta, targets)
    net = MLPOracle(params, BOX_CENTRE, BOX_HALF)
    want_loss, want = net.gradients(theta, targets)
    assert loss == pytest.approx(want_loss, rel=1e-2)
    for k, ((gW, gb), (wW, wb)) in enumerate(zip(grads, want)):
        for g, w in ((gW, wW), (gb, wb)):
            g = g.astype(np.float64).ravel()
            w = w.ravel()
            rel = np.linalg.norm(g - w) / np.linalg.norm(w)
            cos = g @ w / (np.linalg.norm(g) * np.linalg.norm(w))
            assert rel <= 3e-2 and cos >= 0.999, (k, rel, cos)


def test_adam_first_step(sur):
    s, params = sur
    rng = np.random.default_rng(44)
    theta = workloads.theta_box(128, 45)
    targets = rng.normal(size=(128, 2048)).astype(np.float32)
    s.set_weights(params)  # fresh Adam moments
    _, g = s.gradients(theta, targets)
    lr = 1e-3
    s.train_step(theta, targets, lr)
    new = s.weights()
    for (W0, b0), (gW, gb), (W1, b1) in zip(params, g, new):
        for w0, gg, w1 in ((W0, gW, W1), (b0, gb, b1)):
            want = w0.astype(np.float64) - lr * gg / (np.abs(gg.astype(np.float64)) + 1e-8)
            assert np.max(np.abs(w1 - want)) <= 1e-6 * lr + 1e-7 * np.max(np.abs(w0)), np.max(np.abs(w1 - want))
    s.set_weights(params)


def test_training_reduces_the_loss(sur):
    # a learnable target: another network of the same shape (a teacher)
    s, params = sur
    teacher = MLPOracle(init_weights(2048, seed=9), BOX_CENTRE, BOX_HALF)
    theta = workloads.theta_box(1024, 46)
    targets, _ = teacher.forward(theta)
    targets = (targets / targets.std()).astype(np.float32)
    s.set_weights(params)
    first = s.train_step(theta, targets, 1e-3)
    for _ in range(60):
        last = s.train_step(theta, targets, 1e-3)
    assert last < 0.5 * first, (first, last)
    s.set_weights(params)
