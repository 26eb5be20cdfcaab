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


# ---------------------------------------------------------------- Sobol points
def test_sobol_points_match_oracle(sur):
    from oracle.sobol import sobol_points
    s, _ = sur
    got = s.sobol(1000, 4096)
    u = sobol_points(1000, 4096, 5)
    want = (BOX_CENTRE - BOX_HALF).astype(np.float64) + 2.0 * BOX_HALF.astype(np.float64) * u
    np.testing.assert_allclose(got, want, rtol=0, atol=4e-7)  # the FP32 map from [0, 1)


# ---------------------------------------------------------------- training on the exact path
@pytest.fixture(scope="module")
def trained(srw, solar_lk):
    params = init_weights(2048, seed=5)
    s = srw.Surrogate(solar_lk, params, BOX_CENTRE, BOX_HALF)
    theta = workloads.theta_box(1 << 20, 55)
    losses = s.fit(theta, epochs=40, batch=4096, lr=2e-3, lr_final=2e-5)
    yield s, losses
    s.close()


def test_fit_reduces_the_loss(trained):
    s, losses = trained
    print("epoch losses:", " ".join("%.2e" % x for x in losses))
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 1e-2 * losses[0], losses


def test_surrogate_likelihood_epilogue(trained, solar_lk):
    # The fused epilogue (exp, Poisson deviance, FP64 partial sums) against the
    # oracle's formula applied to the same network output.  The epilogue works
    # in FP32 on lm = log mu: rounding lm (|lm| <= ~10, 2^-24 relative) and the
    # fast exponential (at most 2 + 1.17 |lm| ulp) give mu a relative error
    # below 2e-6, and t = mu - n lm + (n ln n - n) adds FP32 roundings of its
    # three terms; per point |d| <= 2 sum_j [2e-6 |mu_j - n_j| + 1.2e-7
    # (mu_j + n_j |lm_j| + |n_j ln n_j - n_j|)] + 1e-3.
    from oracle.mlp_oracle import data_constant, surrogate_neg2lnl
    s, _ = trained
    counts = workloads.load_counts("solar_set_4096")
    theta = workloads.theta_box(257, 56)
    y = s.forward(theta).astype(np.float64)
    m, sd = s.standardization()
    want = surrogate_neg2lnl(y, m, sd, counts, data_constant(counts))
    got = s.loglik(theta)
    lm = m + sd * y
    mu = np.exp(lm)
    c = np.where(counts > 0, counts * np.log(np.where(counts > 0, counts, 1.0)) - counts, 0.0)
    bound = 2.0 * np.sum(2e-6 * np.abs(mu - counts) + 1.2e-7 * (mu + counts * np.abs(lm) + np.abs(c)), axis=1) + 1e-3
    assert np.all(np.abs(got - want) <= bound), np.max(np.abs(got - want) / bound)


def test_surrogate_against_exact_path(trained, solar_lk, srw):
    s, _ = trained
    theta = workloads.theta_box(2048, 57)
    exact = solar_lk.loglik(theta, srw.SRW_FP16X3)
    sur_v = s.loglik(theta)
    d = np.abs(sur_v - exact)
    rel = d / exact
    print("surrogate vs exact: median |d| %.3g, 90%% %.3g, median rel %.3g, max rel %.3g" % (
        np.median(d), np.quantile(d, 0.9), np.median(rel), rel.max()))
    assert np.all(np.isfinite(sur_v))
    assert np.median(rel) < 0.02


@pytest.mark.parametrize("rule", ["cells", "error_bars"])
def test_scan_finds_the_exact_minimum(trained, srw, rule):
    # The gain of the trained network: the pre-screened scan must return the
    # exact scan's minimum (same point, same exact value) while re-evaluating
    # fewer points.  The literal rule re-evaluates every flagged cell; the
    # error-bar rule re-evaluates only points that could still beat the best
    # exact value within twice their cell's held-out error.
    s, _ = trained
    n = 1 << 21
    ex = s.scan_exact(n)
    check = workloads.theta_box(10000, 58)
    code = srw.SRW_SCAN_FLAG_CELLS if rule == "cells" else srw.SRW_SCAN_ERROR_BARS
    s.scan(n, check_theta=check, rule=code)  # first call makes the buffers
    r = s.scan(n, keep_frac=0.01, check_theta=check, tol=0.05, cells_per_dim=4, rule=code, margin_factor=2.0)
    t_pre = r["ms_check"] + r["ms_surrogate"] + r["ms_select"] + r["ms_exact"]
    print("%s: exact scan %.2f ms; pre-screened %.2f ms (surrogate %.2f), re-evaluated %d of %d (%d flagged cells)"
          % (rule, ex["ms"], t_pre, r["ms_surrogate"], r["n_selected"], n, r["n_flagged_cells"]))
    assert r["n_selected"] >= r["n_kept"] >= 0.01 * n
    assert r["best_index"] == ex["best_index"] and r["best_value"] == ex["best_value"]
    if rule == "error_bars":
        assert r["n_selected"] < 0.1 * n
        assert t_pre < ex["ms"]
