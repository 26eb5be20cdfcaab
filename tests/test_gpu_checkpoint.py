"""Checkpoint and resume of the surrogate's training and of long scans.

* A fit interrupted after some epochs and resumed from its checkpoint (in a
  new surrogate object, starting from other weights) ends with exactly the
  weights, Adam state and standardization of the uninterrupted fit: the
  batches come in a fixed order and every kernel of a training step is
  deterministic.
* A checkpoint of another network, or a damaged one, is refused.
* A chunked scan stopped after some chunks and continued from its state file
  gives the result of the uninterrupted chunked scan, and its minimum is the
  exact minimum over all points, as the single-call scan's is.
"""

import os

import numpy as np
import pytest

import workloads
from workloads.mlp import BOX_CENTRE, BOX_HALF, init_weights

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
def be7_lk(srw):
    wl = workloads.be7_line_workload()
    lk = srw.Likelihood(wl, workloads.load_counts(wl["name"]))
    yield lk
    lk.close()


FIT = dict(batch=512, lr=2e-3, lr_final=2e-5)


def _state(sur, tmp_path, name):
    p = str(tmp_path / name)
    sur.save(p)
    return open(p, "rb").read()


def test_interrupted_fit_resumes_to_the_same_weights(srw, be7_lk, tmp_path):
    theta = workloads.theta_box(4096, 61)
    with srw.Surrogate(be7_lk, init_weights(128, seed=7), BOX_CENTRE, BOX_HALF) as a:
        la = a.fit(theta, epochs=4, **FIT)
        full = _state(a, tmp_path, "full.ckpt")
        wa = a.weights()
    ck = str(tmp_path / "run.ckpt")
    with srw.Surrogate(be7_lk, init_weights(128, seed=7), BOX_CENTRE, BOX_HALF) as b:
        lb1 = b.fit_resumable(theta, 4, ck, stop_after=2, **FIT)  # "interrupted" after epoch 2
    assert os.path.exists(ck)
    with srw.Surrogate(be7_lk, init_weights(128, seed=99), BOX_CENTRE, BOX_HALF) as c:  # other start weights
        lc = c.fit_resumable(theta, 4, ck, **FIT)
        assert c.load(ck) == 4
        wc = c.weights()
        resumed = _state(c, tmp_path, "resumed.ckpt")
    # the reported losses sum over warps with atomics (order varies); the weights do not
    np.testing.assert_allclose(np.concatenate([lb1, lc]), la, rtol=1e-9)
    for (W1, b1), (W2, b2) in zip(wa, wc):
        np.testing.assert_array_equal(W1, W2)
        np.testing.assert_array_equal(b1, b2)
    assert resumed == full  # Adam moments, step count and standardization included


def test_checkpoint_of_another_network_or_damaged_is_refused(srw, be7_lk, tmp_path):
    p = str(tmp_path / "a.ckpt")
    with srw.Surrogate(be7_lk, init_weights(128, seed=7), BOX_CENTRE, BOX_HALF) as a:
        a.save(p)
        raw = bytearray(open(p, "rb").read())
        raw[-5] ^= 0xFF
        bad = str(tmp_path / "bad.ckpt")
        open(bad, "wb").write(bytes(raw))
        with pytest.raises(srw.SrwError):
            a.load(bad)
        with pytest.raises(srw.SrwError):
            a.load(str(tmp_path / "missing.ckpt"))
        assert a.load(p) == 0
    with srw.Surrogate(be7_lk, init_weights(128, seed=7), BOX_CENTRE, BOX_HALF * 2) as other:
        with pytest.raises(srw.SrwError):
            other.load(p)


def test_interrupted_scan_resumes(srw, be7_lk, tmp_path):
    theta = workloads.theta_box(4096, 62)
    check = workloads.theta_box(2000, 63)
    with srw.Surrogate(be7_lk, init_weights(128, seed=7), BOX_CENTRE, BOX_HALF) as s:
        s.fit(theta, epochs=3, **FIT)
        opts = dict(keep_frac=0.02, check_theta=check, tol=0.05, cells_per_dim=2, rule=srw.SRW_SCAN_ERROR_BARS)
        n, chunk = 1 << 17, 1 << 15
        whole = s.scan(n, **opts)
        st1 = str(tmp_path / "scan_a.txt")
        ref, done = s.scan_chunked(n, st1, chunk, **opts)
        assert done
        st2 = str(tmp_path / "scan_b.txt")
        part, done = s.scan_chunked(n, st2, chunk, max_new_chunks=2, **opts)  # stopped after two chunks
        assert not done
        assert len(open(st2).read().splitlines()) == 3  # options line + two chunks
        res, done = s.scan_chunked(n, st2, chunk, **opts)
        assert done
        for k in ("best_value", "best_index", "n_kept", "n_selected", "surrogate_min"):
            assert res[k] == ref[k], k
        exact = s.scan_exact(n)  # the true minimum over all n points
        assert res["best_index"] == exact["best_index"] and res["best_value"] == exact["best_value"]
        assert whole["best_index"] == exact["best_index"] and whole["best_value"] == exact["best_value"]
        with pytest.raises(srw.SrwError):  # another scan's state file
            s.scan_chunked(n // 2, st2, chunk, **opts)
