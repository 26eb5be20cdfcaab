"""Host-array checks of the binding's create, data and surrogate calls.

The C calls read host arrays whose sizes they take from other arguments
(n_rec, the binning, the node counts, the handle), so the binding checks
every array's shape first and raises ValueError.  These tests run on the CPU
with a stand-in library: every workload the GPU tests and the benchmark use
passes the checks, and each kind of wrong array is refused before the
library is called.  A Likelihood whose data are refused releases its handle.
"""

import ctypes

import numpy as np
import pytest

import workloads
from workloads.mlp import BOX_CENTRE, BOX_HALF, init_weights
from paper_2607_00488_gb300 import srw as binding

HANDLE = 0x1000


class FakeLib:
    """Records the entry points called; returns SRW_OK and a non-null handle."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        if not name.startswith("srw_"):
            raise AttributeError(name)

        def call(*a):
            self.calls.append(name)
            if name in ("srw_create", "srw_create_joint", "srw_surrogate_create", "srw_group_create"):
                a[-1]._obj.value = HANDLE
            return binding.SRW_OK
        return call


@pytest.fixture
def fake(monkeypatch):
    f = FakeLib()
    monkeypatch.setattr(binding, "lib", lambda: f)
    return f


def _info(monkeypatch, wl):
    n_rec, n_t = (wl["hist"][0] if "hist" in wl else wl["R"]).shape
    monkeypatch.setattr(binding, "srw_info", lambda h: {"n_t": n_t, "n_rec": n_rec})
    return n_rec, n_t


@pytest.mark.parametrize("make", [workloads.be7_line_workload, workloads.solar_set_workload])
def test_workloads_pass(fake, monkeypatch, make):
    wl = make()
    n_rec, n_t = _info(monkeypatch, wl)
    counts = workloads.load_counts(wl["name"])
    lk = binding.Likelihood(wl, counts, mask=np.ones(n_rec, np.uint8), e_true_sm=np.ones(n_t))
    assert fake.calls == ["srw_create", "srw_set_data"]
    sg = binding.Surrogate(lk, init_weights(n_rec), BOX_CENTRE, BOX_HALF)
    assert fake.calls[-1] == "srw_surrogate_create"
    sg.set_weights(init_weights(n_rec, seed=9))
    sg.handle = lk.handle = None  # the stand-in handles are not the library's


def test_uneven_groups_pass(fake, monkeypatch):
    gw = workloads.uneven_groups_workload(n_groups=4, scale=0.25)
    for g in range(4):
        wl = workloads.uneven_group_inputs(gw, g)
        _info(monkeypatch, wl)
        lk = binding.Likelihood(wl, np.zeros(wl["R"].shape[0]))
        lk.handle = None


def test_joint_workload_passes(fake, monkeypatch):
    wl = workloads.solar_joint_workload()
    n_rec, _ = _info(monkeypatch, wl)
    lk = binding.Likelihood(wl, workloads.load_counts(wl["name"]))
    assert fake.calls == ["srw_create_joint", "srw_set_data"]
    lk.handle = None
    ev = [1.0] * len(wl["hist"])
    binding.srw_create_joint(wl["t_edges"], wl["components"], wl["hist"], wl["exposure"], mask=wl.get("mc_mask"),
                             scale=wl.get("scale"), live=wl.get("live"), events=ev, t_min=wl["t_min"])


def test_create_refuses_wrong_arrays(fake):
    wl = workloads.be7_line_workload()
    r = wl["R"]
    args = (wl["t_edges"], r.shape[0], wl["sources"])
    with pytest.raises(ValueError, match="R must be"):
        binding.srw_create(*args, r[:, :-1], wl["exposure"])
    with pytest.raises(ValueError, match="R must be"):
        binding.srw_create(wl["t_edges"], r.shape[0] + 1, wl["sources"], r, wl["exposure"])
    with pytest.raises(ValueError, match="e_true_sm"):
        binding.srw_create(*args, r, wl["exposure"], e_true_sm=np.ones(r.shape[1] - 1))
    bad = [dict(s) for s in wl["sources"]]
    bad[0]["pee"] = np.append(bad[0]["pee"], 0.5)
    with pytest.raises(ValueError, match="same number"):
        binding.srw_create(wl["t_edges"], r.shape[0], bad, r, wl["exposure"])
    assert not fake.calls


def test_create_joint_refuses_wrong_arrays(fake):
    t_edges = np.linspace(0.0, 1.0, 9)
    comps = workloads.be7_line_workload()["sources"] * 2
    hist = [np.ones((5, 8)), np.ones((5, 8))]
    binding.srw_create_joint(t_edges, comps, hist, 1.0e4)
    fake.calls.clear()
    cases = [
        (dict(hist=[np.ones((5, 8)), np.ones((5, 7))]), "hist\\[1\\]"),
        (dict(hist=[np.ones((5, 7)), np.ones((5, 7))]), "hist\\[0\\]"),
        (dict(mask=[None, np.ones(4)]), "mask\\[1\\]"),
        (dict(mask=[None]), "one live-time"),
        (dict(scale=np.ones(3)), "scale"),
        (dict(events=np.ones(1)), "events"),
        (dict(live=np.ones(4)), "live"),
    ]
    for kw, match in cases:
        a = dict(hist=hist)
        a.update(kw)
        h = a.pop("hist")
        with pytest.raises(ValueError, match=match):
            binding.srw_create_joint(t_edges, comps, h, 1.0e4, **a)
    assert not fake.calls


def test_set_data_refuses_wrong_arrays(fake, monkeypatch):
    monkeypatch.setattr(binding, "srw_info", lambda h: {"n_t": 8, "n_rec": 5})
    h = ctypes.c_void_p(HANDLE)
    binding.srw_set_data(h, np.zeros(5), np.ones((2, 5)), np.ones(5, np.uint8))
    binding.srw_set_data(h, np.zeros(5), np.ones(5))  # one template as a 1-D array
    fake.calls.clear()
    for args, match in [((np.zeros(4),), "counts"), ((np.zeros(5), np.ones((2, 4))), "bkg"),
                        ((np.zeros(5), None, np.ones(6, np.uint8)), "mask")]:
        with pytest.raises(ValueError, match=match):
            binding.srw_set_data(h, *args)
    assert not fake.calls


def test_likelihood_releases_its_handle_when_the_data_are_refused(fake, monkeypatch):
    wl = workloads.be7_line_workload()
    _info(monkeypatch, wl)
    with pytest.raises(ValueError, match="counts"):
        binding.Likelihood(wl, np.zeros(wl["R"].shape[0] + 3))
    assert fake.calls == ["srw_create", "srw_destroy"]


def test_surrogate_refuses_wrong_weights_and_targets(fake, monkeypatch):
    monkeypatch.setattr(binding, "srw_info", lambda h: {"n_t": 256, "n_rec": 128})
    h = ctypes.c_void_p(HANDLE)
    w = init_weights(128)
    for k, bad in [(0, np.ones((256, 4))), (3, np.ones((127, 256)))]:
        p = list(w)
        p[k] = (bad, p[k][1])
        with pytest.raises(ValueError, match="layer %d: W" % (k + 1)):
            binding.srw_surrogate_create(h, BOX_CENTRE, BOX_HALF, p)
    p = list(w)
    p[1] = (p[1][0], np.ones(255))
    with pytest.raises(ValueError, match="layer 2: b"):
        binding.srw_surrogate_create(h, BOX_CENTRE, BOX_HALF, p)
    with pytest.raises(ValueError, match="four layers"):
        binding.srw_surrogate_create(h, BOX_CENTRE, BOX_HALF, w[:3])
    with pytest.raises(ValueError, match="centre"):
        binding.srw_surrogate_create(h, BOX_CENTRE[:4], BOX_HALF, w)
    with pytest.raises(ValueError, match="targets"):
        binding.srw_surrogate_gradients(h, np.zeros((3, 5)), np.zeros((3, 127)), w)
    with pytest.raises(ValueError, match="targets"):
        binding.srw_surrogate_train_step(h, np.zeros((3, 5)), np.zeros((2, 128)), 1e-3, n_out=128)
    assert not fake.calls


def test_group_create_needs_one_count_per_handle(fake):
    hs = [ctypes.c_void_p(HANDLE), ctypes.c_void_p(HANDLE + 8)]
    with pytest.raises(ValueError, match="one point count per handle"):
        binding.srw_group_create(hs, [4])
    assert not fake.calls
    binding.srw_group_create(hs, [4, 0])
    assert fake.calls == ["srw_group_create"]
