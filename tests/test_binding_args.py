"""Host-side buffer checks of the binding's entry points.

The library takes every size from its integer arguments and the handle, so
the binding checks the buffers behind the pointers first: device arguments
must be contiguous CUDA tensors of the right dtype, long enough, on one
device; host ``out`` arrays must be writeable contiguous numpy arrays of the
right dtype and length.  The checks run before any library call; these tests
give them stand-ins that look like CUDA tensors and a stand-in library that
records the calls it receives (no GPU needed).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2607_00488_gb300 import srw as binding  # noqa: E402
from test_noalloc_args import FakeCuda  # noqa: E402


class FakeLib:
    """Records every entry-point call and returns SRW_OK."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        if not name.startswith("srw_"):
            raise AttributeError(name)

        def call(*a):
            self.calls.append((name, a))
            return binding.SRW_OK
        return call


@pytest.fixture
def fake(monkeypatch):
    f = FakeLib()
    monkeypatch.setattr(binding, "lib", lambda: f)
    monkeypatch.setattr(binding, "srw_info", lambda h: {"n_t": 96, "n_rec": 48})
    return f


def dev(t, **kw):
    return FakeCuda(t, **kw)


def theta(P, dtype=torch.float32):
    return dev(torch.zeros((P, 5), dtype=dtype))


H = object()  # a handle the stand-in library never looks at


def test_device_loglik_valid_call_reaches_the_library(fake):
    out = dev(torch.zeros(7, dtype=torch.float64))
    binding.srw_loglik(H, theta(7), binding.SRW_FP16X3, out=out, stream=0)
    name, a = fake.calls[-1]
    assert name == "srw_loglik" and a[2] == 7 and a[4] == binding.SRW_DEVICE and a[5] == binding.SRW_FP16X3


@pytest.mark.parametrize("bad,match", [
    (lambda: dict(theta=theta(4, torch.float64)), "float32"),
    (lambda: dict(theta=dev(torch.zeros(7, dtype=torch.float32))), "5 values a point"),
    (lambda: dict(theta=dev(torch.zeros((4, 5)), contiguous=False)), "contiguous"),
    (lambda: dict(out=dev(torch.zeros(4, dtype=torch.float32))), "float64"),
    (lambda: dict(out=dev(torch.zeros(3, dtype=torch.float64))), "holds 3 values"),
    (lambda: dict(out=torch.zeros(4, dtype=torch.float64)), "CUDA tensor"),
    (lambda: dict(out=dev(torch.zeros(4, dtype=torch.float64), dev="cuda:1")), "one device"),
])
def test_device_loglik_rejects(fake, bad, match):
    a = dict(theta=theta(4), out=dev(torch.zeros(4, dtype=torch.float64)))
    a.update(bad())
    with pytest.raises(ValueError, match=match):
        binding.srw_loglik(H, a["theta"], binding.SRW_FP32, out=a["out"], stream=0)
    with pytest.raises(ValueError, match=match):
        binding.srw_loglik_points(H, a["theta"], out=a["out"], stream=0)
    assert not fake.calls


@pytest.mark.parametrize("out,match", [
    (np.zeros(4, dtype=np.float32), "float64"),
    (np.zeros(3, dtype=np.float64), "holds 3 values"),
    (np.zeros(8, dtype=np.float64)[::2], "contiguous"),
    (torch.zeros(4, dtype=torch.float64), "numpy"),
])
def test_host_loglik_rejects_out(fake, out, match):
    with pytest.raises(ValueError, match=match):
        binding.srw_loglik(H, np.zeros((4, 5), dtype=np.float32), binding.SRW_FP32, out=out)
    assert not fake.calls


def test_host_loglik_rejects_read_only_out(fake):
    out = np.zeros(4, dtype=np.float64)
    out.setflags(write=False)
    with pytest.raises(ValueError, match="writeable"):
        binding.srw_loglik(H, np.zeros((4, 5), dtype=np.float32), out=out)


def test_host_loglik_accepts_a_longer_out(fake):
    out = np.zeros(6, dtype=np.float64)
    assert binding.srw_loglik(H, np.zeros((4, 5), dtype=np.float32), out=out) is out
    assert fake.calls[-1][1][2] == 4


@pytest.mark.parametrize("stage,n", [(0, 96), (1, 96), (2, 48), (3, 48)])
def test_spectrum_out_length_follows_the_stage(fake, stage, n):
    th = dev(torch.zeros(5, dtype=torch.float32))
    with pytest.raises(ValueError, match="holds %d values, the call needs %d" % (n - 1, n)):
        binding.srw_spectrum(H, th, stage, out=dev(torch.zeros(n - 1, dtype=torch.float32)), stream=0)
    binding.srw_spectrum(H, th, stage, out=dev(torch.zeros(n, dtype=torch.float32)), stream=0)
    with pytest.raises(ValueError, match="holds"):
        binding.srw_spectrum(H, np.zeros(5, dtype=np.float32), stage, out=np.zeros(n - 1, dtype=np.float32))
    assert [c[0] for c in fake.calls] == ["srw_spectrum"]


def test_spectrum_rejects_a_bad_stage_and_a_short_theta(fake):
    with pytest.raises(ValueError, match="stage"):
        binding.srw_spectrum(H, np.zeros(5, dtype=np.float32), 4)
    with pytest.raises(ValueError, match="holds 4 values"):
        binding.srw_spectrum(H, dev(torch.zeros(4, dtype=torch.float32)), 1,
                             out=dev(torch.zeros(96, dtype=torch.float32)), stream=0)
    assert not fake.calls


def test_spectrum_batch_out_holds_every_point(fake):
    with pytest.raises(ValueError, match="the call needs %d" % (3 * 48)):
        binding.srw_spectrum_batch(H, theta(3), out=dev(torch.zeros((2, 48), dtype=torch.float32)), stream=0)
    with pytest.raises(ValueError, match="the call needs %d" % (3 * 48)):
        binding.srw_spectrum_batch(H, np.zeros((3, 5), dtype=np.float32), out=np.zeros((2, 48), dtype=np.float32))
    binding.srw_spectrum_batch(H, theta(3), out=dev(torch.zeros((3, 48), dtype=torch.float32)), stream=0)
    assert [c[0] for c in fake.calls] == ["srw_spectrum_batch"]


def test_linear_gradient_buffer(fake):
    out = dev(torch.zeros(4, dtype=torch.float64))
    with pytest.raises(ValueError, match="grad_out holds 16 values, the call needs 20"):
        binding.srw_loglik_linear(H, theta(4), out=out, grad_out=dev(torch.zeros((4, 4), dtype=torch.float64)),
                                  stream=0)
    with pytest.raises(ValueError, match="grad_out must be float64"):
        binding.srw_loglik_linear(H, theta(4), out=out, grad_out=dev(torch.zeros((4, 5), dtype=torch.float32)),
                                  stream=0)
    with pytest.raises(ValueError, match="grad_out"):
        binding.srw_loglik_linear(H, np.zeros((4, 5), dtype=np.float32), grad_out=np.zeros((3, 5)))
    assert not fake.calls
    res, g = binding.srw_loglik_linear(H, np.zeros((4, 5), dtype=np.float32), grad_out=np.zeros((4, 5)))
    assert g.shape == (4, 5) and fake.calls[-1][1][4] is not None


def test_group_point_count(fake):
    with pytest.raises(ValueError, match="theta holds 4 points, the group 6"):
        binding.srw_group_loglik(H, theta(4), out=dev(torch.zeros(4, dtype=torch.float64)), stream=0, n_points=6)
    with pytest.raises(ValueError, match="theta holds 4 points, the group 6"):
        binding.srw_group_loglik(H, np.zeros((4, 5), dtype=np.float32), n_points=6)
    with pytest.raises(ValueError, match="holds 5 values"):
        binding.srw_group_loglik(H, theta(6), out=dev(torch.zeros(5, dtype=torch.float64)), stream=0, n_points=6)
    assert not fake.calls
    binding.srw_group_loglik(H, theta(6), out=dev(torch.zeros(6, dtype=torch.float64)), stream=0, n_points=6)
    assert fake.calls[-1][0] == "srw_group_loglik"


def test_grouped_likelihood_passes_its_point_count(fake):
    class Lk:
        handle = None
    grp = binding.GroupedLikelihood([Lk(), Lk()], [3, 4])
    with pytest.raises(ValueError, match="the group 7"):
        grp.loglik(np.zeros((6, 5), dtype=np.float32))
    grp.handle = None  # the stand-in handle is not the library's
