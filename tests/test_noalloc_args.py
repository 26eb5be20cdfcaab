"""Host-side argument checks of the allocation-free entry point's binding.

srw_loglik_point_noalloc reads every size from n_rec and ld, so the binding
rejects tensors that would make the kernels read past an end or fold with the
wrong stride.  The checks run before any device work; these tests give them
stand-ins that look like CUDA tensors (no GPU needed) and expect ValueError
for each wrong argument.
"""

import pytest

torch = pytest.importorskip("torch")

from paper_2607_00488_gb300 import srw as binding  # noqa: E402


class FakeCuda:
    """A CPU tensor that reports itself as a CUDA tensor on device `dev`."""

    def __init__(self, t, dev="cuda:0", contiguous=None):
        self.t = t
        self.is_cuda = True
        self.device = torch.device(dev)
        self._contig = t.is_contiguous() if contiguous is None else contiguous
        self.dtype = t.dtype
        self.shape = t.shape

    def data_ptr(self):
        return self.t.data_ptr()

    def is_contiguous(self):
        return self._contig

    def dim(self):
        return self.t.dim()

    def numel(self):
        return self.t.numel()


def args(n_rec=8, ld=64):
    return dict(R=FakeCuda(torch.zeros((n_rec, ld), dtype=torch.float32)),
                W=FakeCuda(torch.zeros(ld, dtype=torch.float32)),
                counts=FakeCuda(torch.zeros(n_rec, dtype=torch.float64)),
                out=FakeCuda(torch.zeros(1, dtype=torch.float64)),
                bkg=FakeCuda(torch.zeros(n_rec, dtype=torch.float64)),
                mask=FakeCuda(torch.ones(n_rec, dtype=torch.uint8)))


def check(a):
    binding._check_noalloc_args(a["R"], a["W"], a["counts"], a["out"], a["bkg"], a["mask"])


def test_valid_arguments_pass():
    check(args())
    a = args()
    a["bkg"] = a["mask"] = None
    check(a)


@pytest.mark.parametrize("name", ["R", "W", "counts", "out", "bkg", "mask"])
def test_rejects_host_tensor(name):
    a = args()
    a[name] = a[name].t
    with pytest.raises(ValueError, match="CUDA"):
        check(a)


@pytest.mark.parametrize("name,dtype", [("R", torch.float64), ("W", torch.float64), ("counts", torch.float32),
                                        ("bkg", torch.float32), ("out", torch.float32), ("mask", torch.bool)])
def test_rejects_wrong_dtype(name, dtype):
    a = args()
    a[name] = FakeCuda(a[name].t.to(dtype))
    with pytest.raises(ValueError, match="must be"):
        check(a)


def test_rejects_float32_counts_of_the_default_dtype():
    a = args()
    a["counts"] = FakeCuda(torch.zeros(8))  # torch's default float32
    with pytest.raises(ValueError, match="float64"):
        check(a)


def test_rejects_non_contiguous_response():
    a = args()
    a["R"] = FakeCuda(torch.zeros((8, 128), dtype=torch.float32)[:, :64], contiguous=False)
    with pytest.raises(ValueError, match="contiguous"):
        check(a)


def test_rejects_mixed_devices():
    a = args()
    a["W"] = FakeCuda(a["W"].t, dev="cuda:1")
    with pytest.raises(ValueError, match="one device"):
        check(a)


def test_rejects_short_weights():
    a = args()
    a["W"] = FakeCuda(torch.zeros(32, dtype=torch.float32))
    with pytest.raises(ValueError, match="W holds"):
        check(a)


@pytest.mark.parametrize("name", ["counts", "bkg", "mask"])
def test_rejects_per_bin_arrays_of_the_wrong_length(name):
    a = args()
    a[name] = FakeCuda(a[name].t[:5].clone())
    with pytest.raises(ValueError, match="n_rec"):
        check(a)


def test_rejects_empty_out():
    a = args()
    a["out"] = FakeCuda(torch.zeros(0, dtype=torch.float64))
    with pytest.raises(ValueError, match="out"):
        check(a)


def test_rejects_one_dimensional_response():
    a = args()
    a["R"] = FakeCuda(torch.zeros(64, dtype=torch.float32))
    with pytest.raises(ValueError, match="2-D"):
        check(a)
