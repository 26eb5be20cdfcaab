"""The C-ABI library: builds, loads, exports every declared entry point, and
rejects invalid arguments on the host before touching a device."""

import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def srw():
    from paper_2607_00488_gb300 import build
    build.build()
    import paper_2607_00488_gb300 as pkg
    pkg.lib()
    return pkg


def _declared():
    text = open(os.path.join(ROOT, "include", "srw.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(srw_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("srw_create", "srw_set_data", "srw_spectrum", "srw_loglik", "srw_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(srw):
    lib = srw.lib()
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(srw.EXPORTS) >= set(_declared())


def test_status_strings(srw):
    lib = srw.lib()
    assert lib.srw_status_string(0) == b"ok"
    assert lib.srw_status_string(5).startswith(b"expected count")


def _args(**kw):
    wl = {
        "t_edges": np.linspace(0.0, 1.0, 9),
        "n_rec": 4,
        "sources": [{"e": np.array([0.862]), "w": np.array([1.0]), "pee": np.array([0.55])}],
        "R": np.full((4, 8), 0.2, dtype=np.float32),
        "exposure": 100.0,
    }
    wl.update(kw)
    return wl


@pytest.mark.parametrize("bad", [
    {"t_edges": np.array([0.0, 0.5, 0.4, 1.0])},                      # not ascending
    {"t_edges": np.array([0.0, np.nan, 1.0])},                         # NaN edge
    {"R": np.full((4, 8), -0.1, dtype=np.float32)},                    # negative response
    {"exposure": 0.0},
    {"sources": [{"e": np.array([-1.0]), "w": np.array([1.0]), "pee": np.array([0.5])}]},
    {"sources": [{"e": np.array([1.0]), "w": np.array([1.0]), "pee": np.array([1.5])}]},
    {"n_rec": 0},
])
def test_create_rejects_invalid_arguments(srw, bad):
    a = _args(**bad)
    # R shaped n_rec x n_t, so that the binding's shape check passes and the
    # library's own checks decide
    n_t = a["t_edges"].size - 1
    r = a["R"] if "R" in bad else np.full((a["n_rec"], n_t), 0.2, dtype=np.float32)
    with pytest.raises(srw.SrwError) as ei:
        srw.srw_create(a["t_edges"], a["n_rec"], a["sources"], r, a["exposure"])
    assert ei.value.status == 1  # SRW_EINVAL, raised before any device call


@pytest.mark.parametrize("handles,P", [([], []), ([None], [4]), ([None, None], [1, 2])])
def test_group_create_rejects_invalid_arguments(srw, handles, P):
    with pytest.raises(srw.SrwError) as ei:
        srw.srw_group_create(handles, P)
    assert ei.value.status == 1  # SRW_EINVAL, raised before any device call


def _joint(**kw):
    a = {
        "t_edges": np.linspace(0.0, 1.0, 9),
        "components": [{"e": np.array([0.862]), "w": np.array([1.0]), "pee": np.array([0.55])}],
        "hist": [np.full((4, 8), 3.0)],
        "exposure": 100.0,
    }
    a.update(kw)
    return a


@pytest.mark.parametrize("bad", [
    {"hist": [np.full((4, 8), -1.0)]},                       # negative histogram
    {"hist": [np.full((4, 8), np.nan)]},                     # NaN histogram
    {"mask": [np.zeros(4)]},                                 # live-time correction 0
    {"scale": np.array([0.0])},
    {"events": np.array([-5.0])},
    {"live": np.array([1.0, -1.0, 1.0, 1.0])},
    {"exposure": np.inf},
    {"t_edges": np.array([0.0, 0.5, 0.4, 1.0])},
])
def test_create_joint_rejects_invalid_arguments(srw, bad):
    a = _joint(**bad)
    t = a.pop("t_edges")
    comps, hist, expo = a.pop("components"), a.pop("hist"), a.pop("exposure")
    if len(t) != 9:
        hist = [np.full((4, len(t) - 1), 3.0)]
    with pytest.raises(srw.SrwError) as ei:
        srw.srw_create_joint(t, comps, hist, expo, **a)
    assert ei.value.status == 1  # SRW_EINVAL, raised before any device call


def test_missing_library_fails_loudly(srw, monkeypatch):
    # the binding has no fallback: without the built library every call raises
    from paper_2607_00488_gb300 import srw as binding
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB_PATH", os.path.join(ROOT, "no_such_dir", "libsrw.so"))
    with pytest.raises(RuntimeError, match="not built"):
        binding.lib()
    a = _args()
    with pytest.raises(RuntimeError, match="not built"):
        binding.srw_create(a["t_edges"], a["n_rec"], a["sources"], a["R"], a["exposure"])


def test_valid_create_without_a_device_fails_loudly(srw):
    # valid arguments and no usable sm_103 device: an error status, never a CPU path
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    a = _args()
    with pytest.raises(srw.SrwError) as ei:
        srw.srw_create(a["t_edges"], a["n_rec"], a["sources"], a["R"], a["exposure"])
    assert ei.value.status in (3, 7)  # SRW_ECUDA, SRW_EUNSUPPORTED


def test_debug_build_exports_every_declared_symbol():
    """libsrw_debug.so (bounds checks compiled in) builds and exports the same
    boundary as the release library."""
    import ctypes
    from paper_2607_00488_gb300 import build
    path = build.build(debug=True)
    assert path.endswith("libsrw_debug.so")
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
