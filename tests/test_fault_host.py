"""Host-side fault injection: specification parsing, arming and the
environment variable (no GPU needed; the GPU tests in test_gpu_fault.py
check that an armed fault makes each failure path run and that the handle
stays usable)."""

import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def srw():
    from paper_2607_00488_gb300 import build
    build.build()
    import paper_2607_00488_gb300 as pkg
    pkg.srw_fault_inject("none")
    yield pkg
    pkg.srw_fault_inject("none")


@pytest.mark.parametrize("spec,kind,skip", [("alloc", 1, 0), ("launch", 2, 0), ("timeout", 3, 0),
                                            ("alloc:0", 1, 0), ("launch:7", 2, 7), ("timeout:12", 3, 12)])
def test_parse_valid(srw, spec, kind, skip):
    assert srw.srw_fault_parse(spec) == (kind, skip)


@pytest.mark.parametrize("spec", ["", "none", "alloc:", "alloc:-1", "alloc:3x", "alloc3", "Alloc", "launch:1:2",
                                  "timeouts", " alloc"])
def test_parse_rejects(srw, spec):
    with pytest.raises(srw.SrwError):
        srw.srw_fault_parse(spec)


def test_inject_arms_and_none_disarms(srw):
    srw.srw_fault_inject("launch", 4)
    assert srw.srw_fault_pending() == srw.srw.SRW_FAULT_LAUNCH
    srw.srw_fault_inject("none")
    assert srw.srw_fault_pending() == 0


def test_inject_rejects_bad_arguments(srw):
    with pytest.raises(srw.SrwError):
        srw.srw_fault_inject(7)
    with pytest.raises(srw.SrwError):
        srw.srw_fault_inject("alloc", -1)
    assert srw.srw_fault_pending() == 0


@pytest.mark.parametrize("env,kind", [("timeout:2", 3), ("alloc", 1), ("bogus", 0)])
def test_environment_arms_once_per_process(env, kind):
    code = ("import sys; sys.path.insert(0, %r); import paper_2607_00488_gb300 as p; "
            "print(p.srw_fault_pending())" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, SRW_FAULT=env, CUDA_VISIBLE_DEVICES=""),
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert int(r.stdout.strip().splitlines()[-1]) == kind
