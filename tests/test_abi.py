"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/dd.h declares.  No compute call is made (no GPU here)."""
import os
import re

import pytest

from paper_1107_2516_gb300 import build as ddbuild
import paper_1107_2516_gb300 as dd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"DD_API\s+[\w\s\*]+?\b(dd_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    ddbuild.build()
    return dd.load()


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert declared, "no DD_API declarations found"
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(dd.EXPORTS)


def test_exported_symbols_via_nm(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", dd.dd.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (dd_\w+)", out))
    assert _declared() <= exported


def test_version_and_argument_errors(lib):
    assert "sm_103a" in dd.dd_version()
    # invalid arguments are rejected on the host before any CUDA call
    with pytest.raises(dd.DDError) as e:
        dd.dd_plan_create(0, 150.0, -0.1, 1e-4, [0.0], [1], 6.0, dd.DD_F32, 1000)
    assert e.value.code == 1 and "nchans" in str(e.value)
    with pytest.raises(dd.DDError):
        dd.dd_plan_create(16, 150.0, -0.1, 1e-4, [0.0], [], 6.0, dd.DD_F32, 1000)
    with pytest.raises(dd.DDError):
        dd.dd_plan_create(16, 150.0, -0.1, 1e-4, [-1.0], [1], 6.0, dd.DD_F32, 1000)
    with pytest.raises(dd.DDError):
        dd.dd_plan_create(2000, 150.0, -0.1, 1e-4, [0.0], [1], 6.0, dd.DD_F32, 1000)
    with pytest.raises(dd.DDError):
        dd.dd_plan_create(16, 150.0, -0.1, 1e-4, [0.0], [1], 6.0, 7, 1000)
    # maxshift >= nsamp_in is refused (Eq. 2: n outputs need n + maxshift inputs)
    with pytest.raises(dd.DDError) as e:
        dd.dd_plan_create(128, 150.0, -0.1953125, 327.68e-6, [6.3], [1], 6.0, dd.DD_F32, 1544)
    assert "maxshift" in str(e.value)


def test_candidate_layout():
    assert dd.CANDIDATE_DTYPE.itemsize == 32
    assert dd.CANDIDATE_DTYPE.fields["t"][1] == 8
    assert dd.CANDIDATE_DTYPE.fields["value"][1] == 24
