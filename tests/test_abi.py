"""The C-ABI library builds for sm_103a, loads, and exports what spmc.h
declares.  No compute calls: these run on a host without a GPU."""
import ctypes
import re
import shutil
import subprocess

import numpy as np
import pytest

from paper_2604_13929_gb300 import build, spmc


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not build.up_to_date():
        pytest.skip("nvcc not available to build libspmc")
    build.build()
    return spmc.load()


def test_library_exports_every_declared_function(lib):
    declared = spmc.declared_functions()
    assert len(declared) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", spmc.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (sp_mc_\w+)", out))
    assert set(declared) <= exported, set(declared) - exported
    for name in declared:
        assert hasattr(lib, name)


def test_result_layout_matches_binding(lib):
    assert lib.sp_mc_result_size() == ctypes.sizeof(spmc.Result)


def test_version_string(lib):
    assert "sm_103a" in spmc.sp_mc_version()


def test_invalid_arguments_are_rejected_before_any_device_work(lib):
    m = np.ones((4, 4, 4), np.uint8)
    with pytest.raises(spmc.SpmcError) as e:
        spmc.sp_mc_create(m, 4, 4, 4, 1.0, 0.5, 0.005, 1.0)
    assert e.value.code == spmc.SP_EINVAL
    with pytest.raises(spmc.SpmcError):
        spmc.sp_mc_create(m, 4, 4, 4, -1.0, 0.5, 0.005, 0.5)
    with pytest.raises(spmc.SpmcError):
        spmc.sp_mc_create(m, 4, 4, 4, 1.0, -0.5, 0.005, 0.5)
    assert lib.sp_mc_create(None, 4, 4, 4, 1.0, 0.5, 0.005, 0.5) is None
    assert "NULL" in spmc.sp_mc_last_error()
    assert lib.sp_mc_run(None, 10, 1, None) == spmc.SP_EINVAL
    assert lib.sp_mc_tallies(None, None, None) == spmc.SP_EINVAL


def test_no_cpu_fallback_without_a_device(lib):
    """On a host without a GPU the library fails loudly instead of falling
    back to any CPU path."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(spmc.SpmcError) as e:
        spmc.Simulation(np.ones((4, 4, 4), np.uint8), 0.5, 0.005, 0.7)
    assert e.value.code == spmc.SP_ECUDA


def test_product_code_never_uses_the_oracle():
    """The package and the C ABI neither import, include nor link oracle/."""
    import os
    import paper_2604_13929_gb300
    pkg = os.path.dirname(paper_2604_13929_gb300.__file__)
    pat = re.compile(r"^\s*(from\s+oracle|import\s+oracle|#\s*include\s*[<\"].*oracle)",
                     re.M)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                assert not pat.search(open(os.path.join(root, f)).read()), f
    out = subprocess.run(["nm", "-D", spmc.LIB_PATH], capture_output=True, text=True).stdout
    assert "or_run" not in out and "or_philox" not in out
