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


@pytest.fixture(scope="module")
def nnlib():
    if shutil.which("nvcc") is None and not build.up_to_date():
        pytest.skip("nvcc not available to build libspnn")
    build.build()
    from paper_2604_13929_gb300 import spnn
    return spnn.load()


def test_surrogate_library_exports_every_declared_function(nnlib):
    from paper_2604_13929_gb300 import spnn
    declared = spnn.declared_symbols()
    assert len(declared) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", spnn.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (spnn_\w+)", out))
    assert set(declared) <= exported, set(declared) - exported


def test_surrogate_rejects_bad_shapes_before_device_work(nnlib):
    from paper_2604_13929_gb300 import spnn
    assert nnlib.spnn_unet_create(24, 64, 4) is None          # c0 must be 16 or 32
    assert "c0" in nnlib.spnn_last_error().decode()
    assert nnlib.spnn_unet_create(32, 48, 4) is None          # n must be a power of two
    # channel counts must be multiples of 16; checked before any launch
    assert nnlib.spnn_pack_weights(0, 24, 32, 0, None, None, None) == spnn.SPNN_EINVAL
    assert nnlib.spnn_layer_forward(0, 1, 8, 8, 8, None, 16, None, 0, None, None, 32, 1, None,
                                    None, None, None, None) == spnn.SPNN_EINVAL
    assert nnlib.spnn_layer_wgrad(1, 1, 8, 8, 8, None, 16, None, 0, None, 32, None, None, None) == spnn.SPNN_EINVAL


def test_surrogate_options_are_validated_without_a_device(nnlib):
    """Launch-tuning options reject values outside their sets before any device work."""
    from paper_2604_13929_gb300 import spnn
    assert nnlib.spnn_set_option(spnn.OPT["conv_subtiles"], 3) == spnn.SPNN_EINVAL
    assert nnlib.spnn_set_option(spnn.OPT["conv_planes"], 8) == spnn.SPNN_EINVAL
    assert nnlib.spnn_set_option(spnn.OPT["stage_kb"], 500) == spnn.SPNN_EINVAL
    assert nnlib.spnn_set_option(99, 1) == spnn.SPNN_EINVAL
    assert nnlib.spnn_set_option(spnn.OPT["conv_subtiles"], -1) == spnn.SPNN_EINVAL
    assert nnlib.spnn_set_option(spnn.OPT["rows_persistent"], -1) == spnn.SPNN_EINVAL
    assert nnlib.spnn_set_option(spnn.OPT["rows_persistent"], 17) == spnn.SPNN_EINVAL
    assert nnlib.spnn_set_option(spnn.OPT["wgrad_halo"], 3) == spnn.SPNN_EINVAL
    assert nnlib.spnn_set_option(spnn.OPT["loss_fluence_weight"], 2) == spnn.SPNN_EINVAL
    assert nnlib.spnn_set_option(spnn.OPT["loss_fluence_weight"], 0) == spnn.SPNN_OK
    for key in ("conv_subtiles", "conv_planes", "stage_kb", "wgrad_halo", "conv_full_halo", "rows_persistent"):
        assert nnlib.spnn_set_option(spnn.OPT[key], 0) == spnn.SPNN_OK
    assert nnlib.spnn_set_option(spnn.OPT["wgrad_halo"], 2) == spnn.SPNN_OK
    assert nnlib.spnn_set_option(spnn.OPT["wgrad_halo"], 1) == spnn.SPNN_OK
    assert nnlib.spnn_set_option(spnn.OPT["rows_persistent"], 2) == spnn.SPNN_OK


def _header_constants(path, prefix):
    """NAME -> value of every `prefix`* constant a header defines (#define or enum)."""
    text = re.sub(r"/\*.*?\*/", " ", open(path).read(), flags=re.S)   # drop comments
    out = {m.group(1): int(m.group(2)) for m in re.finditer(rf"#define\s+({prefix}\w*)\s+\(?(-?\d+)\)?", text)}
    out.update({m.group(1): int(m.group(2)) for m in re.finditer(rf"\b({prefix}\w*)\s*=\s*(-?\d+)", text)})
    return out


def test_binding_option_keys_match_the_headers():
    import os
    from paper_2604_13929_gb300 import spnn
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sp = _header_constants(os.path.join(root, "include", "spmc.h"), "SP_OPT_")
    nn = _header_constants(os.path.join(root, "include", "spnn.h"), "SPNN_OPT_")
    assert {"SP_OPT_" + k.upper(): v for k, v in spmc.OPT.items()} == sp
    assert {"SPNN_OPT_" + k.upper(): v for k, v in spnn.OPT.items()} == nn


def test_binding_status_codes_match_the_headers():
    import os
    from paper_2604_13929_gb300 import spnn
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sp = _header_constants(os.path.join(root, "include", "spmc.h"), "SP_E")
    sp.update(_header_constants(os.path.join(root, "include", "spmc.h"), "SP_OK"))
    nn = _header_constants(os.path.join(root, "include", "spnn.h"), "SPNN_E")
    nn.update(_header_constants(os.path.join(root, "include", "spnn.h"), "SPNN_OK"))
    assert sp == {n: getattr(spmc, n) for n in ("SP_OK", "SP_EINVAL", "SP_ENOMEM", "SP_ECUDA", "SP_ESTEPLIMIT",
                                                 "SP_EOVERFLOW")}
    assert nn == {n: getattr(spnn, n) for n in ("SPNN_OK", "SPNN_EINVAL", "SPNN_ENOMEM", "SPNN_ECUDA")}
