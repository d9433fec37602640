"""CPU checks of the C-ABI boundary: the library builds, loads without a GPU and exports every
call include/pothole.h declares; the binding exposes the same names."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:pd_status|const char\*|size_t)\s+(pd_\w+)\s*\(", txt, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2012_10802_gb300 import build
    return build.build()


def test_header_declares_the_pipeline_calls():
    names = _declared()
    for n in ["pd_warp", "pd_cost", "pd_aggregate", "pd_disparity", "pd_transform",
              "pd_superpixels", "pd_pothole_mask", "pd_sgm", "pd_run_pipeline"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_has_the_same_names(libpath):
    from paper_2012_10802_gb300 import binding
    for n in _declared():
        assert n in binding.SIGNATURES or n in binding.EXTRA or n == "pd_last_error", n
    for n in binding.SIGNATURES:
        if n not in ("pd_create", "pd_destroy", "pd_set_stream", "pd_default_params",
                     "pd_cnn_create", "pd_cnn_destroy"):  # wrapped by Context and Cnn
            assert hasattr(binding, n), n


def test_default_params_without_gpu(libpath):
    from paper_2012_10802_gb300 import binding
    p = binding.default_params()
    assert (p.D, p.paths, p.P1, p.P2, p.lr_tol) == (128, 8, 4, 32, 1)
    assert abs(p.delta_pd - 2.36) < 1e-6


def test_create_without_gpu_fails_cleanly(libpath):
    from paper_2012_10802_gb300 import binding
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert binding.lib().pd_create(ctypes.byref(h), 0, None) == binding.PD_ERR_INVALID_ARG
    assert binding.lib().pd_destroy(None) == binding.PD_OK


def test_null_handles_are_rejected_without_a_launch(libpath):
    """Calls that take a context or a network reject NULL handles before touching a device."""
    from paper_2012_10802_gb300 import binding
    L = binding.lib()
    assert L.pd_cnn_check(None, None) == binding.PD_ERR_INVALID_ARG
    assert L.pd_cnn_probe_timeout(None, None, 1000) == binding.PD_ERR_INVALID_ARG
    assert L.pd_pipeline_config(None, 1) == binding.PD_ERR_INVALID_ARG
    assert L.pd_cnn_destroy(None) == binding.PD_OK
    h = ctypes.c_void_p()
    assert L.pd_cnn_create(ctypes.byref(h), 0, 0, 8, 8) == binding.PD_ERR_INVALID_ARG  # batch 0
    assert L.pd_cnn_create(None, 0, 1, 8, 8) == binding.PD_ERR_INVALID_ARG
    assert binding.pd_cnn_num_params() == 19682
