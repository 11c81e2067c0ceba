"""The C-ABI library builds, loads and exports every function that
include/pic.h declares; host-only calls behave without a GPU."""
import ctypes as C
import os
import re
import subprocess

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "pic.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2507_10727_gb300 import build as b
    path = b.build()
    return C.CDLL(path), path


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("pic_create", "pic_step", "pic_diagnostics", "pic_get_particles",
                 "pic_set_particles", "pic_get_fields", "pic_save", "pic_load", "pic_destroy",
                 "pic_last_error", "pic_poisson_solve"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    _, path = lib
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (pic_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_config_struct_matches_abi(lib):
    import paper_2507_10727_gb300 as pg
    import pic_inputs
    cfg = pg.PicConfig.from_params(pic_inputs.params_rz32() | dict(cap_e=10, cap_i=10, birth_cap=10))
    assert cfg.struct_size == C.sizeof(pg.PicConfig)
    # the C struct ends with two int32 after three int64: 8-byte aligned total
    assert C.sizeof(pg.PicConfig) % 8 == 0


def test_host_only_calls_without_gpu(lib):
    L, _ = lib
    L.pic_poisson_workspace_bytes.restype = C.c_size_t
    L.pic_poisson_workspace_bytes.argtypes = [C.c_int, C.c_int]
    assert L.pic_poisson_workspace_bytes(256, 256) > 257 * 257 * 8 * 4
    assert L.pic_poisson_workspace_bytes(1, 5) == 0
    # an invalid configuration is rejected before any device call
    import paper_2507_10727_gb300 as pg
    import pic_inputs
    p = pic_inputs.params_rz32() | dict(cap_e=10, cap_i=10, birth_cap=10)
    p["nr"] = 31  # odd: invalid
    cfg = pg.PicConfig.from_params(p)
    out = C.c_void_p()
    L.pic_create.argtypes = [C.POINTER(pg.PicConfig), C.c_int, C.c_void_p, C.c_void_p,
                             C.POINTER(C.c_void_p)]
    assert L.pic_create(C.byref(cfg), 1, None, None, C.byref(out)) == -1
    assert out.value is None


def test_binding_fails_loudly_without_library(tmp_path):
    import paper_2507_10727_gb300.pic as pic
    saved = pic._lib
    pic._lib = None
    try:
        with pytest.raises(RuntimeError):
            pic.load_library(str(tmp_path / "missing.so"))
    finally:
        pic._lib = saved


def test_network_parameter_count_matches_reference(lib):
    import paper_2507_10727_gb300 as pg
    from oracle import unet
    assert pg.pic_unet_param_count() == unet.n_params(unet.init_params(0))


def test_invalid_options_rejected_without_gpu(lib):
    """Each option outside its documented range is rejected by pic_create
    before any device call (PIC_ERR_INVALID, no handle)."""
    L, _ = lib
    import paper_2507_10727_gb300 as pg
    import pic_inputs
    L.pic_create.argtypes = [C.POINTER(pg.PicConfig), C.c_int, C.c_void_p, C.c_void_p,
                             C.POINTER(C.c_void_p)]
    base = pic_inputs.params_rz32() | dict(cap_e=10, cap_i=10, birth_cap=10)
    for bad in (dict(phi_extrapolate=2), dict(phi_extrapolate=-1), dict(sort_every=0),
                dict(sort_every=65), dict(ied_bins=-1), dict(ied_bins=65537),
                dict(ied_bins=10, ied_emax=0.0)):
        cfg = pg.PicConfig.from_params(base | bad)
        out = C.c_void_p()
        assert L.pic_create(C.byref(cfg), 1, None, None, C.byref(out)) == -1, bad
        assert out.value is None, bad
