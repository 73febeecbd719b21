"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/pic.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_2406_01939_b300 import build as pic_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*[\w\s\*]*?\b(pic_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for want in ("pic_create_instance", "pic_instance_load", "pic_destroy_instance",
                 "pic_simulate", "pic_create_batch", "pic_simulate_batch", "pic_policy_grad",
                 "pic_last_error", "pic_owmr_create", "pic_owmr_simulate", "pic_owmr_destroy"):
        assert want in names


def test_library_loads_and_exports_every_declared_symbol():
    path = pic_build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_last_error_is_empty_string_initially():
    lib = ctypes.CDLL(pic_build.build())
    lib.pic_last_error.restype = ctypes.c_char_p
    assert lib.pic_last_error() == b""


def test_null_arguments_rejected_without_gpu():
    """Argument checks run before any device work."""
    import paper_2406_01939_b300 as pic
    L = pic.lib()
    h = ctypes.c_void_p()
    assert L.pic_create_instance(None, ctypes.byref(h)) == pic.PIC_ERR_INVALID_ARG
    assert "descriptor" in pic.pic_last_error()
    assert L.pic_simulate(None, None, None, None, None, None) == pic.PIC_ERR_INVALID_ARG
    assert L.pic_create_batch(None, 3, ctypes.byref(h)) == pic.PIC_ERR_INVALID_ARG
    assert L.pic_simulate_batch(None, None, None, None, None, None, None) == pic.PIC_ERR_INVALID_ARG
    assert "batch" in pic.pic_last_error()
    assert L.pic_policy_grad(None, None, None, None, None, None) == pic.PIC_ERR_INVALID_ARG
    assert L.pic_batch_load(None, None, 2) == pic.PIC_ERR_INVALID_ARG
    assert "batch" in pic.pic_last_error()


def test_owmr_null_and_shape_arguments_rejected_without_gpu():
    """pic_owmr_create checks its descriptor before any device work."""
    import paper_2406_01939_b300 as pic
    from paper_2406_01939_b300 import owmr
    L = owmr._lib()
    h = ctypes.c_void_p()
    assert L.pic_owmr_create(None, ctypes.byref(h)) == pic.PIC_ERR_INVALID_ARG
    d = owmr.pic_owmr_desc(10, 0)  # N = 0
    assert L.pic_owmr_create(ctypes.byref(d), ctypes.byref(h)) == pic.PIC_ERR_INVALID_ARG
    assert "N" in pic.pic_last_error()


def test_no_cpu_fallback_without_a_device():
    """Without a CUDA device the library and the session fail with an error:
    nothing behind the C-ABI or the Python binding simulates on the host."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    import paper_2406_01939_b300 as pic
    from paper_2406_01939_b300 import synth
    from paper_2406_01939_b300.session import DeviceInstance
    inst = synth.greedy_small(0, T=64)
    d = pic.make_desc(inst.T, inst.N, inst.K, inst.R, inst.prod, inst.reg, inst.x0, inst.cost,
                      mem=pic.PIC_MEM_HOST)
    with pytest.raises(pic.PicError) as e:
        pic.pic_create_instance(d)
    assert e.value.status == pic.PIC_ERR_CUDA and pic.pic_last_error()
    with pytest.raises(pic.PicError) as e:
        pic.pic_create_batch([d, d])
    assert e.value.status == pic.PIC_ERR_CUDA
    with pytest.raises(RuntimeError):
        DeviceInstance(inst)
