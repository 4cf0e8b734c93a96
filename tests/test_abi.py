"""Host-side checks of the C ABI (no GPU needed).

The library must build for sm_103a, load, and export every entry point that
include/*.h declare; without a GPU, creating a simulator must fail
cleanly with FFSRL_E_CUDA (no CPU fallback), and bad arguments must be
rejected before any device work.
"""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2503_18616_gb300 import build, ffsrl, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ffsrl.load_library()


def _declared_functions():
    inc = os.path.join(ROOT, "include")
    names = set()
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            text = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, f)).read(), flags=re.S)
            names |= set(re.findall(r"\b(ffsrl_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    declared = _declared_functions()
    assert len(declared) >= 12
    assert sorted(ffsrl.EXPORTS) == declared
    out = subprocess.run(["nm", "-D", "--defined-only", ffsrl.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (ffsrl_[a-z_0-9]+)", out))
    for name in declared:
        assert name in exported, name
        getattr(lib, name)


def test_library_targets_sm_103a_only(lib):
    out = subprocess.run(["cuobjdump", "--list-elf", ffsrl.LIB_PATH], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    archs = set(re.findall(r"sm_(\d+a?)", out.stdout))
    assert archs == {"103a"}


def _params_struct(**over):
    return ffsrl.make_params(inputs.default_params(**over))


def _create(lib, params, n_env=1, mesh=None):
    rest, w, tets = mesh if mesh is not None else inputs.grid_block(3, 3, 2)
    keep = [np.ascontiguousarray(rest, np.float64), np.ascontiguousarray(w, np.float64),
            np.ascontiguousarray(tets, np.int32)]
    m = ffsrl.ffsrl_mesh(len(rest), len(tets), keep[0].ctypes.data, keep[1].ctypes.data, keep[2].ctypes.data)
    h = ctypes.c_void_p()
    rc = lib.ffsrl_create(ctypes.byref(m), 1, None, None, n_env, ctypes.byref(params), None, ctypes.byref(h))
    return rc, h


def test_bad_arguments_are_rejected_before_device_work(lib):
    p = _params_struct(n_obs=4)
    p.substeps = 0
    rc, h = _create(lib, p)
    assert rc == -1 and not h.value
    assert b"substeps" in lib.ffsrl_last_error()
    p = _params_struct(n_obs=4)
    p.block_threads = 100
    rc, h = _create(lib, p)
    assert rc == -1
    p = _params_struct(n_obs=4)
    rc, h = _create(lib, p, n_env=0)
    assert rc == -1
    assert lib.ffsrl_step(None, None, None, None, None) == -1
    assert lib.ffsrl_destroy(None) == -1


def test_no_gpu_means_cuda_error_not_fallback(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rc, h = _create(lib, _params_struct(n_obs=4))
    assert rc == -2 and not h.value


def test_header_constants_match_the_binding():
    text = open(os.path.join(ROOT, "include", "ffsrl.h")).read()
    consts = dict(re.findall(r"#define (FFSRL_[A-Z_0-9]+) \(?([0-9]+)", text))
    assert int(consts["FFSRL_NET_PARAMS"]) == ffsrl.NET_PARAMS == 5379
    assert int(consts["FFSRL_NET_NORM"]) == ffsrl.NET_NORM == 36
    assert ffsrl.NOALLOC_SCRATCH_BYTES == 32 << 20
