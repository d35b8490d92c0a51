"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every function that include/*.h declares (no compute calls here)."""
import ctypes as C
import glob
import os
import re

import pytest

from paper_2511_21264_gb300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*?[\s\*]+([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return sorted(n for n in names if n not in ("if", "while", "return"))


@pytest.fixture(scope="module")
def libmppi():
    native.build()
    return C.CDLL(native.LIB_PATH)


def test_header_declares_the_boundary():
    d = _declared()
    for name in ("mppi_model_load", "mppi_create", "mppi_step", "rollout_batch", "sim_step", "mppi_solve"):
        assert name in d


def test_every_declared_symbol_is_exported(libmppi):
    missing = [n for n in _declared() if not hasattr(libmppi, n)]
    assert not missing, missing


def test_binding_declares_every_export():
    native.lib()
    assert set(_declared()) <= set(native.EXPORTS) | {"mppi_batch_desc"}


def test_strerror_and_argument_checks_without_gpu(libmppi):
    libmppi.mppi_strerror.restype = C.c_char_p
    assert libmppi.mppi_strerror(0) == b"ok"
    assert libmppi.mppi_strerror(4).startswith(b"non-finite")
    # argument validation happens before any device call
    h = C.c_void_p()
    assert libmppi.mppi_model_load(None, 0, C.byref(h)) == 1
    assert libmppi.mppi_create(None, 64, 8, C.c_float(0.1), None, C.c_uint64(0), C.byref(h)) == 1
    assert libmppi.mppi_step(None, None, None, None, None) == 1


def test_malformed_blob_rejected_before_upload(libmppi):
    from paper_2511_21264_gb300 import scenes
    blob = bytearray(scenes.config(1).to_blob())
    blob[4] = 9  # version
    h = C.c_void_p()
    buf = C.create_string_buffer(bytes(blob), len(blob))
    assert libmppi.mppi_model_load(buf, len(blob), C.byref(h)) == 1
