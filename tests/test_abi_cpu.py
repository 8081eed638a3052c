"""Host-side checks of the C ABI (no GPU needed): the library builds for sm_103a,
loads, exports every entry point declared in include/*.h, and rejects invalid
problems with QC_EINVAL before touching the device."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

from paper_2412_10072_gb300 import build as qbuild
from paper_2412_10072_gb300 import qc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(qc_[A-Za-z0-9_]+)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    qbuild.build()
    return qc.load()


def test_header_declares_the_abi():
    names = declared_functions()
    for must in ("qc_create", "qc_solve", "qc_residual", "qc_destroy", "qc_last_error", "qc_version"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_version_string(lib):
    assert b"sm_103a" in lib.qc_version()


def _problem(**over):
    n_row, n_chan = 6, 3
    data = np.zeros((n_row, n_chan, 4), np.complex64)
    weight = np.ones((n_row, n_chan, 4), np.float32)
    a1 = np.array([0, 0, 1, 0, 0, 1], np.int32)
    a2 = np.array([1, 2, 2, 1, 2, 2], np.int32)
    t = np.array([0, 0, 0, 1, 1, 1], np.int32)
    keep = dict(data=data, model=data.copy(), weight=weight, a1=a1, a2=a2, t=t)
    fields = dict(n_row=n_row, n_chan=n_chan, n_corr=4, n_ant=3, n_dir=1, n_time=2, memory=0, model_fp16=0)
    fields.update(over)
    p = qc._Problem(fields["n_row"], fields["n_chan"], fields["n_corr"], fields["n_ant"], fields["n_dir"],
                    fields["n_time"], keep["data"].ctypes.data, keep["model"].ctypes.data,
                    keep["weight"].ctypes.data, None, keep["a1"].ctypes.data, keep["a2"].ctypes.data,
                    keep["t"].ctypes.data, fields["memory"], fields["model_fp16"])
    return p, keep


@pytest.mark.parametrize("over", [dict(n_corr=2), dict(n_dir=0), dict(n_dir=65), dict(n_dir=2, model_fp16=1),
                                  dict(n_ant=1), dict(n_chan=0), dict(n_time=0), dict(memory=7), dict(n_ant=2),
                                  dict(n_time=1)])
def test_create_rejects_invalid_problems(lib, over):
    p, keep = _problem(**over)
    h = C.c_void_p()
    rc = lib.qc_create(C.byref(p), C.byref(h))
    assert rc == qc.QC_EINVAL
    assert not h.value
    assert lib.qc_last_error(None)


def test_create_rejects_null_arguments(lib):
    h = C.c_void_p()
    assert lib.qc_create(None, C.byref(h)) == qc.QC_EINVAL
    p, keep = _problem()
    assert lib.qc_create(C.byref(p), None) == qc.QC_EINVAL


def test_destroy_is_null_safe(lib):
    lib.qc_destroy(None)


def _batch(**over):
    b = dict(n_prob=2, row_offset=np.array([0, 3, 6], np.int64), vis_offset=np.array([0, 6, 12], np.int64),
             n_chan=np.array([2, 2], np.int32), n_ant=np.array([3, 3], np.int32))
    b.update(over)
    data = np.zeros((12, 4), np.complex64)
    keep = dict(data=data, model=data.copy(), weight=np.ones((12, 4), np.float32),
                a1=np.array([0, 0, 1, 0, 0, 1], np.int32), a2=np.array([1, 2, 2, 1, 2, 2], np.int32), **b)
    p = qc._BatchProblem(b["n_prob"], keep["row_offset"].ctypes.data, keep["vis_offset"].ctypes.data,
                         keep["n_chan"].ctypes.data, keep["n_ant"].ctypes.data, keep["data"].ctypes.data,
                         keep["model"].ctypes.data, keep["weight"].ctypes.data, None, keep["a1"].ctypes.data,
                         keep["a2"].ctypes.data, 0, 0)
    return p, keep


@pytest.mark.parametrize("over", [dict(n_prob=0), dict(vis_offset=np.array([0, 5, 12], np.int64)),
                                  dict(n_ant=np.array([3, 2], np.int32)), dict(n_ant=np.array([3, 300], np.int32)),
                                  dict(row_offset=np.array([1, 3, 6], np.int64)),
                                  dict(n_chan=np.array([2, 0], np.int32))])
def test_batch_create_rejects_invalid(lib, over):
    qc._load_batch(lib)
    p, keep = _batch(**over)
    h = C.c_void_p()
    assert lib.qc_batch_create(C.byref(p), C.byref(h)) == qc.QC_EINVAL
    assert lib.qc_batch_last_error(None)
    lib.qc_batch_destroy(None)


def test_new_entry_points_reject_a_null_context(lib):
    """qc_delay_init and qc_mad_flag return QC_EINVAL for a NULL context before any device work."""
    assert lib.qc_delay_init(None, None, 0, 0) == qc.QC_EINVAL
    n = C.c_int64(0)
    assert lib.qc_mad_flag(None, None, 0, 5.0, 0, None, 0, C.byref(n)) == qc.QC_EINVAL


def test_delay_term_needs_channel_frequencies():
    with pytest.raises(ValueError):
        qc.Term("delay", np.zeros(2, np.int32), np.zeros(4, np.int32), 1, 1, 3)
    t = qc.Term("delay", np.zeros(2, np.int32), np.zeros(4, np.int32), 1, 1, 3, chan_freq=np.linspace(1, 2, 4))
    assert t.gains.shape == (1, 1, 3, 4) and t.gains.dtype == np.float32 and not t.gains.any()
    assert t._c().chan_freq == t.chan_freq.ctypes.data
