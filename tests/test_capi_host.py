"""Host-side checks of the C ABI that need no GPU: the library loads, exports every
function declared in include/nnp.h, and rejects invalid parameter sets before any
CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2002_00054_b300 import _capi, build as nnp_build
import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    nnp_build.build()
    return _capi.load()


def _declared():
    txt = open(os.path.join(ROOT, "include", "nnp.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(nnp_[a-z_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_capi.SIGNATURES)


def test_status_strings(lib):
    assert lib.nnp_status_string(0) == b"NNP_OK"
    assert lib.nnp_status_string(3) == b"NNP_ENEIGH_OVERFLOW"


class _P:
    """Keeps the ctypes buffers of a params struct alive."""

    def __init__(self, model, **kw):
        sf = model["sf"]
        rows = [d for e in sf for d in e]
        code = {"radial": 2, "narrow": 3, "wide": 4}
        self.sf = (_capi.SfDesc * len(rows))(*[
            _capi.SfDesc(code[d["type"]], d.get("e1", -1), d.get("e2", -1), d["eta"], d.get("rs", 0.0),
                         d.get("zeta", 1.0), d.get("lambda", 1.0)) for d in rows])
        self.m = np.ascontiguousarray(model["masses"], np.float64)
        self.nsf = np.ascontiguousarray([len(e) for e in sf], np.int32)
        self.mu = np.ascontiguousarray(np.concatenate(model["sf_mu"]))
        self.s = np.ascontiguousarray(np.concatenate(model["sf_s"]))
        self.wd = np.ascontiguousarray(model["widths"], np.int32)
        self.w = np.ascontiguousarray(np.concatenate(model["weights"]))
        p = _capi.Params()
        p.n_elements = len(sf)
        p.masses_amu = self.m.ctypes.data_as(_capi.c_double_p)
        p.cutoff = model["cutoff"]
        p.skin = 1.0
        p.n_sf = self.nsf.ctypes.data_as(_capi.c_int_p)
        p.sf = self.sf
        p.sf_shift = self.mu.ctypes.data_as(_capi.c_double_p)
        p.sf_scale = self.s.ctypes.data_as(_capi.c_double_p)
        p.n_layers = len(self.wd) - 1
        p.widths = self.wd.ctypes.data_as(_capi.c_int_p)
        p.weights = self.w.ctypes.data_as(_capi.c_double_p)
        p.mlp_precision = 0
        p.max_neighbors = 192
        for k, v in kw.items():
            setattr(p, k, v)
        self.p = p


def _create(lib, P, device=0):
    h = ctypes.c_void_p()
    rc = lib.nnp_create(ctypes.byref(P.p), device, ctypes.byref(h))
    return rc, h, lib.nnp_last_error(None).decode()


@pytest.mark.parametrize("field,value,code", [
    ("n_elements", 0, _capi.NNP_EINVAL),
    ("cutoff", -1.0, _capi.NNP_EINVAL),
    ("skin", -0.5, _capi.NNP_EINVAL),
    ("max_neighbors", 8, _capi.NNP_EINVAL),
    ("n_layers", 1, _capi.NNP_EINVAL),
    ("mlp_precision", 7, _capi.NNP_EINVAL),
])
def test_create_rejects_bad_params(lib, field, value, code):
    P = _P(workloads.water_model(), **{field: value})
    rc, h, msg = _create(lib, P)
    assert rc == code and not h.value and msg


def test_create_rejects_bad_descriptors(lib):
    m = workloads.water_model()
    m["sf"][0][20] = dict(m["sf"][0][20], zeta=3.0)
    rc, h, msg = _create(lib, _P(m))
    assert rc == _capi.NNP_EUNSUPPORTED and "zeta" in msg
    m = workloads.water_model()
    m["sf"][1][18] = dict(m["sf"][1][18], e1=0, e2=2)   # element 2 does not exist
    rc, h, msg = _create(lib, _P(m))
    assert rc == _capi.NNP_EINVAL and "out of range" in msg
    m = workloads.water_model()
    m["sf"][1][18] = dict(m["sf"][1][18], type="wide")   # narrow and wide in one model
    rc, h, msg = _create(lib, _P(m))
    assert rc == _capi.NNP_EUNSUPPORTED and "narrow and wide" in msg
    m = workloads.water_model()
    m["sf_s"][0] = np.array(m["sf_s"][0]); m["sf_s"][0][3] = 0.0
    rc, h, msg = _create(lib, _P(m))
    assert rc == _capi.NNP_EINVAL and "sf_scale" in msg


def test_null_handle_calls(lib):
    assert lib.nnp_destroy(None) == 0
    assert lib.nnp_compute(None, 0, None, None, None, 0.0, None, None, None, None, None) == _capi.NNP_EINVAL
    assert lib.nnp_num_params(None) == 0


def test_create_without_device_fails_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rc, h, msg = _create(lib, _P(workloads.water_model()))
    assert rc == _capi.NNP_ECUDA and not h.value


def test_create_rejects_bf16_network_shape(lib):
    m = workloads.water_model(hidden=(25,))
    rc, h, msg = _create(lib, _P(m, mlp_precision=_capi.NNP_BF16))
    assert rc == _capi.NNP_EUNSUPPORTED and "n_layers = 3" in msg
