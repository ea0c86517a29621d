"""C ABI checks that need no GPU: the library builds, loads, exports every
function include/tb.h declares, and its host-side setup arithmetic (row a10:
FD weights, CFL step, sponge, Ricker) agrees with the oracle and with the
closed forms."""
from __future__ import annotations

import ctypes
import math
import os
from fractions import Fraction as F

import numpy as np
import pytest

import oracle
from paper_2010_10248_gb300 import _tb
from paper_2010_10248_gb300 import build as tbbuild
from paper_2010_10248_gb300 import workloads as wl


@pytest.fixture(scope="module")
def lib():
    path = tbbuild.build()
    return _tb.load(path)


def test_exports_every_declared_function(lib):
    declared = _tb.header_functions()
    assert "tb_forward" in declared and "tb_create" in declared
    raw = ctypes.CDLL(_tb.LIB_PATH)
    for name in declared:
        assert hasattr(raw, name), name
    # the binding marshals exactly the declared functions
    assert set(declared) == set(_tb._SIGS)


def test_no_oracle_in_product_path():
    pkg = os.path.dirname(_tb.__file__)
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "tb_oracle" not in txt, f


@pytest.mark.parametrize("so", [4, 8, 12])
def test_fd_weights_closed_rationals(lib, so):
    golden = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "fd_weights.txt")):
        if line.startswith("#") or not line.strip():
            continue
        kind, s, *cs = line.split()
        golden[(kind, int(s))] = [float(F(c)) for c in cs]
    np.testing.assert_allclose(_tb.tb_fd_weights(so), golden[("d2", so)], rtol=1e-14, atol=1e-16)


@pytest.mark.parametrize("so", [4, 8, 12])
def test_cfl_matches_oracle(lib, oracle_lib, so):
    for h, v in (((10.0, 10.0, 10.0), 4500.0), ((20.0, 10.0, 15.0), 1500.0)):
        assert _tb.tb_cfl_dt_max(so, h, v) == pytest.approx(oracle.cfl_dt_max(so, h, v), rel=1e-14)
    assert _tb.tb_cfl_dt_max(4, (10.0, 10.0, 10.0), 1500.0) == pytest.approx(1 / 300, rel=1e-14)


@pytest.mark.parametrize("so", [4, 8, 12])
def test_tti_and_elastic_stability_limits_match_oracle(lib, oracle_lib, so):
    """Both sides sample the same trigonometric symbol maximum (the oracle
    densely, the library densely plus a golden-section refinement): agreement
    to 1e-9; so4 elastic is the closed form 7/3 of the oracle pins."""
    for h, v, e in (((10.0, 10.0, 10.0), 4500.0, 0.3), ((20.0, 10.0, 15.0), 1500.0, 0.0)):
        assert _tb.tb_tti_dt_max(so, h, v, e) == pytest.approx(oracle.tti_dt_max(so, h, v, e), rel=1e-9)
        assert _tb.tb_elastic_dt_max(so, h, v) == pytest.approx(oracle.elastic_dt_max(so, h, v), rel=1e-9)
    assert _tb.tb_tti_dt_max(so, (10.0,) * 3, 3000.0, 0.1) < _tb.tb_tti_dt_max(so, (10.0,) * 3, 3000.0, 0.0)
    assert _tb.tb_elastic_dt_max(so, (10.0, 10.0, 0.0), 3000.0) == -1.0


def test_sponge_matches_oracle(lib, oracle_lib):
    for n, nbl, h, v in ((64, 10, 10.0, 1500.0), (512, 40, 10.0, 4500.0), (30, 0, 5.0, 2000.0)):
        np.testing.assert_allclose(_tb.tb_sponge_profile(n, nbl, h, v),
                                   oracle.damping_axis(n, nbl, h, v), rtol=1e-14, atol=0)


def test_ricker_matches_input_generator(lib):
    got = np.array(_tb.tb_ricker(15.0, 8e-4, 500))
    want = wl.ricker(15.0, 8e-4, 500)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-7)
    assert abs(got.max() - 1.0) < 1e-3 and int(np.argmax(got)) == round((1 / 15.0) / 8e-4)


def test_invalid_arguments_rejected_without_gpu(lib):
    with pytest.raises(_tb.TBError):
        _tb.tb_fd_weights(5)
    assert _tb.tb_cfl_dt_max(8, (10.0, 0.0, 10.0), 1500.0) < 0
    with pytest.raises(_tb.TBError) as e:
        _tb.tb_create((64, 64, 64), (10.0, 10.0, 10.0), 6)  # unsupported space order
    assert e.value.status == _tb.TB_EINVAL
    with pytest.raises(_tb.TBError):
        _tb.tb_create((8, 64, 64), (10.0, 10.0, 10.0), 8)  # too thin for so8
    assert math.isfinite(_tb.tb_cfl_dt_max(12, (10.0, 10.0, 10.0), 1500.0))
