"""The C ABI library loads and exports every symbol include/*.h declares (no GPU).

Only host-side logic runs here: no kernel launch and no device allocation.
"""

import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "esp.h")
MLP_HEADER = os.path.join(ROOT, "include", "esp_mlp.h")
LIB = os.path.join(ROOT, "paper_2601_00161_gb300", "libesp.so")


def declared_functions(header=HEADER):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(esp_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        import __graft_entry__

        __graft_entry__.build()
    return ctypes.CDLL(LIB)


def test_every_declared_symbol_is_exported(lib):
    headers = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))
    assert HEADER in headers and MLP_HEADER in headers
    names = [n for h in headers for n in declared_functions(h)]
    assert len(names) >= 25
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    import paper_2601_00161_gb300 as esp
    from paper_2601_00161_gb300 import mlp

    assert sorted(esp.EXPORTS) == declared_functions()
    for n in esp.EXPORTS:
        assert callable(getattr(esp, n))
    assert sorted(mlp.EXPORTS) == declared_functions(MLP_HEADER)
    for n in mlp.EXPORTS:
        assert callable(getattr(mlp, n))


def test_mlp_rejects_bad_sizes_without_a_device():
    from paper_2601_00161_gb300 import mlp

    assert mlp.esp_mlp_n_params(7, 64, 4) == 64 * 7 + 64 + 64 * 64 + 64 + 4 * 64 + 4
    with pytest.raises(mlp.MLPError):
        mlp.MLP(0, 64, 4, 16)


def test_c_from_tolerance_host_logic(lib):
    import paper_2601_00161_gb300 as esp

    c = esp.esp_c_from_tolerance(1e-5)
    assert 13.5 < c < 14.5
    # the library's tuning rule (Sturm bisection + its own series at x = 1) against the
    # oracle's (library eigensolver + its series)
    from oracle.pswf import c_from_tolerance

    for k in range(3, 12):
        ref = c_from_tolerance(10.0 ** -k)
        assert abs(esp.esp_c_from_tolerance(10.0 ** -k) / ref - 1.0) < 1e-12, k
    assert esp.esp_c_from_tolerance(1e-7) > c
    with pytest.raises(esp.ESPError):
        esp.esp_c_from_tolerance(2.0)


def test_plan_rejects_bad_arguments_before_touching_the_device():
    import numpy as np

    import paper_2601_00161_gb300 as esp

    cell = np.eye(3) * 20.0
    cases = [
        (dict(cell=-cell), esp.ESP_ERR_CELL),
        (dict(cell=np.array([[1.0, 2, 3], [2, 4, 6], [0, 0, 1]])), esp.ESP_ERR_CELL),
        (dict(grid=(8, 8, 8), w=8), esp.ESP_ERR_SUPPORT),
        (dict(w=2), esp.ESP_ERR_ARG),
        (dict(w=13), esp.ESP_ERR_ARG),
        (dict(c=-1.0), esp.ESP_ERR_ARG),
        (dict(alpha=0.0), esp.ESP_ERR_ARG),
        (dict(n=-5), esp.ESP_ERR_ARG),
        (dict(grid=(8, 24, 24)), esp.ESP_ERR_GRID),  # 20 * 14 / (pi * 5) = 17.8 > 8
        (dict(precision=7), esp.ESP_ERR_ARG),
    ]
    for kw, code in cases:
        args = dict(cell=cell, n=10, grid=(24, 24, 24), w=6, c=14.0, alpha=5.0, precision=0)
        args.update(kw)
        with pytest.raises(esp.ESPError) as ei:
            esp.esp_plan(args["cell"], args["n"], args["grid"], args["w"], args["c"],
                         args["alpha"], args["precision"])
        assert ei.value.code == code, (kw, ei.value)
