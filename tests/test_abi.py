"""The C-ABI library loads without a GPU and exports every function that
include/rix.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rix.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rix_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib_path = os.path.join(ROOT, "paper_2507_22128_gb300", "librix.so")
    if not os.path.exists(lib_path):
        from paper_2507_22128_gb300 import build
        build.build()
    lib = ctypes.CDLL(lib_path)
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_the_abi():
    pytest.importorskip("torch")
    from paper_2507_22128_gb300 import rix
    assert set(rix.EXPORTED) == set(_declared())


def test_workspace_query_and_invalid_desc_need_no_gpu():
    from paper_2507_22128_gb300 import rix
    ok = rix.job_workspace_bytes(1024, 4.85e-6, 16, [1.3e9, 1.5e9], rix.FP32, 2, 1000)
    assert ok > 0
    assert rix.job_workspace_bytes(1000, 4.85e-6, 16, [1.3e9], rix.FP32, 2, 1000) == 0      # n not a power of 2
    assert rix.job_workspace_bytes(1024, 4.85e-6, 4, [1.3e9], rix.FP32, 2, 1000) == 0       # too few w-planes


def test_library_daubechies_filters():
    """The library forms db1..db8 with its own root finder; they agree with the
    oracle's spectral factorisation and with the db2 closed form."""
    import numpy as np
    from oracle import wavelet
    from paper_2507_22128_gb300 import rix
    for p in range(1, 9):
        h = np.array(rix.daubechies_lowpass(p))
        assert h.shape == (2 * p,)
        assert np.max(np.abs(h - wavelet.daubechies(p))) < 1e-11
    s3 = np.sqrt(3.0)
    want = np.array([1 + s3, 3 + s3, 3 - s3, 1 - s3]) / (4 * np.sqrt(2.0))
    assert np.max(np.abs(np.array(rix.daubechies_lowpass(2)) - want)) < 1e-15
    with pytest.raises(rix.RixError):
        rix.daubechies_lowpass(9)
