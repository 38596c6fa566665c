"""The C-ABI library loads and exports every symbol that ``include/*.h`` declares (no GPU needed)."""
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b((?:helm|oras|gmres)_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def helm_lib():
    from paper_2103_14921_gb300 import build, helm
    build.build()
    return helm.lib()


def test_every_declared_symbol_is_exported(helm_lib):
    names = _declared_functions()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(helm_lib, n)]
    assert not missing, missing


def test_create_without_gpu_fails_cleanly(helm_lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import ctypes as C
    h = C.c_void_p()
    st = helm_lib.helm_create(C.byref(h), 0, None, 0)
    assert st != 0 and not h.value
    assert b"device" in helm_lib.helm_last_error(None).lower()


def test_library_weight_fit_matches_oracle_quality(helm_lib):
    """The library's own fit (host code) reaches the oracle fit's dispersion error."""
    from paper_2103_14921_gb300 import helm
    from oracle.weights import fit_weights, dispersion_residuals
    w_lib = helm.fit_weights()
    w_or = fit_weights()
    assert abs(sum(w_lib[:3]) - 1) < 1e-12 and min(w_lib) >= 0
    e_lib = np.abs(dispersion_residuals(w_lib)).max()
    e_or = np.abs(dispersion_residuals(w_or)).max()
    assert e_lib < 1.2 * e_or + 1e-4
