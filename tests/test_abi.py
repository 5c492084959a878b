"""The C-ABI library loads, exports every symbol include/usbs.h declares, and rejects
bad arguments before any device work (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2312_11801_gb300 import build as B
from paper_2312_11801_gb300 import instances as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def U():
    B.build()
    from paper_2312_11801_gb300 import usbs
    usbs.load()
    return usbs


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "usbs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(usbs_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ["usbs_create", "usbs_extreme_eigs", "usbs_step", "usbs_solve", "usbs_get_sketch",
                 "usbs_get_dual", "usbs_get_state", "usbs_set_state", "usbs_grow", "usbs_destroy"]:
        assert must in names


def test_library_exports_every_declared_symbol(U):
    lib = ctypes.CDLL(U.LIB_PATH)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    bound = {name for name, _, _ in U.SIGNATURES}
    assert set(declared_symbols()) <= bound


def test_param_defaults_and_version(U):
    p = U.params_default()
    assert p.rho == 0.01 and p.beta == 0.25 and p.k_c == 8 and p.k_p == 0
    assert p.lanczos_restarts == 10 and p.ipm_mu_tol == 1e-7 and p.max_alt == 50
    assert p.certify_restarts == 0 and p.obj_gap_tol == 0.0 and p.model_value_ipm == 0
    assert U.load().usbs_abi_version() == 5


def _expect_einval(U, prob, match, **kw):
    with pytest.raises(U.USBSError) as ei:
        U.usbs_create(prob, **kw)
    assert ei.value.code == U.USBS_EINVAL
    assert match in str(ei.value)


def test_invalid_arguments_rejected_on_the_host(U):
    p = I.maxcut_er(40, 4, seed=1)
    _expect_einval(U, p, "k_p", k_p=1)          # k_c = 8 leaves no room in V's 8 columns
    _expect_einval(U, p, "k_p", k_c=6, k_p=-1)
    _expect_einval(U, p, "k_c", k_c=9)
    _expect_einval(U, p, "certify_restarts", certify_restarts=-1)
    _expect_einval(U, p, "Psi", r=4)
    small = I.maxcut_er(28, 4, seed=1)
    _expect_einval(U, small, "n >= 32")
    bad = I.maxcut_er(40, 4, seed=1)
    bad.A_i = bad.A_i.copy(); bad.A_i[3] = 40
    _expect_einval(U, bad, "A index out of range")
    bad = I.maxcut_er(40, 4, seed=1)
    bad.C_col = bad.C_col.copy(); bad.C_col[0] = -1
    _expect_einval(U, bad, "C_col out of range")
    # an inequality-only problem does not fix the trace: the caller must give it
    cl = I.clustering_sdp(40, 60, 0)
    cl.is_ineq = np.ones_like(cl.is_ineq)
    _expect_einval(U, cl, "trace_hint")
