"""The C-ABI library builds, loads and exports every function include/*.h declares.
No compute call is made here (CPU only)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "subadmm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sim_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("sim_create", "sim_add_subsystem", "sim_add_interface", "sim_step",
                     "sim_residuals"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2302_14344_gb300 import subadmm
    L = subadmm.load()
    for name in _declared():
        assert hasattr(L, name), name
    assert set(_declared()) == set(subadmm.EXPORTS)


def test_library_exports_every_warm_start_network_symbol():
    from paper_2302_14344_gb300 import subadmm, warmstart
    txt = open(os.path.join(ROOT, "include", "warmstart.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = sorted(set(re.findall(r"\b(wsn_[a-z_]+)\s*\(", txt)))
    L = subadmm.load()
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(warmstart.EXPORTS)


def test_default_options_are_the_documented_ones():
    from paper_2302_14344_gb300 import subadmm
    o = subadmm.sim_default_options()
    assert o.h == 1e-3 and list(o.gravity) == [0.0, 0.0, -9.81] and o.baumgarte == 0.2
    assert o.beta_mode == subadmm.SIM_BETA_TRACE and o.warm == subadmm.SIM_WARM_PREV
    assert o.tol_primal == 1e-6 and o.max_iters == 1000 and o.stream is None


def test_create_without_a_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2302_14344_gb300 import subadmm
    with pytest.raises(subadmm.SimError) as ei:
        subadmm.sim_create(subadmm.sim_default_options())
    assert ei.value.code in (subadmm.SIM_ECUDA, subadmm.SIM_EINVAL)
