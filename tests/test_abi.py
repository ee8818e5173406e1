"""Host-side checks of the C ABI (no GPU): the library builds for sm_103a, loads, and exports
every entry point declared in include/hphi_gpu.h; host-only argument validation works."""
import ctypes
import os
import re

import pytest

import paper_1703_03637_gb300 as hp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "hphi_gpu.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hphi_[A-Za-z0-9_]+)\s*\(", txt)))


def test_header_declares_binding_symbols():
    assert _declared() == sorted(hp.EXPORTS)


def test_library_exports_every_declared_symbol():
    L = hp.load()
    for name in _declared():
        assert hasattr(L, name), name


def test_host_validation_without_gpu():
    L = hp.load()
    h = ctypes.c_void_p()
    assert L.hphi_create(ctypes.byref(h), 7, 4) == -1
    assert b"kind" in L.hphi_last_error(None)
    assert L.hphi_create(ctypes.byref(h), hp.SPIN_HALF, 0) == -1
    assert L.hphi_create(ctypes.byref(h), hp.SPIN_HALF, 4) == 0
    J = (ctypes.c_double * 9)(1, 0, 0, 0, 1, 0, 0, 0, 1)
    assert L.hphi_add_spin_coupling(h, 0, 0, J) == -1          # i == j
    assert L.hphi_add_spin_coupling(h, 0, 4, J) == -1          # out of range
    assert L.hphi_add_spin_coupling(h, 0, 1, J) == 0
    assert L.hphi_add_hopping(h, 0, 1, 0, 1.0, 0.0) == -1      # hopping on a spin model
    assert L.hphi_set_basis(h, hp.BASIS_NUMBER, 1, 1) == -1    # spin models take FULL / SZ
    assert L.hphi_set_basis(h, hp.BASIS_SZ, 5, 0) == -1
    assert L.hphi_set_basis(h, hp.BASIS_SZ, 2, 0) == 0
    assert L.hphi_dim(h) == -4                                  # not built
    assert L.hphi_apply_H(h, None, None, 1, 0, None) == -4
    assert L.hphi_set_window_bits(h, -2) == -1                  # window size: -1, 0 or 1..32
    assert L.hphi_set_window_bits(h, 33) == -1
    assert L.hphi_set_window_bits(h, 6) == 0 and L.hphi_set_window_bits(h, -1) == 0
    assert L.hphi_set_window_bits(None, 6) == -1
    assert L.hphi_tpq_run(h, None, None, None) == -4            # not built before the arguments
    L.hphi_destroy(h)


def test_no_cpu_fallback_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(hp.LibraryError):
        hp.Model(hp.SPIN_HALF, 4).build()


def _header_struct_fields(name):
    """Field names of `typedef struct { ... } name;` in include/hphi_gpu.h, in order."""
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "hphi_gpu.h")).read(), flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", text)
    assert m, name
    body = m.group(1)
    out = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        field = re.search(r"([A-Za-z_][A-Za-z0-9_]*)\s*(\[[^\]]*\])?$", decl).group(1)
        out.append(field)
    return out


@pytest.mark.parametrize("cname,pyname", [
    ("hphi_lanczos_params", "LanczosParams"), ("hphi_lanczos_result", "LanczosResult"),
    ("hphi_tpq_params", "TpqParams"), ("hphi_tpq_result", "TpqResult"), ("hphi_tune_result", "TuneResult"),
    ("hphi_invit_params", "InvitParams"), ("hphi_invit_result", "InvitResult"),
])
def test_binding_structs_follow_header(cname, pyname):
    """The ctypes structures list the header's fields in the header's order."""
    import paper_1703_03637_gb300 as hp
    py = [f[0] for f in getattr(hp, pyname)._fields_]
    assert py == _header_struct_fields(cname)
