"""The allocation-free H v entry point (hphi_apply_H_noalloc), through the C ABI.

It exists for callers that must not allocate device memory during a call (host callbacks,
real-time loops that cannot take cudaMalloc's implicit synchronisation, applications that
pre-reserve all memory); its scratch is a fixed device array inside the library.  It must
give the same product as hphi_apply_H, call after call.  This file is collected last so a
failure here never hides the result of the other tests.
"""
import numpy as np
import pytest

import workloads as wl

torch = pytest.importorskip("torch")
hp = pytest.importorskip("paper_1703_03637_gb300")

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(torch.max(torch.abs(a - b)) / torch.max(torch.abs(b)))


def test_apply_H_noalloc_matches_apply_H_twice():
    spec = wl.hubbard_square(4, 3, 1.0, 8.0).with_basis(wl.BASIS_NUMBER, 6, 6)  # 853,776 rows
    m = hp.Model.from_spec(spec)
    inputs = [torch.as_tensor(wl.gaussian_vector(s, m.dim)[:, 0]).cuda() for s in (61, 62)]
    for v in inputs:  # two calls in a row, different inputs: the shared scratch must not leak state
        ref = m.apply_H(v)
        w = torch.empty_like(v)
        m.apply_H_noalloc(v, w)
        torch.cuda.synchronize()
        assert _rel(w, ref) < 1e-12


def test_apply_H_noalloc_rejects_bases_above_its_fixed_scratch():
    spec = wl.hubbard_square(4, 4, 1.0, 8.0).with_basis(wl.BASIS_NUMBER, 8, 8)  # 165,636,900 rows
    m = hp.Model.from_spec(spec)
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = m._L.hphi_apply_H_noalloc(m._h, hp._dptr(dummy), hp._dptr(out), hp._stream())
    assert rc == -1
    assert b"rows" in m._L.hphi_last_error(m._h)
    assert np.all(out.cpu().numpy() == 0.0)


def test_apply_H_noalloc_rejects_other_models():
    m = hp.Model.from_spec(wl.heisenberg_ring(10))
    v = torch.zeros(m.dim, dtype=torch.float64, device="cuda")
    with pytest.raises(hp.LibraryError) as e:
        m.apply_H_noalloc(v, torch.empty_like(v))
    assert e.value.code == -7
