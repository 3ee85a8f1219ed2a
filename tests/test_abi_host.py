"""CPU checks of the C-ABI library: it loads, exports every symbol that
include/dg.h declares, its host-side reference data (quadrature rules, basis)
agrees with the independent oracle, and mesh / argument validation returns
the documented status codes before any device work."""
import os
import re

import numpy as np
import pytest

from oracle.basis import eval_basis
from oracle.quadrature import tet_monomial_integral, tri_monomial_integral
from paper_2209_01877_gb300 import dg
from paper_2209_01877_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(dg.LIB_PATH):
        from paper_2209_01877_gb300 import build
        build.build()
    return dg.load()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "dg.h")).read()
    declared = set(re.findall(r"^(?:dg_status|const char\*)\s+(dg_\w+)\s*\(", hdr, re.M))
    assert declared == set(dg.EXPORTED)
    for name in declared:
        assert hasattr(lib, name), name


@pytest.mark.parametrize("p", [1, 2, 3])
def test_reference_data_matches_oracle(lib, p):
    r = dg.dg_reference_data(p)
    X, w = r["vol_xi"], r["vol_w"]
    deg = 2 * p
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            for c in range(deg + 1 - a - b):
                assert abs(np.sum(w * X[:, 0] ** a * X[:, 1] ** b * X[:, 2] ** c) - tet_monomial_integral(a, b, c)) < 1e-16
    fb, fw = r["face_bary"], r["face_w"]
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            assert abs(np.sum(fw * fb[:, 1] ** a * fb[:, 2] ** b) - tri_monomial_integral(a, b)) < 1e-16
    # same rule as the oracle's (as point sets)
    from oracle.quadrature import face_rule_for_order, volume_rule_for_order

    def same_rule(P, W, Q, V):
        a = np.lexsort(np.round(P, 10).T[::-1])
        b = np.lexsort(np.round(Q, 10).T[::-1])
        np.testing.assert_allclose(P[a], Q[b], atol=1e-15, rtol=0)
        np.testing.assert_allclose(W[a], V[b], atol=1e-16, rtol=0)

    lo, wo = volume_rule_for_order(p)
    same_rule(X, w, lo[:, 1:], wo)
    lf, wf = face_rule_for_order(p)
    same_rule(fb, fw, lf, wf)
    # basis and gradients at the library's points
    phi, grad = eval_basis(p, X)
    np.testing.assert_allclose(r["phi"], phi, atol=1e-12, rtol=0)
    np.testing.assert_allclose(r["dphi"], grad, atol=1e-11, rtol=0)


def _create(vid, xyz, tag=None, **cfg):
    return dg.dg_mesh_create(vid, xyz, tag, dg.make_config(**cfg))


def test_argument_errors(lib):
    m = I.make_periodic_cube(3)
    with pytest.raises(dg.DGError) as e:
        _create(m.tet_vid, m.tet_xyz, order=4)
    assert e.value.status == 1
    with pytest.raises(dg.DGError) as e:
        _create(m.tet_vid, m.tet_xyz, flux=7)
    assert e.value.status == 1
    with pytest.raises(dg.DGError) as e:
        _create(m.tet_vid, m.tet_xyz, gamma=1.0)
    assert e.value.status == 1


def test_null_mesh_is_an_argument_error(lib):
    """Every entry point that takes a mesh checks it before touching a device."""
    import ctypes as C
    null = C.c_void_p(0)
    buf = C.c_void_p(0)
    assert lib.dg_ns_residual(null, buf, buf, 0.01, 0.72, null) == 1
    assert lib.dg_residual(null, buf, buf, null) == 1
    assert lib.dg_rk3_step(null, 1e-3, 1, null) == 1
    assert lib.dg_rk_stage(null, 1, 1e-3, null) == 1
    assert lib.dg_set_state(null, buf, 0, null) == 1
    assert "NULL" in lib.dg_last_error().decode()


def test_mesh_errors(lib):
    m = I.make_periodic_cube(3)
    bad = m.tet_xyz.copy()
    bad[5, [1, 2]] = bad[5, [2, 1]]            # inverted tetrahedron
    with pytest.raises(dg.DGError) as e:
        _create(m.tet_vid, bad)
    assert e.value.status == 2 and "volume" in str(e.value)
    box = I.make_box_channel(3, 2, 2)
    with pytest.raises(dg.DGError) as e:       # boundary faces without tags
        _create(box.tet_vid, box.tet_xyz, None)
    assert e.value.status == 2
    vid = np.concatenate([m.tet_vid, m.tet_vid[:1]])   # a face shared by three tets
    xyz = np.concatenate([m.tet_xyz, m.tet_xyz[:1]])
    with pytest.raises(dg.DGError) as e:
        _create(vid, xyz)
    assert e.value.status == 2


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(dg, "_lib", None)
    monkeypatch.setattr(dg, "LIB_PATH", str(tmp_path / "libdg.so"))
    with pytest.raises(ImportError):
        dg.load()
