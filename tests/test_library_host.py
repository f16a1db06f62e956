"""Host-side checks of libhpsi: it loads, exports what include/hpsi.h declares, and its G-sphere
(a host-only entry point) equals the oracle's bit for bit.  No GPU needed."""
import os
import re

import numpy as np
import pytest

import oracle
import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    from paper_0906_2569_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    binding.load()
    return binding


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^HPSI_API\s+[\w\s\*]*?\b(\w+)\s*\(", src, flags=re.M)
    return names


def test_exports_every_declared_symbol(B):
    lib = B.load()
    names = declared_functions()
    assert len(names) >= 11
    for n in names:
        assert hasattr(lib, n), f"libhpsi.so does not export {n}"
    assert set(B.EXPORTS) <= set(names)


@pytest.mark.parametrize("cfg", ["c1", "c2", "c4a"])
def test_gsphere_bit_exact(B, cfg):
    p = workloads.CONFIGS[cfg]()
    for k in p.kpts[:4]:
        got = B.hpsi_gsphere(p.lattice, p.ecut, k)
        ref = oracle.gsphere.gsphere(p.lattice, p.ecut, k)
        assert got.dtype == np.int32 and np.array_equal(got, ref)


def test_gsphere_cells_and_oblique(B):
    for c in workloads.config4b()[:6]:
        assert np.array_equal(B.hpsi_gsphere(c.lattice, c.ecut, c.kpts[0]),
                              oracle.gsphere.gsphere(c.lattice, c.ecut, c.kpts[0]))
    lat = np.array([[6.0, 0.5, 0.0], [0.3, 7.0, 0.2], [0.0, -0.4, 8.0]])
    k = np.array([0.05, 0.1, -0.2])
    assert np.array_equal(B.hpsi_gsphere(lat, 3.5, k), oracle.gsphere.gsphere(lat, 3.5, k))


def test_gsphere_errors(B):
    with pytest.raises(B.HpsiError) as e:
        B.hpsi_gsphere(np.eye(3) * 10, -1.0, np.zeros(3))
    assert e.value.status == B.HPSI_EINVAL
    with pytest.raises(B.HpsiError):
        B.hpsi_gsphere(np.zeros((3, 3)), 1.0, np.zeros(3))
    with pytest.raises(B.HpsiError):
        B.hpsi_gsphere(np.eye(3) * 10, 1e9, np.zeros(3))


def test_binding_constants_match_header(B):
    """Every HPSI_* enumerator the binding names has the value include/hpsi.h gives it."""
    src = open(os.path.join(ROOT, "include", "hpsi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    declared = {n: int(v) for n, v in re.findall(r"\b(HPSI_[A-Z0-9_]+)\s*=\s*(-?\d+)", src)}
    named = [n for n in dir(B) if n.startswith("HPSI_OPT_") or n.startswith("HPSI_E")
             or n in ("HPSI_OK", "HPSI_FP64", "HPSI_MIXED")]
    assert len([n for n in named if n.startswith("HPSI_OPT_")]) >= 16
    for n in named:
        assert n in declared, f"{n} is not declared in hpsi.h"
        assert getattr(B, n) == declared[n], n


def test_every_declared_option_is_handled():
    """Each hpsi_option enumerator in hpsi.h has a branch in hpsi_set_option (static check of
    csrc/api.cu), so no declared option falls through to the 'unknown option' error."""
    src = open(os.path.join(ROOT, "include", "hpsi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = src[src.index("enum hpsi_option"):]
    body = body[:body.index("};")]
    opts = re.findall(r"\b(HPSI_OPT_[A-Z0-9_]+)\s*=", body)
    api = open(os.path.join(ROOT, "paper_0906_2569_gb300", "csrc", "api.cu")).read()
    assert len(opts) >= 18
    for o in opts:
        assert f"option == {o}" in api, f"{o} has no branch in hpsi_set_option"
