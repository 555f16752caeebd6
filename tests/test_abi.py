"""The C-ABI library builds, loads and exports every entry point include/psvd.h declares;
host-only logic (defaults, status strings, argument validation, workspace sizing) is
exercised without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(psvd_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    import paper_2609_32505_gb300 as P
    P.build()
    return P.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 12
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_defaults_and_status(lib):
    import paper_2609_32505_gb300 as P
    o = P.Opts()
    lib.psvd_default_opts(ctypes.byref(o))
    assert (o.precision, o.schedule, o.pre_iters, o.max_iter) == (0, 0, 2, 50)
    assert abs(o.delta - 0.99) < 1e-15 and abs(o.tol - 1e-5) < 1e-20 and abs(o.eps_qr - 1e-5) < 1e-20
    for code in (0, 1, -1, -2, -3, -4, -5, -6):
        assert lib.psvd_status_string(code)


def test_argument_errors_before_any_device_call(lib):
    import paper_2609_32505_gb300 as P
    o = P.Opts()
    lib.psvd_default_opts(ctypes.byref(o))
    fake = ctypes.c_void_p(0x1000)
    # m < n, null pointers, bad batch: rejected on the host
    assert lib.psvd_svd_fwd(fake, fake, fake, fake, 1, 4, 8, ctypes.byref(o), fake, 1 << 30, None, None) == -1
    assert lib.psvd_svd_fwd(None, fake, fake, fake, 1, 8, 4, ctypes.byref(o), fake, 1 << 30, None, None) == -1
    assert lib.psvd_polar_fwd(fake, fake, None, 0, 8, 4, ctypes.byref(o), fake, 1 << 30, None, None) == -1
    assert lib.psvd_svd_bwd(fake, fake, fake, fake, None, None, None, fake, 1, 8, 4, 1e-8, 3, fake, 1 << 30,
                            None) == -1
    assert lib.psvd_svd_bwd(fake, fake, fake, fake, None, None, None, fake, 1, 8, 4, 0.0, 0, fake, 1 << 30,
                            None) == -1
    assert lib.psvd_gemm_tn(fake, fake, fake, 1, 4, 4, 4, 7, fake, 1 << 30, None) == -1
    # learned schedule without bounds
    o.schedule = 1
    assert lib.psvd_polar_fwd(fake, fake, None, 1, 8, 4, ctypes.byref(o), fake, 1 << 30, None, None) == -1


def test_workspace_queries_scale(lib):
    import paper_2609_32505_gb300 as P
    o = P.Opts()
    lib.psvd_default_opts(ctypes.byref(o))
    a = lib.psvd_svd_workspace_bytes(1, 256, 256, ctypes.byref(o))
    b = lib.psvd_svd_workspace_bytes(2, 256, 256, ctypes.byref(o))
    assert 0 < a < b
    o.precision = 1
    assert lib.psvd_polar_workspace_bytes(1, 256, 256, ctypes.byref(o)) > \
        lib.psvd_polar_workspace_bytes(1, 256, 200, ctypes.byref(o))
    assert lib.psvd_svd_bwd_workspace_bytes(1, 300, 200) > 0
    assert lib.psvd_eigh_workspace_bytes(3, 100) > lib.psvd_eigh_workspace_bytes(1, 100)
    assert lib.psvd_svd_workspace_bytes(0, 4, 4, ctypes.byref(o)) == 0


def _header():
    txt = open(os.path.join(ROOT, "include", "psvd.h")).read()
    defines = {k: float(v) for k, v in re.findall(r"#define\s+(PSVD_[A-Z0-9_]+)\s+(-?[0-9.eE+-]+)\b", txt)}
    body = re.search(r"typedef struct psvd_info \{(.*?)\} psvd_info;", txt, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(int|float)\s+([a-z0-9_]+)\s*;", body)
    return defines, fields


def test_python_mirrors_of_header_constants():
    # the binding's copies of the header's codes and thresholds, and the psvd_info layout
    # the binding decodes (its int fields first, then its float fields)
    import paper_2609_32505_gb300 as P
    d, fields = _header()
    assert (P.PREC_FP32, P.PREC_MIXED, P.PREC_MIXED_BF16) == (d["PSVD_PREC_FP32"], d["PSVD_PREC_MIXED"],
                                                              d["PSVD_PREC_MIXED_BF16"])
    assert (P.SCHED_CANS, P.SCHED_LEARNED, P.SCHED_NS, P.SCHED_PE) == (
        d["PSVD_SCHED_CANS"], d["PSVD_SCHED_LEARNED"], d["PSVD_SCHED_NS"], d["PSVD_SCHED_PE"])
    assert P.MIXED_CORR_MAX == d["PSVD_MIXED_CORR_MAX"]
    assert P.MIXED_RECON_MAX == d["PSVD_MIXED_RECON_MAX"]
    assert P.MIXED_LB_MIN == d["PSVD_MIXED_LB_MIN"]
    assert [name for _, name in fields] == P.INFO_FIELDS
    assert [t for t, _ in fields] == ["int"] * P.INFO_INTS + ["float"] * (P.INFO_WORDS - P.INFO_INTS)


def test_python_opts_mirror_header_struct():
    # the binding's ctypes psvd_opts: same fields, same order, same C types as the header
    import paper_2609_32505_gb300 as P
    txt = open(os.path.join(ROOT, "include", "psvd.h")).read()
    body = re.search(r"typedef struct psvd_opts \{(.*?)\} psvd_opts;", txt, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(int|double|const float)\s*(\*?)\s*([a-z0-9_]+)\s*;", body)
    names = [n for _, _, n in fields]
    assert names == [f for f, _ in P.Opts._fields_]
    kinds = {"int": ctypes.c_int, "double": ctypes.c_double}
    for (t, star, name), (fname, ct) in zip(fields, P.Opts._fields_):
        assert ct is (ctypes.c_void_p if star else kinds[t]), name
