"""The C ABI library loads and exports every entry point that include/pcamg.h
declares (no GPU needed: nothing here launches a kernel)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pcamg.h")).read()
    return sorted(set(re.findall(r"PCAMG_API\s+[\w\s\*]*?\b(pcamg_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    from paper_1806_07028_gb300.build import build
    return build()


def test_every_declared_symbol_is_exported(built):
    names = _declared()
    assert len(names) >= 20
    lib = C.CDLL(built)
    for nm in names:
        assert hasattr(lib, nm), nm
    from paper_1806_07028_gb300 import native as N
    assert sorted(N.EXPORTS) == names


def test_default_params_follow_section4(built):
    from paper_1806_07028_gb300 import default_params, native as N
    p = default_params()
    assert (p.tol, p.threshold, p.numW, p.iterW, p.iterV) == (1e-8, 0.4, 2, 7, 4)
    assert p.precision == N.FP64 and p.p1_mode == N.P1_E_SCALED
    assert N.status_name(N.ERR_NOT_LAPLACIAN) == "NOT_LAPLACIAN"


def test_null_arguments_are_rejected_without_gpu(built):
    from paper_1806_07028_gb300 import native as N
    L = N.lib()
    h = C.c_void_p()
    assert L.pcamg_setup(C.byref(h), None, 10, 30, None, None, None, None, None) == N.ERR_INVALID
    assert L.pcamg_adapt(None, None) == N.ERR_INVALID
    assert L.pcamg_solve(None, None, None, None) == N.ERR_INVALID
    assert L.pcamg_num_hierarchies(None) == -1
    assert b"null" in L.pcamg_last_error(None)


def test_struct_layout_matches_header(built):
    from paper_1806_07028_gb300 import native as N
    src = open(os.path.join(ROOT, "include", "pcamg.h")).read()
    body = re.search(r"typedef struct \{(.*?)\} pcamg_params;", src, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(?:double|int32_t|uint64_t|pcamg_mpnn)\s+([\w\s,]+);", body)
    names = [f.strip() for grp in fields for f in grp.split(",")]
    assert names == [f for f, _ in N.Params._fields_]


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # no CPU fallback: without the built library the first call raises
    from paper_1806_07028_gb300 import native as N
    monkeypatch.setattr(N, "LIB_PATH", str(tmp_path / "libpcamg.so"))
    monkeypatch.setattr(N, "_lib", None)
    with pytest.raises(N.NativeLibraryMissing):
        N.lib()
    from paper_1806_07028_gb300 import solver
    with pytest.raises(N.NativeLibraryMissing):
        solver.default_params()
