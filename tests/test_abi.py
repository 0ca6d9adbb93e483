"""CPU checks of the C ABI: the library loads, exports every entry point the
header declares, and rejects invalid arguments on the host (no GPU needed:
argument checking happens before any CUDA call), except the dose-rate
matrix, whose values the assembly kernel checks (one GPU test)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lgk():
    from paper_2509_08602_b300 import build
    build.build()
    from paper_2509_08602_b300 import lgk as mod
    return mod


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lgk_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol(lgk):
    lib = ctypes.CDLL(lgk._LIB_PATH)
    names = declared_functions()
    assert "lgk_create_case" in names and "lgk_solve_weightings" in names
    for n in names:
        assert hasattr(lib, n), n


def _tiny(nan=False, bad_kind=False, bad_target=False):
    phi = np.full((3, 24), 0.1)
    if nan:
        phi[1, 5] = np.nan
    kind = np.array([0, 1, 2 if not bad_kind else 9], np.uint8)
    sid = np.array([0, 0, 0 if not bad_target else 3], np.uint16)
    return phi, kind, sid


@pytest.mark.parametrize("kw", [dict(bad_kind=True), dict(bad_target=True)])
def test_create_case_rejects_bad_inputs(lgk, kw):
    phi, kind, sid = _tiny(**kw)
    with pytest.raises(lgk.LgkError) as e:
        lgk.create_case(phi, kind, sid, 1, [20.0], [1.0], [1.0], 10.0, 5.0, 3.0)
    assert e.value.code == 1


@pytest.mark.gpu
@pytest.mark.parametrize("bad", [np.nan, np.inf, -1e-3])
def test_create_case_rejects_bad_phi_on_the_device(lgk, bad):
    """phi (up to GBs) is validated by the assembly kernel, not by a host
    scan: a NaN, infinite or negative dose rate still gives LGK_EINVAL."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    phi, kind, sid = _tiny()
    phi[2, 17] = bad
    with pytest.raises(lgk.LgkError) as e:
        lgk.create_case(phi, kind, sid, 1, [20.0], [1.0], [1.0], 10.0, 5.0, 3.0)
    assert e.value.code == 1 and "phi" in str(e.value)
    lgk.create_case(*_tiny()[:3], 1, [20.0], [1.0], [1.0], 10.0, 5.0, 3.0).close()


def test_create_case_rejects_bad_thresholds(lgk):
    phi, kind, sid = _tiny()
    with pytest.raises(lgk.LgkError) as e:
        lgk.create_case(phi, kind, sid, 1, [0.0], [1.0], [1.0], 10.0, 5.0, 3.0)
    assert e.value.code == 1
    with pytest.raises(lgk.LgkError) as e:
        lgk.create_case(phi[:, :23], kind, sid, 1, [20.0], [1.0], [1.0], 10.0, 5.0, 3.0)
    assert e.value.code == 1


def test_default_params(lgk):
    p = lgk.default_params()
    assert p.precision == lgk.PREC_BF16X3 and p.check_every == 10 and p.normalize_rows == 1
    assert p.scale_bot == 1 and p.eps_abs == 1e-12 and p.hbm_budget == 0 and p.lo_refresh == 1
    assert p.lo_refresh_iters == 8000


def test_create_case_rejects_bad_params(lgk):
    phi, kind, sid = _tiny()
    for kw in (dict(lo_refresh=3), dict(lo_refresh_iters=-1), dict(check_every=0), dict(precision=7)):
        with pytest.raises(lgk.LgkError) as e:
            lgk.create_case(phi, kind, sid, 1, [20.0], [1.0], [1.0], 10.0, 5.0, 3.0,
                            params=lgk.default_params(**kw))
        assert e.value.code == 1, kw


def test_null_arguments_are_errors_not_crashes(lgk):
    lib = lgk._lib
    h = ctypes.c_void_p()
    assert lib.lgk_create_case(None, None, ctypes.byref(h)) == 1
    assert lib.lgk_solve_weightings(None, 1, None, None, 0.0, 0.0, 0.0, 1, ctypes.byref(h)) == 1
    assert lib.lgk_fetch_times(None, None, None) == 1
    assert lib.lgk_fetch_stats(None, None, None, None, None, None) == 1
    assert lib.lgk_default_params(None) == 1
    assert lib.lgk_fetch_metrics(None, None, 0, None, None, None, None, None) == 1
    assert lib.lgk_low_dose_volumes(None, None, 0, 0, None, None, None, None) == 1
    assert lib.lgk_two_pass(None, None, 1, None, 0.0, 0.0, 0.0, 1, None, None, ctypes.byref(h),
                            ctypes.byref(h), None, None) == 1
    assert lib.lgk_solve_weightings_masked(None, 1, None, None, 0.0, 0.0, 0.0, 1, None, None, None,
                                           ctypes.byref(h)) == 1
    assert lib.lgk_solve_stream(None, 1, None, None, 0.0, 0.0, 0.0, 1, 1, None, None, None, None, None,
                                None, None, None, None, None) == 1
    assert lib.lgk_fetch_check(None, None) == 1
    assert lib.lgk_solve_weightings_async(None, 1, None, None, 0.0, 0.0, 0.0, 1, ctypes.byref(h)) == 1
    assert lib.lgk_wait(None, 0) == 1
    outs = (ctypes.c_void_p * 4)()
    assert lib.lgk_solve_group(2, None, None, None, None, 0.0, None, 1e-4, 10, outs) == 1
    assert lib.lgk_solve_group(0, None, None, None, None, 0.0, None, 1e-4, 10, outs) == 1
    assert lib.lgk_solve_group(5, None, None, None, None, 0.0, None, 1e-4, 10, outs) == 1
    assert lib.lgk_solve_group(1, None, None, None, None, 0.0, None, 1e-4, 10, None) == 1
    cid = ctypes.c_longlong()
    assert lib.lgk_server_open(None, None, ctypes.byref(cid)) == 1
    assert lib.lgk_server_submit_to(None, 0, 1, None, ctypes.byref(cid)) == 1
    assert lib.lgk_server_close(None, 0) == 1
    lib.lgk_free_result(None)
    lib.lgk_destroy_case(None)
    assert b"NULL" in lib.lgk_last_error() or len(lib.lgk_last_error()) > 0


def test_header_is_plain_c(tmp_path):
    """The boundary is a C ABI: include/lgk.h compiles as C99 on its own
    (no C++ or CUDA types in the declarations)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_lgk.c"
    src.write_text('#include "lgk.h"\n'
                   "int main(void) { lgk_params p; return lgk_default_params(&p); }\n")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-fsyntax-only", "-I",
                        os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
