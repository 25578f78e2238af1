"""The C-ABI library loads, exports every declared symbol, and its host-only logic is right (CPU)."""
import os

import numpy as np
import pytest

from paper_2205_06690_gb300 import binding as B
from oracle import tdh


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(B.LIB_PATH):
        from paper_2205_06690_gb300 import build
        build.build()
    return B.load()


def test_every_declared_symbol_is_exported(lib):
    names = B.header_symbols()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


@pytest.mark.parametrize("dist", [B.SBSE_COEFF_SIGN, B.SBSE_COEFF_GAUSSIAN])
def test_library_coefficients_match_oracle_generator(lib, dist):
    """Both sides implement the splitmix64 stream of Eq. (14)'s coefficients independently."""
    name = "sign" if dist == B.SBSE_COEFF_SIGN else "gaussian"
    for seed in (0, 1, 2**63 + 12345):
        got = B.sbse_coefficients(seed, 10, 37, dist)
        ref = tdh.stochastic_coefficients(seed, 10, 37, name)
        if dist == B.SBSE_COEFF_SIGN:
            assert np.array_equal(got, ref)
        else:
            assert np.max(np.abs(got - ref)) <= 4e-15 * np.max(np.abs(ref))


def test_host_side_argument_errors(lib):
    out = np.empty(4)
    assert lib.sbse_coefficients(0, 0, 4, 0, B._dptr(out)) == B.SBSE_ERR_INVALID_ARG
    assert lib.sbse_coefficients(0, 2, 2, 7, B._dptr(out)) == B.SBSE_ERR_INVALID_ARG
    assert lib.sbse_create(None, 0, 0) == B.SBSE_ERR_INVALID_ARG
    import ctypes as C
    h = C.c_void_p()
    assert lib.sbse_create(C.byref(h), 0, 5) == B.SBSE_ERR_INVALID_ARG
    assert "precision" in B.sbse_last_error(None)
    assert lib.sbse_set_grid(None, 16, 8.0, None) == B.SBSE_ERR_INVALID_ARG
    assert lib.sbse_apply_W(None, None, 0, None, None, None, None) == B.SBSE_ERR_INVALID_ARG
    lib.sbse_destroy(None)


def test_header_is_plain_c(tmp_path):
    """include/sbse.h compiles as C99 (no C++ types cross the boundary) and as C++."""
    import shutil
    import subprocess
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "use.c"
    src.write_text('#include "sbse.h"\nint main(void) { sbse_ctx *c = 0; (void)c; return 0; }\n')
    for lang in (["-std=c99", "-x", "c"], ["-std=c++17", "-x", "c++"]):
        r = subprocess.run([cc, *lang, "-Wall", "-Werror", "-I", os.path.join(root, "include"), "-c", str(src),
                            "-o", str(tmp_path / "use.o")], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_release_build_has_no_debug_bounds_checks():
    """The release library reports that it carries no device-side bounds checks (the call needs no
    GPU: the release build registers no records to read)."""
    from paper_2205_06690_gb300 import binding as B
    if B.LIB_PATH.endswith("libsbse_dbg.so"):
        pytest.skip("the debug build is loaded")
    assert B.sbse_debug_bounds() == (False, 0)
