"""The C ABI library loads on the host and exports every entry point that include/fthms.h declares
(no compute calls: those need a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built_library():
    """Build libfthms.so (nvcc cross-compiles for sm_103a without a GPU) if this checkout has none."""
    lib = os.path.join(ROOT, "paper_2507_05725_gb300", "lib", "libfthms.so")
    if not os.path.exists(lib):
        from paper_2507_05725_gb300.build import build
        build()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "fthms.h")).read()
    return sorted(set(re.findall(r"^\s*(?:fthms_status|const char\*)\s+(fthms_\w+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ["fthms_create", "fthms_destroy", "fthms_submit", "fthms_poll", "fthms_wait", "fthms_traces",
              "fthms_densities", "fthms_stats", "fthms_release", "fthms_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2507_05725_gb300 import fthms as F
    for n in declared_symbols():
        assert hasattr(F.LIB, n), n
        assert n in F.EXPORTED, n


def test_host_validation_without_gpu():
    """Argument checks run before any device call."""
    import ctypes as C

    from paper_2507_05725_gb300 import fthms as F
    assert F.LIB.fthms_create(None, 0, 0, None) == F.FTHMS_EINVAL
    assert "NULL" in F.fthms_last_error()
    assert F.LIB.fthms_bessel0(None, None, None, None, -1, None) == F.FTHMS_EINVAL
    assert F.LIB.fthms_release(None) == F.FTHMS_EINVAL
    assert F.LIB.fthms_wait(None, 0) == F.FTHMS_EINVAL
    assert F.LIB.fthms_set_shapes(None, None) == F.FTHMS_EINVAL
    d = C.c_int()
    assert F.LIB.fthms_poll(None, C.byref(d)) == F.FTHMS_EINVAL


def test_header_is_plain_c(tmp_path):
    """The boundary is a C ABI: include/fthms.h compiles as C11 on its own (no C++ or CUDA types), and a C
    program that calls every declared entry point links against the library."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_abi.c"
    calls = "\n".join(f"  (void)&{n};" for n in declared_symbols())
    src.write_text('#include "fthms.h"\nint main(void) {\n' + calls + "\n  return 0;\n}\n")
    lib_dir = os.path.join(ROOT, "paper_2507_05725_gb300", "lib")
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                        str(src), "-L", lib_dir, "-lfthms", "-o", str(tmp_path / "use_abi")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
