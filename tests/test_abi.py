"""The C-ABI library loads and exports every entry point include/deconv.h
declares, and host-side validation rejects bad arguments before touching a
GPU (no device calls here)."""
import ctypes
import os
import re

import pytest

import paper_1602_01410_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1602_01410_gb300 import build
    build.build()
    return pkg.load()


def declared():
    txt = open(os.path.join(ROOT, "include", "deconv.h")).read()
    return sorted(set(re.findall(r"^\s*(?:deconv_status|const char \*)\s*(deconv_\w+)\s*\(", txt, re.M)))


def test_header_declares_expected_entry_points():
    names = declared()
    assert set(pkg.EXPORTS) == set(names)


def test_library_exports_every_declared_symbol(lib):
    for name in declared():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    assert pkg.deconv_status_string(0) == "ok"
    assert "workspace" in pkg.deconv_status_string(pkg.DECONV_ENOMEM)


def size(rows, cols, K, **kw):
    d, keep = pkg.make_dims(rows, cols, K, **kw)
    n = ctypes.c_size_t(0)
    st = pkg.load().deconv_workspace_size(ctypes.byref(d), ctypes.byref(n))
    return st, n.value


def test_workspace_size_validation(lib):
    st, n = size([1024], [1024], 21)
    assert st == 0 and n > 1024 * 1024 * 4 * 8
    assert size([64], [64], 8)[0] == pkg.DECONV_EINVAL           # even kernel (Sec. I-A: (2b+1)^2 support)
    assert size([64], [7 * 16], 5)[0] == pkg.DECONV_EUNSUPPORTED  # prime factor 7
    assert size([4], [64], 5)[0] == pkg.DECONV_EINVAL             # grid smaller than the kernel
    assert size([64], [64], 5, channels=2)[0] == pkg.DECONV_EINVAL
    assert size([64], [64], 5, relax=2.5)[0] == pkg.DECONV_EINVAL
    assert size([64], [64], 5, dtype=7)[0] == pkg.DECONV_EINVAL


def test_workspace_grows_with_batch_and_precision(lib):
    a = size([256], [256], 9)[1]
    b = size([256, 256], [256, 256], 9)[1]
    c = size([256], [256], 9, dtype=pkg.DECONV_F64)[1]
    assert b > a and c > a


def test_plan_create_rejects_bad_scalars_without_a_gpu(lib):
    d, keep = pkg.make_dims([64], [64], 5)
    plan = ctypes.c_void_p()
    fake = 256  # never dereferenced: validation fails first
    for lam, mu in ((-1.0, 1e-3), (1e-3, 0.0), (float("nan"), 1e-3)):
        st = lib.deconv_plan_create(ctypes.byref(plan), ctypes.byref(d), fake, fake, lam, mu, fake, 1 << 30, None)
        assert st == pkg.DECONV_EINVAL
    st = lib.deconv_plan_create(ctypes.byref(plan), ctypes.byref(d), fake, fake, 1e-3, 1e-3, fake + 1, 1 << 30, None)
    assert st == pkg.DECONV_EINVAL  # misaligned workspace
    st = lib.deconv_plan_create(ctypes.byref(plan), ctypes.byref(d), fake, fake, 1e-3, 1e-3, fake, 16, None)
    assert st == pkg.DECONV_ENOMEM


def test_solve_rejects_null_plan(lib):
    assert lib.deconv_solve(None, None, None, 1, 0, None) == pkg.DECONV_EINVAL
    assert lib.deconv_plan_destroy(None) == pkg.DECONV_EINVAL


def test_header_is_plain_c(tmp_path):
    # The boundary is a C ABI: the header compiles as C99 and C11 with every
    # warning an error, and a C caller can take the address of each entry point.
    import subprocess
    names = declared()
    src = tmp_path / "use.c"
    src.write_text('#include "deconv.h"\ntypedef void (*entry)(void);\nentry entry_points[] = {\n' +
                   "".join(f"  (entry){n},\n" for n in names) + "};\n")
    for std in ("c99", "c11"):
        r = subprocess.run(["gcc", f"-std={std}", "-Wall", "-Wextra", "-Werror", "-pedantic-errors",
                            "-Wno-cast-function-type", "-I", os.path.join(ROOT, "include"), "-c", str(src),
                            "-o", str(tmp_path / f"use_{std}.o")], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
