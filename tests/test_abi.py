"""CPU checks of the boundary: the library builds, loads, and exports every
entry point include/dcg.h declares; the binding declares each of them."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\**(dcg_\w+)\s*\(", src, flags=re.M))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_1706_00241_gb300 import build
    return build.build()


def test_header_declares_core_calls():
    names = _declared()
    for core in ("dcg_create", "dcg_solve", "dcg_update_subspace", "dcg_destroy",
                 "dcg_set_operator_dense", "dcg_set_subspace", "dcg_get_subspace"):
        assert core in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header(lib_path):
    from paper_1706_00241_gb300 import _lib
    assert set(_lib.SIGNATURES) == _declared()
    lib = _lib.load()
    assert lib.dcg_status_string(0) == b"ok"
    assert b"breakdown" in lib.dcg_status_string(4)


def test_config_struct_layout():
    from paper_1706_00241_gb300 import _lib
    # int64 n, twelve int32 fields, int32 reserved[4], then a double: 8 + 64 + 8
    assert ctypes.sizeof(_lib.DcgConfig) == 80
    assert _lib.DcgConfig.extraction.offset == 48
    assert _lib.DcgConfig.fg_form.offset == 52
    assert _lib.DcgConfig.tol.offset == 72
    assert ctypes.sizeof(_lib.DcgSolveInfo) == 64


def test_create_rejects_bad_config_without_gpu(lib_path):
    # argument validation happens before any CUDA call
    from paper_1706_00241_gb300 import _lib
    lib = _lib.load()
    cfg = _lib.DcgConfig()
    cfg.n = 0
    cfg.max_iter = 10
    cfg.tol = 1e-6
    ctx = ctypes.c_void_p()
    assert lib.dcg_create(ctypes.byref(cfg), None, ctypes.byref(ctx)) == 1
    assert b"n out of range" in lib.dcg_last_error(None)
    cfg.n = 10
    cfg.tol = 0.0
    assert lib.dcg_create(ctypes.byref(cfg), None, ctypes.byref(ctx)) == 1
    cfg.tol = 1e-6
    cfg.k = 200
    assert lib.dcg_create(ctypes.byref(cfg), None, ctypes.byref(ctx)) in (1, 9)


def test_create_reports_build_limits_without_gpu(lib_path):
    # k <= 96 and ell <= 128 in this build (UNSUPPORTED = 9), checked before
    # any allocation; k > n stays an argument error (INVALID_ARG = 1)
    from paper_1706_00241_gb300 import _lib
    lib = _lib.load()
    cfg = _lib.DcgConfig()
    cfg.n = 1000
    cfg.max_iter = 10
    cfg.tol = 1e-6
    cfg.window = 1
    ctx = ctypes.c_void_p()
    cfg.k, cfg.ell = 97, 32
    assert lib.dcg_create(ctypes.byref(cfg), None, ctypes.byref(ctx)) == 9
    assert b"k <= 96" in lib.dcg_last_error(None)
    cfg.k, cfg.ell = 32, 129
    assert lib.dcg_create(ctypes.byref(cfg), None, ctypes.byref(ctx)) == 9
    cfg.n, cfg.k, cfg.ell = 20, 21, 4
    assert lib.dcg_create(ctypes.byref(cfg), None, ctypes.byref(ctx)) == 1
    assert not ctx.value


def test_create_rejects_unknown_extraction_without_gpu(lib_path):
    from paper_1706_00241_gb300 import _lib
    lib = _lib.load()
    cfg = _lib.DcgConfig()
    cfg.n, cfg.k, cfg.ell, cfg.max_iter, cfg.tol = 100, 4, 8, 10, 1e-6
    ctx = ctypes.c_void_p()
    cfg.extraction = 2
    assert lib.dcg_create(ctypes.byref(cfg), None, ctypes.byref(ctx)) == 1
    assert b"bad extraction" in lib.dcg_last_error(None)
    cfg.extraction = 0
    cfg.fg_form = 2
    assert lib.dcg_create(ctypes.byref(cfg), None, ctypes.byref(ctx)) == 1
    assert b"bad fg_form" in lib.dcg_last_error(None)
    cfg.fg_form, cfg.extraction = 1, 1
    assert lib.dcg_create(ctypes.byref(cfg), None, ctypes.byref(ctx)) == 1
    assert b"harmonic" in lib.dcg_last_error(None)
    cfg.fg_form, cfg.extraction = 0, 0
    cfg.reserved[3] = 1
    assert lib.dcg_create(ctypes.byref(cfg), None, ctypes.byref(ctx)) == 1
    assert b"reserved" in lib.dcg_last_error(None)
    assert not ctx.value


def test_form_rbf_dense_rejects_bad_arguments_with_a_message(lib_path):
    # every case fails the argument checks, which run before any CUDA call, so
    # the placeholder addresses are never dereferenced
    from paper_1706_00241_gb300 import _lib
    lib = _lib.load()
    P = ctypes.c_void_p
    fake = P(0x1000)
    cases = [
        ((None, 16, 4, 1.0, 1.0, 0.1, fake, 16, None), b"X and A are required"),
        ((fake, 0, 4, 1.0, 1.0, 0.1, fake, 16, None), b"lda >= n"),
        ((fake, 16, 4, 1.0, 1.0, 0.1, fake, 8, None), b"lda >= n"),
        ((fake, 16, 0, 1.0, 1.0, 0.1, fake, 16, None), b"d must be in [1, 4096]"),
        ((fake, 16, 4, -1.0, 1.0, 0.1, fake, 16, None), b"lengthscale > 0"),
        ((fake, 16, 4, 1.0, float("nan"), 0.1, fake, 16, None), b"finite"),
    ]
    for args, msg in cases:
        assert lib.dcg_form_rbf_dense(*args) == 1, args
        assert msg in lib.dcg_last_error(None), (args, lib.dcg_last_error(None))


def test_context_free_error_message_is_per_thread(lib_path):
    # a failing dcg_create on another host thread leaves this thread's message
    import threading
    from paper_1706_00241_gb300 import _lib
    lib = _lib.load()
    cfg = _lib.DcgConfig()
    cfg.n, cfg.max_iter, cfg.tol = 10, 10, 0.0
    ctx = ctypes.c_void_p()
    assert lib.dcg_create(ctypes.byref(cfg), None, ctypes.byref(ctx)) == 1
    assert b"tol must be > 0" in lib.dcg_last_error(None)
    other = []

    def worker():
        c2 = _lib.DcgConfig()
        c2.n, c2.max_iter, c2.tol = 0, 10, 1e-6
        lib.dcg_create(ctypes.byref(c2), None, ctypes.byref(ctypes.c_void_p()))
        other.append(lib.dcg_last_error(None))

    t = threading.Thread(target=worker)
    t.start()
    t.join()
    assert b"n out of range" in other[0]
    assert b"tol must be > 0" in lib.dcg_last_error(None)


def test_header_is_plain_c_and_links(lib_path, tmp_path):
    # the boundary is a C ABI: a C99 translation unit that includes the header
    # and references the core calls compiles with gcc and links against the
    # library (it is not run: no GPU is needed)
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not available")
    src = tmp_path / "use_dcg.c"
    src.write_text(
        '#include "dcg.h"\n'
        "#include <stddef.h>\n"
        "/* the ctypes binding's offsets, checked at compile time */\n"
        "typedef char extraction_at_48[offsetof(dcg_config, extraction) == 48 ? 1 : -1];\n"
        "typedef char tol_at_72[offsetof(dcg_config, tol) == 72 ? 1 : -1];\n"
        "typedef char config_is_80[sizeof(dcg_config) == 80 ? 1 : -1];\n"
        "int main(void) {\n"
        "  dcg_config cfg = {0};\n"
        "  dcg_ctx* ctx = NULL;\n"
        "  cfg.n = 16; cfg.k = 2; cfg.ell = 4; cfg.max_iter = 10; cfg.tol = 1e-6;\n"
        "  dcg_status s = dcg_create(&cfg, NULL, &ctx);\n"
        "  if (s == DCG_OK) {\n"
        "    dcg_solve_info info;\n"
        "    (void)dcg_solve(ctx, NULL, NULL, &info);\n"
        "    (void)dcg_update_subspace(ctx, NULL);\n"
        "    (void)dcg_destroy(ctx);\n"
        "  }\n"
        "  return (int)s;\n"
        "}\n")
    exe = tmp_path / "use_dcg"
    libdir = os.path.dirname(lib_path)
    libname = os.path.basename(lib_path)
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-o", str(exe), os.path.join(libdir, libname), f"-Wl,-rpath,{libdir}"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_library_resolves_every_symbol_at_load(lib_path):
    # RTLD_NOW binds every undefined symbol when the library loads (lazy
    # binding would defer a missing one to its first call on a GPU machine)
    import ctypes
    ctypes.CDLL(lib_path, mode=os.RTLD_NOW)
