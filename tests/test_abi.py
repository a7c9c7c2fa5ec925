"""The C ABI library builds, loads without a GPU and exports every entry point
that include/h3d.h declares.  No compute call is made here."""
import ctypes
import os
import re

from paper_2307_16303_gb300 import api, build_ext

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "h3d.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(h3d_[a-z_A-Z0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    path = build_ext.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(api.EXPORTS) == names


def test_status_strings_and_defaults_without_gpu():
    build_ext.build()
    L = api.lib()
    assert L.h3d_status_string(0) == b"ok"
    assert b"domain" in L.h3d_status_string(2)
    opt = api.Options()
    L.h3d_default_options(ctypes.byref(opt))
    assert opt.precision == 2 and opt.rank_cap == 512 and opt.side == 2.0 and list(opt.lo) == [-1.0] * 3
    # argument validation happens before any device work
    h = ctypes.c_void_p()
    assert L.h3d_build(None, 10, 0, 64, 1e-7, None, None, ctypes.byref(h)) == 1
    assert L.h3d_matvec(None, None, None, 1, None) == 1
    assert L.h3d_free(None) == 0


def test_oracle_shares_nothing_with_the_cuda_path():
    # the oracle is C compiled by gcc from oracle/ only, and imports nothing from the package
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".c", ".py")):
            s = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_2307_16303_gb300" not in s and "csrc" not in s and "h3d.h" not in s
    for f in os.listdir(os.path.join(ROOT, "paper_2307_16303_gb300", "csrc")):
        s = open(os.path.join(ROOT, "paper_2307_16303_gb300", "csrc", f)).read()
        assert "oracle" not in s
    for f in ("api.py", "build_ext.py", "inputs.py", "__init__.py"):
        s = open(os.path.join(ROOT, "paper_2307_16303_gb300", f)).read()
        assert "import oracle" not in s and "from oracle" not in s


def test_new_entry_points_reject_bad_arguments_without_a_gpu():
    """Argument checks happen before any device work, so they run on the CPU."""
    import ctypes as C
    from paper_2307_16303_gb300 import api
    L = api.lib()
    d = C.c_double()
    assert L.h3d_energy(None, None, C.byref(d), None, None) == 1        # H3D_ERR_ARG
    assert L.h3d_forces(None, None, None, None, None) == 1
    out = C.c_void_p()
    assert L.h3d_batch_create(None, 0, C.byref(out)) == 1
    assert L.h3d_batch_matvec(None, None, None, None) == 1
    assert L.h3d_batch_configure(None, 1, 0, 0, 0, -1) == 1
    assert L.h3d_batch_info(None, None, None, None) == 1
    assert L.h3d_batch_free(None) == 0                                  # freeing nothing is fine
    assert L.h3d_import_pivots(None, None, None, None, None) == 1
    assert L.h3d_set_points(None, None, None) == 1
    assert L.h3d_batch_set_wait_limit(None, 10 ** 6) == 1
    n = C.c_int64()
    assert L.h3d_batch_get_queue(None, None, 0, C.byref(n)) == 1
    assert L.h3d_batch_set_queue(None, None, 0) == 1
    L.h3d_debug_fail_alloc(-1)                                          # switching the hook off is a no-op
