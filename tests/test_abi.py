"""CPU-side checks of the C ABI: the library builds, loads, and exports every
function that include/*.h declares.  No compute call is made (no GPU here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(mmf_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_cs_0610046_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_entry_points():
    names = _declared()
    for required in ("mmf_filter1d", "mmf_filter1d_ex", "mmf_last_error", "mmf_device_status"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_host_only_calls(lib):
    lib.mmf_output_length.restype = ctypes.c_int64
    lib.mmf_output_length.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int]
    assert lib.mmf_output_length(10, 3, 0) == 8
    assert lib.mmf_output_length(10, 11, 0) == 0
    assert lib.mmf_output_length(10, 0, 0) == -1
    assert lib.mmf_output_length(10, 4, 1) == 10
    assert lib.mmf_output_length(-1, 4, 1) == -1
    lib.mmf_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.mmf_version()


def test_argument_errors_need_no_gpu(lib):
    """Invalid arguments are rejected before any CUDA call."""
    f = lib.mmf_filter1d
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    lib.mmf_last_error.restype = ctypes.c_char_p
    assert f(16, 10, 3, 0, 0, None, None, None) == 1            # both outputs NULL
    assert f(None, 10, 3, 0, 0, 16, None, None) == 1            # NULL input, n > 0
    assert f(16, 10, 0, 0, 0, 16, None, None) == 1              # w < 1
    assert f(16, -1, 3, 0, 0, 16, None, None) == 1              # n < 0
    assert f(16, 10, 3, 9, 0, 16, None, None) == 1              # bad dtype
    assert f(16, 10, 3, 0, 7, 16, None, None) == 1              # bad mode
    assert f(18, 10, 3, 0, 0, 16, None, None) == 1              # misaligned f32 pointer
    assert f(16, 2, 3, 0, 0, 16, 32, None) == 0                 # w > n: nothing to do
    assert f(None, 0, 3, 0, 0, None, None, None) == 0           # empty input
    assert f(16, 10 ** 9, 2048 * 1100, 0, 0, 16, None, None) == 7  # window beyond the limit
    assert len(lib.mmf_last_error()) > 0


def test_argfilter_and_w3_argument_errors_need_no_gpu(lib):
    """The arg filter and the window-3 entry points reject bad arguments (and
    kernels that compute no locations) before any CUDA call."""
    a = lib.mmf_argfilter1d_ex
    a.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int] + [ctypes.c_void_p] * 5 + \
        [ctypes.c_int]
    a.restype = ctypes.c_int
    assert a(16, 10, 3, 0, None, None, None, None, None, 0) == 1      # every output NULL
    assert a(16, 10, 0, 0, 16, None, None, None, None, 0) == 1        # w < 1
    assert a(16, 10, 3, 9, 16, None, None, None, None, 0) == 1        # bad dtype
    assert a(16, 10, 3, 0, 16, None, 20, None, None, 0) == 1          # misaligned positions
    assert a(16, 10, 3, 0, 16, None, None, None, None, 2) == 7        # the slide has no locations
    assert a(16, 1000, 497, 0, 16, None, None, None, None, 3) == 7    # wedge window limit
    assert a(16, 2, 3, 0, 16, None, None, None, None, 0) == 0         # w > n: nothing to do
    assert a(16, -1, 3, 0, 16, None, None, None, None, 0) == 1        # n < 0
    assert a(16, 10, 2 ** 31, 0, 16, None, None, None, None, 0) == 0  # any window (here w > n)
    f = lib.mmf_filter1d_w3
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int] + [ctypes.c_void_p] * 4
    f.restype = ctypes.c_int
    assert f(16, 10, 0, None, None, None, None) == 1                  # every output NULL
    assert f(None, 10, 0, 16, None, None, None) == 1                  # NULL input
    assert f(16, -1, 0, 16, None, None, None) == 1                    # n < 0
    assert f(16, 10, 9, 16, None, None, None) == 1                    # bad dtype
    assert f(16, 10, 0, 16, None, 12, None) == 1                      # misaligned counter
    assert f(16, 2, 0, 16, None, None, None) == 0                     # no window of 3


def test_extreme_sizes_need_no_gpu(lib):
    """Sizes near 2^63 are refused (or give nothing) on the host, before any
    byte count could wrap around."""
    f = lib.mmf_filter1d
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    assert f(None, 0, 2 ** 62, 0, 1, None, None, None) == 0      # empty envelope, any radius
    assert f(None, 0, 2 ** 63 - 1, 0, 0, None, None, None) == 0  # empty valid filter, any window
    ws = lib.mmf_filter2d_workspace
    ws.argtypes = [ctypes.c_int64] * 5 + [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
    ws.restype = ctypes.c_int
    nbytes = ctypes.c_size_t(0)
    # a column window whose ring size would not fit an int: refused
    assert ws(1, 2 ** 40, 1, 2 ** 35 + 1, 1, 0, -1, ctypes.byref(nbytes)) == 7
    assert ws(1, 4096, 4096, 3, 3, 0, 0, ctypes.byref(nbytes)) == 0 and nbytes.value > 0


def test_product_path_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_cs_0610046_gb300 as mmf
    monkeypatch.setattr(mmf, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(mmf, "_lib", None)
    with pytest.raises(RuntimeError):
        mmf.load()


def test_plain_c_program_uses_the_abi(lib, tmp_path):
    """The header is plain C (C99, pedantic) and a C program links the shared
    library and makes host-only calls through it."""
    import shutil
    import subprocess
    from paper_cs_0610046_gb300 import build
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_mmf.c"
    src.write_text(r"""
#include <stdio.h>
#include <string.h>
#include "mmf.h"
int main(void) {
    if (mmf_output_length(10, 3, MMF_VALID) != 8) return 1;
    if (mmf_output_length(10, 4, MMF_CENTERED_CLIPPED) != 10) return 2;
    if (mmf_filter1d((const void *)16, 10, 0, MMF_F32, MMF_VALID, (void *)16, NULL, NULL) != MMF_EINVAL) return 3;
    if (strlen(mmf_last_error()) == 0) return 4;
    if (strstr(mmf_version(), "sm_103a") == NULL) return 5;
    printf("ok\n");
    return 0;
}
""")
    exe = tmp_path / "use_mmf"
    libdir = os.path.dirname(build.LIB)
    libname = os.path.basename(build.LIB)
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
           str(src), "-o", str(exe), os.path.join(libdir, libname), f"-Wl,-rpath,{libdir}"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", (out.returncode, out.stdout, out.stderr)


def test_binding_refuses_host_tensors_for_device_calls():
    """The device entry points take CUDA tensors only: a CPU tensor is refused
    before any library call (there is no CPU fallback to fall into)."""
    import torch
    import paper_cs_0610046_gb300 as mmf
    x = torch.arange(100, dtype=torch.float32)
    for call in (lambda: mmf.filter1d(x, 3), lambda: mmf.filter1d(x, 3, mode="envelope"),
                 lambda: mmf.argfilter1d(x, 3), lambda: mmf.filter1d_w3(x),
                 lambda: mmf.filter2d(x.reshape(10, 10), 3, 3)):
        with pytest.raises(TypeError):
            call()
    with pytest.raises(TypeError):
        mmf.filter1d(torch.arange(100, dtype=torch.int32), 3)  # an unsupported type as well


def test_wait_fault_hook_checks_its_bound(lib):
    """The timeout test hook takes a bound of 1000 .. 2e9 clocks and can always
    be switched off (host-side state only; no CUDA call)."""
    f = lib.mmf_test_set_wait_fault
    f.argtypes = [ctypes.c_int, ctypes.c_int64]
    f.restype = ctypes.c_int
    assert f(1, 10) == 1 and f(1, 3_000_000_000) == 1
    assert f(1, 200_000) == 0
    assert f(0, 0) == 0


def test_input_clip_hook_is_host_only(lib):
    f = lib.mmf_test_set_input_clip
    f.argtypes = [ctypes.c_int64]
    f.restype = ctypes.c_int
    assert f(-1) == 1 and f(1 << 20) == 0 and f(0) == 0
