"""The C ABI library loads and exports every entry point include/quapi.h declares (CPU only)."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "quapi.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = set(re.findall(r"\b(quapi_[a-z_0-9]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_1205_6872_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("quapi_setup", "quapi_setup_eta", "quapi_propagate", "quapi_query_memory",
              "quapi_propagate_batch", "quapi_last_error", "quapi_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for n in sorted(_declared()):
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (quapi_[a-z_0-9]+)\b", out))
    assert _declared() <= exported


def test_binding_names_match_header(lib_path):
    from paper_1205_6872_gb300 import quapi
    assert set(quapi.EXPORTED) == _declared()
    for n in quapi.EXPORTED:
        assert callable(getattr(quapi, n))


def test_query_memory_host_only(lib_path):
    from paper_1205_6872_gb300 import quapi
    t, tot = quapi.quapi_query_memory(2, 14, quapi.QUAPI_FP32)
    assert t == 2 * 4 ** 14 * 8
    assert tot > t
    t64, _ = quapi.quapi_query_memory(2, 14, quapi.QUAPI_FP64)
    assert t64 == 2 * 4 ** 14 * 16
    t3, _ = quapi.quapi_query_memory(3, 8, quapi.QUAPI_FP64)
    assert t3 == 2 * 9 ** 8 * 16
    with pytest.raises(quapi.QuapiError):
        quapi.quapi_query_memory(4, 3, quapi.QUAPI_FP64)
    with pytest.raises(quapi.QuapiError):
        quapi.quapi_query_memory(2, 0, quapi.QUAPI_FP64)
    with pytest.raises(quapi.QuapiError):
        quapi.quapi_query_memory(2, 17, quapi.QUAPI_FP64)
    with pytest.raises(quapi.QuapiError):
        quapi.quapi_query_memory(2, 3, 16)


def test_opts_defaults(lib_path):
    from paper_1205_6872_gb300 import quapi
    o = quapi.quapi_opts_init()
    assert o.precision == quapi.QUAPI_FP64 and o.endpoint_mode == quapi.QUAPI_ENDPOINT_STRANG
    assert not o.workspace and o.workspace_bytes == 0


def test_struct_layouts_match_binding(tmp_path):
    """sizeof / offsetof of the ABI structs from a C compiler against the ctypes binding."""
    from paper_1205_6872_gb300 import quapi
    src = tmp_path / "layout.c"
    src.write_text(r"""
#include <stddef.h>
#include <stdio.h>
#include "quapi.h"
int main(void) {
    printf("spectral %zu %zu %zu %zu %zu %zu %zu\n", sizeof(quapi_spectral), offsetof(quapi_spectral, kind),
           offsetof(quapi_spectral, a), offsetof(quapi_spectral, wc), offsetof(quapi_spectral, omega),
           offsetof(quapi_spectral, values), offsetof(quapi_spectral, n));
    printf("opts %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(quapi_opts), offsetof(quapi_opts, precision),
           offsetof(quapi_opts, endpoint_mode), offsetof(quapi_opts, cuda_stream), offsetof(quapi_opts, tune),
           offsetof(quapi_opts, workspace), offsetof(quapi_opts, workspace_bytes), offsetof(quapi_opts, hermitian));
    return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    lines = dict(l.split(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.strip().splitlines())
    S = quapi.quapi_spectral
    want_s = [ctypes.sizeof(S)] + [getattr(S, f).offset for f in ("kind", "a", "wc", "omega", "values", "n")]
    assert [int(x) for x in lines["spectral"].split()] == want_s
    O = quapi.quapi_opts
    want_o = [ctypes.sizeof(O)] + [getattr(O, f).offset for f in ("precision", "endpoint_mode", "cuda_stream", "tune",
                                                                    "workspace", "workspace_bytes", "hermitian")]
    assert [int(x) for x in lines["opts"].split()] == want_o


def test_query_memory_opts_host_only(lib_path):
    """Exact tensor bytes per layout and precision, for M = 2 and M = 3."""
    from paper_1205_6872_gb300 import layout, quapi
    for M, L in ((2, 14), (3, 8), (3, 1)):
        for prec, elt in ((quapi.QUAPI_FP32, 8), (quapi.QUAPI_FP64, 16), (quapi.QUAPI_DF64, 16)):
            full, full_tot = quapi.quapi_query_memory_opts(M, L, quapi.quapi_opts_init(precision=prec))
            assert (full, full_tot) == quapi.quapi_query_memory(M, L, prec)
            half, half_tot = quapi.quapi_query_memory_opts(M, L, quapi.quapi_opts_init(precision=prec, hermitian=1))
            assert half == 2 * layout.count(L, M) * elt
            assert half_tot - half == full_tot - full  # the same tables and scratch
    with pytest.raises(quapi.QuapiError) as e:
        quapi.quapi_query_memory_opts(2, 0, quapi.quapi_opts_init(hermitian=1))
    assert e.value.status == quapi.QUAPI_ERR_ARG
