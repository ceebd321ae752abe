"""The C-ABI library: it builds, loads, exports every symbol include/mad.h
declares, the binding mirrors the header's structs, and argument errors are
reported before any GPU work (no GPU needed)."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mad.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2008_13447_gb300 import build
    build.build()
    import paper_2008_13447_gb300 as mad
    return mad.library()


def declared_functions():
    src = open(HEADER).read()
    return re.findall(r"MAD_API\s+[\w\s\*]+?\b(mad_\w+)\s*\(", src)


def test_header_declares_the_abi():
    import paper_2008_13447_gb300 as mad
    names = declared_functions()
    assert set(names) == set(mad.ABI_FUNCTIONS)
    assert len(names) == len(set(names))


def test_library_exports_every_declared_symbol(lib):
    import paper_2008_13447_gb300 as mad
    out = subprocess.run(["nm", "-D", "--defined-only", mad.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(mad_\w+)", out))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)
    # nothing else leaks out of the library under the ABI's prefix
    assert exported == set(declared_functions())


def test_struct_layouts_match_header():
    import paper_2008_13447_gb300 as mad
    # compile a tiny C program against the header and compare sizes/offsets
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "mad.h"
int main(void){
  printf("%zu %zu %zu\n", sizeof(mad_options), offsetof(mad_options, stream), offsetof(mad_options, keep_profiles));
  printf("%zu %zu\n", sizeof(mad_motif), offsetof(mad_motif, dist_recheck));
  printf("%zu %zu\n", sizeof(mad_discord), offsetof(mad_discord, dist_recheck));
  printf("%zu %zu %zu\n", sizeof(mad_length_stats), offsetof(mad_length_stats, passes), offsetof(mad_length_stats, fp32_dq_max));
  return 0; }
'''
    import tempfile
    d = tempfile.mkdtemp()
    src = os.path.join(d, "t.c")
    open(src, "w").write(prog)
    exe = os.path.join(d, "t")
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", exe, src])
    got = subprocess.run([exe], capture_output=True, text=True).stdout.split()
    want = [C.sizeof(mad.mad_options), mad.mad_options.stream.offset, mad.mad_options.keep_profiles.offset,
            C.sizeof(mad.mad_motif), mad.mad_motif.dist_recheck.offset,
            C.sizeof(mad.mad_discord), mad.mad_discord.dist_recheck.offset,
            C.sizeof(mad.mad_length_stats), mad.mad_length_stats.passes.offset,
            mad.mad_length_stats.fp32_dq_max.offset]
    assert [int(g) for g in got] == want


def test_argument_errors_before_gpu_work(lib):
    import paper_2008_13447_gb300 as mad
    ctx = C.c_void_p()
    o = mad._options()
    assert lib.mad_create(None, 100, C.byref(o), C.byref(ctx)) == mad.MAD_EINVAL
    assert "NULL" in mad.mad_last_error()
    x = np.zeros(3)
    assert lib.mad_create(mad._p(x), 3, C.byref(o), C.byref(ctx)) == mad.MAD_EINVAL
    assert lib.mad_create(mad._p(x), 3, C.byref(o), None) == mad.MAD_EINVAL
    assert lib.mad_profile(None, 8, 16, 5) == mad.MAD_EINVAL
    assert lib.mad_motifs(None, 0, 5, None, None) == mad.MAD_EINVAL
    for fn in (lib.mad_discords, lib.mad_discords_global, lib.mad_discords_streamed):
        assert fn(None, 0, 2, 1, None, None) == mad.MAD_EINVAL
    assert lib.mad_motif_sets(None, 0, 2, 1.0, 8, None, None, None) == mad.MAD_EINVAL
    assert lib.mad_observe(None, 0, None, None) == mad.MAD_EINVAL
    lib.mad_destroy(None)   # NULL-safe
    assert isinstance(lib.mad_last_error(None), bytes)


def test_binding_has_no_fallback(monkeypatch):
    import paper_2008_13447_gb300 as mad
    monkeypatch.setattr(mad, "_lib", None)
    monkeypatch.setattr(mad, "LIB_PATH", "/nonexistent/libmad.so")
    with pytest.raises(ImportError):
        mad.library()
