"""The C-ABI library loads and exports every entry point include/kann.h
declares; argument validation that happens before any CUDA call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "kann.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kann_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("kann_index_upload", "kann_search", "kann_exact_knn", "kann_index_destroy", "kann_status_str",
                 "kann_search_batch", "kann_search_sparse", "kann_quantize", "kann_hnsw_build_dense"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_2501_06121_b300 import build
    lib = ctypes.CDLL(build.build())
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert missing == []


def test_status_strings_and_host_validation():
    from paper_2501_06121_b300 import kann as K
    L = K._lib()
    for s in range(6):
        assert L.kann_status_str(s)
    assert L.kann_status_str(99) == b"unknown status"
    # null index / null out-pointer: rejected on the host, nothing launched
    assert L.kann_search(None, None, 0, 10, 10, None, None, None) == K.KANN_EINVAL
    assert L.kann_index_upload(None, None, None, None, None, None, 0) == K.KANN_EINVAL
    assert L.kann_index_destroy(None) == K.KANN_OK
    assert L.kann_exact_knn(None, None, 1, 10, 8, 0, 0, 0, None, None, None, 0, None) == K.KANN_EINVAL
    assert L.kann_quantize(None, 1, 8, K.KANN_F16, None, None, None) == K.KANN_EINVAL
    assert L.kann_hnsw_levels(-1, 16, 0, None, None, None) == K.KANN_EINVAL


def test_upload_rejects_inconsistent_graph_on_host():
    from paper_2501_06121_b300 import kann as K
    L = K._lib()
    fake = ctypes.c_void_p(16)  # never dereferenced: host checks fail first
    g = K.kann_graph_desc(100, 16, 40, 0, 0, 0, fake.value, fake.value, fake.value, None)  # M0 > 2M allowed? cap 64 ok
    v = K.kann_vectors_desc(K.KANN_F32, 128, K.KANN_L2, 0, 16, None, 512)
    h = ctypes.c_void_p()
    bad_M = K.kann_graph_desc(100, 33, 66, 0, 0, 0, fake.value, fake.value, fake.value, None)
    assert L.kann_index_upload(ctypes.byref(h), ctypes.byref(bad_M), ctypes.byref(v), None, None, None, 0) == K.KANN_EFORMAT
    bad_entry = K.kann_graph_desc(100, 16, 32, 0, 100, 0, fake.value, fake.value, fake.value, None)
    assert L.kann_index_upload(ctypes.byref(h), ctypes.byref(bad_entry), ctypes.byref(v), None, None, None, 0) == K.KANN_EFORMAT
    bad_stride = K.kann_vectors_desc(K.KANN_F32, 128, K.KANN_L2, 0, 16, None, 500)
    assert L.kann_index_upload(ctypes.byref(h), ctypes.byref(g), ctypes.byref(bad_stride), None, None, None, 0) == K.KANN_EINVAL
    two_sources = K.kann_pq_desc(4, 256, 4, 0, 16, 16)
    assert L.kann_index_upload(ctypes.byref(h), ctypes.byref(g), ctypes.byref(v), ctypes.byref(two_sources), None, None, 0) == K.KANN_EINVAL
    e4m3_no_scale = K.kann_vectors_desc(K.KANN_E4M3, 128, K.KANN_L2, 0, 16, None, 128)
    assert L.kann_index_upload(ctypes.byref(h), ctypes.byref(g), ctypes.byref(e4m3_no_scale), None, None, None, 0) == K.KANN_EINVAL


def test_binding_struct_layouts_match_the_header(tmp_path):
    # every struct the binding passes by pointer has the header's size and
    # field offsets (a field appended on one side only would shift nothing
    # visible until a search read garbage options)
    import subprocess
    from paper_2501_06121_b300 import kann as K
    structs = [K.kann_graph_desc, K.kann_vectors_desc, K.kann_pq_desc, K.kann_sparse_desc, K.kann_search_opts]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "kann.h"', "int main(void) {"]
    for S in structs:
        lines.append('  printf("%%s %%zu\\n", "%s", sizeof(%s));' % (S.__name__, S.__name__))
        for name, _ in S._fields_:
            lines.append('  printf("%%s.%%s %%zu\\n", "%s", "%s", offsetof(%s, %s));' % (S.__name__, name, S.__name__, name))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                        text=True).stdout.split("\n") if l)
    for S in structs:
        assert int(got[S.__name__]) == ctypes.sizeof(S), S.__name__
        for name, _ in S._fields_:
            assert int(got["%s.%s" % (S.__name__, name)]) == getattr(S, name).offset, (S.__name__, name)
