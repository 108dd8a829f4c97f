"""The C-ABI library builds, loads and exports every entry point of include/*.h (CPU only:
no compute call is made without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(pmh_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2511_16576_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pmh_poly_upload", "pmh_minhash_sign", "pmh_lsh_build", "pmh_lsh_query",
                     "pmh_jaccard_estimate"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2511_16576_gb300 import binding
    assert set(declared_functions()) <= set(binding.exported_names())


def test_error_path_without_gpu_or_bad_args(lib):
    lib.pmh_last_error.restype = ctypes.c_char_p
    lib.pmh_version.restype = ctypes.c_int
    assert lib.pmh_version() >= 10000
    # null out-pointer is rejected before any CUDA call
    assert lib.pmh_create(None, 0) == -1
    assert b"null" in lib.pmh_last_error()
    assert lib.pmh_polys_destroy(None) == 0
    assert lib.pmh_index_destroy(None) == 0


def test_params_struct_layout():
    from paper_2511_16576_gb300 import binding
    assert ctypes.sizeof(binding.Params) == 40
    p = binding.make_params(128, 16)
    assert (p.K, p.bands, p.rows, p.T) == (128, 16, 8, 1 << 24)


def test_header_layout_and_constants_match_the_binding(tmp_path):
    """The header compiled by a plain C compiler: pmh_params and pmh_qgraph_config field
    offsets and the shared constants equal the binding's ctypes view of them."""
    import shutil
    import subprocess
    from paper_2511_16576_gb300 import binding
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "polyminhash.h"
int main(void) {
    printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(pmh_params),
           offsetof(pmh_params, seed), offsetof(pmh_params, K), offsetof(pmh_params, T),
           offsetof(pmh_params, bands), offsetof(pmh_params, rows),
           offsetof(pmh_params, lsh_seed), offsetof(pmh_params, flags),
           offsetof(pmh_params, reserved));
    printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(pmh_qgraph_config),
           offsetof(pmh_qgraph_config, max_queries), offsetof(pmh_qgraph_config, max_vertices),
           offsetof(pmh_qgraph_config, cand_capacity), offsetof(pmh_qgraph_config, m),
           offsetof(pmh_qgraph_config, k), offsetof(pmh_qgraph_config, db),
           offsetof(pmh_qgraph_config, rerank), offsetof(pmh_qgraph_config, shortlist),
           offsetof(pmh_qgraph_config, options));
    printf("%d %d %d %d %d %u %u %d %d\n", PMH_SIGN_VARIANTS, PMH_RERANK_IN, PMH_RERANK_HIDDEN,
           PMH_RERANK_PARAMS, PMH_NOALLOC_MAX_POLYS, PMH_FLAG_STREAM_INDEX,
           PMH_FLAG_COVERAGE_MASK, PMH_ERR_CAPACITY, PMH_QGRAPH_FUSED_SELECT);
    return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    lines = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    sizes = [int(v) for v in lines[0].split()]
    P = binding.Params
    assert sizes[0] == ctypes.sizeof(P)
    for off, (name, _) in zip(sizes[1:], P._fields_):
        assert off == getattr(P, name).offset, name
    gsizes = [int(v) for v in lines[1].split()]
    G = binding.QGraphConfig
    assert gsizes[0] == ctypes.sizeof(G)
    for off, (name, _) in zip(gsizes[1:], G._fields_):
        assert off == getattr(G, name).offset, name
    consts = [int(v) for v in lines[2].split()]
    assert consts == [binding.SIGN_VARIANTS, binding.RERANK_IN, binding.RERANK_HIDDEN,
                      binding.RERANK_PARAMS, binding.NOALLOC_MAX_POLYS, binding.FLAG_STREAM_INDEX,
                      binding.FLAG_COVERAGE_MASK, binding.PMH_ERR_CAPACITY, binding.QGRAPH_FUSED_SELECT]
