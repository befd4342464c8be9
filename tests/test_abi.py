"""The C-ABI library builds, loads and exports every declared entry point
(CPU only: no compute call is made)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+(gp_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gp_create", "gp_destroy", "gp_submit_drawcall", "gp_sync", "gp_stats", "gp_partition"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_1805_08893_gb300 as gp
    lib = ctypes.CDLL(gp.library_path())
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", gp.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (gp_[a-z0-9_]+)", out))
    assert set(declared_functions()) <= exported


def test_pure_host_entry_points():
    import paper_1805_08893_gb300 as gp
    assert gp.gp_out_floats(gp.GP_SHADER_MVP) == 7
    assert gp.gp_out_floats(gp.GP_SHADER_ENVELOPE) == 8
    assert gp.gp_out_floats(99) == 0
    assert gp.gp_status_string(gp.GP_ERR_INDEX_RANGE) == "GP_ERR_INDEX_RANGE"


def test_uniform_struct_sizes_match_header():
    import paper_1805_08893_gb300 as gp
    assert ctypes.sizeof(gp.gp_uniforms_mvp) == 100
    assert ctypes.sizeof(gp.gp_uniforms_skin) == 100 + 768 * 4
    assert ctypes.sizeof(gp.gp_uniforms_envelope) == 8 + 48 * 4
    assert ctypes.sizeof(gp.gp_uniforms_load) == 104
    assert ctypes.sizeof(gp.gp_config) == 64
    # compile a C probe against the header and compare sizeof()
    src = r'''
#include <stdio.h>
#include "gp.h"
int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(gp_config), sizeof(gp_index_buf),
 sizeof(gp_vertex_buf), sizeof(gp_out_buf), sizeof(gp_uniforms_mvp), sizeof(gp_uniforms_skin),
 sizeof(gp_uniforms_envelope), sizeof(gp_stats_t), sizeof(gp_draw_desc), sizeof(gp_draw_config),
 sizeof(gp_autotune_entry), sizeof(gp_serve_config), sizeof(gp_serve_stats), sizeof(gp_walk_desc), sizeof(gp_loop_desc)); return 0;}
'''
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        exe = os.path.join(d, "p")
        open(c, "w").write(src)
        r = subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], capture_output=True, text=True)
        if r.returncode != 0:
            pytest.skip("no C compiler: " + r.stderr[:200])
        sizes = [int(x) for x in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    py = [ctypes.sizeof(t) for t in (gp.gp_config, gp.gp_index_buf, gp.gp_vertex_buf, gp.gp_out_buf,
                                     gp.gp_uniforms_mvp, gp.gp_uniforms_skin, gp.gp_uniforms_envelope,
                                     gp.gp_stats_t, gp.gp_draw_desc, gp.gp_draw_config, gp.gp_autotune_entry,
                                     gp.gp_serve_config, gp.gp_serve_stats, gp.gp_walk_desc, gp.gp_loop_desc)]
    assert sizes == py


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1805_08893_gb300 as gp
    with pytest.raises(gp.GpError) as e:
        gp.gp_create("hash")
    assert e.value.status == gp.GP_ERR_CUDA
