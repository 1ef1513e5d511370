"""The C ABI library loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "graphvine.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(gv_[a-z_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2306_08252_gb300 import build as b
    try:
        b.build()
    except RuntimeError as e:
        pytest.skip(f"cannot build the CUDA library here: {e}")
    return ctypes.CDLL(b.LIB)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["gv_create", "gv_bulk_build", "gv_insert_edges", "gv_delete_edges", "gv_insert_vertices",
                     "gv_delete_vertices", "gv_query_edges", "gv_neighbors", "gv_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2306_08252_gb300 import graphvine
    assert set(_declared()) == set(graphvine.SIGNATURES)


def test_status_strings_without_gpu(lib):
    from paper_2306_08252_gb300 import graphvine
    l = graphvine.load()
    assert l.gv_status_string(0) == b"GV_OK"
    assert l.gv_status_string(2) == b"GV_ERR_OUT_OF_MEMORY"


def test_null_arguments_rejected_on_host(lib):
    from paper_2306_08252_gb300 import graphvine
    l = graphvine.load()
    # NULL graph handles are rejected before any CUDA call
    assert l.gv_insert_edges(None, None, None, 0, None, None) == graphvine.GV_ERR_INVALID_ARG
    assert l.gv_delete_edges(None, None, None, 0, None, None) == graphvine.GV_ERR_INVALID_ARG
    assert l.gv_sync(None) == graphvine.GV_ERR_INVALID_ARG
    assert l.gv_create(None, 4, None, None) == graphvine.GV_ERR_INVALID_ARG
    assert l.gv_destroy(None) == graphvine.GV_OK


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2306_08252_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "gv_oracle" not in src, f


def test_multiply_shift_division_by_block_capacity_is_exact():
    # The kernels divide by C as (x * ceil(2^40 / C)) >> 40; exact for every
    # x < 2^31 and every allowed C (multiple of 4, 4..512).
    import random
    rng = random.Random(7)
    for C in range(4, 513, 4):
        M = ((1 << 40) + C - 1) // C
        xs = [0, 1, C - 1, C, C + 1, (1 << 31) - 1, (1 << 31) - C] + [rng.randrange(1 << 31) for _ in range(300)]
        xs += [k * C + r for k in (1, 7, 1 << 20, (1 << 31) // C - 1) for r in (0, C - 1)]
        for x in xs:
            assert (x * M) >> 40 == x // C, (C, x)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # no CPU fallback: without the CUDA library every entry point raises
    import paper_2306_08252_gb300.graphvine as gvb
    monkeypatch.setattr(gvb, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        gvb.load(str(tmp_path / "libgraphvine.so"))


def test_header_is_plain_c_and_links(lib, tmp_path):
    # a C99 caller: the header compiles without C++ (-pedantic, warnings as
    # errors), links against the library and makes calls that need no GPU
    import os
    import shutil
    import subprocess
    from paper_2306_08252_gb300 import build as b
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "caller.c"
    src.write_text(
        '#include "graphvine.h"\n'
        "#include <stdio.h>\n"
        "#include <string.h>\n"
        "int main(void) {\n"
        "    gv_graph *g = (gv_graph *)0;\n"
        "    if (gv_create((const gv_config *)0, 16, (void *)0, (gv_graph **)0) != GV_ERR_INVALID_ARG) return 1;\n"
        "    if (gv_sync(g) != GV_ERR_INVALID_ARG) return 2;\n"
        "    if (gv_destroy(g) != GV_OK) return 3;\n"
        "    if (strcmp(gv_status_string(GV_ERR_OUT_OF_MEMORY), \"\") == 0) return 4;\n"
        "    printf(\"%s\\n\", gv_status_string(GV_OK));\n"
        "    return 0;\n"
        "}\n")
    exe = tmp_path / "caller"
    libdir = os.path.dirname(b.LIB)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(root, "include"),
                    str(src), "-L", libdir, "-lgraphvine", f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.returncode, r.stderr)
    assert r.stdout.strip()


def test_binding_structs_match_header(tmp_path):
    # the ctypes mirrors of the header's structs have its size
    # and field offsets (a C program compiled against the header prints them)
    import ctypes
    import os
    import shutil
    import subprocess
    import paper_2306_08252_gb300.graphvine as gvb
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    lines = ['#include "graphvine.h"', "#include <stddef.h>", "#include <stdio.h>", "int main(void) {"]
    for cls, name in [(gvb.gv_config, "gv_config"), (gvb.gv_stats_t, "gv_stats_t"), (gvb.gv_serve_request, "gv_serve_request"), (gvb.gv_serve_config, "gv_serve_config")]:
        lines.append(f'    printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'    printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                          check=True).stdout.split("\n") if l)
    for cls, name in [(gvb.gv_config, "gv_config"), (gvb.gv_stats_t, "gv_stats_t"), (gvb.gv_serve_request, "gv_serve_request"), (gvb.gv_serve_config, "gv_serve_config")]:
        assert int(out[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(out[f"{name}.{f}"]) == getattr(cls, f).offset, (name, f)
