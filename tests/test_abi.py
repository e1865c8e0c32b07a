"""The C-ABI library builds, loads without a GPU and exports every entry point include/pipnn.h
declares; the binding fails loudly rather than falling back when the library is absent."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pipnn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pipnn_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2602_21247_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("pipnn_build", "pipnn_free", "pipnn_sketch", "pipnn_partition", "pipnn_leaf_pick",
              "pipnn_hashprune", "pipnn_final_prune", "pipnn_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in _declared():
        assert hasattr(lib, name), name
    import paper_2602_21247_gb300 as pk
    assert sorted(pk.EXPORTS) == _declared()


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2602_21247_gb300 as pk
    monkeypatch.setattr(pk, "_lib", None)
    monkeypatch.setattr(pk, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        pk.lib()


def test_params_struct_matches_header_layout():
    import paper_2602_21247_gb300 as pk
    # 3 x u32, f32, 4 x u32, 6 x u32/f32, 3 x i32, pointer (8-byte aligned), u32 replicas, tail
    # padding to the pointer's alignment
    assert pk.pipnn_params.hyperplanes.offset == 4 * (3 + 1 + 4 + 1 + 4 + 1 + 1 + 2) + 4 == 72
    assert pk.pipnn_params.replicas.offset == 80
    assert pk.pipnn_params.prec.offset == 84
    assert pk.pipnn_params.wave_members.offset == 88
    assert pk.pipnn_params.pick_direction.offset == 96
    assert pk.pipnn_params.merge_waves.offset == 100
    assert ctypes.sizeof(pk.pipnn_params) == 104


def test_batched_build_argument_checks_need_no_gpu():
    # the binding validates the index list before it calls the library
    import numpy as np

    import paper_2602_21247_gb300 as pk

    a = np.zeros((10, 8), np.uint8)
    bp = pk.params(dtype=pk.PIPNN_U8)
    with pytest.raises(ValueError):
        pk.pipnn_build_batched([a, a], bp, [1])                       # one seed per index
    with pytest.raises(ValueError):
        pk.pipnn_build_batched([a, np.zeros((10, 9), np.uint8)], bp, [1, 2])    # one dimension
    with pytest.raises(ValueError):
        pk.pipnn_build_batched([a, np.zeros((10, 8), np.int8)], bp, [1, 2])     # one dtype


def test_every_struct_matches_the_header_compiled_by_the_c_compiler(tmp_path):
    """Field offsets and sizes of the header's structs, as a C compiler lays them out, equal the
    binding's ctypes mirrors."""
    import shutil
    import subprocess

    import paper_2602_21247_gb300 as pk

    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    structs = [pk.pipnn_params, pk.pipnn_stats, pk.pipnn_leaves, pk.pipnn_edges, pk.pipnn_graph]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pipnn.h"', "int main(void) {"]
    for s in structs:
        lines.append(f'printf("%s size %zu\\n", "{s.__name__}", sizeof({s.__name__}));')
        for f, _ in s._fields_:
            lines.append(f'printf("%s %s %zu\\n", "{s.__name__}", "{f}", offsetof({s.__name__}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(line.split()[:2]): int(line.split()[2]) for line in out if line}
    for s in structs:
        assert got[(s.__name__, "size")] == ctypes.sizeof(s), s.__name__
        for f, _ in s._fields_:
            assert got[(s.__name__, f)] == getattr(s, f).offset, (s.__name__, f)
