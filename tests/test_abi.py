"""The C-ABI library without a GPU: it loads, exports every declared symbol,
and its host-side logic (planner formula, file format, argument checks) works."""
import ctypes
import os
import re
import struct

import numpy as np
import pytest

import oracle
from paper_1905_09624_gb300 import cobs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(cobs_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    L = cobs.lib()
    names = _declared_functions()
    assert len(names) >= 25
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing
    # and the binding covers the same names
    assert names <= set(cobs._PROTOS), sorted(names - set(cobs._PROTOS))


def test_bloom_width_matches_oracle():
    for h, p in [(1, 0.3), (3, 0.1), (2, 0.05)]:
        for v in (0, 1, 5, 99, 4970, 123457, 9_999_991):
            assert cobs.bloom_width(h, v, p) == oracle.bloom_width(h, v, p)


def _write_index_file(path, params, blocks, perm, nterms, rows):
    with open(path, "wb") as f:
        f.write(b"COBSGPU2")
        f.write(bytes(params))
        f.write(struct.pack("<QQQ", len(perm), len(blocks), len(rows)))
        for b in blocks:
            f.write(struct.pack("<6Q", b["n_docs"], b["doc_begin"], b["w"], b["rowbytes"], b["row_offset"],
                                b["max_terms"]))
        f.write(np.asarray(perm, np.uint64).tobytes())
        f.write(np.asarray(nterms, np.uint64).tobytes())
        f.write(np.asarray(rows, np.uint8).tobytes())


def test_index_file_roundtrip_and_format_errors(tmp_path):
    P = cobs.make_params(term_kind=0, q=31, num_hashes=1, fpr=0.3, block_docs=2, score_bits=32)
    blocks = [dict(n_docs=2, doc_begin=0, w=5, rowbytes=16, row_offset=0, max_terms=2),
              dict(n_docs=1, doc_begin=2, w=3, rowbytes=16, row_offset=80, max_terms=1)]
    rows = np.arange(128, dtype=np.uint8)
    p = str(tmp_path / "a.idx")
    _write_index_file(p, P, blocks, [1, 2, 0], [2, 2, 1], rows)
    ix = cobs.HostIndex.load(p)
    info = ix.info()
    assert info["n_docs"] == 3 and info["blocks"] == blocks
    assert list(info["perm"]) == [1, 2, 0] and np.array_equal(info["rows"], rows)
    q = str(tmp_path / "b.idx")
    ix.save(q)
    assert open(p, "rb").read() == open(q, "rb").read()
    # truncated, wrong magic, inconsistent table
    data = open(p, "rb").read()
    for bad in (data[:-1], b"XOBSGPU2" + data[8:]):
        open(p, "wb").write(bad)
        with pytest.raises(cobs.CobsError) as e:
            cobs.HostIndex.load(p)
        assert e.value.status == cobs.COBS_ERR_FORMAT
    blocks[1]["row_offset"] = 64
    _write_index_file(p, P, blocks, [1, 2, 0], [2, 2, 1], rows)
    with pytest.raises(cobs.CobsError) as e:
        cobs.HostIndex.load(p)
    assert e.value.status == cobs.COBS_ERR_FORMAT


def test_argument_errors_without_gpu():
    L = cobs.lib()
    res = ctypes.POINTER(cobs.cobs_result)()
    assert L.cobs_query_batch(None, None, None, None, 0, cobs.COBS_BATCHED, None, ctypes.byref(res)) == \
        cobs.COBS_ERR_ARG
    assert b"NULL" in L.cobs_last_error()
    bad = cobs.make_params(term_kind=2, q=9)
    h = ctypes.c_void_p()
    off = np.zeros(1, np.uint64)
    assert L.cobs_build_device(ctypes.byref(bad), None, off.ctypes.data, 0, 0, None, ctypes.byref(h)) == \
        cobs.COBS_ERR_ARG
    assert L.cobs_index_load(b"/nonexistent/file", ctypes.byref(h)) == cobs.COBS_ERR_ARG


def test_product_path_does_not_touch_the_oracle():
    # The CUDA library and its binding never import, link or name the oracle.
    pkg = os.path.join(ROOT, "paper_1905_09624_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_lib" in dirpath:
            continue
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in src and "orc_" not in src and "liboracle" not in src, fn


def test_header_is_plain_c(tmp_path):
    # the boundary header compiles as C99 and as C++ with every warning an error,
    # and a C program that takes the address of every declared function links
    # against the library
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    names = sorted(_declared_functions())
    body = "\n".join(f"    (any_fn)&{n}," for n in names)
    src = tmp_path / "use_header.c"
    src.write_text('#include "cobs_gpu.h"\n#include <stdio.h>\ntypedef void (*any_fn)(void);\n'
                   f"static const any_fn fns[] = {{\n{body}\n}};\n"
                   'int main(void) { printf("%d\\n", (int)(sizeof fns / sizeof fns[0])); return 0; }\n')
    inc = os.path.join(ROOT, "include")
    lib = cobs.lib()._name
    exe = tmp_path / "use_header"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", inc, str(src),
                        lib, "-o", str(exe), f"-Wl,-rpath,{os.path.dirname(lib)}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and int(r.stdout) == len(names), r.stdout + r.stderr
    cpp = tmp_path / "use_header.cpp"
    cpp.write_text('#include "cobs_gpu.h"\nint main() { return 0; }\n')
    r = subprocess.run(["g++", "-std=c++17", "-Wall", "-Wextra", "-Werror", "-I", inc, "-c", str(cpp), "-o",
                        str(tmp_path / "use_header.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_host_index_close(tmp_path):
    # close() and with-blocks release a host index at once (no GPU involved)
    import oracle as orc
    import synth
    lens = synth.lognormal_lengths(3, 10, 300, 0.3, 50, 600)
    docs, off = synth.dna_docs(3, lens)
    ix = orc.build_index(orc.make_params(block_docs=4), docs, off)
    path = str(tmp_path / "x.idx")
    _write_index_file(path, cobs.make_params(block_docs=4), ix.blocks(), ix.perm(), ix.nterms(), ix.rows())
    with cobs.HostIndex.load(path) as h:
        assert h.info()["n_docs"] == 10
    assert h.h is None
    h.close()  # closing twice is harmless


def test_abi_version_matches_header_and_binding():
    src = open(os.path.join(ROOT, "include", "cobs_gpu.h")).read()
    m = re.search(r"#define COBS_GPU_ABI_VERSION (\d+)u", src)
    assert m and int(m.group(1)) == cobs.ABI_VERSION == cobs.lib().cobs_abi_version()
