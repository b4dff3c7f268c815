"""The library's host code under AddressSanitizer + UBSan, without a GPU.

A variant of libcobs_gpu.so whose host code is compiled with
-fsanitize=address,undefined (device code unchanged) runs the CPU tests of the
index file format (round trip, truncated and corrupt files), the index merge,
the argument checks and the Bloom-size formula in a child process; any
sanitizer report fails the test.
"""
import os
import shutil
import subprocess
import sys

import pytest

from paper_1905_09624_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")


def test_host_code_under_address_and_ub_sanitizers():
    libasan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not os.path.isabs(libasan) or not os.path.exists(libasan):
        pytest.skip("libasan not installed")
    # one option per -Xcompiler: nvcc splits its argument at commas
    sanitize = ["-Xcompiler", "-fsanitize=address", "-Xcompiler", "-fsanitize=undefined"]
    san = sanitize + ["-Xcompiler", "-fno-omit-frame-pointer", "-Xcompiler", "-fno-sanitize-recover=all"]
    out = os.path.join(os.path.dirname(_build.LIB), "sanitize", "libcobs_gpu.so")
    path = _build.build(extra_flags=san, lib_path=out, link_flags=sanitize)
    env = dict(os.environ, LD_PRELOAD=libasan, COBS_TEST_LIBRARY=path,
               ASAN_OPTIONS="detect_leaks=0:verify_asan_link_order=0", UBSAN_OPTIONS="print_stacktrace=1")
    tests = ["tests/test_merge.py", "tests/test_abi.py::test_index_file_roundtrip_and_format_errors",
             "tests/test_abi.py::test_argument_errors_without_gpu", "tests/test_abi.py::test_bloom_width_matches_oracle"]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider"] + tests, cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=900)
    log = r.stdout[-4000:] + r.stderr[-4000:]
    assert r.returncode == 0, log
    assert "ERROR: AddressSanitizer" not in r.stderr and "runtime error" not in r.stderr, log
    assert " passed" in r.stdout, log
