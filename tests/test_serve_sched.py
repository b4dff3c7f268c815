"""The serve scheduler on the host alone, and sanitizer runs of the host code.

The scheduler of the serve loop (``serve_core.cpp``) is built with g++ together
with a test backend (``tests/native/serve_mock.cpp``) whose waves run on no
device: admission by the score budget, back-pressure, FIFO order, cancellation,
launch and wave failures and the bounded wait (timeout) are checked through the
same C entry points the library exports (``cobs_serve_submit`` / ``poll`` /
``cancel`` / ``stop``).  The same scheduler under ThreadSanitizer and
AddressSanitizer + UBSan (several client threads submitting, polling and
cancelling), and the CPU oracle under AddressSanitizer + UBSan, must run without
a report.  No GPU is involved.
"""
import ctypes
import os
import shutil
import subprocess
import time

import numpy as np
import pytest

from paper_1905_09624_gb300 import cobs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1905_09624_gb300", "csrc")
NATIVE = os.path.join(ROOT, "tests", "native")
SCHED_SRC = [os.path.join(CSRC, "serve_core.cpp"), os.path.join(CSRC, "status.cpp")]
INC = ["-I", os.path.join(ROOT, "include"), "-I", CSRC]

pytestmark = pytest.mark.skipif(shutil.which("g++") is None, reason="g++ not available")


class MockCfg(ctypes.Structure):
    _fields_ = [("n_slots", ctypes.c_uint32), ("q", ctypes.c_uint32), ("wave_us", ctypes.c_uint32),
                ("fail_launch_wave", ctypes.c_int32), ("fail_wave", ctypes.c_int32), ("hang_wave", ctypes.c_int32),
                ("cost_base", ctypes.c_uint64), ("cost_per_byte", ctypes.c_uint64), ("max_windows", ctypes.c_uint64)]


class MockStats(ctypes.Structure):
    _fields_ = [("launched_waves", ctypes.c_uint64), ("launched_requests", ctypes.c_uint64),
                ("finished_waves", ctypes.c_uint64), ("inflight_cost", ctypes.c_uint64),
                ("max_inflight_cost", ctypes.c_uint64), ("max_wave_requests", ctypes.c_uint64),
                ("launch_order_ok", ctypes.c_uint64)]


def _compile(out, srcs, flags):
    cmd = ["g++", "-std=c++17", "-pthread"] + INC + flags + srcs + ["-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    return r


@pytest.fixture(scope="module")
def mock_lib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("serve_mock") / "libserve_mock.so")
    r = _compile(out, SCHED_SRC + [os.path.join(NATIVE, "serve_mock.cpp")],
                 ["-O2", "-g", "-fPIC", "-shared", "-Wl,-Bsymbolic"])
    assert r.returncode == 0, r.stderr
    L = ctypes.CDLL(out)
    for name, (res, args) in cobs.SERVE_PROTOS.items():
        f = getattr(L, name)
        f.restype, f.argtypes = res, args
    L.mock_serve_start.restype = ctypes.c_int
    L.mock_serve_start.argtypes = [ctypes.POINTER(cobs.cobs_serve_cfg), ctypes.POINTER(MockCfg),
                                   ctypes.POINTER(ctypes.c_void_p)]
    L.mock_get_stats.argtypes = [ctypes.POINTER(MockStats)]
    L.mock_release_hang.argtypes = []
    return L


Q = 4


def start(L, budget=1 << 30, slots=2, wave_us=200, fail_launch=-1, fail_wave=-1, hang=-1, cost_base=100,
          per_byte=1, max_windows=0, wave_max=0, timeout_ms=0):
    cfg = cobs.cobs_serve_cfg(budget, 0, wave_max, timeout_ms, 0)
    mc = MockCfg(slots, Q, wave_us, fail_launch, fail_wave, hang, cost_base, per_byte, max_windows)
    h = ctypes.c_void_p()
    assert L.mock_serve_start(ctypes.byref(cfg), ctypes.byref(mc), ctypes.byref(h)) == cobs.COBS_OK
    return cobs.Server.attach(L, h)


def stats(L):
    s = MockStats()
    L.mock_get_stats(ctypes.byref(s))
    return s


def fnv1a(b):
    h = 2166136261
    for c in b:
        h = ((h ^ c) * 16777619) & 0xFFFFFFFF
    return h


def expected(q, thr):
    nt = max(0, len(q) - Q + 1)
    mn = (thr * nt + 999) // 1000
    i = fnv1a(q) % 1000
    return nt, mn, [i, i + 1], [nt, mn]


def wait(srv, t, limit_s=10.0):
    t0 = time.time()
    while True:
        r = srv.poll(t)
        if r is not None:
            return r
        assert time.time() - t0 < limit_s, f"ticket {t} still pending"
        time.sleep(0.0005)


def status_of(srv, t, limit_s=10.0):
    t0 = time.time()
    while True:
        try:
            r = srv.poll(t)
        except cobs.CobsError as e:
            return e.status
        if r is not None:
            return cobs.COBS_OK
        assert time.time() - t0 < limit_s, f"ticket {t} still pending"
        time.sleep(0.0005)


def queries(n, seed=0):
    rng = np.random.default_rng(seed)
    return [bytes(rng.choice(list(b"ACGT"), size=int(rng.integers(0, 200))).astype(np.uint8)) for _ in range(n)]


def test_results_per_ticket_and_fifo(mock_lib):
    srv = start(mock_lib, wave_max=7)
    qs = queries(100)
    thr = [(i * 37) % 1000 + 1 for i in range(100)]
    tickets = [srv.submit(q, t) for q, t in zip(qs, thr)]
    assert tickets == sorted(tickets) and len(set(tickets)) == 100
    for q, th, t in zip(qs, thr, tickets):
        nt, mn, ids, sc = wait(srv, t)
        e = expected(q, th)
        assert (nt, mn, list(ids), list(sc)) == (e[0], e[1], e[2], e[3])
    st = stats(mock_lib)
    assert st.launch_order_ok == 1 and st.max_wave_requests <= 7 and st.launched_requests == 100
    s = srv.stop()
    assert s["completed"] == 100 and s["failed"] == 0 and s["cancelled"] == 0
    assert s["p50_ms"] <= s["p99_ms"] <= s["max_ms"]


def test_budget_back_pressure(mock_lib):
    # every query costs 100 + len; the budget admits about three at a time
    srv = start(mock_lib, budget=1000, slots=3, wave_us=2000)
    qs = queries(60, seed=1)
    tickets = [srv.submit(q, 500) for q in qs]
    for q, t in zip(qs, tickets):
        assert wait(srv, t)[0] == max(0, len(q) - Q + 1)
    st = stats(mock_lib)
    assert 0 < st.max_inflight_cost <= 1000
    assert st.launched_requests == 60
    srv.stop()


def test_rejections(mock_lib):
    srv = start(mock_lib, budget=500, max_windows=1000)
    with pytest.raises(cobs.CobsError) as e:
        srv.submit(b"A" * 450, 500)  # cost 550 > 500: can never be admitted
    assert e.value.status == cobs.COBS_ERR_BUDGET
    with pytest.raises(cobs.CobsError) as e:
        srv.submit(b"A" * 1100, 500)  # 1097 windows > 1000 (checked before the budget)
    assert e.value.status == cobs.COBS_ERR_OVERFLOW
    for bad in (0, 1001):
        with pytest.raises(cobs.CobsError) as e:
            srv.submit(b"ACGT", bad)
        assert e.value.status == cobs.COBS_ERR_ARG
    with pytest.raises(cobs.CobsError) as e:
        srv.poll(12345)
    assert e.value.status == cobs.COBS_ERR_NOT_FOUND
    with pytest.raises(cobs.CobsError) as e:
        srv.cancel(12345)
    assert e.value.status == cobs.COBS_ERR_NOT_FOUND
    assert srv.stop()["rejected"] == 1


def test_cancel_queued_and_in_flight(mock_lib):
    # one slot; wave 0 hangs until released, so later tickets wait in the queue
    srv = start(mock_lib, slots=1, hang=0, wave_max=1)
    t0 = srv.submit(b"ACGTACGT", 500)
    deadline = time.time() + 10
    while stats(mock_lib).launched_waves < 1:  # wave 0 (t0) is on the device
        assert time.time() < deadline
        time.sleep(0.001)
    queued = [srv.submit(b"ACGTAC" + bytes([65 + i]), 500) for i in range(5)]
    srv.cancel(t0)         # on the device: result dropped when its wave ends
    srv.cancel(queued[1])  # in the queue: never launched
    srv.cancel(queued[1])  # cancelling twice is harmless
    assert status_of(srv, t0) == cobs.COBS_ERR_CANCELLED
    assert status_of(srv, queued[1]) == cobs.COBS_ERR_CANCELLED
    srv.release(queued[1])
    with pytest.raises(cobs.CobsError) as e:
        srv.poll(queued[1])
    assert e.value.status == cobs.COBS_ERR_NOT_FOUND
    mock_lib.mock_release_hang()
    for i, t in enumerate(queued):
        if i != 1:
            assert wait(srv, t)[0] == 4
    assert status_of(srv, t0) == cobs.COBS_ERR_CANCELLED  # still cancelled after its wave ended
    st = stats(mock_lib)
    assert st.launched_requests == 5  # t0 and four queued; the cancelled queued one never ran
    s = srv.stop()
    assert s["cancelled"] == 2 and s["completed"] == 4


def test_cancel_after_finish_drops_result(mock_lib):
    srv = start(mock_lib)
    t = srv.submit(b"ACGTACGT", 500)
    time.sleep(0.05)
    srv.cancel(t)
    assert status_of(srv, t) == cobs.COBS_ERR_CANCELLED
    srv.stop()


def test_launch_failure_and_wave_failure(mock_lib):
    # wave 0 fails at launch (as an allocation failure does), wave 2 fails on the device
    srv = start(mock_lib, slots=1, fail_launch=0, fail_wave=2, wave_max=1)
    tickets = [srv.submit(b"ACGTACGTAC", 500) for _ in range(5)]
    got = [status_of(srv, t) for t in tickets]
    assert got[0] == cobs.COBS_ERR_OOM
    assert got.count(cobs.COBS_ERR_CUDA) == 1
    assert got.count(cobs.COBS_OK) == 3
    s = srv.stop()
    assert s["failed"] == 2


def test_timeout_and_slot_recovery(mock_lib):
    # wave 0 never finishes: its ticket times out, the other slot keeps serving,
    # and the first slot is usable again once its wave ends
    srv = start(mock_lib, slots=2, hang=0, wave_max=1, timeout_ms=100)
    t0 = srv.submit(b"ACGTACGT", 500)
    t_start = time.time()
    deadline = t_start + 10
    while stats(mock_lib).launched_waves < 1:  # wave 0 (t0) hangs on the first slot
        assert time.time() < deadline
        time.sleep(0.001)
    others = [srv.submit(b"ACGTACG" + bytes([65 + i % 4]), 500) for i in range(10)]
    for t in others:
        assert wait(srv, t)[0] == 5
    assert status_of(srv, t0) == cobs.COBS_ERR_TIMEOUT
    assert time.time() - t_start >= 0.09
    mock_lib.mock_release_hang()
    time.sleep(0.01)
    more = [srv.submit(b"ACGTACGT", 500) for _ in range(10)]
    for t in more:
        assert wait(srv, t)[0] == 5
    s = srv.stop()
    assert s["failed"] == 1 and s["completed"] == 20


def test_stop_finishes_queued_work(mock_lib):
    srv = start(mock_lib, slots=1, wave_us=1000, wave_max=2)
    tickets = [srv.submit(b"ACGTACGT", 500) for _ in range(12)]
    s = srv.stop()  # returns once the queue is empty and every wave has ended
    assert s["completed"] == 12 and s["waves"] >= 6 and len(tickets) == 12


# ------------------------------------------------------------- sanitizers

def _sanitized_run(tmp_path, name, srcs, san, env=None):
    exe = str(tmp_path / name)
    r = _compile(exe, srcs, ["-O1", "-g", "-fno-omit-frame-pointer", f"-fsanitize={san}"]
                 + (["-fno-sanitize-recover=all"] if "undefined" in san else []))
    if r.returncode != 0 and ("cannot find" in r.stderr or "-lasan" in r.stderr or "-ltsan" in r.stderr):
        pytest.skip(f"sanitizer runtime not installed: {r.stderr.strip().splitlines()[-1]}")
    assert r.returncode == 0, r.stderr
    e = dict(os.environ)
    e.update(env or {})
    p = subprocess.run([exe], capture_output=True, text=True, timeout=300, env=e)
    assert p.returncode == 0, p.stdout + p.stderr
    assert "WARNING: ThreadSanitizer" not in p.stderr and "ERROR: AddressSanitizer" not in p.stderr, p.stderr
    assert "runtime error" not in p.stderr, p.stderr
    return p.stdout


def test_scheduler_threadsanitizer(tmp_path):
    out = _sanitized_run(tmp_path, "stress_tsan",
                         SCHED_SRC + [os.path.join(NATIVE, "serve_mock.cpp"), os.path.join(NATIVE, "serve_stress.cpp")],
                         "thread", {"TSAN_OPTIONS": "halt_on_error=1 exitcode=66"})
    assert "errors 0" in out


def test_scheduler_address_ub_sanitizer(tmp_path):
    out = _sanitized_run(tmp_path, "stress_asan",
                         SCHED_SRC + [os.path.join(NATIVE, "serve_mock.cpp"), os.path.join(NATIVE, "serve_stress.cpp")],
                         "address,undefined", {"ASAN_OPTIONS": "detect_leaks=1"})
    assert "errors 0" in out


def test_oracle_address_ub_sanitizer(tmp_path):
    out = _sanitized_run(tmp_path, "oracle_asan",
                         [os.path.join(ROOT, "oracle", "cobs_oracle.cpp"), os.path.join(NATIVE, "oracle_sanitize.cpp")],
                         "address,undefined", {"ASAN_OPTIONS": "detect_leaks=1"})
    assert "0 errors" in out
