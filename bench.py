"""Benchmark of the COBS query path on GB300.

A step = one pass of the whole query path (distinct terms + hashes + row
indices, gather/AND/ADD with the fused threshold, hit compaction and sort) over
one batch of queries, with the index and the queries resident in HBM.

Default workload: the compact 10,000-document index (log-normal lengths,
median 100 kb), 10,000 queries of 1,000 bases with 1% substitutions, k = 31
canonical, h = 1, p = 0.3, blocks of 8,192, thresholds 0.5 / 0.8 / 1.0
(query i gets the (i mod 3)-th).  Inputs are seeded synthetic data.

Prints ONE JSON line (rank 0).  --impl reference times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "query k-mers/s (batched form, index and queries resident in HBM)"
UNIT = "k-mers/s"
L2_FLUSH_BYTES = 512 << 20


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def workload(name, path=None):
    """The named workload of the JSON workload file (synth/workloads.json unless
    --workloads names another)."""
    import synth
    return synth.workload(name, path)


def describe(wl, name):
    lens = np.diff(wl.q_off)
    return {"workload": f"{name}: {wl.name}", "n_docs": wl.n_docs, "doc_bytes": int(wl.doc_off[-1]),
            "n_queries": wl.n_queries, "query_bytes": int(wl.q_off[-1]),
            "query_len_min": int(lens.min()), "query_len_max": int(lens.max()),
            "term_kind": wl.term_kind, "q": wl.q, "num_hashes": wl.num_hashes, "fpr": wl.fpr,
            "block_docs": wl.block_docs, "score_bits": wl.score_bits,
            "thresholds_permille": sorted(set(int(t) for t in wl.thresholds))}


def run_config(wl, name, world):
    """The `config` object of the JSON line: the same keys and values in both
    arms (the workload, how L2 is handled between GPU steps, the parallelism);
    launch details of the GPU arm go to its `launch` object."""
    return dict(describe(wl, name),
                l2="GPU arm: a 512 MB write flushes L2 between timed steps, outside the timed events "
                   "(the CPU reference arm has no GPU)",
                parallelism=f"replicas x{world}" if world > 1 else "1 GPU")


def l2_read_peak(cobs, torch, stream, nbytes=64 << 20, reps=150, trials=5, ctas_per_sm=0):
    """Read bandwidth of the L2 cache measured here: cobs_probe_l2_read over a
    buffer well inside L2 (16-byte loads that bypass L1, a full grid), best of
    `trials` launches after a warming one, CUDA events on the launching stream."""
    buf = torch.ones(nbytes, dtype=torch.uint8, device="cuda")
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    best = 0.0
    for t in range(trials + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cobs.probe_l2_read(buf.data_ptr(), nbytes, reps, sink.data_ptr(), ctas_per_sm, stream.cuda_stream)
        e1.record(stream)
        e1.synchronize()
        if t:
            best = max(best, nbytes * reps / (e0.elapsed_time(e1) / 1e3) / 1e9)
    del buf, sink
    return best


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append((time.time(), ln.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        sm, mx, reasons = [], 0.0, set()
        for t, ln in self.lines:
            if not (t0 - 0.25 <= t <= t1 + 0.25):
                continue
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 10:
                continue
            try:
                sm.append(float(p[2]))
                mx = max(mx, float(p[3]))
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for nm, v in zip(names, p[6:10]):
                if v.lower() in ("active", "0x1", "1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def traffic_record(kernel_srcs, record="gather_batched_cfg2_dram.txt"):
    """A committed ncu record of a gather kernel on a bench workload (DRAM bytes
    per launch, L2 figures), or None when the kernel's sources changed since the
    counters were taken."""
    p = os.path.join(ROOT, "profiles", record)
    if not os.path.exists(p):
        return None
    kv = {}
    for ln in open(p):
        if "=" in ln and not ln.startswith("#"):
            k, v = ln.split("=", 1)
            kv[k.strip()] = v.strip()
    h = hashlib.sha256()
    for p_src in kernel_srcs:
        h.update(open(p_src, "rb").read())
    digest = h.hexdigest()[:16]
    if kv.get("kernel_sources_sha256_16") != digest:
        return None
    try:
        opt = lambda k: float(kv[k]) if k in kv else None  # noqa: E731  (L2 figures: not in every record)
        return {"dram_bytes": float(kv["dram_bytes_per_launch_full"]),
                "l2_hit_pct": opt("lts_t_sector_hit_rate_pct"),
                "l2_sector_lookups_pct_of_peak": opt("lts_t_sectors_srcunit_tex_pct_of_peak"),
                "slice_bytes": int(kv.get("slice_bytes", "128"))}
    except (KeyError, ValueError):
        return None


# ------------------------------------------------------------------ CPU oracle
def oracle_baseline(wl, sample_queries, budget_s=20.0, nthreads=None):
    """The oracle as it stands: its index built with the oracle functions on
    disjoint document ranges (threads, untimed), then single-threaded queries of
    a bounded sample timed."""
    import oracle
    t0 = time.perf_counter()
    ix = oracle.build_index_threaded(oracle.make_params(**wl.params()), wl.docs, wl.doc_off, nthreads)
    t_setup = time.perf_counter() - t0
    ql = wl.query_list()
    terms, n, t = 0, 0, 0.0
    for i in sample_queries:
        s = time.perf_counter()
        ell, _, _, _ = ix.query(ql[i], int(wl.thresholds[i]))
        t += time.perf_counter() - s
        terms += ell
        n += 1
        if t > budget_s:
            break
    # the same queries over all host cores: disjoint queries per thread, the
    # partitioned scoring of Sec. 2.3 (the oracle's query releases the GIL)
    from concurrent.futures import ThreadPoolExecutor
    ncores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    done = list(sample_queries[:n])
    s = time.perf_counter()
    with ThreadPoolExecutor(ncores) as ex:
        list(ex.map(lambda i: ix.query(ql[i], int(wl.thresholds[i])), done))
    t_all = time.perf_counter() - s
    return ix, {"value": terms / t if t else None, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"{n} queries of the workload (first {n} of a seeded sample), single thread; "
                          f"oracle index built untimed in {t_setup:.1f} s",
                "seconds": t, "terms": terms,
                "all_cores": {"value": terms / t_all if t_all else None, "cores": ncores, "seconds": t_all,
                              "sample": "the same queries, one thread per host core"}}


def run_l2_sweep(args):
    """--l2-sweep: the L2 read probe over buffer sizes and passes per launch
    (one JSON line per point); the bench's own ceiling is l2_read_peak."""
    import torch
    from paper_1905_09624_gb300 import cobs
    if not torch.cuda.is_available():
        raise SystemExit("--l2-sweep needs a CUDA GPU")
    stream = torch.cuda.Stream()
    for mb in (8, 16, 32, 48, 64, 96, 256, 1024):
        for reps in (10, 40):
            for cps in (0, 4):
                gbs = l2_read_peak(cobs, torch, stream, nbytes=mb << 20, reps=reps, trials=5, ctas_per_sm=cps)
                print(json.dumps({"buffer_mb": mb, "reps": reps, "ctas_per_sm": cps or 8, "gbs": gbs}), flush=True)
    print(json.dumps({"bench_l2_read_peak_gbs": l2_read_peak(cobs, torch, stream)}), flush=True)
    return 0


def run_reference(args):
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    wl = workload(args.config, args.workloads)
    import oracle
    ix = oracle.build_index_threaded(oracle.make_params(**wl.params()), wl.docs, wl.doc_off)
    ql = wl.query_list()
    rng = np.random.default_rng(12345)
    order = rng.permutation(wl.n_queries)
    per_step = max(1, args.ref_queries_per_step)
    pos = 0
    step_times, step_terms = [], []
    for s in range(args.warmup + args.steps):
        idx = [int(order[(pos + j) % wl.n_queries]) for j in range(per_step)]
        pos += per_step
        t0 = time.perf_counter()
        terms = 0
        for i in idx:
            terms += ix.query(ql[i], int(wl.thresholds[i]))[0]
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            step_times.append(dt)
            step_terms.append(terms)
    T = sum(step_times)
    value = sum(step_terms) / T
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / len(step_times),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
           "data": "synthetic (seeded)", "config": run_config(wl, args.config, args.gpus),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"{per_step} queries per step, single thread, oracle index built untimed"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def aggregate_over_ranks(seconds, units, dist=None, device="cpu"):
    """Whole-job throughput of N independent replicas: the slowest rank's time
    (max over ranks) and the units all ranks processed (sum).  With one process
    (dist None) it is (seconds, units)."""
    if dist is None:
        return float(seconds), float(units)
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ------------------------------------------------------------------ sharding
def gather_id_maps(gids, dist):
    """Every rank's shard id map, on rank 0 (None elsewhere); once per run."""
    if dist is None:
        return [gids]
    parts = [None] * dist.get_world_size() if dist.get_rank() == 0 else None
    dist.gather_object(gids, parts, dst=0)
    return parts


def exchange_and_merge(res, id_maps, dist):
    """The exchange step of the sharded path: every rank's hit lists of a batch
    (hit_offsets, shard-local ids, scores) go to rank 0, which merges them into
    the order of the unsharded index (cobs_hits_merge).  Returns the merged
    (hit_offsets, ids, scores) on rank 0, None elsewhere."""
    from paper_1905_09624_gb300 import cobs
    if dist is None:
        parts = [res]
    else:
        parts = [None] * dist.get_world_size() if dist.get_rank() == 0 else None
        dist.gather_object(res, parts, dst=0)
        if dist.get_rank() != 0:
            return None
    return cobs.hits_merge(parts, id_maps)


# -------------------------------------------------------------------- serve
def run_serve(dix, wl, rates, seconds, verify_oracle=None, inflight=3, wave_max=4096, workloads=None, form=0):
    """Poisson arrivals (cfg5 recipe on the given index) submitted at their
    arrival times from one thread, results polled from another; p50/p99 are the
    library's submit-to-visible latencies.  form COBS_PLAIN: every wave is one
    query in the plain form (the one-query-per-launch baseline).  Optionally
    checks a seeded 1% sample of the results against the oracle index."""
    import synth
    from paper_1905_09624_gb300 import cobs
    out = []
    for rate in rates:
        n = max(50, int(rate * seconds))
        params = dict(synth.serving_params("cfg5", workloads), n_q=n, rate=rate)
        qb, qo, thr, src, t_arr = synth.config5_queries(wl, **params)
        ql = [bytes(qb[int(qo[i]):int(qo[i + 1])]) for i in range(n)]
        srv = cobs.Server(dix, max_inflight_waves=inflight, max_wave_queries=wave_max, form=form)
        tickets = [None] * n
        results = [None] * n
        done_evt = threading.Event()

        def poller():
            pending = 0
            while True:
                progressed = False
                for i in range(pending, n):
                    if tickets[i] is None:
                        break
                    if results[i] is None:
                        r = srv.poll(tickets[i])
                        if r is None:
                            break
                        results[i] = r
                        progressed = True
                    if i == pending:
                        pending += 1
                if pending >= n:
                    done_evt.set()
                    return
                if not progressed:
                    time.sleep(0.0002)

        th = threading.Thread(target=poller, daemon=True)
        th.start()
        t0 = time.perf_counter()
        for i in range(n):
            while time.perf_counter() - t0 < t_arr[i]:
                pass
            tickets[i] = srv.submit(ql[i], int(thr[i]))
        done_evt.wait(timeout=120)
        stats = srv.stop()
        terms = sum(int(r[0]) for r in results if r is not None)
        rec = {"rate_qps": rate, "queries": n, "completed": int(stats["completed"]), "waves": int(stats["waves"]),
               "p50_ms": stats["p50_ms"], "p99_ms": stats["p99_ms"], "qps": stats["qps"],
               "kmers_per_s": terms / stats["seconds"] if stats["seconds"] else None,
               "mean_wave_queries": stats["mean_wave_queries"], "mean_wave_ms": stats["mean_wave_ms"],
               "max_wave_ms": stats["max_wave_ms"], "inflight_waves": inflight,
               "form": "plain (one query per wave and launch)" if form == cobs.COBS_PLAIN else "batched waves"}
        if verify_oracle is not None:
            # a seeded 1% sample of the requests, each an independent single-threaded
            # oracle query (run side by side on the host cores)
            from concurrent.futures import ThreadPoolExecutor
            sample = np.random.default_rng(5000 + int(rate)).choice(n, max(1, n // 100), replace=False)

            def same(i):
                ell, mn, ids, sc = verify_oracle.query(ql[i], int(thr[i]))
                r = results[i]
                return int(r is not None and r[0] == ell and r[1] == mn and np.array_equal(r[2], ids)
                           and np.array_equal(r[3], sc))

            with ThreadPoolExecutor(os.cpu_count() or 4) as ex:
                ok = sum(ex.map(same, sample.tolist()))
            rec["oracle_sample"] = f"{ok}/{len(sample)} identical"
        out.append(rec)
    return out


# ------------------------------------------------------------ other configs
HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e, nominal (the measured copy peak is the roofline)
CONFIG_RECORDS = {  # committed ncu records of the gather on a config's full workload
    "cfg4": ("gather_pipe_h3_cfg4_dram.txt", ["gather_h.cu", "gather_common.cuh"]),
    "cfg3": ("gather_pipe_cfg3_dram.txt", ["gather.cu", "gather_common.cuh"]),
}
PLAIN_SAMPLE = {"cfg1": 200, "cfg3": 1000, "cfg4": 10000}   # queries run in the plain form
ORACLE_SAMPLE = {"cfg1": 200, "cfg4": 200}                 # queries compared with the oracle


def _same_query(a, b, i, j):
    """Query i of result arrays a equals query j of result arrays b."""
    if a[0][i] != b[0][j] or a[1][i] != b[1][j]:
        return False
    sa = slice(int(a[2][i]), int(a[2][i + 1]))
    sb = slice(int(b[2][j]), int(b[2][j + 1]))
    return np.array_equal(a[3][sa], b[3][sb]) and np.array_equal(a[4][sa], b[4][sb])


def measure_config(name, args, cobs, torch, stream, flush, device, hbm_peak, l2_peak):
    """One more workload on this GPU: device build, the batched form as a
    captured graph (L2 flushed between steps), the plain form on a sample of
    its queries, and a sample compared with the oracle."""
    wl = workload(name, args.workloads)
    sh = stream.cuda_stream
    P = cobs.make_params(**wl.params())
    d_docs = torch.from_numpy(wl.docs).to("cuda")
    d_doff = torch.from_numpy(wl.doc_off.view(np.int64)).to("cuda")
    torch.cuda.synchronize()
    build_ms = []
    dix = None
    for rep in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        dix = None
        e0.record(stream)
        dix = cobs.DeviceIndex.build_resident(P, d_docs, d_doff, wl.doc_off, stream=sh)
        e1.record(stream)
        e1.synchronize()
        build_ms.append(e0.elapsed_time(e1))
    del d_docs, d_doff
    torch.cuda.empty_cache()
    info = dix.info()
    d_q = torch.from_numpy(wl.queries).to("cuda")
    d_off = torch.from_numpy(wl.q_off.view(np.int64)).to("cuda")
    d_thr = torch.from_numpy(wl.thresholds.view(np.int16)).to("cuda")
    torch.cuda.synchronize()
    eng = cobs.Engine(dix, stream=sh)
    tuned = None
    if name in [c for c in args.autotune_configs.split(",") if c]:
        t0 = time.perf_counter()
        tuned = eng.autotune(d_q, d_off, wl.q_off, d_thr)
        tuned["seconds"] = time.perf_counter() - t0
    steps = args.cfg3_steps if name == "cfg3" else args.config_steps
    ms, gms, terms, rows, launches = [], [], 0, 0, 0
    for i in range(3 + steps):
        with torch.cuda.stream(stream):
            flush.fill_(i & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        eng.query_device(d_q, d_off, wl.q_off, d_thr, cobs.COBS_GRAPH)
        e1.record(stream)
        st = eng.stats()
        if i >= 3:
            ms.append(e0.elapsed_time(e1))
            gms.append(st["ms_gather"])
            terms += st["terms"]
            rows += st["row_bytes"]
            launches += st["launches"]
    batched = eng.download_arrays()
    t_step = float(np.mean(ms)) / 1e3
    g_step = float(np.mean(gms)) / 1e3
    value = terms / steps / t_step
    logical = rows / steps / g_step / 1e9
    # the plain form on the first m queries, as its own batch
    m = min(wl.n_queries, PLAIN_SAMPLE.get(name, 1000))
    qo = wl.q_off[:m + 1].copy()
    sub_q = torch.from_numpy(wl.queries[:int(qo[-1])]).to("cuda")
    sub_off = torch.from_numpy(qo.view(np.int64)).to("cuda")
    sub_thr = torch.from_numpy(wl.thresholds[:m].view(np.int16)).to("cuda")
    torch.cuda.synchronize()
    pms, pst = [], None
    for rep in range(2):
        with torch.cuda.stream(stream):
            flush.fill_(rep)
        eng.query_device(sub_q, sub_off, qo, sub_thr, cobs.COBS_PLAIN)
        pst = eng.stats()
        pms.append(pst["ms_total"])
    plain_res = eng.download_arrays()
    plain_same = all(_same_query(plain_res, batched, i, i) for i in range(m))
    plain_value = pst["terms"] / (min(pms) / 1e3)
    st = eng.stats()
    out = {"workload": describe(wl, name), "steps": steps, "warmup": 3, "form": "graph",
           "launch": {"slice_bytes": st["slice_bytes"], "ctas_per_sm": st["ctas_per_sm"], "autotuned": tuned},
           "value": value, "unit": UNIT, "ms_per_step": 1e3 * t_step, "gather_ms_per_step": 1e3 * g_step,
           "gpu_launches_per_step": launches / steps,
           "row_gbs_logical": logical, "row_frac_of_l2_peak": logical / l2_peak if l2_peak else None,
           "reuse": logical / hbm_peak,
           "plain": {"value": plain_value, "unit": UNIT, "queries": m, "ms": min(pms),
                     "results_identical_to_batched": bool(plain_same)},
           "speedup_batched_over_plain": value / plain_value if plain_value else None,
           "build": {"ms_device": min(build_ms), "input_bytes": int(wl.doc_off[-1]),
                     "gbs_device": int(wl.doc_off[-1]) / (min(build_ms) / 1e3) / 1e9,
                     "index_bytes": info["rows_bytes"], "blocks": len(info["blocks"])}}
    rec_name = CONFIG_RECORDS.get(name)
    rec = None
    if rec_name:
        csrc = os.path.join(ROOT, "paper_1905_09624_gb300", "csrc")
        rec = traffic_record([os.path.join(csrc, f) for f in rec_name[1]], rec_name[0])
    out["row_gbs_physical"] = rec["dram_bytes"] / g_step / 1e9 if rec else None
    out["physical_note"] = (f"ncu DRAM bytes of one step's gather launches (profiles/{rec_name[0]}) over the "
                            "live gather time"
                            if rec else "no current ncu record of this workload's gather")
    del eng, sub_q, sub_off, sub_thr, d_q, d_off, d_thr
    ns = ORACLE_SAMPLE.get(name, 0)
    if ns and not args.skip_cpu:
        import oracle
        ix = oracle.build_index_threaded(oracle.make_params(**wl.params()), wl.docs, wl.doc_off)
        ql = wl.query_list()
        sample = np.random.default_rng(909).choice(wl.n_queries, min(ns, wl.n_queries), replace=False)
        ok, t_cpu, cpu_terms = 0, 0.0, 0
        for i in sample.tolist():
            t0 = time.perf_counter()
            ell, mn, ids, sc = ix.query(ql[i], int(wl.thresholds[i]))
            t_cpu += time.perf_counter() - t0
            cpu_terms += ell
            h0, h1 = int(batched[2][i]), int(batched[2][i + 1])
            ok += int(batched[0][i] == ell and batched[1][i] == mn and np.array_equal(batched[3][h0:h1], ids)
                      and np.array_equal(batched[4][h0:h1], sc))
        out["oracle_sample"] = f"{ok}/{len(sample)} identical (batched graph form vs the oracle)"
        out["cpu_baseline"] = {"value": cpu_terms / t_cpu if t_cpu else None, "unit": UNIT, "cores": 1,
                               "kind": "oracle", "sample": f"the same {len(sample)} queries, single thread"}
        del ix
    else:
        out["oracle_sample"] = ("not run in the bench (the oracle's index of this workload takes minutes on the "
                                "host cores); full-size parity is in tests/test_gpu_fullsize.py")
    del dix, wl
    torch.cuda.empty_cache()
    return out


# --------------------------------------------------------------- sharded GPU
def run_gpu_sharded(args):
    """--shard: document-block sharding over the ranks (one GPU each).  Every
    rank builds the index, keeps the blocks of its shard (cobs_shard_plan /
    cobs_index_shard) and answers every query of the batch over its documents
    (graph form); a step ends with the exchange: the ranks' hit lists to rank 0,
    merged into the order of the unsharded index.  The batch and the index are
    fixed as N grows ("scaling": "strong"); value = distinct query terms of the
    batch (each over the whole index) / the slowest rank's step time."""
    import torch
    from paper_1905_09624_gb300 import cobs
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the CUDA library has no CPU path)")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    wl = workload(args.config, args.workloads)
    stream = torch.cuda.Stream()
    P = cobs.make_params(**wl.params())
    host = cobs.DeviceIndex.build(P, wl.docs, wl.doc_off, device=local).download()
    plan, shard_bytes = host.shard_plan(world)
    sub, gids = host.shard(plan, rank)
    sdix = cobs.DeviceIndex.load(sub, device=local)
    del host
    maps = gather_id_maps(gids, dist)
    eng = cobs.Engine(sdix, stream=stream.cuda_stream)
    d_q = torch.from_numpy(wl.queries).to("cuda")
    d_off = torch.from_numpy(wl.q_off.view(np.int64)).to("cuda")
    d_thr = torch.from_numpy(wl.thresholds.view(np.int16)).to("cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()

    def step():
        with torch.cuda.stream(stream):
            flush.fill_(rank + 1)
        eng.query_device(d_q, d_off, wl.q_off, d_thr, cobs.COBS_GRAPH)
        res = eng.download_arrays()
        merged = exchange_and_merge((res[2], res[3], res[4]), maps, dist)
        return res, merged

    for _ in range(args.warmup):
        step()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    terms = 0
    for _ in range(args.steps):
        res, merged = step()
        terms += int(np.sum(res[0]))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    dt = time.perf_counter() - t0
    T, _ = aggregate_over_ranks(dt, terms, dist, device="cuda")
    if rank == 0:
        out = {"metric": METRIC + ", document blocks sharded over the GPUs", "value": terms / T, "unit": UNIT,
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
               "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "u32",
               "data": "synthetic (seeded)", "config": dict(run_config(wl, args.config, world),
                                                            parallelism=f"document-block shards x{world}"),
               "shards": {"block_shard": plan.tolist(), "shard_bytes": shard_bytes.tolist(),
                          "exchange": "hit lists gathered to rank 0 (gather_object), cobs_hits_merge",
                          "hits_per_step": int(merged[0][-1])},
               "timing": "wall clock per step (query, hit download, exchange, merge), barriers on both sides, "
                         "max over ranks"}
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------- GPU
def run_gpu(args):
    import torch
    from paper_1905_09624_gb300 import cobs

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the CUDA library has no CPU path)")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    wl = workload(args.config, args.workloads)
    L = cobs.lib()
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream

    # ---- device build (documents already in HBM), and with the H2D copy
    P = cobs.make_params(**wl.params())
    d_docs = torch.from_numpy(wl.docs).to("cuda")
    d_doff = torch.from_numpy(wl.doc_off.view(np.int64)).to("cuda")
    torch.cuda.synchronize()
    build_ms = []
    dix = None
    for rep in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            dix = cobs.DeviceIndex.build_resident(P, d_docs, d_doff, wl.doc_off, stream=sh)
            e1.record(stream)
        e1.synchronize()
        build_ms.append(e0.elapsed_time(e1))
    build_h2d = []
    for rep in range(2):  # best of two, as the device-resident build
        t0 = time.perf_counter()
        dix_h2d = cobs.DeviceIndex.build(P, wl.docs, wl.doc_off, device=local)
        build_h2d.append(time.perf_counter() - t0)
        del dix_h2d
    build_h2d_s = min(build_h2d)
    del d_docs, d_doff
    info = dix.info()
    rows_per_term = sum(b["rowbytes"] for b in info["blocks"]) * wl.num_hashes

    # ---- queries resident in HBM
    d_q = torch.from_numpy(wl.queries).to("cuda")
    d_off = torch.from_numpy(wl.q_off.view(np.int64)).to("cuda")
    d_thr = torch.from_numpy(wl.thresholds.view(np.int16)).to("cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()

    eng = cobs.Engine(dix, stream=sh, slice_bytes=args.slice_bytes, ctas_per_sm=args.ctas_per_sm,
                     gather_feed=args.gather_feed, l2_hints=args.l2_hints)
    tuned = None
    if args.autotune:
        tuned = eng.autotune(d_q, d_off, wl.q_off, d_thr)

    def step(flags):
        eng.query_device(d_q, d_off, wl.q_off, d_thr, flags)

    def flush_l2():
        with torch.cuda.stream(stream):
            flush.fill_(rank + 1)

    form = cobs.COBS_GRAPH if args.form == "graph" else cobs.COBS_BATCHED
    for _ in range(args.warmup):
        flush_l2()
        step(form)
        eng.stats()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier()
    stream.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    gather_ms, launches, terms_total, row_bytes_total = [], 0, 0, 0
    t_wall0 = time.time()
    for i in range(args.steps):
        flush_l2()
        ev[i][0].record(stream)
        step(form)
        ev[i][1].record(stream)
        st = eng.stats()  # synchronises this step
        gather_ms.append(st["ms_gather"])
        launches += st["launches"]
        terms_total += st["terms"]
        row_bytes_total += st["row_bytes"]
    stream.synchronize()
    barrier()
    t_wall1 = time.time()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    # ---- the L2 read ceiling of the gather, measured now (clocks sampled meanwhile)
    t_l2_0 = time.time()
    l2_peak = l2_read_peak(cobs, torch, stream)
    t_l2_1 = time.time()
    T, terms_all = aggregate_over_ranks(sum(step_ms) / 1e3, terms_total, dist, device="cuda")
    value = terms_all / T

    phases = {k: st[k] for k in ("ms_terms", "ms_gather", "ms_hits", "ms_total", "ms_host")}
    # ---- results of the timed form, kept for the plain comparison
    batched_res = eng.download_arrays()

    # ---- end to end through the public host-buffer API (H2D + query + D2H)
    e2e_times = []
    h2d = int(wl.q_off[-1]) + wl.q_off.nbytes + wl.thresholds.nbytes
    d2h = 0
    # the step's inputs sit in page-locked host memory, as a serving front end keeps them
    pin_q = torch.empty(len(wl.queries), dtype=torch.uint8, pin_memory=True).numpy()
    pin_q[:] = wl.queries
    for i in range(max(2, args.e2e_steps) + 1):
        t0 = time.perf_counter()
        res = eng.query_host_arrays(pin_q, wl.q_off, wl.thresholds, form)
        dt = time.perf_counter() - t0
        if i:
            e2e_times.append(dt)
        # per query: terms, threshold, hit offset; per hit: id, score
        d2h = wl.n_queries * 4 * 2 + (wl.n_queries + 1) * 8 + len(res[3]) * 8
    e2e_sync_value = terms_total / args.steps / float(np.mean(e2e_times))
    # pipelined: E engines (own streams) take batches in turn, E - 1 batches in
    # flight, so one batch's copies and host planning overlap the others' kernels;
    # with --e2e-streams 1 they share the first engine's stream (their kernels
    # then queue behind each other instead of sharing the GPU)
    n_eng = max(2, args.e2e_engines)
    extra = [cobs.Engine(dix, stream=(torch.cuda.Stream() if args.e2e_streams == 2 else stream).cuda_stream,
                         slice_bytes=args.slice_bytes, ctas_per_sm=args.ctas_per_sm, gather_feed=args.gather_feed,
                         l2_hints=args.l2_hints) for _ in range(n_eng - 1)]
    engs = [eng] + extra
    n_pipe = max(20, args.e2e_steps)
    for e in engs:  # warm all (graph capture, buffers)
        e.submit_host(pin_q, wl.q_off, wl.thresholds, form)
        e.download_arrays()
    t0 = time.perf_counter()
    for i in range(n_pipe + n_eng - 1):
        if i < n_pipe:
            engs[i % n_eng].submit_host(pin_q, wl.q_off, wl.thresholds, form)
        j = i - (n_eng - 1)
        if j >= 0:
            res = engs[j % n_eng].download_arrays()
    pipe_s = (time.perf_counter() - t0) / n_pipe
    e2e_value = terms_total / args.steps / pipe_s
    del extra, engs

    # ---- plain form (one query per kernel sequence) on the same batch
    plain = None
    if not args.skip_plain:
        pr = []
        for rep in range(2):
            flush_l2()
            step(cobs.COBS_PLAIN)
            pr.append(eng.stats())
        plain_res = eng.download_arrays()
        same = all(np.array_equal(a, b) for a, b in zip(plain_res, batched_res))
        pt = min(p["ms_total"] for p in pr) / 1e3
        # the same batch in the plain form through the host-buffer API (H2D of the
        # queries, one query per launch, D2H of the hits)
        t0 = time.perf_counter()
        plain_host = eng.query_host_arrays(pin_q, wl.q_off, wl.thresholds, cobs.COBS_PLAIN)
        pe2e = time.perf_counter() - t0
        same_host = all(np.array_equal(a, b) for a, b in zip(plain_host, batched_res))
        plain = {"value": pr[0]["terms"] / pt, "unit": UNIT, "ms": pt * 1e3,
                 "us_per_query": pt * 1e6 / wl.n_queries,
                 "row_gbs_logical": pr[0]["row_bytes"] / pt / 1e9,
                 "launches": pr[0]["launches"], "results_identical_to_batched": bool(same and same_host),
                 "e2e": {"value": pr[0]["terms"] / pe2e, "unit": UNIT, "ms": pe2e * 1e3,
                         "h2d_bytes": h2d, "path": "query_host_arrays, plain form"}}
    # ---- hit emission under many hits: the first 1,000 queries at K = 1 permille
    # (min score 1: nearly every document is a hit) against the same queries at
    # the workload's thresholds, batched form, gather and hit phases
    low_k = None
    if not args.skip_low_k:
        m = min(1000, wl.n_queries)
        qo = wl.q_off[:m + 1].copy()
        sq = torch.from_numpy(wl.queries[:int(qo[-1])]).to("cuda")
        so = torch.from_numpy(qo.view(np.int64)).to("cuda")
        low_k = {"queries": m}
        for label, thr_host in (("workload_thresholds", wl.thresholds[:m].copy()),
                                ("k_1_permille", np.ones(m, np.uint16))):
            st_thr = torch.from_numpy(thr_host.view(np.int16)).to("cuda")
            torch.cuda.synchronize()
            runs = []
            for rep in range(4):
                flush_l2()
                eng.query_device(sq, so, qo, st_thr, cobs.COBS_BATCHED)
                runs.append(eng.stats())
            hits = int(eng.download_arrays()[2][-1])
            best = min(runs[1:], key=lambda r: r["ms_gather"])
            low_k[label] = {"ms_gather": best["ms_gather"], "ms_hits": best["ms_hits"], "hits": hits}
        del sq, so, st_thr
    # ---- the same batch on a streamed copy of the index: rows in pinned host
    # memory, copied block by block into a ring of device slots every step
    streamed = None
    if not args.skip_streamed:
        sdix = cobs.DeviceIndex.load_streamed(dix.download(), device=local)
        seng = cobs.Engine(sdix, stream=sh, slice_bytes=args.slice_bytes, ctas_per_sm=args.ctas_per_sm,
                     gather_feed=args.gather_feed, l2_hints=args.l2_hints,
                           stage_bytes=args.stage_bytes)
        for _ in range(3):
            flush_l2()
            seng.query_device(d_q, d_off, wl.q_off, d_thr, form)
            seng.stats()
        s_ms, s_terms = [], 0
        for i in range(args.streamed_steps):
            flush_l2()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            seng.query_device(d_q, d_off, wl.q_off, d_thr, form)
            e1.record(stream)
            sst = seng.stats()
            s_ms.append(e0.elapsed_time(e1))
            s_terms += sst["terms"]
        same = all(np.array_equal(a, b) for a, b in zip(seng.download_arrays(), batched_res))
        slot = max(b["w"] * b["rowbytes"] for b in info["blocks"])
        slot = (slot + 255) // 256 * 256
        n_slots = min(len(info["blocks"]), args.stage_bytes // slot if args.stage_bytes else 2)
        sm = float(np.mean(s_ms))
        # the host link's ceiling: one 512 MB copy from pinned memory, best of 5
        lk_h = torch.empty(512 << 20, dtype=torch.uint8, pin_memory=True)
        lk_d = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
        lk = []
        with torch.cuda.stream(stream):
            for i in range(6):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                lk_d.copy_(lk_h, non_blocking=True)
                e1.record(stream)
                e1.synchronize()
                if i:
                    lk.append(e0.elapsed_time(e1))
        link_gbs = lk_d.numel() / (min(lk) / 1e3) / 1e9
        del lk_h, lk_d
        h2d_gbs = sst["h2d_index_bytes"] / (sm / 1e3) / 1e9
        streamed = {"value": s_terms / args.streamed_steps / (sm / 1e3), "unit": UNIT, "ms_per_step": sm,
                    "steps": args.streamed_steps, "h2d_index_bytes_per_step": sst["h2d_index_bytes"],
                    "h2d_index_gbs": h2d_gbs, "link_gbs": link_gbs, "link_frac": h2d_gbs / link_gbs,
                    "link_rule": "index bytes copied per step / step time, over one 512 MB pinned copy's rate",
                    "stage_slots": n_slots, "rows_host_numa_node": sst["stream_numa_node"],
                    "stage_bytes": n_slots * slot, "index_bytes": info["rows_bytes"],
                    "results_identical_to_resident": bool(same)}
        del seng, sdix
    # ---- multi-index querying: a view over two indexes of half the documents each
    multi = None
    if not args.skip_multi and wl.n_docs >= 2:
        half = wl.n_docs // 2
        parts = []
        for lo, hi in ((0, half), (half, wl.n_docs)):
            o = wl.doc_off[lo:hi + 1] - wl.doc_off[lo]
            parts.append(cobs.DeviceIndex.build(P, wl.docs[int(wl.doc_off[lo]):int(wl.doc_off[hi])], o,
                                                device=local))
        view = cobs.DeviceIndex.multi(parts)
        meng = cobs.Engine(view, stream=sh, slice_bytes=args.slice_bytes, ctas_per_sm=args.ctas_per_sm,
                     gather_feed=args.gather_feed, l2_hints=args.l2_hints)
        for _ in range(3):
            flush_l2()
            meng.query_device(d_q, d_off, wl.q_off, d_thr, form)
            meng.stats()
        m_ms, m_terms, m_rows = [], 0, 0
        for i in range(args.streamed_steps):
            flush_l2()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            meng.query_device(d_q, d_off, wl.q_off, d_thr, form)
            e1.record(stream)
            mst = meng.stats()
            m_ms.append(e0.elapsed_time(e1))
            m_terms += mst["terms"]
            m_rows += mst["row_bytes"]
        mm = float(np.mean(m_ms))
        multi = {"value": m_terms / args.streamed_steps / (mm / 1e3), "unit": UNIT, "ms_per_step": mm,
                 "steps": args.streamed_steps, "parts": 2, "blocks": len(view.info()["blocks"]),
                 "row_gbs_logical": m_rows / args.streamed_steps / (mm / 1e3) / 1e9}
        del meng, view, parts
    # ---- incremental insertion: 5 % more documents of the same length law
    insert = None
    if not args.skip_insert and wl.n_docs >= 20:
        import synth
        n_new = max(1, wl.n_docs // 20)
        lens = (wl.doc_off[1:] - wl.doc_off[:-1]).astype(np.int64)
        rng = np.random.default_rng(4242)
        new_lens = rng.choice(lens, n_new)
        if wl.term_kind == 2:
            words, word_off = synth.vocab(4244, 2000)
            new_docs, new_off = synth.text_docs(4243, new_lens.astype(np.uint64), words, word_off)
        else:
            new_docs, new_off = synth.dna_docs(4243, new_lens.astype(np.uint64))
        host_ix = dix.download()
        t0 = time.perf_counter()
        ins = host_ix.insert(new_docs, new_off, device=local)
        t_ins = time.perf_counter() - t0
        ii = ins.info()
        insert = {"new_docs": int(n_new), "new_bytes": int(new_off[-1]), "seconds": t_ins,
                  "blocks_before": len(info["blocks"]), "blocks_after": len(ii["blocks"]),
                  "into_free_columns": int(sum(b["n_docs"] for b in ii["blocks"][:len(info["blocks"])]) - wl.n_docs),
                  "note": "cobs_index_insert on the host index: the time includes copying the index to the "
                          "device and back"}
        del ins, host_ix
    sampler.stop()
    clocks = sampler.summary(t_wall0, t_wall1)

    peak, peak_kind = measured_peaks()
    g_ms = float(np.mean(gather_ms))
    alg_bytes = row_bytes_total / args.steps
    achieved = alg_bytes / (g_ms / 1e3) / 1e9 if g_ms > 0 else None
    # the committed ncu record covers the bench workload (cfg2) in the default
    # launch configuration only
    default_launch = args.slice_bytes == 0 and args.ctas_per_sm == 0 and not args.autotune \
        and args.gather_feed == 0 and args.l2_hints == 0
    csrc = os.path.join(ROOT, "paper_1905_09624_gb300", "csrc")
    rec = traffic_record([os.path.join(csrc, "gather.cu"), os.path.join(csrc, "gather_common.cuh")]) \
        if args.config == "cfg2" and default_launch else None
    if rec and rec["slice_bytes"] != eng.stats()["slice_bytes"]:
        rec = None  # taken with another slice width
    kname = "k_gather_pipe" if wl.num_hashes == 1 else "k_gather_pipe_h" if wl.num_hashes <= 4 else "k_gather_batched"
    hbm_kind = (f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                else "fallback")
    # The gather reads every row slice of a batch through L2 many times (each
    # distinct row once from HBM per residency): its logical row bytes are bound
    # by the L2's read bandwidth, measured in this run; the DRAM side is the ncu
    # traffic of the same launch over the live launch time.
    dram_gbs = rec["dram_bytes"] / (g_ms / 1e3) / 1e9 if rec and g_ms > 0 else None
    roofline = {"bound": "l2", "kernel": kname, "achieved": achieved, "peak": l2_peak, "unit": "GB/s",
                "frac": achieved / l2_peak if achieved and l2_peak else None,
                "peak_kind": "measured in this run: L2 read bandwidth (cobs_probe_l2_read: 64 MB buffer read "
                             "150 times per launch, 16-byte L1-bypassing loads, best of 5 launches, CUDA events)",
                "traffic": rec["dram_bytes"] if rec else None, "algorithmic_bytes_per_launch": alg_bytes,
                "launch_ms": g_ms, "bytes_rule": "sum over distinct query terms and blocks of h * rowbytes_b",
                "dram_gbs": dram_gbs, "dram_frac": dram_gbs / peak if dram_gbs else None,
                "hbm_peak": peak, "hbm_peak_kind": hbm_kind,
                "dram_frac_of_nominal": dram_gbs / HBM_NOMINAL_GBS if dram_gbs else None,
                "hbm_nominal": HBM_NOMINAL_GBS,
                "reuse": achieved / peak if achieved else None,
                "reuse_rule": "logical row bytes per second over the HBM peak: above 1 only through L2 reuse",
                "l2_hit_pct": rec["l2_hit_pct"] if rec else None,
                "l2_sector_lookups_pct_of_peak": rec["l2_sector_lookups_pct_of_peak"] if rec else None,
                "l2_probe_clocks": sampler.summary(t_l2_0, t_l2_1)}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded)",
           "config": run_config(wl, args.config, world),
           "launch": {"form": args.form, "slice_bytes": eng.stats()["slice_bytes"],
                      "ctas_per_sm": eng.stats()["ctas_per_sm"], "autotuned": tuned},
           "row_gbs_logical": row_bytes_total / T / 1e9,
           "roofline": roofline,
           "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                   "ms_per_step": 1e3 * pipe_s, "steps": n_pipe,
                   "mode": f"{n_eng} engines on {args.e2e_streams if args.e2e_streams == 1 else n_eng} stream(s) taking "
                           "batches in turn with cobs_engine_submit_host / cobs_engine_download "
                           "(pinned query bytes); every step copies its inputs in and its hits out",
                   "one_call_at_a_time": {"value": e2e_sync_value, "ms_per_step": 1e3 * float(np.mean(e2e_times)),
                                          "call": "cobs_engine_query_host"}},
           "gpu_launches": launches, "clocks": clocks, "phases_ms_last_step": phases, "plain": plain,
           "build": {"ms_device": min(build_ms), "input_bytes": int(wl.doc_off[-1]),
                     "gbs_device": int(wl.doc_off[-1]) / (min(build_ms) / 1e3) / 1e9,
                     "gbs_with_h2d": int(wl.doc_off[-1]) / build_h2d_s / 1e9,
                     "index_bytes": info["rows_bytes"], "blocks": len(info["blocks"])},
           "speedup_batched_over_plain": (value / plain["value"]) if plain else None,
           "streamed": streamed, "multi_index": multi, "insert": insert, "many_hits": low_k}
    if plain:
        out["plain"]["frac_of_hbm_peak"] = plain["row_gbs_logical"] / peak

    oracle_ix = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        rng = np.random.default_rng(777)
        sample = rng.permutation(wl.n_queries)[:args.cpu_queries].tolist()
        oracle_ix, cpu = oracle_baseline(wl, sample, budget_s=args.cpu_budget_s)
        out["cpu_baseline"] = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample", "all_cores")}
    if args.serve_rates and args.config == "cfg2":
        del eng
        rates = [float(r) for r in args.serve_rates.split(",") if r]
        out["serve"] = run_serve(dix, wl, rates, args.serve_seconds, verify_oracle=oracle_ix,
                                 inflight=args.serve_inflight, wave_max=args.serve_wave_max,
                                 workloads=args.workloads)
        # the same arrivals served by the plain form: one query per wave and
        # launch, one wave at a time
        out["serve_plain"] = run_serve(dix, wl, rates, args.serve_seconds, verify_oracle=oracle_ix, inflight=1,
                                       wave_max=1, workloads=args.workloads, form=cobs.COBS_PLAIN)
    del dix, oracle_ix
    if args.configs and world == 1:
        out["configs"] = {}
        for name in [c for c in args.configs.split(",") if c and c != args.config]:
            out["configs"][name] = measure_config(name, args, cobs, torch, stream, flush, local, peak, l2_peak)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--config", default="cfg2")
    ap.add_argument("--form", default="graph", choices=["batched", "graph"],
                    help="graph: the batched launch sequence captured once and replayed (default)")
    ap.add_argument("--slice-bytes", type=int, default=0)
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--skip-streamed", action="store_true", help="skip the streamed-index measurement")
    ap.add_argument("--streamed-steps", type=int, default=10, help="timed steps of the streamed and multi-index runs")
    ap.add_argument("--skip-multi", action="store_true", help="skip the multi-index measurement")
    ap.add_argument("--skip-insert", action="store_true", help="skip the incremental-insertion measurement")
    ap.add_argument("--skip-low-k", action="store_true", help="skip the K = 1 permille hit-emission measurement")
    ap.add_argument("--gather-feed", type=int, default=0, help="0 default, 1 cp.async ring, 2 TMA gather")
    ap.add_argument("--l2-hints", type=int, default=0, help="L2 eviction hints of the gather (0 default, 1..4)")
    ap.add_argument("--workloads", default=None,
                    help="JSON file of named workloads (recipe + parameters); default synth/workloads.json")
    ap.add_argument("--e2e-engines", type=int, default=4,
                    help="engines taking end-to-end batches in turn (batches in flight + 1)")
    ap.add_argument("--e2e-streams", type=int, default=2, choices=[1, 2],
                    help="pipelined end to end: every engine on its own stream (2) or all on one (1)")
    ap.add_argument("--stage-bytes", type=int, default=0, help="streamed index: device staging bytes (0 = 2 slots)")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--cpu-queries", type=int, default=400)
    ap.add_argument("--cpu-budget-s", type=float, default=15.0)
    ap.add_argument("--ref-queries-per-step", type=int, default=40)
    ap.add_argument("--serve-rates", default="1000,5000,10000,20000,50000",
                    help="Poisson arrival rates (queries/s) of the serving run on the cfg2 index; '' to skip")
    ap.add_argument("--serve-seconds", type=float, default=1.5)
    ap.add_argument("--serve-inflight", type=int, default=3, help="waves on the device at once")
    ap.add_argument("--serve-wave-max", type=int, default=4096, help="queries per wave at most")
    ap.add_argument("--l2-sweep", action="store_true", help="print the L2 read probe over buffer sizes and exit")
    ap.add_argument("--shard", action="store_true",
                    help="document-block sharding over the ranks instead of replicas (strong scaling)")
    ap.add_argument("--configs", default="cfg1,cfg4,cfg3",
                    help="further workloads measured after the main one ('' to skip): batched graph form, "
                         "plain form on a sample, device build, oracle sample")
    ap.add_argument("--config-steps", type=int, default=10, help="timed steps of each further workload")
    ap.add_argument("--autotune-configs", default="cfg3",
                    help="further workloads whose engine is autotuned on their batch before the timed steps")
    ap.add_argument("--cfg3-steps", type=int, default=3, help="timed steps of cfg3 (about 0.25 s each)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.l2_sweep:
        return run_l2_sweep(args)
    if args.shard:
        return run_gpu_sharded(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
