"""Benchmark: trial-event-ELT evaluations per second of one ARA layer.

Workload (the paper-shaped single layer): a YET of 1,000,000 trials with
Poisson(1000) events drawn uniformly from a catalogue of 2,000,000 event ids,
one layer over 15 ELTs of 10,000 records each (mean ~ LogNormal(10, 2),
exposure = mean * U(2, 20), sigma = mean * U(0.1, 1.0) clipped so both Beta
shapes stay >= 0.05), percentile-set layer terms, Philox seed 0, PML and TVaR
at return periods 100 and 250.  Synthetic stand-in for the paper's
proprietary industry YET/ELTs (Section 5).

One step = the whole hot path: per-layer index build, the fused layer kernel
(YET stream, lookup, Philox, inverse Beta, ELT terms, sum over ELTs,
occurrence terms, FP64 running sum, aggregate terms, YLT), and PML/TVaR by
radix select.  ``value`` is evals / second with the inputs resident in HBM
(the 4 GB YET exceeds the 129 MB L2, so no L2 flush is needed); ``e2e`` is
the same metric through the C ABI with the YET, the ELTs and the results in
host memory, the copies inside the timed region (the YET upload runs beside
the ELT load).

``--impl reference`` times the FP64 CPU oracle (the reference arm: there is
no reference implementation to install, only the paper) on a bounded sample
of the same workload.

Launch: ``python bench.py [--gpus N --steps K --warmup W]``; for N > 1 under
torchrun (one process per GPU, weak scaling: every rank runs its own
1M-trial shard with its own seed; the exact global PML/TVaR comes from each
rank's top m = ceil(N_total / RP) year losses (ara_top_m), one all-gather of
them, and the C-ABI merge ara_merge_top).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "paper-1m"
RETURN_PERIODS = (100.0, 250.0)
METRIC = "trial-event-ELT evals/s (1M-trial ARA)"
UNIT = "evals/s"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _terms():
    with open(os.path.join(ROOT, "tests", "golden", "workload_terms.json")) as fh:
        return json.load(fh)[WORKLOAD]["layer_terms"]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal
LAYER_SOURCES = ("ara_layer.cu", "ara_device_math.cuh", "ara_internal.h")  # what k_gather and k_losses compile from


def _kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1501_06326_gb300", "csrc")
    for f in LAYER_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profiled_layer(key):
    """A per-launch figure of the layer kernels from the committed ncu capture
    (profiles/k_layer_paper-1m.json, beside its summary), if it was taken on the
    current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "k_layer_paper-1m.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != _kernel_source_hash():
        return None
    v = d.get(key)
    return float(v) if v is not None else None


def _profiled_traffic():
    """DRAM bytes per launch of the layer kernels (ncu), or None."""
    return _profiled_layer("dram_bytes_per_full_launch")


def _usable_cores() -> int:
    """Host cores this process may run on (its CPU affinity)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5], parts[6], parts[7], parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        reasons = set()
        for r in rows:
            for name, flag in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), r[2:]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median([r[0] for r in rows])), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


def _memory_nodes(ptr: int, nbytes: int, gpu: int):
    """NUMA nodes of the pages of a host buffer (move_pages on sampled pages) and
    the NUMA node of the GPU's PCI device, or None where the host does not say."""
    import ctypes
    import platform

    out = {"buffer_nodes": None, "gpu_node": None}
    nr = {"aarch64": 239, "x86_64": 279}.get(platform.machine())
    try:
        if nr is not None:
            libc = ctypes.CDLL(None, use_errno=True)
            page = os.sysconf("SC_PAGE_SIZE")
            k = 16
            addrs = (ctypes.c_void_p * k)(*[(ptr + i * (nbytes // k)) // page * page for i in range(k)])
            status = (ctypes.c_int * k)()
            if libc.syscall(nr, 0, k, addrs, None, status, 0) == 0:
                # negative entries are error codes (a page not present), not nodes
                out["buffer_nodes"] = sorted(set(int(v) for v in status if v >= 0))
        bus = subprocess.run(["nvidia-smi", "-i", str(gpu), "--query-gpu=pci.bus_id", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=20).stdout.strip().lower()
        if bus:
            dev = bus[-12:] if len(bus) >= 12 else bus
            with open(f"/sys/bus/pci/devices/{dev}/numa_node") as fh:
                out["gpu_node"] = int(fh.read().strip())
    except (OSError, ValueError, subprocess.SubprocessError):
        pass
    return out


def _algorithmic_bytes(offsets_span: int, n_events: int, n_trials: int, n_records: int) -> int:
    """Bytes the method must move per layer: YET ids (4 B / occurrence), trial
    offsets (8 B / trial), each record of the layer once (16 B: mean, sigma,
    exposure, event id), and the YLT (8 B / trial)."""
    return 4 * n_events + 8 * (n_trials + 1) + 16 * n_records + 8 * n_trials


# ------------------------------------------------------------------ CPU legs (oracle)
def _oracle_leg(yet, pool, terms, seed, sample_trials: int, threads: int = 0):
    import oracle

    trials = np.arange(sample_trials, dtype=np.int64)
    evals = int(yet.offsets[sample_trials] - yet.offsets[0]) * pool.n_elts
    t = time.perf_counter()
    oracle.run_layer(yet, pool, terms, seed=seed, trials=trials, threads=threads)
    dt = time.perf_counter() - t
    return evals / dt, dt, evals


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_1501_06326_gb300 import synth

    n_sample = args.ref_trials
    yet, pool, spec = synth.workload(WORKLOAD, n_trials=n_sample)
    terms = _terms()
    cores = _usable_cores()
    for _ in range(args.warmup):
        _oracle_leg(yet, pool, terms, 0, min(n_sample, 200))
    times, evals = [], 0
    for _ in range(args.steps):
        v, dt, evals = _oracle_leg(yet, pool, terms, 0, n_sample)
        times.append(dt)
    value = evals / float(np.mean(times))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{WORKLOAD} (sample: first {n_sample} trials per step)", "trials": n_sample,
                   "elts": pool.n_elts, "return_periods": list(RETURN_PERIODS)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"first {n_sample} trials of the 1M-trial YET, all 15 ELTs"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import torch

    from paper_1501_06326_gb300 import ara, build, synth

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()

    spec = dict(synth.WORKLOADS[WORKLOAD])
    n_trials = spec["n_trials"] if args.trials is None else int(args.trials)
    seed = 0 + rank  # weak scaling: each rank its own shard / stream
    yet_seed = spec["seed"] + 1000 * rank
    offsets = synth.yet_offsets(n_trials, spec["mean_events"], yet_seed)
    n_events = int(offsets[-1])
    # generate the ids straight into pinned host memory (also the e2e source buffer)
    ids_host = torch.empty(n_events, dtype=torch.int32, pin_memory=True)
    synth.fill_yet_ids(ids_host.numpy(), spec["catalogue"], yet_seed)
    offsets_host = torch.from_numpy(offsets).pin_memory()
    pool = synth.make_elt_pool(spec["n_elts"], spec["entries"], spec["catalogue"], spec["seed"], recipe=spec["recipe"])
    terms = _terms()
    n_recs = int(pool.rec_offsets[-1])
    evals_per_step = n_events * pool.n_elts

    stream = torch.cuda.current_stream(dev)
    eng = ara.Ara(local, 0, stream.cuda_stream)
    eng.load_yet(offsets_host, ids_host, spec["catalogue"])
    eng.load_pool(pool)
    ylt = torch.empty(n_trials, dtype=torch.float64, device=dev)
    rps = np.array(RETURN_PERIODS)
    pml = torch.empty(len(rps), dtype=torch.float64, device=dev)
    tvar = torch.empty(len(rps), dtype=torch.float64, device=dev)

    def step():
        eng.run_layer(pool.elt_ids, terms, seed, 0, n_trials, ylt)
        eng.pml_tvar(ylt, rps, pml, tvar)

    def barrier():
        if ws > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step()
    barrier()
    eng.timing(reset=True)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        barrier()
        start.record(stream)
        for _ in range(args.steps):
            step()
        end.record(stream)
        barrier()
    ms = start.elapsed_time(end) / args.steps
    tm = eng.timing(reset=True)
    st = eng.stats()
    ms_max = ms
    if ws > 1:
        import torch.distributed as dist

        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    value = ws * evals_per_step / (ms_max * 1e-3)

    # ---- global PML/TVaR across ranks: each rank's top m year losses (ara_top_m on the
    # device), one all-gather of them over NCCL, and the merge (ara_merge_top)
    global_pml = None
    if ws > 1:
        import torch.distributed as dist

        total = ws * n_trials
        m_max = int(math.ceil(total / min(RETURN_PERIODS)))
        top_v = torch.empty(m_max, dtype=torch.float64, device=dev)
        top_t = torch.empty(m_max, dtype=torch.int64, device=dev)
        eng.top_m(ylt, m_max, rank * n_trials, top_v, top_t)
        torch.cuda.synchronize(dev)
        gv = [torch.empty_like(top_v) for _ in range(ws)]
        gt = [torch.empty_like(top_t) for _ in range(ws)]
        dist.all_gather(gv, top_v)
        dist.all_gather(gt, top_t)
        global_pml = ara.merge_top(torch.cat(gv).cpu().numpy(), torch.cat(gt).cpu().numpy(), total, RETURN_PERIODS)

    # ---- roofline of the layer kernels (gather + losses: the whole per-layer hot
    # path between the index build and PML/TVaR) against the layer's algorithmic bytes
    calls = max(tm["layer_calls"], 1)
    kernel_ms = tm["kernel_ms"] / calls
    algo = _algorithmic_bytes(n_events, n_events, n_trials, n_recs)
    peak, peak_kind = _peaks()
    achieved = algo / (kernel_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                "traffic": _profiled_traffic(), "kernel": "k_gather+k_losses", "kernel_ms": kernel_ms,
                "gather_ms": tm["gather_ms"] / calls, "losses_ms": tm["losses_ms"] / calls,
                "algorithmic_bytes": algo, "peak_source": f"hbm_gbs of {peak_kind}"}

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        ylt_host = torch.empty(n_trials, dtype=torch.float64, pin_memory=True)
        pml_h, tvar_h = np.zeros(len(rps)), np.zeros(len(rps))
        terms_arr = pool.terms

        def e2e_step():
            # the YET upload (link-bound) runs beside the ELT load (its table build)
            eng.load_yet_async(offsets_host, ids_host, spec["catalogue"])
            eng.load_elts(pool.elt_ids, pool.rec_offsets, pool.event_ids, pool.mean, pool.sigma, pool.exposure,
                          terms_arr)
            eng.run_layer(pool.elt_ids, terms, seed, 0, n_trials, ylt_host)
            eng.pml_tvar(ylt_host, rps, pml_h, tvar_h)

        e2e_step()
        barrier()
        n_e2e = max(2, min(args.steps, 5))
        step_ms = []
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            t_s = time.perf_counter()
            e2e_step()
            step_ms.append((time.perf_counter() - t_s) * 1e3)
        barrier()
        e2e_ms = (time.perf_counter() - t0) * 1e3 / n_e2e
        if ws > 1:
            import torch.distributed as dist

            t = torch.tensor([e2e_ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_ms = float(t.item())
        # its parts alone (wall time): the YET upload, the ELT load with its table build
        def wall(fn, reps=2):
            barrier()
            t = time.perf_counter()
            for _ in range(reps):
                fn()
            barrier()
            return (time.perf_counter() - t) * 1e3 / reps

        upload_ms = wall(lambda: (eng.load_yet_async(offsets_host, ids_host, spec["catalogue"]), eng.finish_yet()))
        elt_ms = wall(lambda: eng.load_elts(pool.elt_ids, pool.rec_offsets, pool.event_ids, pool.mean, pool.sigma,
                                            pool.exposure, terms_arr))
        pool_bytes = (pool.elt_ids.nbytes + pool.rec_offsets.nbytes + pool.event_ids.nbytes + pool.mean.nbytes
                      + pool.sigma.nbytes + pool.exposure.nbytes + pool.terms.nbytes)
        h2d = offsets.nbytes + 4 * n_events + pool_bytes + 8 * n_trials  # ylt host -> device staging for PML
        d2h = 8 * n_trials + 16 * len(rps)
        e2e = {"value": ws * evals_per_step / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms, "ms_steps": step_ms,
               "yet_upload_ms": upload_ms, "yet_upload_gbs": 4 * n_events / (upload_ms * 1e-3) / 1e9,
               "memory_nodes": _memory_nodes(ids_host.data_ptr(), 4 * n_events, local),
               "elt_load_ms": elt_ms,
               "step": "ara_load_yet_async (pinned host YET) beside ara_load_elts (host ELTs, table build), "
                       "ara_run_layer (host YLT), ara_pml_tvar"}

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        yet_view = synth.YET(offsets=offsets, event_ids=ids_host.numpy(), catalogue_size=spec["catalogue"])
        v, dt, ev = _oracle_leg(yet_view, pool, terms, seed, min(args.cpu_trials, n_trials))
        n1 = min(args.cpu_trials // 50, n_trials)
        v1, dt1, ev1 = _oracle_leg(yet_view, pool, terms, seed, n1, threads=1)
        cpu = {"value": v, "unit": UNIT, "cores": _usable_cores(), "kind": "oracle",
               "sample": f"first {min(args.cpu_trials, n_trials)} trials of the workload ({ev} evals, {dt:.1f} s)",
               "single_core": {"value": v1, "sample": f"first {n1} trials ({ev1} evals, {dt1:.1f} s, 1 thread)"}}

    # ---- two-part secondary uncertainty (correlated sigma) on the same layer; the plain
    # layer pass is timed here too, on the same stream, for the comparison
    correlated = events = stress = None
    if ws == 1 and not (args.no_correlated and args.no_events and args.no_stress):
        eng.load_pool(pool)

        def plain_layer():
            eng.run_layer(pool.elt_ids, terms, seed, 0, n_trials, ylt)

        for _ in range(3):
            plain_layer()
        torch.cuda.synchronize(dev)
        steps_c = max(2, min(args.steps, 10))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps_c):
            plain_layer()
        b.record(stream)
        torch.cuda.synchronize(dev)
        ms_plain_layer = a.elapsed_time(b) / steps_c
        if not args.no_correlated:
            correlated = _correlated_leg(eng, synth, torch, dev, stream, spec, terms, n_trials, n_events, seed,
                                         ms_plain_layer, args)
            eng.load_pool(pool)
        if not args.no_events:
            events = _events_leg(eng, torch, dev, stream, pool, terms, n_trials, seed, ms_plain_layer, args)
        if not args.no_stress and n_trials == spec["n_trials"]:
            stress = _stress_leg(eng, synth, torch, dev, stream, n_trials, n_events, ms_plain_layer, args)
            eng.load_pool(pool)

    # ---- batched layers (several layers in one pass over the YET) against one pass per layer
    batched = None
    if ws == 1 and not args.no_batched:
        batched = _batched_leg(eng, synth, torch, dev, stream, n_trials, n_events, seed, args)
    serving = None
    if ws == 1 and not args.no_serving and n_trials == synth.WORKLOADS["serving"]["n_trials"]:
        serving = _serving_leg(eng, synth, offsets, args)

    # ---- the second bound: warp instructions issued (ncu count per launch) against the SMs'
    # issue rate (4 warp instructions per SM per cycle at the sampled SM clock)
    clk = clocks.summary()
    inst = _profiled_layer("warp_instructions_per_full_launch")
    if inst is not None and clk.get("sm_mhz"):
        n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
        issue_peak = n_sms * 4 * clk["sm_mhz"] * 1e6
        roofline["issue"] = {"warp_instructions": inst, "achieved": inst / (kernel_ms * 1e-3), "peak": issue_peak,
                             "unit": "warp instructions/s", "frac": inst / (kernel_ms * 1e-3) / issue_peak,
                             "peak_source": f"{n_sms} SMs x 4 issue slots x {clk['sm_mhz']:.0f} MHz (sampled)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{WORKLOAD}: 1,000,000 trials x Poisson(1000) events, catalogue 2,000,000, "
                                   "one layer of 15 ELTs x 10,000 records, percentile terms, RP 100/250",
                       "trials": n_trials, "events": n_events, "elts": pool.n_elts,
                       "evals_per_step": evals_per_step, "l2": "inputs (4 GB YET) larger than L2; no flush",
                       "accumulation": "FP32 loss arithmetic, FP64 per-trial running sum",
                       "parallelism": f"trial shards x{ws}"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": tm["kernel_launches"] // max(args.steps, 1),
            "clocks": clk,
            "stats": {"index_ms": tm["index_ms"] / max(tm["layer_calls"], 1),
                      "pml_ms": tm["pml_ms"] / max(tm["pml_calls"], 1), "pairs_hit": st["n_pairs_hit"],
                      "nonconverged": st["n_nonconverged"], "newton_pairs": st["n_newton"],
                      "grid": st["grid"], "block": st["block"],
                      "smem_bytes": st["smem_bytes"], "filter_bits": st["filter_bits"]},
        }
        if global_pml is not None:
            line["global_pml_tvar"] = {"pml": list(global_pml[0]), "tvar": list(global_pml[1])}
        if correlated is not None:
            line["correlated"] = correlated
        if events is not None:
            line["events"] = events
        if stress is not None:
            line["stress"] = stress
        if batched is not None:
            line["batched"] = batched
        if serving is not None:
            line["serving"] = serving
        print(json.dumps(line))
    eng.close()
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def _stress_leg(eng, synth, torch, dev, stream, n_trials, n_events, ms_plain, args):
    """The precision-stress workload: the paper-1m YET and 15 ELTs x 10,000 records
    whose Beta shapes are log-uniform over [0.2, 50] (heavy-tailed small shapes
    included), timed with CUDA events like the plain layer, with the count of
    pairs that ran the FP32 Halley iteration.  Its errors against the FP64 oracle
    over all 1M trials are measured by the parity tests, not here."""
    spec = synth.WORKLOADS["stress-1m"]
    pool = synth.make_elt_pool(spec["n_elts"], spec["entries"], spec["catalogue"], spec["elt_seed"],
                               recipe=spec["recipe"])
    with open(os.path.join(ROOT, "tests", "golden", "workload_terms.json")) as fh:
        terms = json.load(fh)["stress-1m"]["layer_terms"]
    eng.load_pool(pool)
    out = torch.empty(n_trials, dtype=torch.float64, device=dev)

    def layer():
        eng.run_layer(pool.elt_ids, terms, 0, 0, n_trials, out)

    for _ in range(3):
        layer()
    torch.cuda.synchronize(dev)
    eng.timing(reset=True)
    steps = max(2, min(args.steps, 10))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        layer()
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / steps
    tm = eng.timing(reset=True)
    calls = max(tm["layer_calls"], 1)
    st = eng.stats()
    return {"workload": "stress-1m: the paper-1m YET, 15 ELTs x 10,000 records, Beta shapes log-uniform in "
                        "[0.2, 50], percentile terms",
            "steps": steps, "ms_layer": ms, "ms_layer_plain": ms_plain,
            "evals_per_s": n_events * pool.n_elts / (ms * 1e-3),
            "gather_ms": tm["gather_ms"] / calls, "losses_ms": tm["losses_ms"] / calls,
            "pairs": st["n_pairs_hit"], "halley_pairs": st["n_newton"], "nonconverged": st["n_nonconverged"],
            "errors": "against the FP64 oracle over all 1M trials: tests/test_gpu_parity.py "
                      "test_stress_1m_layer_full_parity"}


def _batched_leg(eng, synth, torch, dev, stream, n_trials, n_events, seed, args):
    """The batched workload: 16 layers of 1..32 ELTs from a pool of 64, over the same
    YET, as one ara_run_layers pass and as 16 ara_run_layer passes (device buffers,
    CUDA events on the engine's stream)."""
    spec = synth.WORKLOADS["batched-16"]
    with open(os.path.join(ROOT, "tests", "golden", "workload_terms.json")) as fh:
        spec_layers = json.load(fh)["batched-16"]["layers"]
    pool = synth.make_elt_pool(spec["n_elts"], spec["entries"], spec["catalogue"], spec["elt_seed"],
                               recipe=spec["recipe"])
    eng.load_pool(pool)
    layers = [(np.asarray(l["elt_ids"], np.int32), l["layer_terms"]) for l in spec_layers]
    out = torch.empty((len(layers), n_trials), dtype=torch.float64, device=dev)

    def batch_step():
        eng.run_layers(layers, seed, 0, n_trials, out)

    # the default rule's configuration first, then the autotuner's (its first pass measures
    # the candidates and caches the fastest for this shape; later passes reuse it)
    ms_default = None

    def plain_step():
        for l, (ids, terms) in enumerate(layers):
            eng.run_layer(ids, terms, seed, 0, n_trials, out[l])

    def timed(fn, steps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / steps

    from paper_1501_06326_gb300 import ara

    steps = max(2, min(args.steps, 5))
    # each work item pinned (all CTAs an SM holds), then the default rule, without the YET's
    # event-major index and with it (built once, its device time reported), then the autotuner
    items = {"tile": ara.ARA_BATCH_ITEM_TILE, "trial": ara.ARA_BATCH_ITEM_TRIAL, "dense": ara.ARA_BATCH_ITEM_DENSE,
             "indexed": ara.ARA_BATCH_ITEM_INDEXED}
    names = {v: k for k, v in items.items()}
    ms_items = {}
    try:
        for name, item in items.items():
            if item == ara.ARA_BATCH_ITEM_INDEXED:
                continue
            eng.set_batch_config(item, 0)
            ms_items[name] = timed(batch_step, steps)
        eng.set_batch_config(ara.ARA_BATCH_AUTO)
        ms_no_index = timed(batch_step, steps)
        st_no_index = eng.stats()
        eng.build_yet_index()
        index = eng.yet_index_info()
        eng.set_batch_config(ara.ARA_BATCH_ITEM_INDEXED, 0)
        ms_items["indexed"] = timed(batch_step, steps)
    finally:
        eng.set_batch_config(ara.ARA_BATCH_AUTO)
    ms_default = timed(batch_step, steps)
    st_default = eng.stats()
    eng.run_layers(layers, seed, 0, n_trials, out, autotune=True)
    ms_batch = timed(batch_step, steps)
    st = eng.stats()
    ms_plain = timed(plain_step, steps)
    evals = n_events * sum(len(ids) for ids, _ in layers)
    return {"workload": f"batched-16: the {n_trials:,}-trial YET, 16 layers of 1..32 ELTs from a pool of "
                        f"{spec['n_elts']} x {spec['entries']:,} records",
            "layers": len(layers), "steps": steps, "ms_batched": ms_batch, "ms_plain": ms_plain,
            "layers_per_s": len(layers) / (ms_batch * 1e-3), "plain_layers_per_s": len(layers) / (ms_plain * 1e-3),
            "speedup": ms_plain / ms_batch, "evals_per_s": evals / (ms_batch * 1e-3),
            "ms_batched_by_item": ms_items,
            "without_yet_index": {"item": names[st_no_index["batch_item"]], "ms_batched": ms_no_index,
                                  "speedup": ms_plain / ms_no_index},
            "yet_index": {"bytes": index["bytes"], "build_ms": index["build_ms"], "method": index["method"],
                          "note": "built once per YET (ara_build_yet_index); ara_run_layer (ms_plain) streams the YET"},
            "autotuned": {"item": names[st["batch_item"]], "blocks_per_sm": st["batch_blocks_per_sm"],
                          "tuned": bool(st["batch_tuned"])},
            "default_rule": {"item": names[st_default["batch_item"]],
                             "blocks_per_sm": st_default["batch_blocks_per_sm"], "ms_batched": ms_default}}


def _correlated_leg(eng, synth, torch, dev, stream, spec, terms, n_trials, n_events, seed, ms_plain, args):
    """The paper-1m layer with each record's sigma split into an independent and a
    correlated part (sigma_C = sigma u, u ~ U(0, 0.5); the Beta shapes are those of
    the main workload), loaded with ara_load_xelts: layer passes (index, gather,
    losses) timed with CUDA events against the same passes on the plain pool."""
    pool = synth.make_elt_pool(spec["n_elts"], spec["entries"], spec["catalogue"], spec["seed"],
                               recipe=spec["recipe"], correlated=0.5)
    eng.load_pool(pool)
    out = torch.empty(n_trials, dtype=torch.float64, device=dev)

    def layer():
        eng.run_layer(pool.elt_ids, terms, seed, 0, n_trials, out)

    for _ in range(3):
        layer()
    torch.cuda.synchronize(dev)
    eng.timing(reset=True)
    steps = max(2, min(args.steps, 10))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        layer()
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / steps
    tm = eng.timing(reset=True)
    calls = max(tm["layer_calls"], 1)
    evals = n_events * pool.n_elts
    return {"workload": f"{WORKLOAD} with sigma = sigma_I + sigma_C, sigma_C = sigma u, u ~ U(0, 0.5) per record",
            "steps": steps, "ms_layer": ms, "ms_layer_plain": ms_plain, "evals_per_s": evals / (ms * 1e-3),
            "gather_ms": tm["gather_ms"] / calls, "losses_ms": tm["losses_ms"] / calls,
            "newton_pairs": eng.stats()["n_newton"]}


def _events_leg(eng, torch, dev, stream, pool, terms, n_trials, seed, ms_plain, args):
    """The paper-1m layer with its per-event output (ara_run_layer_events): one row
    per hit event (trial, k, event id, O_k, inc_k: 32 bytes) and each trial's largest
    O_k, all in device memory; timed with CUDA events against the plain layer pass."""
    ylt = torch.empty(n_trials, dtype=torch.float64, device=dev)
    n_rows = eng.run_layer_events(pool.elt_ids, terms, seed, 0, n_trials, ylt)
    rows = [torch.empty(n_rows, dtype=dt, device=dev)
            for dt in (torch.int64, torch.int32, torch.int32, torch.float64, torch.float64)]
    max_occ = torch.empty(n_trials, dtype=torch.float64, device=dev)

    def step():
        eng.run_layer_events(pool.elt_ids, terms, seed, 0, n_trials, ylt, *rows, max_occ)

    for _ in range(3):
        step()
    torch.cuda.synchronize(dev)
    steps = max(2, min(args.steps, 10))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        step()
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / steps
    return {"workload": f"{WORKLOAD} layer with per-event rows (YELT) and per-trial max occurrence loss (OEP input)",
            "steps": steps, "rows": n_rows, "row_bytes": 32 * n_rows, "ms_layer_events": ms,
            "ms_layer_plain": ms_plain, "rows_per_s": n_rows / (ms * 1e-3)}


def _serving_leg(eng, synth, offsets, args):
    """The serving workload: requests with Poisson arrivals at several rates, served by
    the continuous-batching loop (ara_submit / ara_serve_step / ara_poll) in real time.
    The host loop submits each request when its arrival time has passed, calls
    ara_serve_step (which launches rounds without waiting for them) and polls the
    pending tickets after a step that finished some; a request's latency is the
    wall time from its arrival to the poll that returns its PML/TVaR."""
    spec = synth.WORKLOADS["serving"]
    pool = synth.make_elt_pool(spec["n_elts"], spec["entries"], spec["catalogue"], spec["elt_seed"],
                               recipe=spec["recipe"])
    eng.load_pool(pool)
    eng.build_yet_index()  # (no-op when the batched leg built it on this YET)
    index = eng.yet_index_info()
    with open(os.path.join(ROOT, "tests", "golden", "serving_terms.json")) as fh:
        st = json.load(fh)
    reqs = synth.serving_requests(spec, args.serve_requests, spec["request_seed"])
    terms = st["layer_terms"][: len(reqs)]
    if len(terms) < len(reqs):
        raise RuntimeError("serving_terms.json holds fewer requests than asked for")
    rps = np.array(RETURN_PERIODS)
    results = []
    for rate in args.serve_rates:
        rng = np.random.default_rng([spec["request_seed"], int(rate)])
        arrivals = np.cumsum(rng.exponential(1.0 / rate, len(reqs)))
        s0 = eng.serve_stats()
        pending, lat, evals = {}, [], 0
        i, max_pending = 0, 0
        t0 = time.perf_counter()
        while i < len(reqs) or pending:
            now = time.perf_counter() - t0
            while i < len(reqs) and arrivals[i] <= now:
                ids, t_end = reqs[i]
                tk = eng.submit(ids, terms[i], 0, t_end, rps)
                pending[tk] = (arrivals[i], int(offsets[t_end]) * len(ids))
                i += 1
            max_pending = max(max_pending, len(pending))
            if eng.serve_step() > 0:
                done_at = time.perf_counter() - t0
                for tk in list(pending):
                    if eng.poll(tk, len(rps)) is not None:
                        arr, ev = pending.pop(tk)
                        lat.append(done_at - arr)
                        evals += ev
            elif not pending and i < len(reqs):
                time.sleep(max(0.0, min(arrivals[i] - (time.perf_counter() - t0), 0.002)))
        wall = time.perf_counter() - t0
        s1 = eng.serve_stats()
        lat_ms = 1e3 * np.asarray(lat)
        passes = s1["passes_launched"] - s0["passes_launched"]
        offered = sum(int(offsets[t_end]) * len(ids) for ids, t_end in reqs) / float(arrivals[-1])
        results.append({"rate_per_s": rate, "requests": len(lat), "p50_ms": float(np.percentile(lat_ms, 50)),
                        "p99_ms": float(np.percentile(lat_ms, 99)), "max_ms": float(lat_ms.max()),
                        "wall_s": wall, "evals_per_s": evals / wall, "offered_evals_per_s": offered,
                        "rounds": s1["rounds_launched"] - s0["rounds_launched"], "passes": passes,
                        "max_pending": max_pending})
    return {"workload": f"serving: the paper-1m YET, a pool of {spec['n_elts']} ELTs x {spec['entries']:,} records, "
                        f"{len(reqs)} requests per rate of |J| ~ U{{1..15}} over trial prefixes log-uniform in "
                        "[1e4, 1e6], RP 100/250, percentile terms per request (tests/golden/serving_terms.json)",
            "time": "real: Poisson arrivals in wall time; latency = arrival to the poll that returns the result",
            "passes": "batched passes through the YET's event-major index (built once per YET, before the sweep)",
            "yet_index": {"bytes": index["bytes"], "build_ms": index["build_ms"], "method": index["method"]},
            "chunk_trials": eng.serve_stats()["chunk_trials"], "rates": results}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("gpu", "reference"), default="gpu")
    ap.add_argument("--cpu-trials", type=int, default=1_000_000,
                    help="trials in the oracle's CPU-baseline sample (about 15 s on 16 cores for the full workload)")
    ap.add_argument("--ref-trials", type=int, default=200_000,
                    help="trials per step of the reference arm (about 3 s per step on 16 cores)")
    ap.add_argument("--trials", type=int, default=None,
                    help="truncate the YET (profiling of a smaller case); the default is the full workload")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-layers comparison")
    ap.add_argument("--no-correlated", action="store_true",
                    help="skip the correlated-sigma layer and the per-event output legs")
    ap.add_argument("--no-events", action="store_true", help="skip the per-event output leg")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-latency sweep")
    ap.add_argument("--no-stress", action="store_true", help="skip the precision-stress layer")
    ap.add_argument("--serve-requests", type=int, default=10_000, help="requests per rate of the serving sweep")
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[200.0, 800.0, 1600.0, 3200.0, 4800.0],
                    help="request arrival rates (per second) of the serving sweep")
    args = ap.parse_args(argv)
    args.warmup = max(3, args.warmup)  # at least three untimed warm-up steps
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
