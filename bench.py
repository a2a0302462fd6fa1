"""Benchmark of the Hoshen-Kopelman labelling path on GB300.

Default workload: critical site percolation on a 1024^3 lattice (float32
phi = u - (1 - 0.3116), u iid uniform, periodic in x, y, z), labelled, sized
and histogrammed per step through the C ABI with phi resident in HBM.  One
JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

--impl reference times the CPU oracle (the serial algorithm of the paper) on
the host cores, on a bounded sample of the same workload.  Under torchrun
(N > 1) every rank labels its own lattice (independent replicas, weak
scaling); only rank 0 runs the reference arm.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gsites/s labelled+sized at 1024^3 p_c; batched vs per-lattice; p50/p99 latency"
P_C = 0.3116
L_HEADLINE = 1024
# kernels of one hk_label call: occupancy, tile_label (fast pass and the pass over
# dense tiles), face_merge, piece_finalize, three scan kernels, lattice_finish, flatten
LAUNCHES_PER_CALL = 10


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=("gb300", "reference"))
    ap.add_argument("--size", type=int, default=L_HEADLINE, help="lattice side (default 1024)")
    ap.add_argument("--tile", default="", help="ty,tz tile override")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-streams", type=int, default=0,
                    help="contexts (each on its own stream) that take alternate steps in the end-to-end run "
                         "(default: 3 on one GPU, 2 per rank with several, to bound the pinned host memory)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="headline config only")
    ap.add_argument("--served-requests", type=int, default=2000)
    ap.add_argument("--capsule-state", action="store_true",
                    help="only the interior state of moving capsules (Sec. 6) at --size, for profiling")
    ap.add_argument("--decompose", action="store_true",
                    help="under torchrun: one --size^3 lattice split into z slabs across the ranks (the domain "
                         "decomposition of Sec. 3, strong scaling) instead of one lattice per rank")
    ap.add_argument("--backend", default="nccl", choices=("nccl", "gloo"),
                    help="process-group backend with several ranks (gloo lets ranks share a GPU)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per lattice site of one
# hk_label call at p_c, per pass, from one ncu capture of a 512^3 call on these kernel
# sources, scaled by the number of sites.  It holds only for the kernel sources it was
# taken on, identified by TRAFFIC_SOURCE_SHA; after any change to them it is reported
# as null.
TRAFFIC_SITES = 512 ** 3
TRAFFIC_BYTES = {"occupancy": 554.3e6, "tile_label": 61.9e6, "face_merge": 37.3e6, "piece_finalize": 30.1e6,
                 "scan": 8.5e6, "lattice_finish": 0.0, "flatten": 630.2e6}
TRAFFIC_SOURCE_SHA = "2a066ea8b3ba4896"
# Warp instructions of one launch of the two instruction-bound passes at 512^3
# (smsp__inst_executed.sum of one ncu capture of these kernel sources), scaled by
# sites like the traffic and held to the same kernel sources.  Their roofline is the
# issue rate: 4 warp schedulers per SM, each issuing at most one warp instruction per
# clock.
INST_PER_LAUNCH = {"tile_label": 340986233, "flatten": 169021401}


# the sources of the passes of one hk_label call and of their launch (the captures above
# measure these kernels; the other sources build other entry points)
KERNEL_SOURCES = ("hk_kernels.cu", "hk_device.cuh", "hk_launch.h", "hk_api.cu")


def kernel_source_sha() -> str:
    files = [os.path.join(ROOT, "paper_1405_1931_gb300", "csrc", f) for f in KERNEL_SOURCES]
    h = hashlib.sha256()
    for f in sorted(files):
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="hk_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "20",
                 "-i", str(self.dev)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.05)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline_oracle(side: int = 512, reps: int = 3):
    """Serial oracle on a bounded sample of the same distribution (one host core)."""
    import oracle
    from paper_1405_1931_gb300 import fields
    oracle.load()
    phi = fields.iid_field(side, side, side, seed=0, occupancy=P_C)
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.label(phi, (1, 1, 1))
    dt = time.perf_counter() - t0
    sites = reps * side ** 3
    return {"value": sites / dt / 1e9, "unit": "Gsites/s", "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{reps} x {side}^3 iid phi at p=0.3116, periodic xyz (serial C oracle, {dt:.1f} s)"}


def cpu_parallel_oracle(side: int = 512, reps: int = 3):
    """The paper's parallel scheme (Sec. 3) on all host cores, one slab per thread, on the
    same sample as the serial baseline; its result equals the serial oracle's."""
    import oracle
    from paper_1405_1931_gb300 import fields
    oracle.load()
    threads = os.cpu_count() or 1
    phi = fields.iid_field(side, side, side, seed=0, occupancy=P_C)
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.label_mt(phi, (1, 1, 1), threads=threads)
    dt = time.perf_counter() - t0
    return {"value": reps * side ** 3 / dt / 1e9, "unit": "Gsites/s", "cores": threads,
            "kind": "the paper's parallel scheme (Sec. 3) on host threads",
            "sample": f"{reps} x {side}^3 iid phi at p=0.3116, periodic xyz ({dt:.1f} s)"}


def max_over_ranks(value: float, dist=None, device="cuda") -> float:
    """The maximum of a per-rank number over all ranks (the value itself for one process)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gsites_per_s(world: int, sites_per_rank: int, ms_per_step: float) -> float:
    """Whole-job throughput: each of the `world` ranks labels its own lattice every step."""
    return world * sites_per_rank / (ms_per_step * 1e-3) / 1e9


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle as it stands, timed per step on a bounded sample."""
    if rank != 0:
        return
    import oracle
    from paper_1405_1931_gb300 import fields
    oracle.load()
    side = 256
    phi = fields.iid_field(side, side, side, seed=0, occupancy=P_C)
    for _ in range(args.warmup):
        oracle.label(phi, (1, 1, 1))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.label(phi, (1, 1, 1))
    dt = time.perf_counter() - t0
    value = args.steps * side ** 3 / dt / 1e9
    sample = f"each step: {side}^3 iid phi at p=0.3116, periodic xyz (the 1024^3 workload's distribution)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gsites/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": f"critical site percolation {side}^3 sample of 1024^3, p=0.3116, periodic xyz"},
            "cpu_baseline": {"value": value, "unit": "Gsites/s", "cores": 1, "host_cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "Gsites/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def flush_l2(buf):
    buf.add_(1)   # rewrites a buffer larger than L2


def time_single(lab, phi, per, reps, flush=None):
    """Device time (ms, trimmed mean) of one hk_label call on a resident lattice, L2
    flushed between reps when `flush` is given, and the latency of a call enqueued only
    once the device is idle (the host's enqueue then counts too).

    For the device time the reps are enqueued back to back (flush, event, call, event),
    so that the host is ahead of the device and each pair of events brackets the call's
    kernels and the gaps between them, not the host's work of enqueueing them."""
    import torch
    out = lab.alloc_outputs(phi.shape, phi.device)
    s = torch.cuda.current_stream()
    for _ in range(3):
        lab.label(phi, per, out=out)
    evs = []
    for _ in range(reps):
        if flush is not None:
            flush_l2(flush)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        lab.label(phi, per, out=out)
        b.record(s)
        evs.append((a, b))
    torch.cuda.synchronize()
    dev = [a.elapsed_time(b) for a, b in evs]
    one = []
    for _ in range(reps):
        if flush is not None:
            flush_l2(flush)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        lab.label(phi, per, out=out)
        b.record(s)
        b.synchronize()
        one.append(a.elapsed_time(b))
    lab.sync_status()
    return trimmed_mean(dev), int(out[3].item()), trimmed_mean(one)


def trimmed_mean(ts, cut=0.1):
    """Mean of the samples without the lowest and highest tenth.  CUDA event times come in
    steps of about 2 us on this device, so a median of short calls can only move by a
    step; a trimmed mean resolves finer changes and still drops outliers."""
    v = np.sort(np.asarray(ts, dtype=np.float64))
    k = int(len(v) * cut)
    return float(v[k:len(v) - k].mean()) if len(v) > 2 * k else float(v.mean())


def extra_configs(args, peak):
    """The other workloads: 32^3, 256^3 emulsion, the block benchmark sweep at 1024^3, capsule
    interiors, the interior state of moving capsules at 1024^3, the uneven batch, the served stream."""
    import torch
    from paper_1405_1931_gb300 import autotune, fields, hk, serve
    res = {}
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")   # 256 MB > L2
    lab = hk.Labeller(0)

    def line(name, n_sites, ms, ncl, workload, cache, ms_one=None, ms_warm=None):
        b = 8 * n_sites + 8 * ncl + 256
        res[name] = {"workload": workload, "gsites_per_s": n_sites / (ms * 1e-3) / 1e9, "ms": ms,
                     "n_clusters": ncl, "roofline_frac": b / (ms * 1e-3) / 1e9 / peak, "cache": cache,
                     "timing": "device time, calls enqueued back to back"}
        if ms_one is not None:   # a call enqueued on an idle device: the host's enqueue included
            res[name]["ms_one_call_idle_device"] = ms_one
        if ms_warm is not None:  # the same calls without the flush: the lattice stays in L2
            res[name]["l2_not_flushed"] = {"ms": ms_warm, "gsites_per_s": n_sites / (ms_warm * 1e-3) / 1e9}

    # 32^3, occupancy 0.3, seed 0
    phi = torch.empty((32, 32, 32), dtype=torch.float32, device="cuda")
    hk.hk_gen_iid(phi.data_ptr(), 32, 32, 32, 0, 0.3, hk._stream_handle(None))
    ms, ncl, ms_one = time_single(lab, phi, (1, 1, 1), 50, flush)
    ms_warm = time_single(lab, phi, (1, 1, 1), 50)[0]
    line("small32", 32 ** 3, ms, ncl, "32^3 iid p=0.3 periodic xyz", "L2 flushed between reps", ms_one, ms_warm)
    # 256^3 emulsion, 600 droplets r in [5, 15]
    L = 256
    phi = torch.empty((L, L, L), dtype=torch.float32, device="cuda")
    c, r = fields.sphere_params(600, (L, L, L), seed=1)
    hk.hk_gen_spheres(phi.data_ptr(), L, L, L, c, r, 8.0, hk._stream_handle(None))
    ms, ncl, ms_one = time_single(lab, phi, (1, 1, 1), 20, flush)
    ms_warm = time_single(lab, phi, (1, 1, 1), 20)[0]
    line("emulsion256", L ** 3, ms, ncl, "256^3 emulsion, 600 droplets r in [5,15], periodic", "L2 flushed between reps",
         ms_one, ms_warm)
    del phi

    # The benchmark of Sec. 3: 1024^3 filled with alternating cubic domains of b^3 sites
    # that touch only at edges and corners, so n_clusters = (1024 / b)^3 / 2 runs from 32
    # (b = 256) to the maximum V / 2 (b = 1, the site checkerboard).
    L = 1024
    sweep = []
    for b in (256, 128, 64, 32, 16, 8, 4, 2, 1):
        phi = fields.block_field_device(L, b)
        ms, ncl, _ = time_single(lab, phi, (1, 1, 1), 5)
        assert ncl == (L // b) ** 3 // 2, (b, ncl)
        sweep.append({"b": b, "n_clusters": ncl, "ms": ms, "gsites_per_s": L ** 3 / (ms * 1e-3) / 1e9})
        del phi
        torch.cuda.empty_cache()
    res["block_sweep1024"] = {"workload": "Sec. 3 benchmark pattern at 1024^3: alternating cubic domains of b^3 "
                                          "sites, periodic; n_clusters from 32 to V/2",
                              "points": sweep, "cache": "inputs larger than L2"}

    # interior/exterior of closed membranes (Sec. 6, steps 3-5): 256^3 index field, 24 capsules
    shape = (256, 256, 256)
    caps = fields.capsule_params(24, shape, seed=12, a_lo=8.0, a_hi=30.0)
    index = torch.from_numpy(fields.capsule_index_field(shape, caps)).cuda()
    out = lab.alloc_outputs(shape, index.device)
    for _ in range(3):
        res_i = lab.label_interior(index, (1, 1, 1), out=out)
    s0 = torch.cuda.current_stream()
    times = {}
    for mode in ("back_to_back", "idle_device"):      # as in time_single
        ts = []
        for _ in range(20):
            flush_l2(flush)
            if mode == "idle_device":
                torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s0)
            res_i = lab.label_interior(index, (1, 1, 1), out=out)
            b.record(s0)
            ts.append((a, b))
            if mode == "idle_device":
                b.synchronize()
        torch.cuda.synchronize()
        times[mode] = trimmed_mean([a.elapsed_time(b) for a, b in ts])
    ms = times["back_to_back"]
    ncl = int(res_i[3].item())
    tags = res_i[4][:ncl].cpu().numpy()
    line("capsule_interior256", 256 ** 3, ms, ncl, f"256^3 index field, {len(caps)} capsules (Sec. 6 steps 3-5), periodic",
         "L2 flushed between reps", times["idle_device"])
    res["capsule_interior256"].update({"interior": int((tags == 1).sum()), "exterior": int((tags == 0).sum()),
                                       "undetermined": int((tags == -1).sum())})
    del index, out, res_i

    # Interior state of moving capsules (Sec. 6): the full identification that
    # initialises or refreshes the state, against the update of the last paragraph of
    # Sec. 6 (dense, from the whole index field, and from the list of near sites) after
    # the capsules move by under half a lattice constant.  1024^3, 700 capsules.
    shape = (1024, 1024, 1024)
    caps = fields.capsule_params(700, shape, seed=21, a_lo=8.0, a_hi=30.0)
    assert len(caps) == 700
    index = torch.from_numpy(fields.capsule_index_field(shape, caps)).cuda()
    state = lab.interior_state(index)
    rng = np.random.default_rng(22)
    caps2 = [((c[0] + d[0], c[1] + d[1], c[2] + d[2]), a)
             for (c, a), d in zip(caps, rng.uniform(-0.25, 0.25, size=(len(caps), 3)))]
    I2 = fields.capsule_index_field(shape, caps2)
    near = ~(I2.reshape(-1) < -0.5)
    sites = torch.from_numpy(np.flatnonzero(near).astype(np.int32)).cuda()
    vals = torch.from_numpy(I2.reshape(-1)[near]).cuda()
    index2 = torch.from_numpy(I2).cuda()
    del I2, near

    def ev_time(fn, reps=10):   # calls enqueued back to back, as in time_single
        ts = []
        for _ in range(reps):
            flush_l2(flush)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s0)
            fn()
            b.record(s0)
            ts.append((a, b))
        torch.cuda.synchronize()
        return trimmed_mean([a.elapsed_time(b) for a, b in ts])

    out_state = torch.empty_like(state)
    for _ in range(2):
        lab.interior_state(index, out=out_state)
    ms_full = ev_time(lambda: lab.interior_state(index, out=out_state))
    upd = torch.empty_like(state)
    ms_dense = ev_time(lambda: hk.interior_update(state, index2, out=upd))
    sp = state.clone()
    ms_sites = ev_time(lambda: hk.interior_update_sites(sp, sites, vals))
    full2 = lab.interior_state(index2)
    assert torch.equal(upd, full2) and torch.equal(sp, full2)     # the update equals a refresh
    n_int = int((full2 == 1).sum().item())
    res["capsule_state1024"] = {
        "workload": "1024^3 index field, 700 capsules (semi-axes U[8,30]), periodic; moved by U[-0.25,0.25] "
                    "per axis for the update",
        "refresh_ms": ms_full, "update_dense_ms": ms_dense, "update_sites_ms": ms_sites,
        "near_sites": int(sites.numel()), "interior_sites": n_int,
        "refresh_gsites_per_s": 1024 ** 3 / (ms_full * 1e-3) / 1e9,
        "update_dense_gb_per_s": 1024 ** 3 * 6 / (ms_dense * 1e-3) / 1e9,
        "cache": "L2 flushed between reps"}
    del index, index2, state, out_state, upd, sp, full2, sites, vals
    torch.cuda.empty_cache()

    # uneven batch of 96 lattices: per-lattice launches vs one batched launch sequence
    params = fields.batch_params(96, master_seed=2)
    s = torch.cuda.Stream()
    items = []
    with torch.cuda.stream(s):
        for prm in params:
            d = torch.empty((prm["nz"], prm["ny"], prm["nx"]), dtype=torch.float32, device="cuda")
            hk.hk_gen_iid(d.data_ptr(), prm["nx"], prm["ny"], prm["nz"], prm["seed"], prm["occupancy"],
                          hk._stream_handle(s))
            items.append((d, prm["periodic"], lab.alloc_outputs(d.shape, d.device)))
    s.synchronize()
    sites = sum(int(d.numel()) for d, _, _ in items)
    tuned = autotune.tune(lab, items, stream=s, reps=2, cache=None)

    def timed(fn, reps=5):
        with torch.cuda.stream(s):
            fn()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            for _ in range(reps):
                fn()
            b.record(s)
        b.synchronize()
        return a.elapsed_time(b) / reps

    per = timed(lambda: [lab.label(d, p_, out=o, stream=s) for d, p_, o in items])
    bat = timed(lambda: lab.label_batched(items, stream=s))
    lab.set_graphs(True)
    gra = timed(lambda: lab.label_batched(items, stream=s))
    lab.set_graphs(False)
    lab.sync_status(s)
    lab.set_tile(16, 16)   # the library's defaults again
    lab.set_merge(1, 1)
    # compulsory bytes of the whole batch: 8 B a site, 8 B a cluster size, 256 B of histogram a lattice
    nclus = sum(int(o[3].item()) for _, _, o in items)
    bbytes = 8 * sites + 8 * nclus + 256 * len(items)
    res["batched96"] = {"workload": "96 lattices, axes in {32,...,384}, p in U[0.15,0.45], random periodic flags",
                        "sites": sites, "n_clusters": nclus, "tile": list(tuned["tile"]),
                        "merge_schedule": {"face_merge_unions_per_lane": tuned["merge"][0],
                                           "finalize_combines_hot_root": bool(tuned["merge"][1])},
                        "autotune_ms": tuned["ms"],
                        "per_lattice_ms": per, "batched_ms": bat, "batched_graph_ms": gra,
                        "per_lattice_gsites_per_s": sites / (per * 1e-3) / 1e9,
                        "batched_gsites_per_s": sites / (bat * 1e-3) / 1e9,
                        "batched_graph_gsites_per_s": sites / (gra * 1e-3) / 1e9,
                        "roofline_frac": {"per_lattice": bbytes / (per * 1e-3) / 1e9 / peak,
                                          "batched": bbytes / (bat * 1e-3) / 1e9 / peak,
                                          "batched_graph": bbytes / (gra * 1e-3) / 1e9 / peak,
                                          "bytes": bbytes}}
    del items
    lab.close()
    torch.cuda.empty_cache()

    # served: Poisson stream, continuous batching vs one launch per request.  The
    # stand-in simulation hands over each field finished at its request's arrival
    # (generated up to 50 ms ahead); the same stream with each field generated only
    # after its request arrives is reported beside it.
    reqs = serve.request_stream(args.served_requests, rate=400.0, seed=3)
    srv = serve.Server(0, cap_bytes=32 * serve.GB, workers=4)
    # one untimed warm-up run of each mode on another seed, as for every timed form here
    for mode in ("continuous", "fifo"):
        srv.serve(serve.request_stream(300, rate=400.0, seed=5), mode=mode)
    cont = srv.serve(reqs)
    reqs = serve.request_stream(args.served_requests, rate=400.0, seed=3)
    fifo = srv.serve(reqs, mode="fifo")
    cont0 = srv.serve(serve.request_stream(args.served_requests, rate=400.0, seed=3), gen_lead_s=0.0)
    fifo0 = srv.serve(serve.request_stream(args.served_requests, rate=400.0, seed=3), mode="fifo", gen_lead_s=0.0)
    # saturated: the same mix arriving far faster than it can be served
    nsat = max(100, args.served_requests // 4)
    sat_c = srv.serve(serve.request_stream(nsat, rate=20000.0, seed=4))
    sat_f = srv.serve(serve.request_stream(nsat, rate=20000.0, seed=4), mode="fifo")
    srv.close()
    for st in (cont, fifo, cont0, fifo0, sat_c, sat_f):
        st.pop("done", None)
        # compulsory bytes per second of the served stream (8 B a site and 256 B of
        # histogram a request; the 8 B cluster sizes are left out: droplet fields hold
        # about one cluster per droplet, far under 0.1 % of the sites)
        st["roofline_frac"] = (8 * st["sites"] + 256 * st["requests"]) / st["wall_s"] / 1e9 / peak if st["wall_s"] else 0.0
    res["served"] = {"workload": f"{args.served_requests} Poisson requests at 400/s, 80% emulsion / 20% capsule, "
                                 "side log-uniform in [64,512], 32 GB admission cap",
                     "warmup": "one run of 300 requests (another seed) in each mode first",
                     "continuous": cont, "fifo": fifo,
                     "generated_on_arrival": {"continuous": cont0, "fifo": fifo0},
                     "saturated": {"workload": f"{nsat} requests of the same mix at 20000/s",
                                   "continuous": sat_c, "fifo": sat_f}}
    torch.cuda.empty_cache()
    return res


def run_capsule_state(args):
    """The interior state of moving capsules alone (Sec. 6): --steps full refreshes and
    dense updates of an L^3 index field with 700 (L / 1024)^3 capsules, one JSON line."""
    import torch
    from paper_1405_1931_gb300 import fields, hk
    L = args.size
    shape = (L, L, L)
    ncap = max(1, round(700 * (L / 1024) ** 3))
    caps = fields.capsule_params(ncap, shape, seed=21, a_lo=8.0, a_hi=30.0)
    index = torch.from_numpy(fields.capsule_index_field(shape, caps)).cuda()
    lab = hk.Labeller(0)
    state = torch.empty(shape, dtype=torch.int8, device="cuda")
    upd = torch.empty_like(state)
    for _ in range(max(args.warmup, 1)):
        lab.interior_state(index, out=state)
        hk.interior_update(state, index, out=upd)
    torch.cuda.synchronize()
    s0 = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record(s0)
    for _ in range(args.steps):
        lab.interior_state(index, out=state)
    ev[1].record(s0)
    for _ in range(args.steps):
        hk.interior_update(state, index, out=upd)
    ev[2].record(s0)
    ev[2].synchronize()
    assert torch.equal(upd, state)                 # a static field: the update changes nothing
    print(json.dumps({"workload": f"{L}^3 index field, {len(caps)} capsules (semi-axes U[8,30]), periodic",
                      "steps": args.steps, "refresh_ms": ev[0].elapsed_time(ev[1]) / args.steps,
                      "update_dense_ms": ev[1].elapsed_time(ev[2]) / args.steps}), flush=True)
    lab.close()


def run_decomposed(args, rank, world, local, dist):
    """One L^3 critical-percolation lattice split into z slabs across the ranks (Sec. 3):
    each step labels every slab and merges them across the slab faces (face data
    exchanged with all_gather).  Whole-job Gsites/s = L^3 / the max over ranks of the
    step time; strong scaling."""
    import torch
    from paper_1405_1931_gb300 import distributed as D
    from paper_1405_1931_gb300 import hk
    L = args.size
    z0, nzr = D.slab_bounds(L, world, rank)
    full = torch.empty((L, L, L), dtype=torch.float32, device="cuda")
    assert hk.hk_gen_iid(full.data_ptr(), L, L, L, 0, P_C, hk._stream_handle(None)) == 0
    slab = full[z0:z0 + nzr].contiguous()
    del full
    torch.cuda.empty_cache()
    lab = hk.Labeller(local)
    per = (1, 1, 1)
    for _ in range(max(args.warmup, 3)):
        res = D.label_slab(lab, slab, z0, L, per)
    dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        res = D.label_slab(lab, slab, z0, L, per)
    torch.cuda.synchronize()
    dist.barrier()
    ms = max_over_ranks((time.perf_counter() - t0) / args.steps * 1e3, dist,
                        device="cuda" if args.backend == "nccl" else "cpu")
    if rank == 0:
        print(json.dumps({"metric": METRIC, "value": L ** 3 / (ms * 1e-3) / 1e9, "unit": "Gsites/s",
                          "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                          "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "int32",
                          "data": "synthetic",
                          "config": {"workload": f"critical site percolation {L}^3, p=0.3116, periodic xyz, split "
                                                 f"into {world} z slabs (Sec. 3 domain decomposition)",
                                     "backend": args.backend, "parallelism": f"z slabs x{world}"},
                          "n_clusters": res.n_clusters, "gpu_launches": None}), flush=True)
    lab.close()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.capsule_state:
        run_capsule_state(args)
        return

    import torch
    from paper_1405_1931_gb300 import hk

    local = local % max(1, torch.cuda.device_count())   # ranks may share a GPU with --backend gloo
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        if args.backend == "nccl":
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
    if args.decompose and world > 1:
        run_decomposed(args, rank, world, local, dist)
        dist.destroy_process_group()
        return
    rdev = "cuda" if args.backend == "nccl" else "cpu"   # where the max over ranks is reduced

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    L = args.size
    N = L ** 3
    lab = hk.Labeller(local)
    if args.tile:
        lab.set_tile(*[int(v) for v in args.tile.split(",")])
    stream = torch.cuda.current_stream()
    phi = torch.empty((L, L, L), dtype=torch.float32, device="cuda")
    rc = hk.hk_gen_iid(phi.data_ptr(), L, L, L, 0, P_C, hk._stream_handle(stream))
    assert rc == 0
    out = lab.alloc_outputs(phi.shape, phi.device)
    per = (1, 1, 1)

    for _ in range(max(args.warmup, 3)):
        lab.label(phi, per, out=out)
    torch.cuda.synchronize()

    hk.hk_set_timing(lab.ctx, True)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(args.steps):
        lab.label(phi, per, out=out)
    t_end.record(stream)
    barrier()
    clk = clocks.stop()
    ms_total = t_start.elapsed_time(t_end)
    passes = hk.hk_get_timing(lab.ctx)
    hk.hk_set_timing(lab.ctx, False)
    lab.sync_status()          # raises if a bounded device loop gave up in the timed calls

    ms_step = max_over_ranks(ms_total / args.steps, dist, device=rdev)
    value = job_gsites_per_s(world, N, ms_step)

    labels, sizes, hist, ncl, cap = out
    n_clusters = int(ncl.item())

    # Roofline.  The compulsory bytes of the path are defined for one whole labelling
    # call (4 B phi read + 4 B label write per site, 8 B per cluster size, 256 B of
    # histogram), so the roofline entry treats one hk_label call -- the launch sequence
    # of all passes on one stream -- as the unit.  Per-kernel entries attribute those
    # bytes to the kernels that move them (occupancy reads phi, flatten writes labels
    # and sizes); the other passes move only workspace bytes.
    peak, peak_kind = read_peaks()
    names = list(hk.PASS_NAMES)
    path_bytes = 8 * N + 8 * n_clusters + 8 * 32
    path_achieved = path_bytes / (ms_step * 1e-3) / 1e9
    attributed = {"occupancy": 4 * N, "flatten": 4 * N + 8 * n_clusters + 8 * 32}
    total_pass_ms = sum(passes)
    # A lattice that takes the one-launch path reports its whole call as the first pass
    # (the other slots hold only the gaps between the timing events); the captured
    # traffic and instructions are those of the tiled passes, so they do not apply.
    one_launch = all(p < 0.01 for p in passes[1:])
    traffic_ok = kernel_source_sha() == TRAFFIC_SOURCE_SHA and not one_launch
    if one_launch:
        names, passes = ["one_launch_small_path"], [total_pass_ms]
        attributed = {"one_launch_small_path": path_bytes}
    kernels = []
    for name, ms in zip(names, passes):
        b = attributed.get(name, 0)
        kernels.append({"kernel": name, "avg_ms": ms, "share": ms / total_pass_ms, "algorithmic_bytes": b,
                        "achieved_gbs": (b / (ms * 1e-3) / 1e9) if b else 0.0,
                        "frac": (b / (ms * 1e-3) / 1e9 / peak) if b else 0.0,
                        "traffic": TRAFFIC_BYTES[name] * N / TRAFFIC_SITES if traffic_ok and name in TRAFFIC_BYTES
                        else None})
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    clk_mhz = clk.get("sm_max_mhz") or 2070.0
    issue_peak = nsm * 4 * clk_mhz * 1e6 / 1e9                  # G warp instructions / s
    for k in kernels:
        if k["kernel"] in INST_PER_LAUNCH:
            inst = INST_PER_LAUNCH[k["kernel"]] * N / TRAFFIC_SITES if traffic_ok else None
            ach = inst / (k["avg_ms"] * 1e-3) / 1e9 if inst else None
            k["issue"] = {"bound": "alu", "unit": "G warp-instr/s", "achieved": ach, "peak": issue_peak,
                          "frac": ach / issue_peak if ach else None, "warp_instructions": inst,
                          "peak_basis": f"{nsm} SMs x 4 schedulers x 1 warp instruction per clock x {clk_mhz:.0f} MHz"}
    dom = max(kernels, key=lambda k: k["avg_ms"])
    path_traffic = sum(TRAFFIC_BYTES.values()) * N / TRAFFIC_SITES if traffic_ok else None
    roofline = {"bound": "hbm", "unit": "GB/s", "achieved": path_achieved, "peak": peak,
                "frac": path_achieved / peak, "traffic": path_traffic, "peak_kind": peak_kind,
                "scope": "one hk_label call (all passes)" if not one_launch else "one hk_label call (one launch)",
                "algorithmic_bytes": path_bytes,
                "dominant_kernel": dom["kernel"], "dominant_share": dom["share"],
                "dominant_kernel_issue": dom.get("issue")}

    # End to end through the host-buffer entry points, every step's copy of phi in and
    # of labels, sizes, histogram and count out inside the timed region.  The headline
    # form streams fields the way a simulation hands over snapshots: the asynchronous
    # entry on --e2e-streams contexts, each on its own stream, taking steps in turn,
    # so that one step's copy in overlaps another's copy out.  The synchronous entry
    # (one step at a time) is reported beside it.
    e2e = None
    if not args.no_e2e:
        k_e2e = max(3, min(args.steps, 20))
        cap_h = 2 * n_clusters + 1024            # host sizes buffers: the count fits with room
        phi_h = torch.empty((L, L, L), dtype=torch.float32, pin_memory=True)
        phi_h.copy_(phi)
        nstr = args.e2e_streams if args.e2e_streams > 0 else (3 if world == 1 else 2)
        outs_h = []
        for _ in range(nstr):       # page-locked output sets; fewer contexts if the host runs short
            try:
                outs_h.append((torch.empty((L, L, L), dtype=torch.int32, pin_memory=True),
                               torch.empty(cap_h, dtype=torch.int64, pin_memory=True),
                               torch.empty(32, dtype=torch.int64, pin_memory=True),
                               torch.empty(1, dtype=torch.int64, pin_memory=True)))
            except RuntimeError:
                if not outs_h:
                    raise
                break
        nstr = len(outs_h)
        more = [hk.Labeller(local) for _ in range(nstr - 1)]
        for m in more:
            if args.tile:
                m.set_tile(*[int(v) for v in args.tile.split(",")])
        labs = [lab] + more
        streams = [stream] + [torch.cuda.Stream() for _ in range(nstr - 1)]

        def async_step(i):
            j = i % nstr
            labs[j].label_host_async(phi_h, *outs_h[j], per, stream=streams[j])

        def sync_step():
            o = outs_h[0]
            rc = hk.hk_label_host(lab.ctx, phi_h.data_ptr(), L, L, L, per, o[0].data_ptr(), o[1].data_ptr(),
                                  cap_h, o[2].data_ptr(), o[3].data_ptr(), hk._stream_handle(stream))
            assert rc == hk.HK_OK, rc

        def timed(run):
            barrier()
            t0 = time.perf_counter()
            run()
            for st in streams:
                st.synchronize()
            barrier()
            return max_over_ranks((time.perf_counter() - t0) / k_e2e * 1e3, dist, device=rdev)

        for i in range(nstr):
            async_step(i)
        torch.cuda.synchronize()
        ms_async = timed(lambda: [async_step(i) for i in range(k_e2e)])
        for o in outs_h:
            assert int(o[3][0]) == n_clusters
        for lb, st in zip(labs, streams):
            lb.sync_status(st)
        assert torch.equal(outs_h[0][0], labels.cpu()) and torch.equal(outs_h[0][1][:n_clusters], sizes[:n_clusters].cpu())
        sync_step()
        ms_sync = timed(lambda: [sync_step() for _ in range(k_e2e)])
        assert int(outs_h[0][3][0]) == n_clusters
        d2h = 4 * N + 8 * n_clusters + 8 * 32 + 8
        e2e = {"value": job_gsites_per_s(world, N, ms_async), "unit": "Gsites/s", "ms_per_step": ms_async,
               "h2d_bytes_per_step": 4 * N, "d2h_bytes_per_step": d2h,
               "entry": f"hk_label_host_async (pinned host buffers), {nstr} contexts on {nstr} streams taking "
                        "steps in turn: one step's copy in overlaps another's copy out",
               "steps": k_e2e,
               "sync": {"value": job_gsites_per_s(world, N, ms_sync), "ms_per_step": ms_sync,
                        "entry": "hk_label_host, one step at a time"}}
        # the host link this run had: 1 GiB pinned copies one way, and both ways at once
        nb = min(N, 1 << 28)
        h_in, d_in = phi_h.reshape(-1)[:nb], torch.empty(nb, dtype=torch.float32, device="cuda")
        h_out, d_out = outs_h[0][0].reshape(-1)[:nb].view(torch.float32), phi.reshape(-1)[:nb]

        def rate(fn, nbytes, reps=3):
            fn()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                fn()
            torch.cuda.synchronize()
            return nbytes * reps / (time.perf_counter() - t0) / 1e9

        def both():
            with torch.cuda.stream(streams[0]):
                d_in.copy_(h_in, non_blocking=True)
            with torch.cuda.stream(streams[-1]):
                h_out.copy_(d_out, non_blocking=True)

        e2e["link_gbs"] = {"h2d": rate(lambda: d_in.copy_(h_in, non_blocking=True), 4 * nb),
                           "d2h": rate(lambda: h_out.copy_(d_out, non_blocking=True), 4 * nb),
                           "duplex_each_way": rate(both, 4 * nb)}
        # the same on the whole buffers the steps use: phi in, and each context's labels
        # out while phi comes in (the pattern of the pipelined steps), one pass each
        del d_in
        d_big = torch.empty(N, dtype=torch.float32, device="cuda")
        whole = {"h2d_phi": rate(lambda: d_big.copy_(phi_h.reshape(-1), non_blocking=True), 4 * N, reps=1)}
        for j, o in enumerate(outs_h):
            h_lab = o[0].reshape(-1).view(torch.float32)

            def pair(h_lab=h_lab):
                with torch.cuda.stream(streams[0]):
                    d_big.copy_(phi_h.reshape(-1), non_blocking=True)
                with torch.cuda.stream(streams[-1]):
                    h_lab.copy_(phi.reshape(-1), non_blocking=True)
            whole[f"d2h_labels{j}"] = rate(lambda h_lab=h_lab: h_lab.copy_(phi.reshape(-1), non_blocking=True), 4 * N, reps=1)
            whole[f"duplex_phi_labels{j}_each_way"] = rate(pair, 4 * N, reps=1)
        e2e["link_gbs"]["whole_buffers"] = whole
        del d_big
        for m in more:
            m.close()
        del phi_h, outs_h

    extra = None
    if rank == 0 and not args.no_extra:
        del out, phi, labels, sizes, hist, ncl
        torch.cuda.empty_cache()
        extra = extra_configs(args, peak)

    cpu = cpu_par = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_oracle()
        # a report beside the baseline, run in a child process: never a reason for this run to fail
        try:
            res = subprocess.run([sys.executable, "-c", "import json, bench; print(json.dumps(bench.cpu_parallel_oracle()))"],
                                 cwd=ROOT, capture_output=True, text=True, timeout=120)
            cpu_par = json.loads(res.stdout.strip().splitlines()[-1]) if res.returncode == 0 else \
                {"error": f"exit {res.returncode}: {res.stderr.strip()[-200:]}"}
        except Exception as exc:
            cpu_par = {"error": str(exc)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "Gsites/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": {"workload": f"critical site percolation {L}^3, p=0.3116, periodic xyz",
                           "nx": L, "ny": L, "nz": L, "tile": [32, lab_tile(lab)[0], lab_tile(lab)[1]],
                           "cache": "inputs larger than L2 (4 B/site phi and labels at 1024^3: 8 GiB per step)",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
                "n_clusters": n_clusters,
                "passes_ms": dict(zip(names, passes)),
                "roofline": roofline, "kernels": kernels, "configs": extra,
                "cpu_baseline": cpu, "cpu_parallel": cpu_par, "e2e": e2e,
                "gpu_launches": LAUNCHES_PER_CALL * args.steps, "clocks": clk}
        print(json.dumps(line), flush=True)
    lab.close()
    if dist is not None:
        dist.destroy_process_group()


def lab_tile(lab):
    return lab.tile


if __name__ == "__main__":
    main()
