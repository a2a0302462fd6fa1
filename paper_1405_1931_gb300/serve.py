"""Serving loop: labelling requests from a running simulation, continuous batching.

A producer stands in for the simulation (Sec. 5 emulsions and Sec. 6
capsules): it generates each request's field on the device, on its own
stream, finishing about when the request arrives (the simulation hands over a
finished field).  The server keeps fields and output
buffers resident on the device and:

* admits requests while their bytes (field, labels, sizes and the per-lattice
  workspace bound) fit under a memory cap;
* batches by size: arrived small requests go together into one batched call
  (``hk_label_batched``) on a free small-request worker stream, and requests
  that arrive while others are on the GPU join the next batch as soon as a
  worker frees up; large requests run one per call, enqueued in arrival order
  on one large-request stream as soon as they arrive, so that they follow each
  other on the device with no host round trip between them and none shares the
  GPU with another large call.  Each worker owns its own library context, so
  calls on different workers overlap on the device;
* detects completion with CUDA events and frees the request's memory; once a
  worker's stream is idle it reads that context's device status word, and a
  request whose batch saw a bounded device loop give up is counted as failed.

Latency is reported two ways: from the request's arrival to the host
observing its completion event, and from its field being ready on the device
to its labels being ready (CUDA events: queueing plus labelling, without the
stand-in simulation's generation time).  ``mode="fifo"`` serves the same stream with one
``hk_label`` launch per request in arrival order on one stream (one worker),
as the baseline.  Results are bit-identical between the modes and to labelling each
request alone (the tests check this).
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import fields, hk

GB = 1 << 30


@dataclass
class Request:
    rid: int
    arrival: float                   # seconds after the stream starts
    kind: str                        # "emulsion" or "capsule"
    L: int
    spheres: tuple | None = None     # (centres (n,3), radii (n,))
    axes: tuple | None = None        # capsule semi-axes
    periodic: tuple = (1, 1, 1)
    # runtime state
    phi: object = None
    out: object = None
    gen_event: object = None
    sphere_ptr: int = 0
    ready_to_done_ms: float = math.nan
    t_done: float = math.nan
    n_clusters: int = -1
    failed: bool = False             # a bounded device loop gave up in its batch

    @property
    def sites(self) -> int:
        return self.L ** 3

    def nbytes(self) -> int:
        n = self.sites
        return 4 * n + 4 * n + 8 * ((n + 1) // 2) + hk.hk_workspace_bytes(self.L, self.L, self.L)


def request_stream(n: int = 2000, rate: float = 400.0, seed: int = 3, frac_emulsion: float = 0.8,
                   l_lo: int = 64, l_hi: int = 512) -> list:
    """Seeded Poisson request stream (exponential gaps, mean 1/rate).

    Request k draws counters 4k..4k+3 of stream `seed`: the gap, the kind
    (emulsion with probability frac_emulsion, else capsule), the side L
    (log-uniform in [l_lo, l_hi]) and a sub-seed.  Emulsions get
    round(0.3 L^3 / (4/3 pi E[r^3])) droplets with r in [5, 15]
    (E[r^3] = 1250), i.e. a droplet volume fraction of about 0.3; capsules get
    semi-axes uniform in [10, 60] clamped to L/2 - 2.
    """
    u = fields.uniform(seed, np.arange(4 * n, dtype=np.uint64)).astype(np.float64).reshape(n, 4)
    t = 0.0
    out = []
    for k in range(n):
        t += -math.log(1.0 - u[k, 0]) / rate
        kind = "emulsion" if u[k, 1] < frac_emulsion else "capsule"
        L = int(round(l_lo * (l_hi / l_lo) ** u[k, 2]))
        sub = 100000 + k
        if kind == "emulsion":
            nd = max(1, int(round(0.3 * L ** 3 / (4.0 / 3.0 * math.pi * 1250.0))))
            centres, radii = fields.sphere_params(nd, (L, L, L), seed=sub)
            out.append(Request(k, t, kind, L, spheres=(centres, radii)))
        else:
            ax = fields.uniform(sub, np.arange(3, dtype=np.uint64)).astype(np.float64)
            axes = tuple(float(min(10.0 + 50.0 * a, L / 2 - 2)) for a in ax)
            out.append(Request(k, t, kind, L, axes=axes))
    return out


def upload_spheres(requests: list):
    """Put every emulsion request's droplets on the device once (the simulation's state).

    Returns the device tensor; each request gets `sphere_ptr` into it (4 floats a droplet).
    """
    import torch
    chunks, offs, total = [], [], 0
    for r in requests:
        if r.kind == "emulsion":
            c, rad = r.spheres
            a = np.concatenate([c, rad[:, None]], axis=1).astype(np.float32).reshape(-1)
            offs.append((r, total))
            chunks.append(a)
            total += a.size
    host = torch.from_numpy(np.concatenate(chunks) if chunks else np.zeros(4, np.float32)).pin_memory()
    dev = host.to("cuda", non_blocking=True)
    torch.cuda.current_stream().synchronize()
    for r, off in offs:
        r.sphere_ptr = dev.data_ptr() + 4 * off
    return dev


def generate(req: Request, stream) -> None:
    """Write the request's phi on the device (the simulation stand-in)."""
    import torch
    L = req.L
    req.phi = torch.empty((L, L, L), dtype=torch.float32, device="cuda")
    h = hk._stream_handle(stream)
    if req.kind == "emulsion" and getattr(req, "sphere_ptr", None):
        rc = hk.hk_gen_spheres_dev(req.phi.data_ptr(), L, L, L, req.sphere_ptr, len(req.spheres[1]), 8.0, h)
    elif req.kind == "emulsion":
        centres, radii = req.spheres
        rc = hk.hk_gen_spheres(req.phi.data_ptr(), L, L, L, centres, radii, 8.0, h)
    else:
        rc = hk.hk_gen_capsule(req.phi.data_ptr(), L, *req.axes, h)
    if rc != 0:
        raise RuntimeError(f"field generation failed ({rc})")


class Server:
    """Continuous-batching server of labelling requests on one GPU.

    Workers are library contexts, each on its own stream, above the producers'
    priority; `small_workers` of them take only small requests (at most
    `small_sites` sites), batched together up to `max_batch` requests and
    `small_batch_sites` sites, so that a small request never waits behind a large
    one.  The first of the other workers takes every large request, one per call,
    in arrival order: it is a queue on its stream, each call enqueued when its
    request arrives, so that a large request waits only for the large ones before
    it, as in FIFO, but for none of the small ones.  Its stream has the highest
    priority, so that the small batches running beside a large call delay it as
    little as possible (the latency tail is the large requests').  Workers with
    nothing in flight take small batches when no small worker is free.  The FIFO
    baseline is every request on the large-request stream.
    """

    def __init__(self, device: int = 0, cap_bytes: int = 32 * GB, workers: int = 4, max_batch: int = 64,
                 max_batch_sites: int = 1 << 28, tile: tuple | None = None, graphs: bool = False,
                 producers: int = 4, small_workers: int = 2, small_sites: int = 1 << 21,
                 small_batch_sites: int = 1 << 23, small_priority: int = -1,
                 large_priority: int = -2, max_side: int = 512):
        import torch
        self.device = device
        self.cap = cap_bytes
        self.max_batch = max_batch
        self.max_batch_sites = max_batch_sites   # bounds each worker's workspace
        self.small_sites = small_sites
        self.small_batch_sites = small_batch_sites
        self.n_small = max(0, min(small_workers, workers - 1))
        # Priorities (a lower number is a higher one, clamped to the device's range): the
        # simulation stand-in's producers run at the default, every labelling worker above
        # them, and the large-request worker above the small ones.
        self.producers = [torch.cuda.Stream(device=device) for _ in range(producers)]
        self.streams = ([torch.cuda.Stream(device=device, priority=small_priority) for _ in range(self.n_small)] +
                        [torch.cuda.Stream(device=device, priority=large_priority) for _ in range(workers - self.n_small)])
        self.labs = [hk.Labeller(device, tile=tile) for _ in range(workers)]
        for lab in self.labs:
            if graphs:
                lab.set_graphs(True)
        self.warm(max_side)

    def warm(self, max_side: int):
        """Grow every worker's workspace for the largest request (a cube of max_side) and
        for a full small batch, run one small call on each worker and each field generator
        once, and have torch's caching allocator reserve the admission cap once, so that
        no call or request in service allocates from the driver (a cudaMalloc synchronises
        the device) or loads kernels."""
        import torch
        try:   # fields and outputs are carved from this one cached segment later
            blk = torch.empty(self.cap, dtype=torch.uint8, device=f"cuda:{self.device}")
            del blk
        except RuntimeError:
            pass
        need = hk.hk_workspace_bytes(max_side, max_side, max_side)
        side = max(1, int(round(self.small_batch_sites ** (1.0 / 3.0))))
        need = max(need, hk.hk_workspace_bytes(side, side, side) * 2)
        phi = torch.full((48, 48, 40), -1.0, dtype=torch.float32, device=f"cuda:{self.device}")
        phi[::2] = 1.0
        for lab, s in zip(self.labs, self.streams):
            lab.reserve(need)
            out = lab.alloc_outputs(phi.shape, phi.device)
            with torch.cuda.stream(s):
                lab.label(phi, (1, 1, 1), out=out, stream=s)
                lab.label_batched([(phi, (1, 1, 1), out), (phi, (0, 1, 0), lab.alloc_outputs(phi.shape, phi.device))],
                                  stream=s)
            lab.sync_status(s)
        # the stand-in simulation's generators, once each, so that their first launch in
        # service does not stall the stream behind it
        side = 64
        em = Request(-1, 0.0, "emulsion", side, spheres=fields.sphere_params(4, (side, side, side), seed=1))
        cap = Request(-2, 0.0, "capsule", side, axes=(10.0, 12.0, 14.0))
        keep = upload_spheres([em])
        prod = self.producers[0]
        with torch.cuda.stream(prod):
            for r in (em, cap):
                generate(r, prod)
        prod.synchronize()
        del keep

    def close(self):
        for lab in self.labs:
            lab.close()

    def serve(self, requests: list, mode: str = "continuous", keep_outputs: bool = False,
              gen_lead_s: float = 0.05) -> dict:
        """Serve `requests` (arrival times in seconds from now) and return statistics.

        The stand-in simulation produces each request's field on a producer stream
        starting `gen_lead_s` before the request's arrival (as memory admits), so that
        a request arrives when the simulation hands over its finished field; a field
        still being written at arrival is waited for on the device.  gen_lead_s = 0
        generates each field only once its request has arrived.  Latency is from
        arrival to the host seeing the request's labels done.
        """
        import torch
        spheres_dev = upload_spheres(requests)   # noqa: F841  (kept alive for the run)
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        generated = deque()      # field generation issued, request not yet arrived
        ready = deque()          # arrived, not yet launched
        inflight = []            # (worker, [requests], end_event)
        # continuous batching uses every worker; the baseline is one launch per
        # request, in arrival order, on a single stream
        fifo = mode == "fifo"
        nbusy = [0] * len(self.streams)          # calls in flight per worker
        used = 0
        peak_used = 0
        done = []
        failed = 0
        unchecked = [[] for _ in self.streams]   # completed requests whose status is not yet read
        nprod = 0
        t0 = time.perf_counter()
        while pending or generated or ready or inflight:
            now = time.perf_counter() - t0
            # 1. completions
            still = []
            for w, batch, ev in inflight:
                if ev.query():
                    tdone = time.perf_counter() - t0
                    for r in batch:
                        r.t_done = tdone
                        r.ready_to_done_ms = r.gen_event.elapsed_time(ev)
                        r.n_clusters = int(r.out[3].item()) if keep_outputs else -1
                        used -= r.nbytes()
                        if not keep_outputs:
                            r.phi = None
                            r.out = None
                        done.append(r)
                    unchecked[w].extend(batch)
                    nbusy[w] -= 1
                else:
                    still.append((w, batch, ev))
            inflight = still
            # The device status word of a worker's context (a bounded loop that gave up)
            # is read once its stream is idle, so that the read waits for nothing; the
            # word is sticky, so a give-up fails every request completed since the last read.
            for w in range(len(self.streams)):
                if unchecked[w] and not any(iw == w for iw, _, _ in inflight):
                    rc = hk.hk_sync_status(self.labs[w].ctx, hk._stream_handle(self.streams[w]))
                    if rc != hk.HK_OK:
                        for r in unchecked[w]:
                            r.failed = True
                        failed += len(unchecked[w])
                    unchecked[w] = []
            # 2. the simulation produces fields ahead of their arrival, admitted by memory
            while pending and pending[0].arrival - gen_lead_s <= now and used + pending[0].nbytes() <= self.cap:
                r = pending.popleft()
                used += r.nbytes()
                peak_used = max(peak_used, used)
                prod = self.producers[nprod % len(self.producers)]
                nprod += 1
                with torch.cuda.stream(prod):
                    generate(r, prod)
                    r.out = hk.Labeller.alloc_outputs(r.phi.shape, r.phi.device)
                    r.gen_event = torch.cuda.Event(enable_timing=True)
                    r.gen_event.record(prod)
                generated.append(r)
            # 3. arrivals
            while generated and generated[0].arrival <= now:
                ready.append(generated.popleft())
            # 4. launches
            if ready:
                if fifo:
                    # every request is its own launch, enqueued back to back on the
                    # large-request stream
                    w, batch = self.n_small, [ready.popleft()]
                else:
                    w, batch = self._pick(ready, nbusy)
                if batch:
                    nbusy[w] += 1
                    s = self.streams[w]
                    for r in batch:
                        s.wait_event(r.gen_event)
                    with torch.cuda.stream(s):
                        if len(batch) == 1:
                            r = batch[0]
                            self.labs[w].label(r.phi, r.periodic, out=r.out, stream=s)
                        else:
                            self.labs[w].label_batched([(r.phi, r.periodic, r.out) for r in batch], stream=s)
                        ev = torch.cuda.Event(enable_timing=True)
                        ev.record(s)
                    inflight.append((w, batch, ev))
                    continue
            nxt = []
            if pending:
                nxt.append(pending[0].arrival - gen_lead_s)
            if generated:
                nxt.append(generated[0].arrival)
            if not inflight and not ready and nxt:
                wait = min(nxt) - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.001))
        wall = max(r.t_done for r in done) if done else 0.0
        lat = np.array([r.t_done - r.arrival for r in done]) * 1e3
        lat_ready = np.array([r.ready_to_done_ms for r in done])
        sites = sum(r.sites for r in done)
        small = np.array([r.sites <= self.small_sites for r in done])
        stats = {"mode": mode, "requests": len(done), "wall_s": wall, "sites": sites,
                 "gsites_per_s": sites / wall / 1e9 if wall > 0 else 0.0,
                 "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                 "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
                 "ready_p50_ms": float(np.percentile(lat_ready, 50)), "ready_p99_ms": float(np.percentile(lat_ready, 99)),
                 "peak_admitted_gb": peak_used / GB, "cap_gb": self.cap / GB,
                 "workers": 1 if fifo else len(self.streams), "failed": failed, "gen_lead_ms": gen_lead_s * 1e3,
                 "done": done}
        if small.any() and (~small).any():
            stats["small_p99_ms"] = float(np.percentile(lat[small], 99))
            stats["large_p99_ms"] = float(np.percentile(lat[~small], 99))
        return stats

    def _pick(self, ready: deque, nbusy: list):
        """Continuous mode: the next batch and its worker, or (-1, []) to wait.

        The oldest large request goes to the large-request worker whether or not it
        has calls in flight (its stream keeps them in arrival order); small requests
        go to a small worker with nothing in flight as one batch, oldest first, up to
        max_batch requests and small_batch_sites sites, else to another idle worker."""
        for r in ready:
            if r.sites > self.small_sites:
                ready.remove(r)
                return self.n_small, [r]
        idle = [w for w in range(len(self.streams)) if nbusy[w] == 0]
        if not idle:
            return -1, []
        # a small worker, else a spare one, else the large-request worker itself
        w = min(idle, key=lambda v: (v >= self.n_small, v == self.n_small, v))
        batch, sites = [], 0
        for r in list(ready):
            if batch and (len(batch) >= self.max_batch or sites + r.sites > self.small_batch_sites):
                break
            batch.append(r)
            sites += r.sites
        for r in batch:
            ready.remove(r)
        return w, batch
