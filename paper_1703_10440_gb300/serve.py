"""Continuous-batching server for A-orthonormal QR requests.

The client of this loop is a projection eigensolver or a block-GMRES code
that asks for many A-orthonormalisations of different sizes.  The server:

* admits arrived requests in arrival order while the device-memory budget
  allows (A, Z, Q, R and, for batched requests, the x/p workspace stay
  resident on the device until the request completes);
* every tick, puts all admitted small requests (m * n^2 <= ``small_work``)
  into ONE ``mgsa_qr_batched`` call (in the form ``small_variant``, by
  default the server's form) -- a persistent kernel in which every CTA
  runs one instance, so requests of different sizes run side by side -- and
  gives each large request its own ``mgsa_qr`` launch over the whole GPU;
* with ``max_large_inflight`` = w > 0, keeps at most w large launches queued
  on the device and launches the waiting large request with the least work
  (m * n^2) next, so medium requests overtake queued big ones;
* with ``slice_ms`` > 0, runs large requests in time slices of about that
  long, so a request that arrives while a long factorisation runs waits for
  one slice, not for the whole factorisation.  By default
  (``large_mode="group"``) each launch is one grouped launch
  (``mgsa_qr_group``): the waiting large requests with the least remaining
  work share the large part of the GPU side by side, each on a gang of CTAs
  sized in proportion to its rows, each for a slice of about ``slice_ms``;
  up to ``max_large_inflight`` such launches are queued on the stream, so the
  GPU never waits for the host between them.  With ``large_mode="slices"``
  each slice is a whole-GPU ``mgsa_qr_steps`` launch of one request on a
  handle of its own from a small pool, least remaining work first;
* with ``small_ctas`` = k > 0, partitions the SMs: large requests run with
  k fewer CTAs than the GPU has SMs, small ones on a second stream and a
  second handle whose batched launches use k CTAs, so the two kinds run side
  by side and small requests do not wait behind large ones;
* keeps ticking while earlier launches run (continuous batching): requests
  that arrive meanwhile are admitted as memory frees up and launched behind
  the work in flight;
* timestamps completion with CUDA events and reports per-request latency
  (arrival to device completion) as p50 / p99 beside throughput.

Inputs are drawn on the device at admission (``workloads.device``) on a side
stream; the QR stream waits for them with an event.  Scheduling is host
Python; every step of the QRs runs in libmgsa's kernels.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time

import numpy as np

from . import mgsa
from .batch import JOB_DTYPE, _round


@dataclasses.dataclass
class Request:
    rid: int
    m: int
    n: int
    kind: str            # 'laplace' | 'banded'
    arrival: float       # seconds after the start of the run
    seed: int = 20170330
    # filled in by the server
    A: tuple | None = None
    Z: object = None
    Q: object = None
    R: object = None
    work: object = None
    nbytes: int = 0
    need: int = 0            # device bytes the request needs once admitted (computed once)
    ready: object = None     # event on the generator stream after its inputs were drawn
    small: bool = False
    t_done: float = math.nan
    info: int = -99
    info_buf: object = None
    handle: int = 0          # sliced large requests: the pool handle holding its state
    next_step: int = 0       # sliced large requests: first step of the next slice
    slice_inflight: bool = False


def poisson_arrivals(rate: float, duration: float, seed: int = 20170330, m_lo: float = 1e3, m_hi: float = 1e6,
                     n_lo: int = 8, n_hi: int = 128) -> list[Request]:
    """Arrivals of a Poisson process of ``rate`` per second over ``duration``
    seconds; m ~ logU[m_lo, m_hi], n ~ U{n_lo..n_hi}, matrix kind 50/50.  The
    sizes and the gaps come from separate streams, so request k has the same
    size at every rate (only its arrival time depends on the rate)."""
    gaps = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 50])))
    sizes = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 51])))
    t, out = 0.0, []
    while True:
        t += gaps.exponential(1.0 / rate)
        if t >= duration:
            break
        m = int(round(math.exp(sizes.uniform(math.log(m_lo), math.log(m_hi)))))
        n = int(sizes.integers(n_lo, n_hi + 1))
        kind = "laplace" if sizes.random() < 0.5 else "banded"
        out.append(Request(len(out), m, n, kind, t, seed))
    return out


class Server:
    def __init__(self, handle: int, variant: str = "hp", budget_bytes: float = 120e9, small_work: float = 2e7,
                 device: int = 0, max_batch: int = 4096, max_m: int = 1_000_000, max_n: int = 128,
                 small_ctas: int = 0, max_large_inflight: int = 0, slice_ms: float = 0.0, large_handles: int = 3,
                 large_mode: str = "group", rows_per_cta: int = 4096, admit_per_tick: int = 0,
                 gang_fill: str = "prefix", small_variant: str | None = None):
        import torch

        self.torch = torch
        self.h = handle
        self.variant = variant
        self.v = mgsa.VARIANTS[variant]
        # Small requests (the batched kernel) may use another form: with one
        # CTA per instance HP is the fastest, on the whole GPU HA usually is.
        self.small_variant = small_variant or variant
        self.vs = mgsa.VARIANTS[self.small_variant]
        self.budget = budget_bytes
        self.small_work = small_work
        self.dev = torch.device("cuda", device)
        self.max_batch = max_batch
        # Requests admitted per turn of the loop (0: as many as the budget
        # allows).  Drawing a request's inputs costs the host about a
        # millisecond; a bounded turn keeps launches flowing under a backlog.
        self.admit_per_tick = admit_per_tick
        self.stream = torch.cuda.Stream(self.dev)
        self.gen_stream = torch.cuda.Stream(self.dev)
        self.small_ctas = small_ctas
        self.max_large_inflight = max_large_inflight
        self.h_small, self.stream_small, self._own_handle = handle, self.stream, 0
        if small_ctas > 0:
            sms = torch.cuda.get_device_properties(self.dev).multi_processor_count
            if not 0 < small_ctas < sms:
                raise ValueError("small_ctas must be in (0, number of SMs)")
            mgsa.mgsa_set_param(handle, mgsa.MGSA_PARAM_MAX_CTAS, sms - small_ctas)
            self._own_handle = mgsa.mgsa_create(device)
            mgsa.mgsa_set_param(self._own_handle, mgsa.MGSA_PARAM_BATCH_CTAS, small_ctas)
            self.h_small = self._own_handle
            self.stream_small = torch.cuda.Stream(self.dev)
        # Large requests share the handle's workspace: size it once, up front.
        mgsa.mgsa_reserve(handle, max_m, max_n, self.v)
        self.shared_ws = mgsa.mgsa_workspace_bytes(handle, max_m, max_n, self.v)
        # Sliced large requests: grouped launches, or one pool handle per
        # request in progress.
        self.slice_ms = slice_ms
        if large_mode not in ("group", "slices"):
            raise ValueError("large_mode: 'group' or 'slices'")
        self.group = slice_ms > 0 and large_mode == "group"
        self.rows_per_cta = rows_per_cta
        if gang_fill not in ("prefix", "greedy"):
            raise ValueError("gang_fill: 'prefix' or 'greedy'")
        self.gang_fill = gang_fill
        self.sms = torch.cuda.get_device_properties(self.dev).multi_processor_count
        self.large_ctas = self.sms - max(small_ctas, 0)
        self._pool: list[int] = []
        if slice_ms > 0 and not self.group:
            sms = torch.cuda.get_device_properties(self.dev).multi_processor_count
            for _ in range(large_handles):
                hh = mgsa.mgsa_create(device)
                if small_ctas > 0:
                    mgsa.mgsa_set_param(hh, mgsa.MGSA_PARAM_MAX_CTAS, sms - small_ctas)
                mgsa.mgsa_reserve(hh, max_m, max_n, self.v)
                self._pool.append(hh)
            self.shared_ws += large_handles * mgsa.mgsa_workspace_bytes(self._pool[0], max_m, max_n, self.v)
        self._all_pool = list(self._pool)

    def close(self):
        """Undo the SM partition (the caller's handle gets its default CTA
        count back) and release the handles the server created."""
        self.torch.cuda.synchronize(self.dev)
        if self._own_handle:
            mgsa.mgsa_set_param(self.h, mgsa.MGSA_PARAM_MAX_CTAS, 0)
            mgsa.mgsa_destroy(self._own_handle)
            self._own_handle = 0
            self.h_small = self.h
        for hh in self._all_pool:
            mgsa.mgsa_destroy(hh)
        self._all_pool, self._pool = [], []

    # -- time slices of large requests --------------------------------------
    # Cost model of one step (seconds): the sweep's FP64 work on the remaining
    # columns at an effective 0.8 TFLOP/s, the per-column MVs of HA / naive,
    # and a fixed 20 us of barriers and reductions.
    # On a gang of c of the GPU's S CTAs the work part scales by S / c.
    def _step_s(self, r: Request, i: int, ctas: int = 0) -> float:
        per_pair = 6.0 if self.variant == "hp" else 4.0
        nnz_row = 5.0 if r.kind == "laplace" else 17.0
        mvs = 0 if self.variant == "hp" else (2 if self.variant == "naive" else 1)
        share = 1.0 if ctas <= 0 else self.sms / ctas
        return share * (per_pair * r.m * (r.n - 1 - i) + mvs * 2.0 * nnz_row * r.m) / 0.8e12 + 20e-6

    def _remaining_s(self, r: Request) -> float:
        k = r.n - r.next_step
        per_pair = 6.0 if self.variant == "hp" else 4.0
        nnz_row = 5.0 if r.kind == "laplace" else 17.0
        mvs = 0 if self.variant == "hp" else (2 if self.variant == "naive" else 1)
        return (per_pair * r.m * k * (k - 1) / 2 + mvs * 2.0 * nnz_row * r.m * k) / 0.8e12 + 20e-6 * k

    def _launch_slice(self, r: Request):
        torch = self.torch
        if r.next_step == 0:  # its inputs come from the generator stream
            ready = torch.cuda.Event()
            ready.record(self.gen_stream)
            self.stream.wait_event(ready)
        first, count, t = r.next_step, 0, 0.0
        while first + count < r.n and (count == 0 or t < self.slice_ms * 1e-3):
            t += self._step_s(r, first + count)
            count += 1
        rowptr, col, val = r.A
        csr = mgsa.make_csr(r.m, col.numel(), rowptr, col, val)
        st = mgsa.mgsa_qr_steps(r.handle, csr, r.Z, r.m, r.n, r.m, self.v, r.Q, r.Q.stride(0), r.R, r.n, first, count,
                                self.stream)
        if st != mgsa.MGSA_OK:
            raise mgsa.MgsaError(st, mgsa.mgsa_last_error())
        r.next_step = first + count
        last = r.next_step >= r.n
        if last:
            mgsa.mgsa_copy_info(r.handle, r.info_buf, self.stream)
        done = torch.cuda.Event(enable_timing=True)
        done.record(self.stream)
        r.slice_inflight = True
        return ("slice", [r], done, last)

    # -- grouped launches of large requests ---------------------------------
    def _gangs(self, cands: list[Request]) -> list[tuple[Request, int]]:
        """The members of the next grouped launch and their CTAs.  Requests
        are taken in the given order (least remaining work first), each with
        the gang it wants or the CTAs still free, until the large part of the
        GPU is taken; every gang is at least one CTA and at most one CTA per
        128 rows (the smallest slab).  CTAs left over (members capped by their
        rows) go to the members with the most rows (with a backlog) or in
        order (otherwise).

        With a backlog (four or more candidates) a gang wants one CTA per
        ``rows_per_cta`` rows, for throughput: every member then has about the
        same rows per CTA, so their slices take about the same time.
        Otherwise it wants one CTA per ``rows_per_cta // 4`` rows, for
        latency, and the request closest to done finishes first."""
        backlog = len(cands) >= 4
        target = self.rows_per_cta if backlog else max(128, self.rows_per_cta // 4)
        left = self.large_ctas
        chosen, ctas, caps = [], [], []
        for r in cands:
            if left <= 0 or len(chosen) == mgsa.MGSA_GROUP_MAX:
                break
            cap = max(1, -(-r.m // 128))
            want = max(1, min(cap, -(-r.m // target)))
            g = min(want, left)
            if g < want and chosen:
                if self.gang_fill == "prefix":  # the first request that does not fit ends the group
                    break
                # "greedy": a gang squeezed below what the request wants must
                # still run one step within a slice (a launch lasts as long as
                # its slowest member), else the request waits.
                if self._step_s(r, r.next_step, g) > self.slice_ms * 1e-3:
                    continue
            chosen.append(r)
            ctas.append(g)
            caps.append(cap)
            left -= g
        order = sorted(range(len(chosen)), key=lambda k: -chosen[k].m) if backlog else range(len(chosen))
        for k in order:
            if left <= 0:
                break
            add = min(left, caps[k] - ctas[k])
            ctas[k] += add
            left -= add
        return list(zip(chosen, ctas))

    def _launch_group(self, cands: list[Request]):
        torch = self.torch
        members = self._gangs(cands)
        for r, _ in members:
            if r.next_step == 0:  # its inputs come from the generator stream
                self.stream.wait_event(r.ready)
        budget = self.slice_ms * 1e-3
        specs, finishing = [], []
        for r, c in members:
            first, count, t = r.next_step, 0, 0.0
            while first + count < r.n and (count == 0 or t < budget):
                t += self._step_s(r, first + count, c)
                count += 1
            rowptr, col, val = r.A
            specs.append(mgsa.group_member(r.m, r.n, self.v, rowptr, col, val, r.Z, r.m, r.Q, r.Q.stride(0), r.R, r.n,
                                           r.work, first, count, c))
            r.next_step = first + count
            if r.next_step >= r.n:
                finishing.append(r)
        st = mgsa.mgsa_qr_group(self.h, self.v, specs, self.stream)
        if st != mgsa.MGSA_OK:
            raise mgsa.MgsaError(st, mgsa.mgsa_last_error())
        with torch.cuda.stream(self.stream):
            for r in finishing:  # the member's status words, as mgsa_copy_info reports them
                r.info_buf.copy_(r.work[:1].view(torch.int32))
        done = torch.cuda.Event(enable_timing=True)
        done.record(self.stream)
        return ("group", finishing, done, len(members))

    # -- admission ---------------------------------------------------------
    def _bytes(self, r: Request) -> int:
        m, n = r.m, r.n
        nnz = 5 * m if r.kind == "laplace" else 17 * m
        b = 12 * nnz + 4 * (m + 1) + 2 * 8 * m * n + 8 * n * n
        if r.m * r.n ** 2 <= self.small_work:
            b += mgsa.mgsa_job_workspace_bytes(m, n, self.vs)
        elif self.group:
            b += mgsa.mgsa_group_workspace_bytes(self.h, m, n, self.v)
        return b

    def _materialize(self, r: Request):
        from workloads import device as wd

        torch = self.torch
        with torch.cuda.stream(self.gen_stream):
            r.A, r.Z, r.m = wd.request_inputs(r.kind, r.m, r.n, r.seed, r.rid, self.dev)
            r.n = r.Z.shape[1]
            r.Q = torch.empty((r.n, _round(r.m)), dtype=torch.float64, device=self.dev)
            r.R = torch.empty((r.n, r.n), dtype=torch.float64, device=self.dev)
            r.small = r.m * r.n ** 2 <= self.small_work
            if r.small:
                r.work = torch.empty(mgsa.mgsa_job_workspace_bytes(r.m, r.n, self.vs) // 8 + 1, dtype=torch.float64,
                                     device=self.dev)
            elif self.group:  # x / p columns, partials and status words of its grouped slices
                r.work = torch.empty(mgsa.mgsa_group_workspace_bytes(self.h, r.m, r.n, self.v) // 8 + 1,
                                     dtype=torch.float64, device=self.dev)
                assert r.work.data_ptr() % 256 == 0
            r.info_buf = torch.zeros(2, dtype=torch.int32, device=self.dev)
            r.ready = torch.cuda.Event()
            r.ready.record(self.gen_stream)

    def _release(self, r: Request):
        r.A = r.Z = r.Q = r.R = r.work = r.info_buf = r.ready = None

    # -- launches ----------------------------------------------------------
    def _launch(self, admitted: list[Request], ref_event):
        torch = self.torch
        ready = torch.cuda.Event()
        ready.record(self.gen_stream)
        self.stream.wait_event(ready)
        if self.stream_small is not self.stream:
            self.stream_small.wait_event(ready)
        groups = []
        small = [r for r in admitted if r.small]
        large = [r for r in admitted if not r.small]
        if small:
            small.sort(key=lambda r: -r.m * r.n ** 2)
            jobs = np.zeros(len(small), dtype=JOB_DTYPE)
            for k, r in enumerate(small):
                rowptr, col, val = r.A
                jobs[k] = (r.m, r.n, self.vs, rowptr.data_ptr(), col.data_ptr(), val.data_ptr(), r.Z.data_ptr(), r.m,
                           r.Q.data_ptr(), r.Q.stride(0), r.R.data_ptr(), r.n, r.work.data_ptr())
            # pinned + non_blocking: the host loop must not wait behind the work in flight
            jobs_host = torch.from_numpy(jobs.view(np.uint8).copy()).pin_memory()
            with torch.cuda.stream(self.stream_small):
                jobs_dev = jobs_host.to(self.dev, non_blocking=True)
                info = torch.zeros(len(small), dtype=torch.int32, device=self.dev)
            st = mgsa.mgsa_qr_batched(self.h_small, len(small), jobs_dev, info, self.stream_small)
            if st != mgsa.MGSA_OK:
                raise mgsa.MgsaError(st, mgsa.mgsa_last_error())
            done = torch.cuda.Event(enable_timing=True)
            done.record(self.stream_small)
            groups.append(("batch", small, done, (jobs_dev, info, jobs_host)))
        for r in large:
            rowptr, col, val = r.A
            csr = mgsa.make_csr(r.m, col.numel(), rowptr, col, val)
            st = mgsa.mgsa_qr(self.h, csr, r.Z, r.m, r.n, r.m, self.v, r.Q, r.Q.stride(0), r.R, r.n, self.stream)
            if st != mgsa.MGSA_OK:
                raise mgsa.MgsaError(st, mgsa.mgsa_last_error())
            mgsa.mgsa_copy_info(self.h, r.info_buf, self.stream)
            done = torch.cuda.Event(enable_timing=True)
            done.record(self.stream)
            groups.append(("single", [r], done, None))
        return groups

    # -- the loop ----------------------------------------------------------
    def run(self, requests: list[Request], realtime: bool = True) -> dict:
        """Serve ``requests`` (arrival times relative to the start).  With
        ``realtime`` False every request is considered arrived at t = 0."""
        torch = self.torch
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting: collections.deque = collections.deque()
        inflight: collections.deque = collections.deque()
        ready_large: list = []  # admitted large requests not yet launched (max_large_inflight > 0 or slicing)
        running: list = []      # sliced large requests with slices still to run
        used = self.shared_ws
        peak = used
        torch.cuda.synchronize(self.dev)
        ref = torch.cuda.Event(enable_timing=True)
        ref.record(self.stream)
        ref.synchronize()
        t0 = time.perf_counter()
        ticks = launches = 0
        window = self.max_large_inflight if self.max_large_inflight > 0 else 2
        launches_box = [0]

        def top_up_groups():
            # Large requests share grouped launches; up to `window` of them are
            # queued on the stream (those whose event has not fired), each
            # formed from the requests with the least remaining work (a
            # request's next slice may follow its current one in the queue:
            # the stream orders them).  One queued launch keeps an arriving
            # request's wait to one slice; with a backlog (four or more
            # requests with slices to run), `window` keep the GPU busy while
            # the host admits requests or notices a completion.
            cands = [r for r in running if r.next_step < r.n]
            group_window = window if len(cands) >= 4 else min(window, 1)
            n_groups = sum(1 for grp in inflight if grp[0] == "group" and not grp[2].query())
            while n_groups < group_window and cands:
                cands.sort(key=lambda r: (self._remaining_s(r), r.arrival))
                inflight.append(self._launch_group(cands))
                launches_box[0] += 1
                n_groups += 1
                cands = [r for r in running if r.next_step < r.n]

        while pending or waiting or inflight or ready_large or running:
            now = time.perf_counter() - t0
            while pending and (not realtime or pending[0].arrival <= now):
                waiting.append(pending.popleft())
            admitted = []
            cap = self.max_batch if self.admit_per_tick <= 0 else min(self.max_batch, self.admit_per_tick)
            while waiting and len(admitted) < cap:
                if not waiting[0].need:
                    waiting[0].need = self._bytes(waiting[0])
                need = waiting[0].need
                if used + need > self.budget and (inflight or admitted or ready_large or running):
                    break
                r = waiting.popleft()
                self._materialize(r)
                r.nbytes = need
                used += need
                admitted.append(r)
                if self.group:  # drawing inputs takes host time: keep the launch queue topped up meanwhile
                    if not r.small:
                        running.append(r)
                    top_up_groups()
            peak = max(peak, used)
            launch_now = admitted
            if self.group:
                launch_now = [r for r in admitted if r.small]
                top_up_groups()
            elif self.slice_ms > 0:
                ready_large.extend(r for r in admitted if not r.small)
                launch_now = [r for r in admitted if r.small]
                n_slices = sum(1 for grp in inflight if grp[0] == "slice")
                # One slice in flight keeps an arriving request's wait to one
                # slice; with a backlog of large requests (four or more
                # waiting), two keep the GPU busy while the host notices a
                # completion.
                slice_window = window if len(ready_large) >= 4 else min(window, 1)
                while n_slices < slice_window:
                    cands = [r for r in running if not r.slice_inflight]
                    if self._pool:
                        cands += ready_large
                    if not cands:
                        break
                    nxt = min(cands, key=lambda r: (self._remaining_s(r), r.arrival))
                    if nxt.next_step == 0 and nxt in ready_large:
                        ready_large.remove(nxt)
                        nxt.handle = self._pool.pop()
                        running.append(nxt)
                    inflight.append(self._launch_slice(nxt))
                    launches += 1
                    n_slices += 1
            elif self.max_large_inflight > 0:
                ready_large.extend(r for r in admitted if not r.small)
                launch_now = [r for r in admitted if r.small]
                n_large = sum(1 for grp in inflight if grp[0] == "single")
                while ready_large and n_large < self.max_large_inflight:
                    nxt = min(ready_large, key=lambda r: (r.m * r.n ** 2, r.arrival))
                    ready_large.remove(nxt)
                    launch_now.append(nxt)
                    n_large += 1
            if launch_now:
                for g in self._launch(launch_now, ref):
                    inflight.append(g)
                    launches += 1
                ticks += 1
            progressed = bool(launch_now)
            finished = [grp for grp in inflight if grp[2].query()]
            if finished:
                inflight = collections.deque(grp for grp in inflight if not any(grp is f for f in finished))
            for kind, reqs, done, extra in finished:
                t_done = ref.elapsed_time(done) / 1e3
                if kind == "slice":
                    r = reqs[0]
                    r.slice_inflight = False
                    progressed = True
                    if not extra:  # more slices to come
                        continue
                    running.remove(r)
                    self._pool.append(r.handle)
                    r.handle = 0
                    infos = [int(r.info_buf[0].item())]
                elif kind == "group":
                    progressed = True
                    for r in reqs:
                        running.remove(r)
                    infos = [int(r.info_buf[0].item()) for r in reqs]
                elif kind == "batch":
                    infos = extra[1].cpu().numpy()
                else:
                    infos = [int(reqs[0].info_buf[0].item())]
                for r, inf in zip(reqs, infos):
                    r.t_done = t_done
                    r.info = int(inf)
                    used -= r.nbytes
                progressed = True
                for r in reqs:
                    self._keep(r)
            if not progressed:
                time.sleep(50e-6)
        launches += launches_box[0]
        torch.cuda.synchronize(self.dev)
        lat = np.array([r.t_done - r.arrival for r in requests])
        first = min(r.arrival for r in requests)
        last = max(r.t_done for r in requests)
        self.last_latency_s = {r.rid: r.t_done - r.arrival for r in requests}
        return {"requests": len(requests), "ok": int(sum(r.info == 0 for r in requests)),
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_ms": float(lat.mean() * 1e3), "qr_per_s": len(requests) / (last - first),
                "makespan_s": last - first, "ticks": ticks, "launches": launches, "peak_bytes": peak,
                "small": int(sum(r.small for r in requests))}

    # Results are dropped after completion unless a subclass keeps them.
    def _keep(self, r: Request):
        self._release(r)


class KeepingServer(Server):
    """Keeps Q and R of every request on the host (for tests)."""

    def __init__(self, *a, **kw):
        super().__init__(*a, **kw)
        self.results = {}

    def _keep(self, r: Request):
        self.results[r.rid] = (r.Q[:, : r.m].T.cpu().numpy(), r.R.T.cpu().numpy(), r.info)
        self._release(r)
