"""Continuous-batching CP-ALS service over the relate C ABI.

Clients submit decomposition requests (a sparse tensor on the host, a rank,
a precision, a stopping rule); the server answers each with the CP model
(lambda, factors, fit). The paper runs CP-ALS one tensor at a time; serving
many tensors on one GPU is layered on top of its method and changes no
arithmetic: every request runs the same encode + CP-ALS path (Sec. 3, Sec.
2.2) as a lone call, through the C ABI.

* Admission. A request's device footprint is what the library says its
  encode and CP-ALS will request (relate_footprint) plus its factors. The
  queue admits requests in arrival order while the admitted footprints fit
  in the budget; when the head does not fit, later requests that do fit may
  go first, at most `max_bypass` times per head (bounded wait). A request
  larger than the whole budget is refused at submission.
* Continuous batching. `workers` host threads, each with its own CUDA
  stream, take admitted requests as soon as they are free: a finishing
  request's slot is refilled at once instead of waiting for a batch to
  drain, and the kernels of different requests share the SMs (a small
  request's launches fill only part of the GPU).
* Launches. Each request's CP-ALS replays one captured CUDA graph per
  iteration (relate_set_cpals_graph), and the library's device memory comes
  from the stream-ordered allocator, so one request's release never waits
  for the other streams.
* Batch lane (small requests). Requests of at most `small_nnz` nonzeros go
  to one lane that runs up to `batch_max` of them in lockstep
  (relate_cpals_batch): per iteration and mode ONE persistent MTTKRP launch
  over the tiles of all of them, one captured CUDA graph per iteration. The
  lane works in chunks of `chunk_iters` iterations: between chunks finished
  requests leave and newly admitted ones join (continuous batching at chunk
  granularity); each request keeps its own stopping rule (its previous fit is
  carried across chunks).

Latency = completion - arrival, including the host-to-device copy of the
tensor, the encoding, CP-ALS and the copy of the factors back to the host.
"""
from __future__ import annotations

import math
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np

from . import relate as rl

_TORCH_DTYPES = {"f64": "float64", "f32": "float32", "bf16": "bfloat16"}


@dataclass
class Request:
    """coords: (N, nnz) uint32 host array; vals: (nnz,) f32 or f64 host array.
    precision is the factor dtype: "f64" (FP64 factors and accumulation),
    "f32" (FP32 factors and accumulation, FP64 normal equations) or "bf16"."""
    coords: np.ndarray
    vals: np.ndarray
    dims: tuple
    R: int
    precision: str = "f32"
    tol: float = 1e-4
    max_iters: int = 50
    init_seed: int = 0
    return_factors: bool = True
    init: list | None = None   # host initial factors; None: drawn on the device from init_seed
    rid: int = -1
    arrival: float = 0.0   # set by submit()

    @property
    def nnz(self) -> int:
        return int(self.coords.shape[1])

    @property
    def nmodes(self) -> int:
        return int(self.coords.shape[0])


@dataclass
class Result:
    rid: int
    fit: float
    iters: int
    status: int
    lam: np.ndarray
    factors: list | None
    nnz: int
    R: int
    nmodes: int
    footprint: int
    t_arrival: float
    t_admit: float
    t_start: float
    t_done: float
    fit_trace: np.ndarray = field(default_factory=lambda: np.zeros(0))

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival

    @property
    def work(self) -> float:
        """nnz * R * N * iterations: the MTTKRP work the request did."""
        return float(self.nnz) * self.R * self.nmodes * self.iters


def initial_factors(dims, R: int, seed: int, device, dtype):
    """U[0,1) initial factors drawn on the device from a seeded generator, in
    FP32 so that every precision starts from the same values (BF16 rounds
    them)."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    return [torch.rand((int(I), R), generator=gen, device=device, dtype=torch.float32).to(dtype).contiguous()
            for I in dims]


def footprint(req: Request) -> int:
    """Device bytes of a request: library allocations (relate_footprint) and
    its factors, plus the staging of the initial factors."""
    fp = rl.relate_footprint(req.dims, req.nnz, req.R, factor_dtype=req.precision,
                             val_dtype="f64" if req.vals.dtype == np.float64 else "f32")
    init = sum(int(I) for I in req.dims) * req.R * 4
    return fp["peak"] + init


class AdmissionQueue:
    """FIFO admission by device-memory footprint (host logic only).

    put(item, nbytes) enqueues; take() blocks until an item is admitted (its
    bytes are then counted as in use) or the queue is closed (returns None);
    release(nbytes) returns an admitted item's bytes."""

    def __init__(self, budget_bytes: int, max_bypass: int = 8):
        self.budget = int(budget_bytes)
        self.max_bypass = int(max_bypass)
        self.in_use = 0
        self.peak_in_use = 0
        self.admitted = 0
        self._items: list = []      # [item, nbytes, bypassed]
        self._closed = False
        self._cv = threading.Condition()

    def put(self, item, nbytes: int) -> None:
        if nbytes > self.budget:
            raise ValueError(f"request needs {nbytes} device bytes, more than the budget {self.budget}")
        with self._cv:
            if self._closed:
                raise RuntimeError("queue closed")
            self._items.append([item, int(nbytes), 0])
            self._cv.notify_all()

    def _pick(self):
        if not self._items:
            return None
        free = self.budget - self.in_use
        head = self._items[0]
        if head[1] <= free:
            return 0
        if head[2] >= self.max_bypass:
            return None     # the head has waited long enough: no more bypassing
        for k in range(1, len(self._items)):
            if self._items[k][1] <= free:
                head[2] += 1
                return k
        return None

    def take(self, timeout: float | None = None):
        deadline = None if timeout is None else time.monotonic() + timeout
        with self._cv:
            while True:
                k = self._pick()
                if k is not None:
                    item, nbytes, _ = self._items.pop(k)
                    self.in_use += nbytes
                    self.peak_in_use = max(self.peak_in_use, self.in_use)
                    self.admitted += 1
                    return item, nbytes
                if self._closed and not self._items:
                    return None
                wait = None if deadline is None else deadline - time.monotonic()
                if wait is not None and wait <= 0:
                    return None
                self._cv.wait(wait)

    def release(self, nbytes: int) -> None:
        with self._cv:
            self.in_use -= int(nbytes)
            assert self.in_use >= 0
            self._cv.notify_all()

    def close(self) -> None:
        with self._cv:
            self._closed = True
            self._cv.notify_all()

    def __len__(self) -> int:
        with self._cv:
            return len(self._items)


def percentile(xs, p: float) -> float:
    """Nearest-rank percentile (p in (0, 100])."""
    s = sorted(xs)
    if not s:
        return float("nan")
    k = max(1, math.ceil(p / 100.0 * len(s)))
    return float(s[k - 1])


class Server:
    """Worker threads (one CUDA stream each) over an AdmissionQueue, and
    optionally a batch lane for small requests (small_nnz > 0)."""

    def __init__(self, workers: int = 8, budget_bytes: int | None = None, device: int = 0,
                 use_graph: bool = True, max_bypass: int = 8, small_nnz: int = 0, batch_max: int = 16,
                 chunk_iters: int = 5, small_budget_frac: float = 0.1, small_tol: float = 1e-4,
                 tune_nnz: int = 0):
        import torch
        self._torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("the CP-ALS service needs a CUDA device")
        self.device = torch.device("cuda", device)
        rl.lib()  # fail loudly here if the library is missing
        if budget_bytes is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            budget_bytes = int(0.5 * free)
        self.small_nnz = int(small_nnz)
        if self.small_nnz > 0:
            small_budget = int(small_budget_frac * budget_bytes)
            self.small_queue = AdmissionQueue(small_budget, max_bypass)
            budget_bytes -= small_budget
        else:
            self.small_queue = None
        self.queue = AdmissionQueue(budget_bytes, max_bypass)
        self.use_graph = use_graph
        self.batch_max = int(batch_max)
        self.chunk_iters = int(chunk_iters)
        self.small_tol = float(small_tol)  # the lane's stopping tolerance (one per lockstep call)
        self.tune_nnz = int(tune_nnz)  # requests this large get their kernel plans tuned first (0: never)
        self._t0 = time.perf_counter()
        self._threads = []
        self._errors = []
        for w in range(workers):
            t = threading.Thread(target=self._worker, name=f"relate-serve-{w}", daemon=True)
            t.start()
            self._threads.append(t)
        if self.small_queue is not None:
            t = threading.Thread(target=self._batch_lane, name="relate-serve-batch", daemon=True)
            t.start()
            self._threads.append(t)

    def now(self) -> float:
        return time.perf_counter() - self._t0

    def submit(self, req: Request) -> Future:
        fut: Future = Future()
        req.arrival = self.now()
        nbytes = footprint(req)
        if (self.small_queue is not None and req.nnz <= self.small_nnz and nbytes <= self.small_queue.budget
                and req.tol == self.small_tol):
            self.small_queue.put((req, fut), nbytes)
        else:
            self.queue.put((req, fut), nbytes)
        return fut

    def close(self) -> None:
        self.queue.close()
        if self.small_queue is not None:
            self.small_queue.close()
        for t in self._threads:
            t.join()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _worker(self) -> None:
        torch = self._torch
        setup_error = None
        try:
            torch.cuda.set_device(self.device)
            stream = torch.cuda.Stream(self.device)
        except BaseException as e:  # every request this worker takes fails with it
            setup_error = e
        while True:
            got = self.queue.take()
            if got is None:
                return
            (req, fut), nbytes = got
            t_admit = self.now()
            try:
                if setup_error is not None:
                    raise setup_error
                with torch.cuda.stream(stream):
                    res = self._run(req, stream, nbytes, t_admit)
                fut.set_result(res)
            except BaseException as e:  # reported through the future
                fut.set_exception(e)
            finally:
                self.queue.release(nbytes)

    def _run(self, req: Request, stream, nbytes: int, t_admit: float) -> Result:
        torch = self._torch
        t_start = self.now()
        tdt = getattr(torch, _TORCH_DTYPES[req.precision])
        if req.init is not None:
            factors = [torch.from_numpy(np.ascontiguousarray(f)).to(self.device).to(tdt).contiguous()
                       for f in req.init]
        else:
            factors = initial_factors(req.dims, req.R, req.init_seed, self.device, tdt)
        h = rl.relate_encode(req.coords, req.vals, req.dims, factor_dtype=req.precision, stream=stream)
        try:
            if self.tune_nnz > 0 and req.nnz >= self.tune_nnz:
                # the per-mode plan search of tune.py, timed on this worker's
                # stream (one launch per plan, no L2 flush); the handle keeps
                # the fastest plans for its CP-ALS
                from .tune import tune_modes
                tune_modes(h, req.dims, req.R, req.precision, factors, reps=1, stream=stream, flush_l2=False)
            if self.use_graph:
                rl.relate_set_cpals_graph(h, True)
            out = rl.relate_cpals(h, req.R, req.max_iters, req.tol, factors)
        finally:
            h.close()
        host = [f.float().cpu().numpy() if req.precision == "bf16" else f.cpu().numpy()
                for f in factors] if req.return_factors else None
        stream.synchronize()
        return Result(req.rid, out["fit"], out["iters"], out["status"], out["lam"], host, req.nnz, req.R,
                      req.nmodes, nbytes, req.arrival, t_admit, t_start, self.now(), out["fit_trace"])


    def _batch_lane(self) -> None:
        """Small requests in lockstep, in chunks of chunk_iters iterations;
        admission between chunks (continuous batching)."""
        torch = self._torch
        q = self.small_queue
        try:
            torch.cuda.set_device(self.device)
            stream = torch.cuda.Stream(self.device)
        except BaseException as e:
            while True:
                got = q.take()
                if got is None:
                    return
                (req, fut), nbytes = got
                fut.set_exception(e)
                q.release(nbytes)
        active = []  # dicts: req, fut, nbytes, h, factors, prev, iters, trace, t_admit, t_start
        closed = False
        while True:
            while not closed and len(active) < self.batch_max:
                got = q.take(timeout=0.0 if active else None)
                if got is None:
                    closed = q._closed and len(q) == 0
                    break
                (req, fut), nbytes = got
                t_admit = self.now()
                try:
                    with torch.cuda.stream(stream):
                        tdt = getattr(torch, _TORCH_DTYPES[req.precision])
                        if req.init is not None:
                            facs = [torch.from_numpy(np.ascontiguousarray(f)).to(self.device).to(tdt).contiguous()
                                    for f in req.init]
                        else:
                            facs = initial_factors(req.dims, req.R, req.init_seed, self.device, tdt)
                        h = rl.relate_encode(req.coords, req.vals, req.dims, factor_dtype=req.precision,
                                             stream=stream)
                    active.append({"req": req, "fut": fut, "nbytes": nbytes, "h": h, "factors": facs,
                                   "prev": float("nan"), "iters": 0, "trace": [], "t_admit": t_admit,
                                   "t_start": t_admit, "status": 0})
                except BaseException as e:
                    fut.set_exception(e)
                    q.release(nbytes)
            if not active:
                if closed or (q._closed and len(q) == 0):
                    return
                continue
            chunk = min([self.chunk_iters] + [a["req"].max_iters - a["iters"] for a in active])
            try:
                with torch.cuda.stream(stream):
                    res, _ = rl.relate_cpals_batch([a["h"] for a in active], [a["req"].R for a in active], chunk,
                                                   self.small_tol, [a["factors"] for a in active], stream,
                                                   prev_fit=[a["prev"] for a in active])
            except BaseException as e:
                for a in active:
                    a["h"].close()
                    a["fut"].set_exception(e)
                    q.release(a["nbytes"])
                active = []
                continue
            still = []
            for a, r in zip(active, res):
                a["iters"] += r["iters"]
                a["trace"].extend(r["fit_trace"].tolist())
                a["prev"] = r["fit"]
                a["lam"] = r["lam"]
                a["status"] = r["status"]
                done = r["status"] != 0 or r["iters"] < chunk or a["iters"] >= a["req"].max_iters
                if not done:
                    still.append(a)
                    continue
                req = a["req"]
                try:
                    host = [f.float().cpu().numpy() if req.precision == "bf16" else f.cpu().numpy()
                            for f in a["factors"]] if req.return_factors else None
                    stream.synchronize()
                    a["fut"].set_result(Result(req.rid, r["fit"], a["iters"], a["status"], a["lam"], host, req.nnz,
                                               req.R, req.nmodes, a["nbytes"], req.arrival, a["t_admit"],
                                               a["t_start"], self.now(), np.array(a["trace"])))
                except BaseException as e:
                    a["fut"].set_exception(e)
                finally:
                    a["h"].close()
                    q.release(a["nbytes"])
            active = still


def summarize(results, makespan: float) -> dict:
    lat = [r.latency for r in results]
    work = sum(r.work for r in results)
    return {"requests": len(results), "makespan_s": makespan,
            "throughput_req_s": len(results) / makespan if makespan > 0 else float("nan"),
            "nnz_R_per_s": work / makespan if makespan > 0 else float("nan"),
            "p50_s": percentile(lat, 50), "p99_s": percentile(lat, 99), "max_s": max(lat) if lat else 0.0,
            "mean_iters": float(np.mean([r.iters for r in results])) if results else 0.0}


def run_mix(requests, arrivals=None, workers: int = 8, budget_bytes: int | None = None,
            use_graph: bool = True, small_nnz: int = 0, batch_max: int = 16, chunk_iters: int = 5,
            small_tol: float = 1e-4, tune_nnz: int = 0):
    """Serves `requests` (Request objects). arrivals: None = closed loop (all
    submitted at t = 0), else the arrival time of each request in seconds.
    small_nnz > 0 routes requests of at most that many nonzeros to the batch
    lane; tune_nnz > 0 tunes the kernel plans of requests of at least that
    many nonzeros. Returns (results in request order, summary dict, queue
    statistics)."""
    srv = Server(workers=workers, budget_bytes=budget_bytes, use_graph=use_graph, small_nnz=small_nnz,
                 batch_max=batch_max, chunk_iters=chunk_iters, small_tol=small_tol, tune_nnz=tune_nnz)
    futs = []
    t0 = srv.now()
    try:
        for k, req in enumerate(requests):
            if arrivals is not None:
                delay = t0 + float(arrivals[k]) - srv.now()
                if delay > 0:
                    time.sleep(delay)
            futs.append(srv.submit(req))
        results = [f.result() for f in futs]
    finally:
        srv.close()
    makespan = max(r.t_done for r in results) - t0 if results else 0.0
    q = {"budget_bytes": srv.queue.budget, "peak_admitted_bytes": srv.queue.peak_in_use,
         "admitted": srv.queue.admitted}
    return results, summarize(results, makespan), q


def make_requests(n: int, seed_base: int = 1000, nnz_range=(1e4, 2e7), tol: float = 1e-4, max_iters: int = 50,
                  return_factors: bool = False):
    """The seeded request mix of a CP-ALS service (synth.serving_request), FP32
    precision; with_precision() gives the same requests at another one."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import synth
    out = []
    for i in range(n):
        spec, R = synth.serving_request(i, seed_base=seed_base, nnz_range=nnz_range)
        c, v = synth.make_tensor(spec)
        out.append(Request(c, v, spec.dims, R, precision="f32", tol=tol, max_iters=max_iters,
                           init_seed=spec.seed, return_factors=return_factors, rid=i))
    return out


def with_precision(requests, precision: str):
    """The same requests at another precision (FP64 values for "f64")."""
    from dataclasses import replace
    return [replace(r, precision=precision, vals=r.vals.astype(np.float64) if precision == "f64" else r.vals)
            for r in requests]


def main(argv=None):
    """Serves the request mix in several forms: the first form closed loop
    measures the service rate S, then every form serves Poisson arrivals at
    0.8 S (and, with --closed-all, also closed loop). A form is
    "precision[:lane][:tuned]": factor precision; ":lane" sends requests of at
    most --small-nnz nonzeros to the batch lane; ":tuned" tunes the kernel
    plans (tune.tune_modes) of requests of at least --tune-nnz nonzeros
    before their CP-ALS. Prints one JSON line per run."""
    import argparse
    import json
    import os
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import synth

    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=128)
    ap.add_argument("--nnz-max", type=float, default=2e7)
    ap.add_argument("--workers", type=int, default=8)
    ap.add_argument("--budget-gb", type=float, default=0.0)
    ap.add_argument("--forms", default="f32:lane,bf16:lane,f64",
                    help="comma-separated precision[:lane] forms; the first one calibrates the arrival rate")
    ap.add_argument("--precisions", default=None, help="(older spelling) comma-separated precisions, no lane")
    ap.add_argument("--small-nnz", type=int, default=200_000)
    ap.add_argument("--batch-max", type=int, default=16)
    ap.add_argument("--chunk-iters", type=int, default=5)
    ap.add_argument("--tune-nnz", type=int, default=2_000_000)
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-open-loop", action="store_true")
    ap.add_argument("--closed-all", action="store_true", help="closed loop for every form, not only the first")
    args = ap.parse_args(argv)
    budget = int(args.budget_gb * 2 ** 30) if args.budget_gb > 0 else None
    forms = args.forms.split(",") if args.precisions is None else args.precisions.split(",")
    rate = None
    lines = []
    all_fits = {}
    t = time.time()
    mix = make_requests(args.requests, nnz_range=(1e4, args.nnz_max))
    gen_s = time.time() - t
    print(json.dumps({"generated": len(mix), "nnz_total": sum(r.nnz for r in mix), "generation_s": gen_s}),
          flush=True)
    for k, form in enumerate(forms):
        prec, *opts = form.split(":")
        lane = "lane" in opts
        tuned = "tuned" in opts
        reqs = with_precision(mix, prec)
        loops = ["closed", "open"] if (k == 0 or args.closed_all) else ["open"]
        for loop in loops:
            if loop == "open" and args.no_open_loop:
                continue
            arr = None if loop == "closed" else synth.poisson_arrivals(len(reqs), rate, seed=0)
            res, summ, q = run_mix(reqs, arr, workers=args.workers, budget_bytes=budget,
                                   use_graph=not args.no_graph, small_nnz=args.small_nnz if lane else 0,
                                   batch_max=args.batch_max, chunk_iters=args.chunk_iters,
                                   small_tol=reqs[0].tol if reqs else 1e-4,
                                   tune_nnz=args.tune_nnz if tuned else 0)
            if loop == "closed" and rate is None:
                rate = 0.8 * summ["throughput_req_s"]
            line = {"serve": prec, "lane": lane, "small_nnz": args.small_nnz if lane else 0,
                    "tune_nnz": args.tune_nnz if tuned else 0, "loop": loop,
                    "workers": args.workers, "graph": not args.no_graph,
                    "arrival_rate_req_s": rate if loop == "open" else None, **summ, **q,
                    "nnz_total": sum(r.nnz for r in reqs), "lane_requests": sum(1 for r in reqs if lane and
                                                                                r.nnz <= args.small_nnz)}
            fits = {r.rid: (r.fit, r.iters) for r in res}
            all_fits[(form, loop)] = fits
            print(json.dumps(line), flush=True)
            lines.append(line)
        del reqs
    # every form's fits against the plain FP64 form's (the acceptance bound is 1e-3)
    ref = next((v for (f, _), v in all_fits.items() if f.partition(":")[0] == "f64"), None)
    if ref is not None:
        diff, gap = {}, {}
        for (f, loop), v in all_fits.items():
            d = np.array([abs(ref[i][0] - v[i][0]) for i in v])
            early = np.array([v[i][1] < ref[i][1] for i in v])
            diff[f"{f}/{loop}"] = float(d.max())
            gap[f"{f}/{loop}"] = {"p50": float(np.percentile(d, 50)), "p99": float(np.percentile(d, 99)),
                                  "max": float(d.max()), "over_1e-3": int((d > 1e-3).sum()), "requests": int(d.size),
                                  "over_1e-3_stopped_earlier": int(((d > 1e-3) & early).sum())}
        print(json.dumps({"max_fit_diff_vs_f64": diff}), flush=True)
        print(json.dumps({"fit_gap_vs_f64": gap}), flush=True)
    return lines


if __name__ == "__main__":
    main()
