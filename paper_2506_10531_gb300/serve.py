"""Request loop over libqaoa's serving API (continuous batching of optimise-and-sample jobs).

`serve_stream` replays a list of requests with arrival times against a `qaoa_server`: it
submits each request once the wall clock reaches its arrival time, ticks the server (every
tick admits what fits and runs one step of every admitted job on the device), collects finished
jobs, and reports per-request latency (completion minus arrival) and throughput. Admission,
batching, the optimiser and sampling all run inside the library; this module only paces the
arrivals and collects results.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import (qaoa_server_clock, qaoa_server_create, qaoa_server_destroy, qaoa_server_poll,
               qaoa_server_stats, qaoa_server_submit, qaoa_server_tick)


@dataclass
class Request:
    n: int
    p: int
    Q: np.ndarray          # n x n float32
    params: np.ndarray     # 2p float32 (gamma then beta)
    steps: int
    lr: float
    arrival: float = 0.0   # seconds after the start of the replay


@dataclass
class StreamReport:
    results: dict = field(default_factory=dict)     # request index -> qaoa_job_result
    latency_s: np.ndarray = None                     # per request, in request order
    elapsed_s: float = 0.0                           # first arrival to last completion
    max_active: int = 0
    ticks: int = 0
    bytes_total: float = 0.0
    gpu_ms: float = 0.0
    launches: int = 0

    @property
    def solves_per_s(self) -> float:
        return len(self.results) / self.elapsed_s if self.elapsed_s > 0 else 0.0


def serve_stream(ctx, requests, scratch_bytes: int, max_jobs: int, k: int, stream=None,
                 server=None) -> StreamReport:
    """Replay `requests` (sorted by arrival) in real time; returns the report."""
    own = server is None
    srv = qaoa_server_create(ctx, scratch_bytes, max_jobs, k) if own else server
    rep = StreamReport()
    try:
        t0 = qaoa_server_clock()
        ids = {}
        nxt = 0
        pending = 0
        while nxt < len(requests) or pending > 0:
            now = qaoa_server_clock() - t0
            while nxt < len(requests) and requests[nxt].arrival <= now:
                r = requests[nxt]
                jid = qaoa_server_submit(srv, r.n, r.p, r.Q, r.params, r.steps, r.lr)
                ids[jid] = nxt
                nxt += 1
                pending += 1
            active, queued = qaoa_server_tick(srv, stream)
            rep.ticks += 1
            rep.max_active = max(rep.max_active, active)
            for res in qaoa_server_poll(srv, wait=(active == 0 and queued == 0 and pending > 0)):
                rep.results[ids[res.job_id]] = res
                pending -= 1
            if pending == 0 and nxt < len(requests):
                # idle until the next arrival
                gap = requests[nxt].arrival - (qaoa_server_clock() - t0)
                if gap > 0:
                    time.sleep(gap)
        arr = np.array([r.arrival for r in requests])
        done = np.array([rep.results[i].t_done - t0 for i in range(len(requests))])
        rep.latency_s = done - arr
        rep.elapsed_s = float(done.max() - arr.min()) if len(requests) else 0.0
        _, _, _, rep.bytes_total, rep.gpu_ms, rep.launches = qaoa_server_stats(srv)
    finally:
        if own:
            qaoa_server_destroy(srv)
    return rep
