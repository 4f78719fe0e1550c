"""Client side of the render server: output-slot pools and the replay of a
timed request stream (the serving workload: Poisson arrivals over resident
soups, forward only with binary opacity, Eq. 3).

``replay(server, soup_ids, reqs, ...)`` submits every request at its arrival
time from the calling thread and collects completions on a second thread;
latency is the server's own done - submit time of each request.  An output
slot (G-buffer + colour of one view) is reused only after the request that
last wrote it has completed.
"""
from __future__ import annotations

import collections
import queue
import threading
import time

import numpy as np

from . import native as N


class SlotPool:
    """Per-resolution free lists of preallocated output buffers."""

    def __init__(self, resolutions, slots: int, C: int, device: str = "cuda"):
        import torch
        self.free = {}
        self.cv = threading.Condition()
        for (w, h) in resolutions:
            self.free[(w, h)] = collections.deque(
                (torch.empty((1, h, w, 4), dtype=torch.int32, device=device),
                 torch.empty((1, C - 1, h, w), dtype=torch.float32, device=device)) for _ in range(slots))

    def take(self, wh):
        with self.cv:
            while not self.free[wh]:
                self.cv.wait()
            return self.free[wh].popleft()

    def give(self, wh, slot):
        with self.cv:
            self.free[wh].append(slot)
            self.cv.notify_all()


def replay(srv: "N.Server", soup_ids, reqs, pool: SlotPool, mode: int = N.DS_MODE_THRESHOLD_HALF, bg=None,
           time_scale: float = 1.0):
    """Submit ``reqs`` = [(t_arrival_s, soup_index, camera, seed)] at their
    arrival times; returns a dict of per-request arrays (latency_ms,
    batch, pixels) and the wall-clock span."""
    done_q: "queue.Queue" = queue.Queue()
    stats = []

    def waiter():
        while True:
            item = done_q.get()
            if item is None:
                return
            tk, wh, slot = item
            st = srv.wait(tk)
            pool.give(wh, slot)
            stats.append((st, wh))

    th = threading.Thread(target=waiter, daemon=True)
    th.start()
    t0 = time.perf_counter()
    for (ta, k, cam, seed) in reqs:
        delay = t0 + ta * time_scale - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        wh = (cam.width, cam.height)
        slot = pool.take(wh)
        tk = srv.submit(soup_ids[k], cam, seed, mode, bg, slot[0], slot[1])
        done_q.put((tk, wh, slot))
    done_q.put(None)
    th.join()
    wall = time.perf_counter() - t0
    lat = np.array([(s["done_ns"] - s["submit_ns"]) / 1e6 for s, _ in stats])
    first = min(s["submit_ns"] for s, _ in stats)
    last = max(s["done_ns"] for s, _ in stats)
    return {"latency_ms": lat, "batch": np.array([s["batch"] for s, _ in stats]),
            "pixels": np.array([w * h for _, (w, h) in stats]), "span_s": (last - first) / 1e9, "wall_s": wall}
