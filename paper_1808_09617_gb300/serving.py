"""Continuous-batching NN-DTW server over resident training sets.

Training sets (and their envelopes, built once on the device) stay resident.
Queries arrive one at a time (``submit``) for any of the sets.  A scheduler
thread keeps up to ``n_slots`` batches in flight, each on its own CUDA stream.
Whenever a slot is free it forms a batch across datasets: it visits the sets
in the order of their oldest waiting query and admits from each as many
waiting queries as fit both ``max_batch`` (queries per batch, all sets
together) and the device-memory budget (the batch's search workspace, query
and result buffers); a set that does not fit ends the batch, so the oldest
query is never passed over.  With ``mix_ratio``, only sets of a similar
cost per query (within that factor of the first set's N L (2W+1)) share a
batch, since every query of a batch completes with its slowest set; the
others wait for the next free slot, where the oldest of them comes first.
On the 16-set serving workload a factor of 4 lowered the median latency at
10,000-20,000 queries/s offered and raised the 99th percentile there, so
the default mixes every set.  The batch's queries are copied to the device and
searched by one ``nn_dtw_search_batched`` call on the slot's stream, every set
of the batch in the same stage launches.  Batches on different slots overlap
on the GPU; queries that arrive while others run are admitted as soon as a
slot and memory free up.  Completed batches are detected by CUDA events, their
results copied back and the futures resolved.  A query's result does not
depend on which batch it joins (the search is exact per query).  A set whose
one-query batch can never fit the budget is refused when the server starts.
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np

from . import nndtw


@dataclass(eq=False)
class _Set:
    train: object
    labels: object
    env: object
    L: int
    W: int
    V: int
    N: int
    flags: int = 0


@dataclass(eq=False)
class _Req:
    query: np.ndarray
    set_id: int
    future: Future
    t_arrival: float


@dataclass(eq=False)
class _Batch:
    parts: list          # [(set_id, [requests], host outputs (idx, label, dist))]
    stream: object
    event: object
    nbytes: int
    t_launch: float
    keep: list = field(default_factory=list)


class Server:
    def __init__(self, sets: dict, n_slots: int = 4, max_batch: int = 512,
                 memory_budget: int = 8 << 30, device: str = "cuda", tune: bool = True,
                 mix_ratio: float = float("inf")):
        """``sets``: {set_id: (train float32 [N, L], labels int32 [N], W, V)}."""
        import torch
        self.torch = torch
        dev = torch.device(device)
        if dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        self.dev = dev
        self.sets: dict[int, _Set] = {}
        for sid, (train, labels, W, V) in sets.items():
            t = torch.from_numpy(np.ascontiguousarray(train, dtype=np.float32)).to(self.dev)
            lab = torch.from_numpy(np.ascontiguousarray(labels, dtype=np.int32)).to(self.dev)
            env = nndtw.nn_dtw_build_envelopes(t, int(W))
            self.sets[sid] = _Set(t, lab, env, t.shape[1], int(W), int(V), t.shape[0])
        torch.cuda.synchronize(self.dev)
        self.n_slots = n_slots
        self.max_batch = max_batch
        self.mix_ratio = float(mix_ratio)
        self.budget = memory_budget
        # a set whose one-query batch does not fit the budget could never be
        # served: refuse it here rather than let its queries wait forever
        for sid, s in self.sets.items():
            if self._batch_bytes(s, 1) > self.budget:
                raise ValueError(f"training set {sid}: one query needs "
                                 f"{self._batch_bytes(s, 1)} bytes, more than the memory "
                                 f"budget of {self.budget}")
        self.in_use = 0
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(n_slots)]
        self.free_slots = list(range(n_slots))
        self.pending: dict[int, collections.deque] = {sid: collections.deque() for sid in self.sets}
        self.inflight: list[_Batch] = []
        self.lock = threading.Lock()
        self.wake = threading.Event()
        self.running = True
        self.latencies: list[float] = []
        self.completed = 0
        self.batches = 0
        self.batch_sets = 0      # datasets over all batches (batches span datasets)
        self.t_first = None
        self.t_last = None
        if tune:
            self._tune()
        self.thread = threading.Thread(target=self._loop, name="nndtw-server", daemon=True)
        self.thread.start()

    # ------------------------------------------------------------- public API
    def submit(self, query, set_id: int, t_arrival: float | None = None) -> Future:
        """Queue one query (float32 [L]) for training set ``set_id``; the future
        resolves to (nn_index, nn_label, nn_dist)."""
        q = np.ascontiguousarray(query, dtype=np.float32)
        if set_id not in self.sets or q.shape != (self.sets[set_id].L,):
            raise ValueError("query shape does not match the training set")
        f: Future = Future()
        r = _Req(q, set_id, f, time.perf_counter() if t_arrival is None else t_arrival)
        with self.lock:
            if not self.thread.is_alive() and self.running is False:
                raise RuntimeError("server is closed")
            self.pending[set_id].append(r)
            if self.t_first is None:
                self.t_first = r.t_arrival
        self.wake.set()
        return f

    def close(self):
        self.running = False
        self.wake.set()
        self.thread.join()

    def latency_stats(self) -> dict:
        with self.lock:
            lat = np.array(self.latencies)
            n = self.completed
            span = (self.t_last - self.t_first) if (self.t_first and self.t_last) else 0.0
        if lat.size == 0:
            return {"completed": 0}
        return {"completed": n, "batches": self.batches,
                "mean_sets_per_batch": self.batch_sets / self.batches if self.batches else None,
                "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_ms": float(lat.mean() * 1e3),
                "throughput_qps": n / span if span > 0 else None}

    # --------------------------------------------------------------- internals
    def _tune(self):
        """Pick the DTW lanes-per-pair per set on a sample batch of its own series."""
        from . import autotune
        for s in self.sets.values():
            q = s.train[: min(64, s.N)]
            g = autotune.tune_search(s.train, s.labels, q, s.W, s.V, reps=2)
            s.flags = nndtw.DTW_GROUP(g) if g else 0

    def _batch_bytes(self, s: _Set, Q: int) -> int:
        """Device bytes of Q queries of set s in a batch: their share of the
        batched search's workspace, the query series and the outputs."""
        return (nndtw.nn_dtw_workspace_size(s.N, Q, s.L, s.W, s.V) + 256 + Q * s.L * 4
                + Q * 16 + 4096)

    @staticmethod
    def _cost(s: _Set) -> float:
        """Work per query of a set, roughly: N series of L (2W+1) band cells."""
        return float(s.N) * s.L * min(2 * s.W + 1, s.L)

    def _pick(self):
        """The batch to launch: [(set_id, n)] in the order of the sets'
        oldest waiting queries, within max_batch and the memory budget."""
        order = sorted((dq[0].t_arrival, sid) for sid, dq in self.pending.items() if dq)
        take, total, used = [], 0, 0
        first_cost = None
        for _, sid in order:
            room = self.max_batch - total
            if room <= 0:
                break
            s = self.sets[sid]
            cost = self._cost(s)
            if first_cost is None:
                first_cost = cost
            elif not (first_cost / self.mix_ratio <= cost <= first_cost * self.mix_ratio):
                continue   # another cost class: the next free slot

            n = min(len(self.pending[sid]), room)
            while n > 0 and self.in_use + used + self._batch_bytes(s, n) > self.budget:
                n //= 2
            if n == 0:
                break   # the next set in line waits for memory: nobody jumps it
            take.append((sid, n))
            total += n
            used += self._batch_bytes(s, n)
        return take, used

    def _launch(self, slot: int, take, nbytes: int):
        torch = self.torch
        stream = self.streams[slot]
        self.in_use += nbytes
        parts, descs, keep = [], [], []
        with torch.cuda.stream(stream):
            for sid, n in take:
                s = self.sets[sid]
                reqs = [self.pending[sid].popleft() for _ in range(n)]
                host_q = torch.from_numpy(np.stack([r.query for r in reqs])).pin_memory()
                dq = host_q.to(self.dev, non_blocking=True)
                out = (torch.empty(n, dtype=torch.int32, device=self.dev),
                       torch.empty(n, dtype=torch.int32, device=self.dev),
                       torch.empty(n, dtype=torch.float64, device=self.dev))
                descs.append(dict(train=s.train, labels=s.labels, test=dq, W=s.W, V=s.V,
                                  env=s.env, flags=s.flags))
                host_out = tuple(torch.empty(o.shape, dtype=o.dtype, pin_memory=True)
                                 for o in out)
                parts.append((sid, reqs, host_out, out))
                keep += [host_q, dq, *out]
            ws = torch.empty(nndtw.nn_dtw_batch_workspace_size(descs), dtype=torch.uint8,
                             device=self.dev)
            nndtw.nn_dtw_search_batched(descs, workspace=ws, outs=[p[3] for p in parts],
                                        stream=stream)
            for _, _, host_out, out in parts:
                for h, o in zip(host_out, out):
                    h.copy_(o, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        keep.append(ws)
        self.inflight.append(_Batch([(sid, reqs, host_out) for sid, reqs, host_out, _ in parts],
                                    stream, ev, nbytes, time.perf_counter(), keep=keep))
        self.batches += 1
        self.batch_sets += len(take)

    def _retire(self, b: _Batch, slot: int):
        now = time.perf_counter()
        for _, reqs, host_out in b.parts:
            idx, lab, dist = (h.numpy() for h in host_out)
            for k, r in enumerate(reqs):
                r.future.set_result((int(idx[k]), int(lab[k]), float(dist[k])))
                self.latencies.append(now - r.t_arrival)
            self.completed += len(reqs)
        self.t_last = now
        self.in_use -= b.nbytes
        self.free_slots.append(slot)

    def _loop(self):
        try:
            self._run()
        except BaseException as e:  # fail every outstanding request rather than hang
            with self.lock:
                self.running = False
                for b in self.inflight:
                    for _, reqs, _ in b.parts:
                        for r in reqs:
                            if not r.future.done():
                                r.future.set_exception(e)
                self.inflight.clear()
                for dq in self.pending.values():
                    while dq:
                        r = dq.popleft()
                        if not r.future.done():
                            r.future.set_exception(e)
            raise

    def _run(self):
        torch = self.torch
        torch.cuda.set_device(self.dev)
        while self.running or self.inflight or any(self.pending.values()):
            progressed = False
            # cleared before the queues are scanned: a submit() after this
            # point sets it again and ends the wait below at once
            self.wake.clear()
            with self.lock:
                # retire finished batches
                for b in list(self.inflight):
                    if b.event.query():
                        self.inflight.remove(b)
                        self._retire(b, self.streams.index(b.stream))
                        progressed = True
                # admit new batches into free slots
                while self.free_slots:
                    take, nbytes = self._pick()
                    if not take:
                        break
                    self._launch(self.free_slots.pop(), take, nbytes)
                    progressed = True
            if not progressed:
                if self.inflight:
                    time.sleep(5e-5)
                else:
                    self.wake.wait(0.01)
