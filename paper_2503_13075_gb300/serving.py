"""Serving loop for constraint-solve requests (orchestration only; all arithmetic runs
in the library's kernels).

A request carries one molecule topology (constrained atom pairs) and its coordinates
(x_old, x_unc, inverse masses, target distances).  The engine

* keeps set-up topologies (programs, schedules, workspaces) resident on the device in an
  LRU cache bounded by an HBM budget; a topology is planned and uploaded on its first
  request (``ilves_setup_topology``) and reused afterwards,
* admits a request only if its topology and its input/output footprint fit the budget
  (otherwise it is rejected with a reason, never queued forever),
* dispatches requests continuously: the requests that have arrived go out together once
  the oldest has waited ``max_wait_s`` (0: on arrival) or ``max_batch`` are waiting, with
  at most ``max_batch`` in flight; their solves are enqueued back to back on a pool of
  CUDA streams, one stream per topology so that solves sharing a topology's workspace stay
  ordered, and each request completes on its own (its stream's event is polled), without
  waiting for the others.  A request's batched kernel launches only the CTAs that own its
  molecules (with the shared memory they use), so solves run side by side on disjoint SMs
  rather than one after another; requests above the partition threshold are solved by
  overlapping domains.  Each ilves_solve reads the request's page-locked host inputs and
  writes its page-locked host outputs in place (no staging copies) and computes the
  diagonal start itself,
* records per-request latency (arrival -> results on the host), iterations and status;
  ``max_relative_violation`` reports the accuracy of returned positions.
"""
from __future__ import annotations

import collections
import hashlib
import time
from dataclasses import dataclass, field

import numpy as np


def topology_key(n_atoms, atom_i, atom_j):
    h = hashlib.sha1()
    h.update(np.int64(n_atoms).tobytes())
    h.update(np.ascontiguousarray(atom_i, np.int32).tobytes())
    h.update(np.ascontiguousarray(atom_j, np.int32).tobytes())
    return h.hexdigest()


def max_relative_violation(x, atom_i, atom_j, d):
    """Host-side accuracy report of returned positions: max_k |(|x_i - x_j|^2 - d_k^2)| / d_k^2."""
    r = x[atom_i] - x[atom_j]
    return float(np.max(np.abs(np.einsum("ij,ij->i", r, r) - d * d) / (d * d))) if len(d) else 0.0


@dataclass
class Request:
    rid: int
    arrival: float  # seconds on the engine clock
    n_atoms: int
    atom_i: np.ndarray
    atom_j: np.ndarray
    x_old: np.ndarray
    x_unc: np.ndarray
    inv_mass: np.ndarray
    d: np.ndarray
    key: str = ""
    host: list = None  # pinned host tensors: x_old, x_unc, inv_mass, d, and result buffers
    # results
    done: float = -1.0
    status: str = "pending"
    x: np.ndarray = None
    iterations: np.ndarray = None
    mol_status: np.ndarray = None

    def io_bytes(self):
        return 8 * (3 * self.n_atoms * 3 + self.n_atoms + 2 * len(self.d)) + 4 * len(self.d)


class TopologyCache:
    """LRU cache of device-resident topologies under a byte budget (host logic only)."""

    def __init__(self, budget_bytes, make_topology, size_of):
        self.budget = int(budget_bytes)
        self.make = make_topology
        self.size_of = size_of
        self.entries = collections.OrderedDict()  # key -> (topology, bytes)
        self.used = 0
        self.hits = self.misses = self.evictions = 0

    def get(self, key, factory_args, reserve=0):
        """Topology for `key`, creating (and evicting LRU entries) as needed.

        Returns None when the topology plus `reserve` bytes cannot fit the budget even
        after evicting everything not in use."""
        if key in self.entries:
            self.entries.move_to_end(key)
            self.hits += 1
            return self.entries[key][0]
        self.misses += 1
        topo = self.make(*factory_args)
        nbytes = int(self.size_of(topo))
        if nbytes + reserve > self.budget:
            return None
        while self.used + nbytes + reserve > self.budget and self.entries:
            _, (old, ob) = self.entries.popitem(last=False)
            self.used -= ob
            self.evictions += 1
            if hasattr(old, "close"):
                old.close()
        self.entries[key] = (topo, nbytes)
        self.used += nbytes
        return topo


@dataclass
class ServingStats:
    latencies: list = field(default_factory=list)
    rejected: int = 0
    completed: int = 0
    atoms: int = 0
    batches: int = 0
    max_violation: float = 0.0
    iterations: list = field(default_factory=list)


class Engine:
    """Dynamic-batching solve engine on one GPU."""

    def __init__(self, hbm_budget_bytes=8 << 30, n_streams=8, max_batch=64, max_wait_s=0.002,
                 precision="mixed", warm_start="diag", tol=1e-12, device="cuda:0", overlap=2):
        import torch

        from . import binding as B

        self.B = B
        self.torch = torch
        self.dev = torch.device(device)
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(n_streams)]
        self.max_batch = max_batch
        self.max_wait_s = max_wait_s
        self.precision = precision
        self.warm_start = warm_start
        self.tol = tol
        self.budget = hbm_budget_bytes
        self.cache = TopologyCache(hbm_budget_bytes, lambda n, i, j: B.Topology(n, i, j, overlap=overlap),
                                   lambda t: t.device_bytes())
        self.stats = ServingStats()
        self.t0 = time.perf_counter()

    def now(self):
        return time.perf_counter() - self.t0

    def prewarm(self, systems):
        """Plan and upload the topologies of a known pool before serving."""
        for sys_ in systems:
            key = topology_key(sys_.n_atoms, sys_.atom_i, sys_.atom_j)
            self.cache.get(key, (sys_.n_atoms, sys_.atom_i, sys_.atom_j))
        self.cache.hits = self.cache.misses = 0

    def pin(self, req):
        """Pinned host buffers of a request (done when the request is created): inputs
        x_old, x_unc, inv_mass, d; outputs x, iterations, status, lambda."""
        torch = self.torch
        req.host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
                    for a in (req.x_old, req.x_unc, req.inv_mass, req.d)]
        n_mol_max = max(1, len(req.d))
        req.host += [torch.empty(req.n_atoms, 3, dtype=torch.float64).pin_memory(),
                     torch.empty(n_mol_max, dtype=torch.int32).pin_memory(),
                     torch.empty(n_mol_max, dtype=torch.int32).pin_memory(),
                     torch.empty(max(1, len(req.d)), dtype=torch.float64).pin_memory()]

    def _launch(self, batch):
        """Enqueues the solves of `batch`; returns (request, event, outputs) per admitted request."""
        torch = self.torch
        jobs = []
        for req in batch:
            topo = self.cache.get(req.key, (req.n_atoms, req.atom_i, req.atom_j), reserve=req.io_bytes())
            if topo is None:
                req.status = "rejected: topology and buffers exceed the HBM budget"
                self.stats.rejected += 1
                continue
            # one stream per topology: solves of one topology share its workspace and must be
            # stream-ordered; different topologies overlap on different streams
            s = self.streams[int(req.key[:8], 16) % len(self.streams)]
            # the kernels read the request's pinned inputs and write its pinned outputs in
            # place (no staging copies); the diagonal start is computed inside the solve
            hx, hi, hs = req.host[4], req.host[5][: topo.n_molecules], req.host[6][: topo.n_molecules]
            hl = req.host[7][: topo.n_constraints]
            topo.solve(*req.host[:4], tol=self.tol, precision=self.precision, x_out=hx, lambda_out=hl,
                       iterations_out=hi, status_out=hs, stream=s,
                       start="diag" if self.warm_start == "diag" else None)
            ev = torch.cuda.Event()
            ev.record(s)
            jobs.append((req, ev, hx, hi, hs))
        return jobs

    def _finish(self, job):
        req, ev, hx, hi, hs = job
        req.done = self.now()
        req.x, req.iterations, req.mol_status = hx.numpy().copy(), hi.numpy().copy(), hs.numpy().copy()
        req.status = "ok" if np.all(req.mol_status == 0) else "not converged"
        self.stats.latencies.append(req.done - req.arrival)
        self.stats.completed += 1
        self.stats.atoms += req.n_atoms
        self.stats.iterations.extend(req.iterations.tolist())

    def serve(self, requests):
        """Serve requests (sorted by arrival time, engine clock) in real time."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        inflight = []
        self.t0 = time.perf_counter()
        while pending or inflight:
            now = self.now()
            ready = 0
            while ready < len(pending) and pending[ready].arrival <= now:
                ready += 1
            room = self.max_batch - len(inflight)
            if ready and room > 0 and (now - pending[0].arrival >= self.max_wait_s or ready >= self.max_batch):
                inflight += self._launch([pending.popleft() for _ in range(min(ready, room))])
                self.stats.batches += 1
                continue
            done, still = [], []
            for job in inflight:
                (done if job[1].query() else still).append(job)
            if done:
                for job in done:
                    self._finish(job)
                inflight = still
                continue
            if not inflight and pending:  # idle: sleep until the next request can go out
                wait = pending[0].arrival + (self.max_wait_s if ready else 0.0) - self.now()
                if wait > 2e-4:
                    time.sleep(wait - 1e-4)
        return self.stats


def make_requests(n_req, rate_hz, seed, n_topologies=32, lo=20, hi=50_000, warm_pool=True):
    """Poisson arrivals; each request picks a molecule of a pool of topologies whose sizes
    are log-uniform in [lo, hi] atoms (tree generator), with fresh coordinates."""
    from . import workloads as wl

    rng = np.random.default_rng(seed)
    sizes = wl.serving_sizes(n_topologies, seed=seed, lo=lo, hi=hi)
    pool = []
    for k, n in enumerate(sizes):
        s = wl.tree_molecules_of_sizes([int(n)], seed=seed * 1000 + k)
        pool.append(s)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n_req))
    reqs = []
    for r in range(n_req):
        s = pool[int(rng.integers(len(pool)))]
        x_unc = s.x_old + rng.normal(0.0, 0.003, size=s.x_old.shape)
        req = Request(r, float(t[r]), s.n_atoms, s.atom_i, s.atom_j, s.x_old, np.ascontiguousarray(x_unc),
                      s.inv_mass, s.d)
        req.key = topology_key(s.n_atoms, s.atom_i, s.atom_j)
        reqs.append(req)
    return reqs, pool
