"""A particle-sharded filter: the host side of the exchange between shards.

Algorithm 1's loops over particles are independent (the paper's
particle-parallel layout, Sec. 3.1), so one filter of N particles can be split
into G contiguous shards, one per GPU.  Each epoch the shards share only what
couples the particles:

* Step 3a: the maximum of the log fitness weights (a max-reduce) and the tile
  totals of the cumulative weights (a gather in slot order);
* Steps 3b-3c: every resampled slot's parent may live on another shard.  The
  outputs whose parent a shard holds form one contiguous range of slots
  (both the thresholds tau_i and the cumulative weights increase), so each
  shard resamples its range and sends each parent's record to the shard that
  holds the output's slot (an all-to-all);
* Steps 5-6: the maximum of the new log weights and the moment sums (added in
  shard order, so every shard commits the same moments).

`ShardedFilter` runs that protocol for one shard (one process or thread per
shard) over a `Comm` (collectives) and an engine that runs the phases on the
shard's particles.  `LibraryShard` is the engine of the CUDA library
(pf_shard_* calls); the collectives are `TorchComm` (torch.distributed: NCCL
between GPUs, gloo on CPU) or `ThreadComm` (several shards driven by threads
of one process, e.g. on one GPU).  This module holds none of the method's
arithmetic on particles: it only plans the output ranges and moves data.
"""
from __future__ import annotations

import threading

import numpy as np


# ------------------------------------------------------------------ planning
def shard_bounds(N: int, G: int, tile: int) -> list:
    """G + 1 slot boundaries 0 = b_0 < ... < b_G = N, interior ones multiples
    of the scan tile, the tiles spread as evenly as possible."""
    nt = (N + tile - 1) // tile
    if G < 1 or G > nt:
        raise ValueError(f"need 1 <= G <= {nt} shards for N = {N}")
    out = [min(N, (q * nt // G) * tile) for q in range(G)] + [N]
    out[0] = 0
    return out


def threshold(i: int, u: float, N: int, total: float) -> float:
    """tau_i = ((i + u) / N) c_{N-1}, in exactly this order of operations
    (the library's and the oracle's)."""
    return (float(i) + u) / float(N) * total


def count_below(b: float, u: float, N: int, total: float) -> int:
    """Number of outputs i in [0, N) with tau_i < b (tau increases with i)."""
    lo, hi = 0, N
    while lo < hi:
        mid = (lo + hi) // 2
        if threshold(mid, u, N, total) < b:
            lo = mid + 1
        else:
            hi = mid
    return lo


def plan_ranges(bounds, tile, tile_end, total, u):
    """The outputs each shard resamples.  With l_i = min{k : c_k > tau_i},
    l_i lies in shard q's slots [b_q, b_{q+1}) exactly when
    c_{b_q - 1} <= tau_i < c_{b_{q+1} - 1}; the outputs whose threshold
    reaches the total, tau_i >= c_{N-1}, take the first k with c_k = c_{N-1},
    which lies in the first shard whose last value is the total.  Returns the
    per-shard [i_lo, i_hi) and i_fb = #{i : tau_i < c_{N-1}}."""
    G = len(bounds) - 1
    N = bounds[-1]
    cend = [total if q == G - 1 else float(tile_end[bounds[q + 1] // tile - 1]) for q in range(G)]
    qstar = next(q for q in range(G) if cend[q] == total)
    i_fb = count_below(total, u, N, total)
    ranges = []
    for q in range(G):
        if q > qstar:
            ranges.append((N, N))
            continue
        lo = 0 if q == 0 else count_below(cend[q - 1], u, N, total)
        hi = N if q == qstar else count_below(cend[q], u, N, total)
        ranges.append((lo, hi))
    return ranges, i_fb


def exchange_counts(ranges, bounds, me):
    """Records shard `me` sends to every shard (its range cut at their slot
    boundaries) and receives from every shard (their ranges cut at its own)."""
    G = len(bounds) - 1
    lo, hi = ranges[me]
    send = [max(0, min(hi, bounds[r + 1]) - max(lo, bounds[r])) for r in range(G)]
    recv = [max(0, min(ranges[q][1], bounds[me + 1]) - max(ranges[q][0], bounds[me]))
            for q in range(G)]
    return send, recv


# --------------------------------------------------------------- collectives
class TorchComm:
    """Collectives over a torch.distributed process group (NCCL between GPUs,
    gloo on CPU).  Scalars and gathers travel as float64 tensors on `device`;
    the record exchange is one all_to_all_single."""

    def __init__(self, group=None, device="cpu"):
        import torch.distributed as dist
        self.dist, self.group, self.device = dist, group, device
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)

    def _t(self, a):
        import torch
        return torch.as_tensor(np.asarray(a, dtype=np.float64), device=self.device)

    def max(self, x: float) -> float:
        t = self._t([x])
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return float(t.cpu()[0])

    def gather(self, a) -> list:
        """Every rank's 1-D array (lengths may differ), in rank order."""
        import torch
        a = np.asarray(a, dtype=np.float64)
        n = self._t([len(a)])
        ns = [torch.zeros_like(n) for _ in range(self.size)]
        self.dist.all_gather(ns, n, group=self.group)
        lens = [int(v.cpu()[0]) for v in ns]
        m = max(lens)
        pad = np.zeros(m)
        pad[:len(a)] = a
        t = self._t(pad)
        outs = [torch.zeros_like(t) for _ in range(self.size)]
        self.dist.all_gather(outs, t, group=self.group)
        return [o.cpu().numpy()[:k].copy() for o, k in zip(outs, lens)]

    def alltoallv(self, send, send_counts, recv, recv_counts, rec):
        """send/recv: float64 tensors (on the group's device), or NumPy
        arrays for a CPU group (shared with the tensors the exchange uses),
        of records of `rec` doubles; counts in records per rank."""
        import torch
        if isinstance(send, np.ndarray):
            send = torch.from_numpy(np.ascontiguousarray(send))
        if isinstance(recv, np.ndarray):
            recv = torch.from_numpy(recv)
        self.dist.all_to_all_single(recv, send, [c * rec for c in recv_counts],
                                    [c * rec for c in send_counts], group=self.group)
        if recv.is_cuda:
            # the receiver's next kernel runs on its filter's own stream
            torch.cuda.current_stream(recv.device).synchronize()


class ThreadComm:
    """Collectives among `size` threads of one process (several shards driven
    side by side, e.g. on one GPU).  Every thread calls each collective in the
    same order; a barrier separates writing the mailbox from reading it."""

    def __init__(self, size: int, timeout: float = 600.0):
        self.size = size
        # a thread that fails calls abort(), so the others leave their wait
        self._bar = threading.Barrier(size, timeout=timeout)
        self._box = [None] * size

    def abort(self):
        self._bar.abort()

    def view(self, rank):
        return _ThreadRank(self, rank)


class _ThreadRank:
    def __init__(self, hub, rank):
        self.hub, self.rank, self.size = hub, rank, hub.size

    def _share(self, obj):
        h = self.hub
        h._bar.wait()
        h._box[self.rank] = obj
        h._bar.wait()
        out = list(h._box)
        h._bar.wait()
        return out

    def max(self, x: float) -> float:
        return max(self._share(float(x)))

    def gather(self, a) -> list:
        return [np.array(v, dtype=np.float64) for v in self._share(np.asarray(a, dtype=np.float64))]

    def alltoallv(self, send, send_counts, recv, recv_counts, rec):
        """Each rank copies its chunks out of every sender's buffer (torch
        tensors on one device, or NumPy arrays)."""
        boxes = self._share((send, list(send_counts)))
        off_in = 0
        for q, (buf, counts) in enumerate(boxes):
            start = sum(counts[:self.rank]) * rec
            n = counts[self.rank] * rec
            assert n == recv_counts[q] * rec
            if n:
                recv[off_in:off_in + n] = buf[start:start + n]
            off_in += n
        if hasattr(recv, "device") and getattr(recv.device, "type", "cpu") == "cuda":
            import torch
            torch.cuda.current_stream(recv.device).synchronize()
        self._share(None)   # every copy out of the send buffers is done


# -------------------------------------------------------------------- engine
class LibraryShard:
    """One shard on the CUDA library (pf_shard_* calls), its record buffers
    CUDA tensors sized for the worst case (every output's parent here)."""

    def __init__(self, pf, w, n_all, first, n, stream=None, device="cuda", filter_id=0, seed=None):
        import torch
        self.f = pf.Filter.from_workload(w, N=n, stream=stream, shard=(n_all, first),
                                         filter_id=filter_id, seed=seed)
        self.info = self.f.pf_shard_info()
        rec = self.info["record"]
        self.send = torch.zeros(n_all * rec, dtype=torch.float64, device=device)
        self.recv = torch.zeros(n * rec, dtype=torch.float64, device=device)
        self.torch = torch

    def stage1(self, t, y):
        return self.f.pf_shard_stage1(t, y)

    def scan(self, lg_max):
        return self.f.pf_shard_scan(lg_max, self.info["tiles"])

    def offsets(self, tiles_all, cl_last):
        return self.f.pf_shard_offsets(tiles_all, cl_last)

    def resample(self, i_lo, i_hi, i_fb, u, total):
        self.f.pf_shard_resample(i_lo, i_hi, i_fb, u, total, self.send.data_ptr())
        return self.send

    def stage2(self):
        return self.f.pf_shard_stage2(self.recv.data_ptr())

    def moments(self, lw_max):
        return self.f.pf_shard_moments(lw_max)

    def commit(self, sums):
        self.f.pf_shard_commit(sums)

    def abort(self):
        self.f.pf_shard_abort()

    def close(self):
        self.f.close()


class DegenerateEpoch(RuntimeError):
    """Every weight of the epoch is zero over the whole ensemble; nothing was
    committed."""


class ShardedFilter:
    """The protocol for one shard.  `engine` runs the phases on its particles
    (LibraryShard, or a stand-in with the same methods), `comm` the
    collectives; `bounds` are the shard boundaries (shard_bounds)."""

    def __init__(self, engine, comm, bounds, tile):
        self.e, self.comm, self.bounds, self.tile = engine, comm, list(bounds), int(tile)
        self.N = self.bounds[-1]
        self.rec = engine.info["record"]
        self._commit(0.0)                       # Step 1's moments

    def _commit(self, lw_max):
        sums = self.comm.gather(self.e.moments(lw_max))
        total = sums[0].copy()
        for s in sums[1:]:
            total = total + s                   # shard order, the same on every shard
        self.e.commit(total)

    def assimilate(self, t, y):
        """One epoch (Steps 2-6) of the whole filter on this shard's slots."""
        e, comm = self.e, self.comm
        M = comm.max(e.stage1(t, y))
        if not np.isfinite(M):
            e.abort()
            raise DegenerateEpoch("every first-stage weight is zero")
        tiles, cl_last = e.scan(M)
        parts = comm.gather(np.concatenate([tiles, [cl_last]]))
        tiles_all = np.concatenate([p[:-1] for p in parts])
        tile_end, total, u = e.offsets(tiles_all, parts[-1][-1])
        ranges, i_fb = plan_ranges(self.bounds, self.tile, tile_end, total, u)
        lo, hi = ranges[comm.rank]
        send = e.resample(lo, hi, i_fb, u, total)
        sc, rc = exchange_counts(ranges, self.bounds, comm.rank)
        comm.alltoallv(send[:(hi - lo) * self.rec], sc, e.recv, rc, self.rec)
        LW = comm.max(e.stage2())
        if not np.isfinite(LW):
            e.abort()
            raise DegenerateEpoch("every new weight is zero")
        self._commit(LW)
        return ranges
