"""Multi-rank plumbing (one process per GPU).

A batch of independent matrices shards with no data-path collective: each rank
takes a share of the matrices chosen by longest-processing-time order on the n^3
cost and sweeps it with its own launch; only timings (and, if wanted, the
per-matrix results) are combined.

A single matrix shards only with a per-step broadcast of the pivot row: the
row-block condensation of Sec. 2.1 / Fig. 6 (`logdet_rowblock`). Each rank owns
a contiguous block of rows; ranks take turns to factor their next row as the
pivot row (the arbitrary pivot row k of Eq. (2)), broadcast it, and every rank
applies the step to its remaining rows; the last row of every rank is gathered
and the small world x world matrix finished on rank 0.
"""
from __future__ import annotations

import heapq
import math

import torch
import torch.distributed as dist


def lpt_partition(sizes, world: int):
    """Indices of a batch split over `world` ranks, balancing sum(n^3):
    largest first, each to the currently lightest rank. Deterministic."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]) ** 3, i))
    heap = [(0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + int(sizes[i]) ** 3, r))
    return [sorted(p) for p in parts]


def world_info():
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def max_over_ranks(x: float, device=None) -> float:
    """Largest value of x over all ranks (the job's time is its slowest rank's)."""
    _, world = world_info()
    if world == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])


def sum_over_ranks(x: float, device=None) -> float:
    _, world = world_info()
    if world == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t[0])


def gather_results(indices, values, count: int, device=None):
    """Scatter each rank's (indices, values) into one length-`count` FP64 tensor
    on every rank (the only exchange, after the timed work)."""
    out = torch.zeros(count, dtype=torch.float64, device=device)
    if len(indices):
        out[torch.as_tensor(indices, dtype=torch.long, device=device)] = torch.as_tensor(
            values, dtype=torch.float64, device=device)
    _, world = world_info()
    if world > 1:
        dist.all_reduce(out, op=dist.ReduceOp.SUM)
    return out


def logdet_batched_distributed(sizes, get_matrix, mode="f32_plain", compute=None, device=None):
    """sign and log|det| of a batch of independent matrices sharded over the ranks.

    Every rank passes the whole batch's `sizes`; `get_matrix(i)` returns matrix i
    on this rank's device and is called only for this rank's share (longest
    processing time first on the n^3 cost, `lpt_partition`). Each rank sweeps its
    share in one ld_logdet_batched call (`compute(mats, mode)` replaces that call,
    e.g. in host-only tests); the (sign, log|det|) pairs are then combined once,
    so every rank returns both full FP64 vectors (length len(sizes)) in batch
    order. No collective runs inside the sweep.
    """
    rank, world = world_info()
    mine = lpt_partition(sizes, world)[rank]
    if compute is None:
        from . import api

        def compute(mats, mode):
            s, l = api.logdet_batched(api.BatchedInputs(mats), mode)
            return s, l
    if mine:
        signs, logabs = compute([get_matrix(i) for i in mine], mode)
        signs = torch.as_tensor(signs, dtype=torch.float64).to(device).tolist()
        logabs = torch.as_tensor(logabs, dtype=torch.float64).to(device).tolist()
    else:
        signs, logabs = [], []
    return (gather_results(mine, signs, len(sizes), device=device),
            gather_results(mine, logabs, len(sizes), device=device))


# ---------------------------------------------------------------------------
# Row-block condensation (Sec. 2.1, Fig. 6)


def rowblock_counts(n: int, world: int):
    """Rows per rank of the block distribution (Fig. 1, left): contiguous blocks
    of near-equal size, the first n mod world ranks one row more. Every rank must
    own a row (n >= world)."""
    if world < 1 or n < world:
        raise ValueError(f"row-block condensation needs n >= world >= 1 (n={n}, world={world})")
    q, r = divmod(n, world)
    return [q + (1 if p < r else 0) for p in range(world)]


def rowblock_schedule(counts):
    """(rank, local row) of every condensation step (Fig. 6 loops): for each local
    row index i, the ranks in turn pivot on their row i, as long as it is not
    their last row. len = sum(counts) - len(counts)."""
    return [(p, i) for i in range(max(counts) - 1) for p, c in enumerate(counts) if i < c - 1]


def step_sign(pivot: float, k: int, l: int, m: int) -> float:
    """Sign factor of one step on an m x m active matrix with pivot row k (its
    position among the active rows) and pivot column position l, the pivot
    column's slot refilled from position m-1 (Sec. 2.4): sgn(p) (-1)^(k+l) from
    the Laplace expansion of Eq. (2), times (-1)^(m-2-l) for moving column m-1
    to position l (no move when l = m-1)."""
    s = -1.0 if pivot < 0 else 1.0
    e = k + (m - 2 if l != m - 1 else l)
    return -s if e & 1 else s


class DeviceSteps:
    """The two halves of a step and the final small sweep on this process's GPU
    (ld_rowblock_factor / ld_rowblock_update / ld_logdet)."""

    def __init__(self, dtype: torch.dtype, stream=None):
        from . import _lib
        if dtype not in (torch.float64, torch.float32):
            raise TypeError("row-block condensation stores FP64 or FP32")
        self._lib = _lib
        self.dtype = dtype
        self.code = _lib.LD_DTYPE_F64 if dtype == torch.float64 else _lib.LD_DTYPE_F32
        self.mode = "f64_plain" if dtype == torch.float64 else "f32_plain"
        self.stream = stream

    def _s(self):
        s = torch.cuda.current_stream() if self.stream is None else self.stream
        return s.cuda_stream

    def factor(self, row, labels, m, step):
        self._lib.check("ld_rowblock_factor", self._lib.ld_rowblock_factor(
            row.data_ptr(), self.code, labels.data_ptr(), m, step.data_ptr(), self._s()))

    def update(self, F, rows, m, r, labels, step):
        self._lib.check("ld_rowblock_update", self._lib.ld_rowblock_update(
            F.data_ptr() if rows > 0 else 0, self.code, rows, F.stride(0), m, r.data_ptr(),
            labels.data_ptr(), step.data_ptr(), self._s()))

    def small(self, M):
        from . import api
        return api.logdet(M.contiguous(), self.mode, stream=self.stream)


class _Emulated:
    """All ranks' blocks in one process; the broadcast and the gather are the
    shared buffer itself (no collective)."""

    def __init__(self, world):
        self.world = world

    def local(self):
        return range(self.world)

    def broadcast(self, buf, src):
        pass

    def gather_rows(self, rows_by_rank):
        return torch.stack([rows_by_rank[p] for p in range(self.world)])

    def share(self, x):
        return x


class _Distributed:
    def __init__(self, rank, world):
        self.rank, self.world = rank, world

    def local(self):
        return (self.rank,)

    def broadcast(self, buf, src):
        dist.broadcast(buf, src=src)

    def gather_rows(self, rows_by_rank):
        mine = rows_by_rank[self.rank].contiguous()
        out = [torch.empty_like(mine) for _ in range(self.world)]
        dist.all_gather(out, mine)
        return torch.stack(out)

    def share(self, x):
        dist.broadcast(x, src=0)
        return x


def _neumaier(values):
    s = c = 0.0
    for v in values:
        t = s + v
        c += (s - t) + v if abs(s) >= abs(v) else (v - t) + s
        s = t
    return s + c


def _rowblock(blocks, counts, n, comm, steps):
    """Fig. 6 on the blocks this process holds (blocks[p] = rank p's rows, shape
    counts[p] x n, modified in place). Returns (sign, log|det|, pivot labels,
    pivot values) on every process."""
    world = len(counts)
    local = list(comm.local())
    ref = blocks[local[0]]
    dev, dt = ref.device, ref.dtype
    es = ref.element_size()
    # one packed buffer per broadcast: 4 FP64 step fields, then the pivot row
    buf = torch.zeros(32 + n * es, dtype=torch.uint8, device=dev)
    step = buf[:32].view(torch.float64)
    row = buf[32:].view(dt)
    labels = {p: torch.arange(n, dtype=torch.int32, device=dev) for p in local}
    sched = rowblock_schedule(counts)
    rec = torch.zeros((len(sched), 4), dtype=torch.float64, device=dev)
    consumed = [0] * world
    ks, ms = [], []
    m = n
    for s, (p, i) in enumerate(sched):
        k = sum(counts[q] - consumed[q] for q in range(p))  # first remaining row of rank p
        if p in blocks and p in local:
            row[:m].copy_(blocks[p][i, :m])
            steps.factor(row, labels[p], m, step)
        comm.broadcast(buf, p)
        consumed[p] += 1
        for q in local:
            F = blocks[q][consumed[q]:]
            steps.update(F, F.shape[0], m, row, labels[q], step)
        rec[s].copy_(step)
        ks.append(k)
        ms.append(m)
        m -= 1
    last = {q: blocks[q][counts[q] - 1, :m] for q in local}
    final = comm.gather_rows(last)
    res = torch.zeros(2, dtype=torch.float64, device=dev)
    if 0 in local:
        fs, fl = steps.small(final)
        res[0], res[1] = float(fs), float(fl)
    res = comm.share(res)
    r = rec.cpu()
    status = r[:, 2]
    labels_seq = [int(x) for x in r[:, 3]]
    pivots = [float(x) for x in r[:, 1]]
    if bool((status == 2).any()):
        return math.nan, math.nan, labels_seq, pivots
    if bool((status == 1).any()):
        return 0.0, -math.inf, labels_seq, pivots
    sign = float(res[0])
    for s in range(len(sched)):
        sign *= step_sign(pivots[s], ks[s], int(r[s, 0]), ms[s])
    logabs = _neumaier([math.log(abs(v)) for v in pivots] + [float(res[1])])
    if sign == 0.0:
        logabs = -math.inf
    return sign, logabs, labels_seq, pivots


def logdet_rowblock(A_local, n: int, steps=None):
    """sign(det A) and log|det A| by row-block condensation over the ranks
    (Sec. 2.1, Fig. 6).

    A_local: this rank's contiguous block of rows of A, shape
    rowblock_counts(n, world)[rank] x n (row-major, FP64 or FP32, on this rank's
    device; overwritten). Ranks pivot on their rows in turn (rowblock_schedule),
    the factored pivot row and its column travel in one broadcast per step, and
    the world x world matrix of every rank's last row is finished on rank 0 with
    the plain sweep. `steps` replaces the device steps (DeviceSteps), e.g. with
    a host stand-in in CPU tests. Returns (sign, log|det|, pivot labels, pivot
    values) on every rank.
    """
    rank, world = world_info()
    counts = rowblock_counts(n, world)
    if tuple(A_local.shape) != (counts[rank], n):
        raise ValueError(f"rank {rank} holds {tuple(A_local.shape)}, expected {(counts[rank], n)}")
    if steps is None:
        steps = DeviceSteps(A_local.dtype)
    comm = _Distributed(rank, world) if world > 1 else _Emulated(1)
    return _rowblock({rank: A_local}, counts, n, comm, steps)


def logdet_rowblock_emulated(A, world: int, steps=None):
    """The row-block condensation of `logdet_rowblock` with all `world` ranks'
    blocks held by this process (one device): the same steps in the same order,
    the broadcast being the shared buffer. A is copied, not modified."""
    n = A.shape[0]
    counts = rowblock_counts(n, world)
    starts = [sum(counts[:p]) for p in range(world)]
    blocks = {p: A[starts[p]:starts[p] + counts[p]].clone() for p in range(world)}
    if steps is None:
        steps = DeviceSteps(A.dtype)
    return _rowblock(blocks, counts, n, _Emulated(world), steps)
