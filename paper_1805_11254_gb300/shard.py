"""Row sharding of one collection across ranks, one process per GPU.

Sketches are independent per set and decisions independent per (query, row)
pair (Sec. 3.2, Alg. 1-2), so a collection is split into contiguous row
ranges, every rank holds the same query batch and compares it with its own
rows, and the only exchange is the final gather of accepted pairs: each
rank's row indices are made global by adding its range start and the union is
put back in (query, row) order.  The result equals a one-rank run exactly.

Throughput runs with a fixed collection per rank (weak scaling) need none of
the exchange; `max_over_ranks` is their only collective, for timing.

A self-join (every pair i < j of one collection) splits by its blocks of
query rows instead: every rank holds the whole collection, takes the blocks
b = rank, rank + world, ... (hoph_self_join_part), and the one exchange is
again the final gather of pairs, whose row indices are global already.
"""
import numpy as np

from .hoph import PAIR_DTYPE


def row_range(n_rows, rank, world):
    """[r0, r1) of rank `rank` among `world`: contiguous, covering, sizes
    differing by at most one (the first n_rows % world ranks take one more)."""
    if world < 1 or not 0 <= rank < world or n_rows < 0:
        raise ValueError("bad shard request: n_rows=%d rank=%d world=%d" % (n_rows, rank, world))
    base, extra = divmod(n_rows, world)
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def globalize(pairs, r0):
    """Copy of `pairs` (PAIR_DTYPE) with local row indices shifted by r0."""
    out = np.array(pairs, dtype=PAIR_DTYPE, copy=True).reshape(-1)
    out["row"] += r0
    return out


def merge_pairs(chunks):
    """Union of pair arrays in (query, row) order, the order hoph_query_batch
    emits within one call."""
    chunks = [np.asarray(c, dtype=PAIR_DTYPE).reshape(-1) for c in chunks]
    if not chunks:
        return np.empty(0, dtype=PAIR_DTYPE)
    allp = np.concatenate(chunks)
    return allp[np.lexsort((allp["row"], allp["query"]))]


def gather_pairs(local_pairs, r0, group=None, dst=None):
    """The exchange: every rank's pairs, made global, to every rank (dst None)
    or to rank dst only (others get None)."""
    import torch.distributed as dist
    mine = globalize(local_pairs, r0).tobytes()
    world = dist.get_world_size(group)
    if dst is None:
        parts = [None] * world
        dist.all_gather_object(parts, mine, group=group)
    else:
        parts = [None] * world if dist.get_rank(group) == dst else None
        dist.gather_object(mine, parts, dst=dst, group=group)
        if parts is None:
            return None
    return merge_pairs([np.frombuffer(p, dtype=PAIR_DTYPE) for p in parts])


def sharded_query(local_query, n_rows, group=None, dst=None):
    """Compare the query batch with this rank's rows and gather the accepted
    pairs.  local_query(r0, r1) returns the pairs (PAIR_DTYPE, rows local to
    r0) of the rows [r0, r1) this rank holds."""
    import torch.distributed as dist
    r0, r1 = row_range(n_rows, dist.get_rank(group), dist.get_world_size(group))
    return gather_pairs(local_query(r0, r1), r0, group, dst)


def self_join_blocks(n_rows, batch, part, parts):
    """The blocks of a self-join over n_rows rows in blocks of `batch` query
    rows that part `part` of `parts` runs (hoph_self_join_part's split): block b
    holds queries b*batch .. b*batch+batch-1 against the rows from b*batch on."""
    if parts < 1 or not 0 <= part < parts or batch < 1 or n_rows < 0:
        raise ValueError("bad self-join split: n_rows=%d batch=%d part=%d parts=%d"
                         % (n_rows, batch, part, parts))
    n_blocks = (n_rows - 1 + batch - 1) // batch if n_rows > 1 else 0
    return list(range(part, n_blocks, parts))


def sharded_self_join(local_self_join, group=None, dst=None):
    """This rank's part of a self-join and the gather of every part's pairs.
    local_self_join(part, parts) returns the pairs (PAIR_DTYPE, global rows) of
    the blocks self_join_blocks(..., part, parts)."""
    import torch.distributed as dist
    mine = local_self_join(dist.get_rank(group), dist.get_world_size(group))
    return gather_pairs(mine, 0, group, dst)


def gpu_local_self_join(plan, mode, planes, n_rows, batch=1536, capacity=1 << 16, stream=None):
    """local_self_join for sharded_self_join on this rank's GPU: `planes` holds
    the whole collection ([G][n_rows][k'], uint32 or compact uint16)."""
    def run(part, parts):
        cap = capacity
        while True:
            pairs, count, _ = plan.self_join(mode, planes, n_rows, batch, cap, stream,
                                             part=part, parts=parts)
            if count <= cap:
                return pairs
            cap = count
    return run


def gpu_local_query(plan, mode, q_planes, n_queries, local_planes, capacity=1 << 16, stream=None):
    """local_query for sharded_query on this rank's GPU: local_planes holds
    the sketches of rows [r0, r1) only ([G][r1 - r0][k'])."""
    def run(r0, r1):
        n = r1 - r0
        cap = capacity
        while True:
            pairs, count, _ = plan.query(mode, q_planes, n_queries, local_planes, n, cap, stream)
            if count <= cap:
                return pairs
            cap = count
    return run


def max_over_ranks(x, group=None, device="cpu"):
    """Max of a host float over the ranks (timing: the slowest rank sets the
    job's time)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
