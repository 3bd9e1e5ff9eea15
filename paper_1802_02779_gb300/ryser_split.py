"""One large matrix by Ryser's formula split over the GPUs of one node.

Ryser's sum (Su & Zheng, arXiv:1802.02779, Section 3.3, Eq. (4); Glynn's
half-size form for complex and 0/1 input) is a sum over Gray codes with no
dependence between ranges of codes, so it shards by code range.  libperm cuts
the codes of an order-n matrix into a fixed number of pieces (perm_ryser_pieces,
a function of n and the element type only).  Here every rank

  1. takes its contiguous, balanced share of the pieces (perm_ryser_split),
  2. computes their partial sums on its own GPU (perm_ryser_partials),
  3. all-gathers the shares in rank order, which is piece order
     (pieces x 32 bytes for complex input: 4 MB at n = 34), and
  4. finishes from the whole array (perm_ryser_finish), which sums the pieces
     in the fixed order perm_batch uses.

So every rank holds the same result, bit-identical to one GPU's perm_batch
with PERM_METHOD_RYSER for any number of ranks.  The all-gather is the one
exchange step; every step of the arithmetic runs in libperm's kernels, and this
module only moves their bytes.
"""
from __future__ import annotations

from typing import Callable, Optional, Sequence

from . import libperm


def shares(pieces: int, world: int) -> Sequence[tuple]:
    """[(begin, end)] of every rank, from perm_ryser_split."""
    return [libperm.ryser_split(pieces, r, world) for r in range(world)]


def gather_in_rank_order(local, sizes: Sequence[int], dist=None, group=None):
    """All-gather 1-D uint8 tensors of per-rank byte sizes `sizes` and return their
    concatenation in rank order (the local tensor alone without a process group)."""
    import torch
    if dist is None or len(sizes) == 1:
        return local
    biggest = max(sizes)
    padded = torch.zeros(biggest, dtype=torch.uint8, device=local.device)
    padded[: local.numel()] = local
    parts = [torch.empty(biggest, dtype=torch.uint8, device=local.device) for _ in sizes]
    dist.all_gather(parts, padded, group=group)
    return torch.cat([p[:s] for p, s in zip(parts, sizes)])


def split_partials(n: int, dtype: str, rank: int, world: int,
                   compute: Callable[[int, int], "torch.Tensor"], dist=None, group=None):
    """Steps 1-3: this rank's share computed by compute(begin, end) (a uint8 tensor of
    (end - begin) * piece bytes), gathered with every other rank's in piece order."""
    pieces, piece_bytes = libperm.ryser_pieces(n, dtype)
    ranges = shares(pieces, world)
    b, e = ranges[rank]
    local = compute(b, e)
    if local.numel() != (e - b) * piece_bytes:
        raise ValueError(f"rank {rank}: {local.numel()} partial-sum bytes for pieces [{b}, {e})")
    full = gather_in_rank_order(local, [(e1 - b1) * piece_bytes for b1, e1 in ranges], dist, group)
    assert full.numel() == pieces * piece_bytes
    return full


def permanent(plan: "libperm.Plan", mat, n: int, dist=None, group=None):
    """The permanent of one order-n device matrix `mat` (a torch tensor of n*n
    elements of the plan's dtype) split over the ranks of `dist` (None: one rank).
    Every rank must call it with the same matrix.  Work runs on the current stream,
    which the all-gather follows.  Returns (out, item_status) device tensors: one
    complex128, or the plan's integer words (int64)."""
    import torch
    rank = dist.get_rank(group) if dist is not None else 0
    world = dist.get_world_size(group) if dist is not None else 1
    _, piece_bytes = libperm.ryser_pieces(n, plan.dtype)

    def compute(b, e):
        buf = torch.empty(max(1, (e - b) * piece_bytes), dtype=torch.uint8, device=mat.device)
        plan.ryser_partials(mat, n, b, e, buf)
        return buf[: (e - b) * piece_bytes]

    full = split_partials(n, plan.dtype, rank, world, compute, dist, group)
    if plan.dtype == "c128":
        out = torch.empty(1, dtype=torch.complex128, device=mat.device)
    else:
        out = torch.empty(plan.describe().get("out_words", 2), dtype=torch.int64, device=mat.device)
    st = torch.empty(1, dtype=torch.int32, device=mat.device)
    plan.ryser_finish(n, full, out, st)
    return out, st
