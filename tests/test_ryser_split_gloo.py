"""Bookkeeping of one matrix's Ryser code range split over ranks, on CPU.

The split (perm_ryser_split) must partition the pieces into contiguous,
balanced shares, and the all-gather must put every rank's partial sums back in
piece order, so that the finishing kernel sees the same array for every number
of ranks.  Here two and three gloo ranks gather stand-in partial sums (bytes
that name their piece), and the gathered array is compared with the one-rank
array byte for byte.  perm_ryser_pieces and perm_ryser_split are host-only C
functions; no GPU is used."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


@pytest.fixture(scope="module")
def lp():
    from paper_1802_02779_gb300 import build
    build.build()
    from paper_1802_02779_gb300 import libperm
    libperm.load()
    return libperm


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _stand_in(b, e, piece_bytes):
    """Bytes of pieces [b, e): byte k of piece p is a hash of (p, k)."""
    p = np.arange(b, e, dtype=np.uint64)[:, None]
    k = np.arange(piece_bytes, dtype=np.uint64)[None, :]
    v = ((p * np.uint64(2654435761) + k * np.uint64(40503) + np.uint64(7)) >> np.uint64(3)) & np.uint64(0xFF)
    return torch.from_numpy(v.astype(np.uint8).reshape(-1))


CASES = [(34, "c128"), (24, "c128"), (30, "u01"), (12, "u01"), (22, "i64")]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1802_02779_gb300 import libperm, ryser_split
    libperm.load()
    out = []
    for n, dtype in CASES:
        _, pb = libperm.ryser_pieces(n, dtype)
        full = ryser_split.split_partials(n, dtype, rank, world, lambda b, e: _stand_in(b, e, pb), dist)
        out.append(full.numpy().tobytes())
    dist.barrier()
    q.put((rank, out))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gather_restores_piece_order(lp, world):
    from paper_1802_02779_gb300 import ryser_split
    want = []
    for n, dtype in CASES:
        _, pb = lp.ryser_pieces(n, dtype)
        one = ryser_split.split_partials(n, dtype, 0, 1, lambda b, e: _stand_in(b, e, pb))
        want.append(one.numpy().tobytes())
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got in res:
        assert got == want, rank


def test_pieces_are_a_function_of_n_and_dtype(lp):
    # complex: Glynn's 2^(n-1) codes, 2^16 per piece; integers: 2^17 codes of Eq. 4 per piece
    assert lp.ryser_pieces(34, "c128") == (1 << 17, 32)
    assert lp.ryser_pieces(17, "c128") == (1, 32)
    assert lp.ryser_pieces(30, "u01") == (1 << 13, 40)
    assert lp.ryser_pieces(8, "i64") == (1, 40)
    for bad in ((0, "c128"), (41, "u01")):
        with pytest.raises(lp.LibpermError):
            lp.ryser_pieces(*bad)


@pytest.mark.parametrize("pieces", [1, 2, 3, 7, 128, 1 << 17, (1 << 17) + 5])
@pytest.mark.parametrize("world", [1, 2, 3, 4, 8, 9])
def test_split_partitions_the_pieces(lp, pieces, world):
    ranges = [lp.ryser_split(pieces, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == pieces
    for (b0, e0), (b1, e1) in zip(ranges, ranges[1:]):
        assert e0 == b1                               # contiguous, in rank order
    sizes = [e - b for b, e in ranges]
    assert min(sizes) >= 0 and max(sizes) - min(sizes) <= 1   # balanced


def test_split_rejects_bad_arguments(lp):
    for args in ((0, 0, 1), (4, -1, 2), (4, 2, 2), (4, 0, 0)):
        with pytest.raises(lp.LibpermError):
            lp.ryser_split(*args)
