"""Host logic of the multi-GPU layout, on CPU with gloo and 2 ranks: rows of
C are independent, so ranks take row blocks of A balanced by product count
(bench.py's partition), compute their blocks without any exchange, and the
blocks reassemble into the full product.  The per-rank block product is the
oracle here (the GPU path computes the same block through the plan's row
range, which the GPU tests check)."""
import os
import socket

import numpy as np
import pytest

from paper_2112_10037_gb300 import gen

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_balanced_row_blocks():
    import bench
    A = gen.rmat(10, 16)
    prod = bench.row_products(A, A)
    for n in (1, 2, 3, 8):
        cuts = bench.balanced_row_blocks(prod, n)
        assert cuts[0] == 0 and cuts[-1] == A.nrows and all(a <= b for a, b in zip(cuts, cuts[1:]))
        parts = [int(prod[a:b].sum()) for a, b in zip(cuts, cuts[1:])]
        assert sum(parts) == int(prod.sum())
        if n > 1:
            assert max(parts) <= prod.sum() / n + prod.max()


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    A = gen.rmat(11, 16)
    prod = bench.row_products(A, A)
    cuts = bench.balanced_row_blocks(prod, world)
    rb, re = cuts[rank], cuts[rank + 1]
    C = oracle.spgemm(oracle.select_rows(A, np.arange(rb, re)), A)
    # no exchange on the data path; gather only to check the reassembly
    blocks = [None] * world
    dist.all_gather_object(blocks, (rb, re, C.row_ptr, C.col_idx, C.vals))
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    pt = torch.tensor([float(prod[rb:re].sum())], dtype=torch.float64)
    dist.all_reduce(pt, op=dist.ReduceOp.SUM)
    if rank == 0:
        rp = [np.zeros(1, np.int64)]
        ci, vals, off = [], [], 0
        for (b0, b1, r, c, v) in blocks:
            rp.append(np.asarray(r[1:], np.int64) + off)
            off += int(r[-1])
            ci.append(c)
            vals.append(v)
        full = oracle.spgemm(A, A)
        ok = (np.array_equal(np.concatenate(rp), full.row_ptr) and
              np.array_equal(np.concatenate(ci), full.col_idx) and
              np.array_equal(np.concatenate(vals), full.vals) and
              t.item() == world and pt.item() == float(prod.sum()))
        with open(out_path, "w") as fh:
            fh.write("ok" if ok else "mismatch")
    dist.destroy_process_group()


def test_two_rank_row_shards_gloo(tmp_path, oracle_mod):
    import torch.multiprocessing as mp
    out = str(tmp_path / "result.txt")
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert open(out).read() == "ok"
