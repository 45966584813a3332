"""Throat lists sharded over ranks (Sec. 4: every pore throat is an independent
simulation, so spreading them over GPUs needs no exchange but the final gather
of their results).  The split is longest processing time first on the
non-solid cells of each box; two gloo ranks on the CPU run a stand-in for the
batch and must reassemble exactly the serial answer.  CPU only."""
import os
import socket

import numpy as np
import pytest

import workloads as W


def test_lpt_partition_properties():
    import paper_1906_04722_gb300 as lbm
    rng = np.random.default_rng(3)
    for parts in (1, 2, 3, 8):
        cost = rng.uniform(1.0, 100.0, 57)
        part, load = lbm.lbm_partition_lpt(cost, parts)
        assert part.min() >= 0 and part.max() < parts
        for q in range(parts):
            assert load[q] == pytest.approx(cost[part == q].sum(), rel=1e-12)
        # Graham's bound for LPT: makespan <= 4/3 of the optimum, and the
        # optimum is at least the mean load and the largest item
        opt_lb = max(cost.sum() / parts, cost.max())
        assert load.max() <= (4.0 / 3.0) * opt_lb + 1e-9
    # worked by hand: costs 5, 4, 3, 3, 3 on two parts -> {5, 3} and {4, 3, 3}
    part, load = lbm.lbm_partition_lpt([5, 4, 3, 3, 3], 2)
    assert list(part) == [0, 1, 1, 0, 1] and list(load) == [8.0, 10.0]


def _fake_batch(th, params, ladder, n_steps, rho_out_w):
    """Stand-in for lbm_run_throat_batch: a result that depends on the throat
    alone (its first sphere's radius), so any mix-up in the gather shows."""
    res = [{"p_ce": float(t[0, 3]) * 0.01, "invaded_at": int(t[0, 3]) % 5, "n_fluid": 0} for t in th]
    rows = [[{"S_w": 1.0 - 0.01 * k - float(t[1, 3]) * 1e-4} for k in range(len(ladder))] for t in th]
    return res, rows


def _worker(rank, world, port, throats, out_dir):
    import torch.distributed as dist
    import paper_1906_04722_gb300 as lbm
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)

    def gather(obj):
        out = [None] * world
        dist.all_gather_object(out, obj)
        return out

    res, rows = lbm.run_throat_batch_sharded(throats, lbm.make_params(), [2.0, 2.05, 2.1], 10, 2.0, rank, world,
                                             gather, run=_fake_batch)
    np.save(os.path.join(out_dir, f"r{rank}.npy"),
            np.array([[r["p_ce"], r["invaded_at"], rows[i][2]["S_w"]] for i, r in enumerate(res)]))
    dist.destroy_process_group()


def test_sharded_batch_two_gloo_ranks(tmp_path):
    import multiprocessing as mp
    pytest.importorskip("torch")
    throats = W.delaunay_throats(W.sample_spheres(128, seed=5), 23, seed=2)
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, 2, port, throats, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    serial_res, serial_rows = _fake_batch(throats, None, [0, 1, 2], 10, 2.0)
    want = np.array([[r["p_ce"], r["invaded_at"], serial_rows[i][2]["S_w"]] for i, r in enumerate(serial_res)])
    for r in range(2):
        assert np.array_equal(np.load(tmp_path / f"r{r}.npy"), want)
