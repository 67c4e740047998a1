"""Instance sharding across ranks: the plan, the per-rank workload, and the
gradient all-reduce of designs shared by tasks on different ranks (Eq. 35).

The multi-rank tests run two gloo ranks on the CPU.  Each rank computes its
instances' gradients with the FP64 oracle, and the result is compared with one
oracle run over the whole batch.
"""
import os
import socket
import tempfile

import numpy as np
import pytest

from paper_2503_22767_gb300 import shard
from paper_2503_22767_gb300 import workloads as W


# ---------------------------------------------------------------------------
# the plan (pure host logic)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_plan_covers_every_instance_once_and_balances(world):
    rng = np.random.default_rng(world)
    counts = [int(c) for c in rng.integers(5000, 40000, size=64)]
    p = shard.plan(counts, None, world)
    seen = sorted(i for r in range(world) for i in p.local[r])
    assert seen == list(range(64))
    for r in range(world):
        assert p.local[r] == sorted(p.local[r])
        assert all(p.owner[i] == r for i in p.local[r])
    loads = [p.load(r) for r in range(world)]
    assert sum(loads) == sum(counts)
    # greedy LPT: the spread between ranks is at most one instance
    assert max(loads) - min(loads) <= max(counts)
    assert p.shared == []  # independent designs never need a collective


def test_plan_shared_design_detection():
    # three tasks of one design, two ranks: the design spans both ranks
    p = shard.plan([100, 100, 100], [0, 0, 0], 2)
    assert p.local == [[0, 2], [1]]
    assert p.shared == [0]
    # two designs with two tasks each on two ranks: equal counts alternate
    p = shard.plan([50, 50, 50, 50], [0, 0, 1, 1], 2)
    assert p.shared == [0, 1]
    # one rank: nothing is shared
    assert shard.plan([100, 100, 100], [0, 0, 0], 1).shared == []


def test_plan_more_ranks_than_instances():
    p = shard.plan([10, 30], None, 4)
    assert p.local == [[1], [0], [], []]
    assert p.load(2) == 0 and p.local_designs(3) == []


def test_plan_rejects_bad_arguments():
    with pytest.raises(ValueError):
        shard.plan([1, 2], None, 0)
    with pytest.raises(ValueError):
        shard.plan([1, 2], [0], 2)


def _multitask(n_tasks=3, n_steps=8):
    """One tiny 2D body, one design, several field schedules and targets."""
    base = W.tiny_2d(seed=11, n_steps=n_steps, phi_lo=0.3, field_scale=0.2, mag_scale=1.0)
    parts = []
    for k in range(n_tasks):
        other = W.tiny_2d(seed=100 + k, n_steps=n_steps, field_scale=0.2)
        parts.append(W.Workload("task", base.cfg, base.x0, base.v0, base.phi, base.mag, other.field,
                                other.target))
    return W.batch(parts, design_of_instance=[0] * n_tasks, name="multitask")


def _independent(n_steps=8):
    """Three tiny 2D bodies of different sizes, each with its own design."""
    parts = [W.tiny_2d(seed=20 + k, n_steps=n_steps, cells=c, phi_lo=0.3, field_scale=0.2, mag_scale=1.0)
             for k, c in enumerate([(4, 2), (6, 2), (2, 2)])]
    return W.batch(parts, name="independent")


def test_local_workload_slices_instances_and_designs():
    w = _independent()
    p = shard.plan(w.cfg.counts, None, 2)
    ioff = np.concatenate([[0], np.cumsum(w.cfg.counts)])
    for r in range(2):
        lw = shard.local_workload(w, p, r)
        assert lw.cfg.counts == [w.cfg.counts[i] for i in p.local[r]]
        assert lw.cfg.design_of_instance is None
        x = np.concatenate([w.x0[:, ioff[i]:ioff[i + 1]] for i in p.local[r]], axis=1)
        np.testing.assert_array_equal(lw.x0, x)
        np.testing.assert_array_equal(lw.field, w.field[p.local[r]])
        phi = np.concatenate([w.phi[ioff[i]:ioff[i + 1]] for i in p.local[r]])
        np.testing.assert_array_equal(lw.phi, phi)
    wm = _multitask()
    pm = shard.plan(wm.cfg.counts, wm.cfg.design_of_instance, 2)
    lw = shard.local_workload(wm, pm, 0)
    assert lw.cfg.design_of_instance == [0, 0] and lw.phi.shape == wm.phi.shape


# ---------------------------------------------------------------------------
# two gloo ranks on the CPU
# ---------------------------------------------------------------------------
def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, case, outdir):
    import torch
    import torch.distributed as dist

    import oracle

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        w = _multitask() if case == "multitask" else _independent()
        p = shard.plan(w.cfg.counts, w.cfg.design_of_instance, world)
        lw = shard.local_workload(w, p, rank)
        g = oracle.backward(lw)
        g_phi = torch.from_numpy(np.ascontiguousarray(g["g_phi"]))
        g_mag = torch.from_numpy(np.ascontiguousarray(g["g_mag"]))
        n_coll = shard.reduce_design_grads(p, rank, w.cfg.dim, g_phi, g_mag)
        np.savez(os.path.join(outdir, f"rank{rank}.npz"), g_phi=g_phi.numpy(), g_mag=g_mag.numpy(),
                 g_field=g["g_field"], n_coll=n_coll)
    finally:
        dist.destroy_process_group()


def _run_ranks(case, world=2):
    import torch.multiprocessing as mp

    out = tempfile.mkdtemp(prefix="shard_")
    mp.start_processes(_rank_main, args=(world, _free_port(), case, out), nprocs=world, join=True,
                       start_method="spawn")
    return [dict(np.load(os.path.join(out, f"rank{r}.npz"))) for r in range(world)]


@pytest.mark.parametrize("case", ["multitask", "independent"])
def test_two_rank_gradients_match_single_process(orc, case):
    w = _multitask() if case == "multitask" else _independent()
    full = orc.backward(w)
    p = shard.plan(w.cfg.counts, w.cfg.design_of_instance, 2)
    res = _run_ranks(case)
    dcounts = w.cfg.design_counts()
    doff = np.concatenate([[0], np.cumsum(dcounts)]).astype(int)
    for r in range(2):
        out = res[r]
        # Eq. 35's exchange only where a design spans ranks
        assert int(out["n_coll"]) == (1 if p.shared else 0)
        gdes = p.local_designs(r)
        want_phi = np.concatenate([full["g_phi"][doff[g]:doff[g + 1]] for g in gdes])
        want_mag = np.concatenate([full["g_mag"][:, doff[g]:doff[g + 1]] for g in gdes], axis=1)
        scale = np.abs(full["g_phi"]).max()
        # only the order of the task sums differs from the single-process run
        np.testing.assert_allclose(out["g_phi"], want_phi, rtol=1e-10, atol=1e-12 * scale)
        np.testing.assert_allclose(out["g_mag"], want_mag, rtol=1e-10,
                                   atol=1e-12 * np.abs(full["g_mag"]).max())
        # per-instance field gradients never cross ranks
        np.testing.assert_array_equal(out["g_field"], full["g_field"][p.local[r]])
    if case == "multitask":
        # the shared design got contributions from both ranks: neither rank's
        # local sum equals the total alone
        single = orc.backward(shard.local_workload(w, p, 1))
        assert not np.allclose(single["g_phi"], full["g_phi"])
