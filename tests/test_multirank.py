"""Multi-rank host logic on CPU: two gloo ranks.

* bench.py: events are independent problems, so ranks share no data: each
  draws its own events (distinct seeds), and the only collective is the max
  over ranks of the timed regions, from which the whole-job rate is formed
  (weak scaling).
* A bank-sharded event: each rank holds half of the bank's rows and evaluates
  the event on its half; one all-gather of each rank's evidence record, row
  count and per-sample marginals, then dotpe_evidence_merge (FP64, host) on
  every rank gives the one-pass ln Z, N_eff, N_eff,int, N_eff,ext, per-sample
  marginals and maximum (Eq. Z_sum; Eqs. posterior_element, int_ess,
  ext_ess).  The shards' records come from the oracle here (no GPU); the
  one-pass reference is the oracle on the whole bank.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank-local timings of two regions (device-resident, end to end)
        got = bench.combine_ranks(dist, (10.0 + rank, 20.0 - rank), torch.device("cpu"))
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.rank_seed(2, rank))
        out[rank] = (got, seeds)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_by_max():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        got, seeds = res[r]
        assert got == [11.0, 20.0]          # each region: the slowest rank
        assert len(set(seeds)) == world      # independent events per rank
    # whole-job rate: every rank's units over the max-over-ranks time
    assert bench.whole_job_rate(world, 1000, 10, 11.0) == pytest.approx(2 * 1000 * 10 / 0.011)


def test_single_process_needs_no_collective():
    assert bench.combine_ranks(None, (3.0, 4.0), None) == [3.0, 4.0]


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    monkeypatch.setenv("RANK", "1")

    class A:
        steps, warmup, gpus = 1, 1, 2
    assert bench.run_reference(A()) is None


def _shard_rank(rank, world, port, out):
    import numpy as np
    import oracle
    import paper_2507_16022_gb300 as dp
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        wl = synth.make_workload(n_int=90, n_ext=24, n_det=2, n_modes=3, n_bins=48, snr=12.0, seed=61,
                                 ln_w="random", n_phi=16)
        cuts = [0, 37, 90]  # uneven row halves
        a, b = cuts[rank], cuts[rank + 1]
        P = oracle.OracleProblem(wl.bank, wl.ext, wl.event, i_slice=slice(a, b))
        grid, _ = P.eval_grid(0.0)
        ev = P.evidence(grid)
        rec = dict(ln_z=ev["ln_z"], n_eff=ev["n_eff"], n_eff_int=ev["n_eff_int"], n_eff_ext=ev["n_eff_ext"],
                   max_lnl_ml=ev["max_lnl_ml"], arg_i=a + int(ev["arg"][0]), arg_e=int(ev["arg"][1]),
                   arg_o=int(ev["arg"][2]), n_marginalised=ev["n_marginalised"], n_pairs=(b - a) * 24,
                   lnl_ml_threshold=float("-inf"), device_status=0, n_refined_tiles=-1)
        shards = [None] * world
        dist.all_gather_object(shards, (rec, b - a, np.asarray(ev["ln_p_ext"], dtype=np.float64)))
        merged, lpe = dp.dotpe_evidence_merge(shards, wl.event.n_phi)
        out[rank] = (merged, lpe.tolist())
    finally:
        dist.destroy_process_group()


def test_bank_sharded_event_merges_to_one_pass():
    import numpy as np
    import oracle
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_shard_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    wl = synth.make_workload(n_int=90, n_ext=24, n_det=2, n_modes=3, n_bins=48, snr=12.0, seed=61,
                             ln_w="random", n_phi=16)
    P = oracle.OracleProblem(wl.bank, wl.ext, wl.event)
    grid, _ = P.eval_grid(0.0)
    ref = P.evidence(grid)
    for r in range(world):
        got, lpe = res[r]
        assert got["ln_z"] == pytest.approx(ref["ln_z"], abs=1e-12)
        for k in ("n_eff", "n_eff_int", "n_eff_ext"):
            assert got[k] == pytest.approx(ref[k], rel=1e-10), k
        assert got["max_lnl_ml"] == ref["max_lnl_ml"]
        assert (got["arg_i"], got["arg_e"], got["arg_o"]) == tuple(int(x) for x in ref["arg"])
        assert got["n_marginalised"] == ref["n_marginalised"] and got["n_pairs"] == 90 * 24
        np.testing.assert_allclose(lpe, ref["ln_p_ext"], rtol=0, atol=1e-12)


def test_evidence_merge_of_one_shard_is_identity():
    import numpy as np
    import paper_2507_16022_gb300 as dp
    rec = dict(ln_z=-1.25, n_eff=37.5, n_eff_int=4.0, n_eff_ext=9.0, max_lnl_ml=12.0, arg_i=3, arg_e=4, arg_o=5,
               n_marginalised=100, n_pairs=200, lnl_ml_threshold=-8.0, device_status=0, n_refined_tiles=7)
    lpe = np.log(np.array([0.5, 1.5, 2.0]))
    got, out = dp.dotpe_evidence_merge([(rec, 20, lpe)], 8)
    assert got["ln_z"] == pytest.approx(rec["ln_z"], abs=1e-14)
    assert got["n_eff"] == pytest.approx(37.5, rel=1e-14) and got["n_eff_int"] == pytest.approx(4.0, rel=1e-14)
    # N_eff,ext is recomputed from the per-sample marginals: S1^2 / sum_e P_e^2
    s1 = np.exp(rec["ln_z"]) * 20 * 3 * 8
    assert got["n_eff_ext"] == pytest.approx(s1 ** 2 / np.sum(np.exp(2 * lpe)), rel=1e-12)
    np.testing.assert_allclose(out, lpe, atol=1e-15)
    assert (got["arg_i"], got["n_refined_tiles"], got["lnl_ml_threshold"]) == (3, 7, -8.0)


def test_evidence_merge_adds_screen_counters():
    """The screening counters of row shards add up; a shard without them (-1, or a
    record that does not carry them) leaves the merged counters unknown (-1)."""
    import numpy as np
    import paper_2507_16022_gb300 as dp
    base = dict(ln_z=-1.0, n_eff=2.0, n_eff_int=2.0, n_eff_ext=2.0, max_lnl_ml=5.0, arg_i=0, arg_e=0, arg_o=0,
                n_marginalised=10, n_pairs=40, lnl_ml_threshold=-15.0, device_status=0, n_refined_tiles=1)
    lpe = np.log(np.array([0.5, 1.5]))
    a = dict(base, n_screen_candidates=30, n_screen_evaluated=4)
    b = dict(base, arg_i=20, n_screen_candidates=12, n_screen_evaluated=3)
    got, _ = dp.dotpe_evidence_merge([(a, 20, lpe), (b, 20, lpe)], 8)
    assert (got["n_screen_candidates"], got["n_screen_evaluated"]) == (42, 7)
    got, _ = dp.dotpe_evidence_merge([(a, 20, lpe), (base, 20, lpe)], 8)
    assert (got["n_screen_candidates"], got["n_screen_evaluated"]) == (-1, -1)
