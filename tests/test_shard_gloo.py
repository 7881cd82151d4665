"""The multi-rank path on CPU: world_size-2 gloo ranks shard a Lambda batch.

Each rank evaluates its block of rows with the FP64 oracle (standing in for its GPU
context: the sharding logic is the same), the blocks are gathered in rank order, and
rank 0 checks the result against one process evaluating the whole batch.  Also checks
the row split, the max over ranks used for the job's time, and a batch whose size is
not a multiple of the world size.  Event shards exchange their parts in one all_gather
and combine them with the library's gwc_merge_parts (its host arithmetic, as on gloo).
"""
import os
import socket

import numpy as np
import pytest


@pytest.fixture(scope="module", autouse=True)
def _library():
    # the event-shard merge runs in libgwc.so (host arithmetic for host rows)
    from paper_2605_23538_gb300 import build
    build.build()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n_rows, result_file):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2605_23538_gb300 import shard, synth
        cat = synth.catalogue(synth.scaled("shard", 4, ("fixed", 200), 4, 128, 2000, "found"))
        lam_all = shard.world_batch(n_rows // world, world, lambda n: synth.lambda_batch(n, purpose=51)) \
            if n_rows % world == 0 else synth.lambda_batch(n_rows, purpose=51)
        mine = shard.rank_rows(lam_all, rank, world)
        r = oracle.loglik(cat, mine, n_threads=1)
        block = torch.tensor(np.column_stack([r["lnL_total"], r["ln_xi"]]), dtype=torch.float64)
        allrows = shard.gather_rows(block, len(lam_all))
        t = shard.max_over_ranks(10.0 + rank)
        if rank == 0:
            np.savez(result_file, gathered=allrows.numpy(), lam=lam_all, tmax=t)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("n_rows", [6, 5])
def test_two_gloo_ranks_reproduce_one_process(tmp_path, n_rows):
    import torch.multiprocessing as mp
    import oracle
    from paper_2605_23538_gb300 import synth
    out = str(tmp_path / "r.npz")
    mp.start_processes(_rank_main, args=(2, _free_port(), n_rows, out), nprocs=2,
                       start_method="spawn", join=True)
    res = np.load(out)
    cat = synth.catalogue(synth.scaled("shard", 4, ("fixed", 200), 4, 128, 2000, "found"))
    ref = oracle.loglik(cat, res["lam"], n_threads=1)
    assert res["gathered"].shape == (n_rows, 2)
    np.testing.assert_array_equal(res["gathered"][:, 0], ref["lnL_total"])
    np.testing.assert_array_equal(res["gathered"][:, 1], ref["ln_xi"])
    assert res["tmax"] == 11.0


def test_row_ranges_cover_the_batch_once():
    from paper_2605_23538_gb300 import shard
    for n in (0, 1, 5, 6, 256, 1001):
        for world in (1, 2, 3, 8):
            spans = [shard.row_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.row_range(4, 2, 2)


def _parts_rank(rank, world, port, result_file):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2605_23538_gb300 import shard, synth
        cat = synth.catalogue(synth.scaled("shard", 4, ("fixed", 200), 4, 128, 2000, "found"))
        lam = synth.lambda_batch(3, purpose=52)
        ne, ni = len(cat["offsets"]) - 1, len(cat["inj_m1"])
        ev = list(range(rank * ne // world, (rank + 1) * ne // world))
        part = synth.subset_events(cat, ev)
        a, b = rank * ni // world, (rank + 1) * ni // world
        for k in ("inj_m1", "inj_m2", "inj_dl", "inj_lnpd"):
            part[k] = cat[k][a:b]
        r = oracle.loglik(part, lam, n_threads=1, neff_min_event=0.0)
        mine = {"sum_events": r["lnL_event"].sum(axis=1), "ln_xi": r["ln_xi"], "neff_sel": r["neff_sel"],
                "flags": r["flags"], "n_events": len(ev)}
        merged = shard.merge_parts_distributed(mine)
        if rank == 0:
            np.savez(result_file, total=merged["lnL_total"], ln_xi=merged["ln_xi"],
                     neff_sel=merged["neff_sel"], lam=lam)
    finally:
        dist.destroy_process_group()


def test_event_shards_on_two_gloo_ranks(tmp_path):
    # each rank evaluates half of the events and half of the injections with the oracle;
    # one exchange reproduces the whole catalogue's ln xi, N_eff,sel and total
    import torch.multiprocessing as mp
    import oracle
    from paper_2605_23538_gb300 import synth
    out = str(tmp_path / "p.npz")
    mp.start_processes(_parts_rank, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    res = np.load(out)
    cat = synth.catalogue(synth.scaled("shard", 4, ("fixed", 200), 4, 128, 2000, "found"))
    ref = oracle.loglik(cat, res["lam"], n_threads=1, neff_min_event=0.0)
    np.testing.assert_allclose(res["ln_xi"], ref["ln_xi"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(res["neff_sel"], ref["neff_sel"], rtol=1e-12)
    np.testing.assert_allclose(res["total"], ref["lnL_total"], rtol=0, atol=1e-10)


def _parts_rank_grad(rank, world, port, result_file):
    # multi-peak (16-entry) Lambda with gradients: the oracle gives this shard's total
    # gradient; its parts are rebuilt from the definition of ln xi
    # (d ln xi = sum_m softmax(ln w)_m d ln w_m) and grad_total = grad_events - n_r d ln xi_r
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2605_23538_gb300 import shard, synth
        cat = synth.catalogue(synth.scaled("shard", 4, ("fixed", 200), 4, 128, 2000, "found"))
        lam = synth.lambda_batch(2, purpose=53, model="multipeak")
        ne, ni = len(cat["offsets"]) - 1, len(cat["inj_m1"])
        ev = list(range(rank * ne // world, (rank + 1) * ne // world))
        part = synth.subset_events(cat, ev)
        a, b = rank * ni // world, (rank + 1) * ni // world
        for k in ("inj_m1", "inj_m2", "inj_dl", "inj_lnpd"):
            part[k] = cat[k][a:b]
        r = oracle.loglik(part, lam, grad=True, neff_min_event=0.0)
        gx = []
        for q in lam:
            lw, dlw, _ = oracle.ln_w_samples(q, part, "inj", grad=True)
            fin = np.isfinite(lw)
            w = np.exp(lw[fin] - lw[fin].max())
            gx.append((w[:, None] * dlw[fin]).sum(axis=0) / w.sum())
        gx = np.array(gx)
        mine = {"sum_events": r["lnL_event"].sum(axis=1), "ln_xi": r["ln_xi"], "neff_sel": r["neff_sel"],
                "flags": r["flags"], "n_events": len(ev),
                "grad_events": r["grad_total"] + len(ev) * gx, "grad_ln_xi": gx}
        merged = shard.merge_parts_distributed(mine)
        if rank == 0:
            np.savez(result_file, total=merged["lnL_total"], grad=merged["grad_total"], lam=lam)
    finally:
        dist.destroy_process_group()


def test_event_shards_merge_multipeak_gradients_on_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    import oracle
    from paper_2605_23538_gb300 import synth
    out = str(tmp_path / "pg.npz")
    mp.start_processes(_parts_rank_grad, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    res = np.load(out)
    cat = synth.catalogue(synth.scaled("shard", 4, ("fixed", 200), 4, 128, 2000, "found"))
    ref = oracle.loglik(cat, res["lam"], grad=True, neff_min_event=0.0)
    assert res["grad"].shape == (2, 16)
    np.testing.assert_allclose(res["total"], ref["lnL_total"], rtol=0, atol=1e-9)
    np.testing.assert_allclose(res["grad"], ref["grad_total"], rtol=1e-8, atol=1e-8 * np.abs(ref["grad_total"]).max())


def test_merge_entry_on_host_rows_matches_the_whole_catalogue(orc):
    # the same entry gloo ranks use, called in one process on three shards' host rows
    # (events and injections split unevenly), against the oracle on the whole catalogue
    from paper_2605_23538_gb300 import shard, synth
    cat = synth.catalogue(synth.scaled("shard", 6, ("fixed", 150), 4, 128, 3000, "found"))
    lam = synth.lambda_batch(3, purpose=54)
    ne, ni = len(cat["offsets"]) - 1, len(cat["inj_m1"])
    cuts_e, cuts_i = [0, 1, 4, ne], [0, ni // 5, ni // 2, ni]
    parts = []
    for r in range(3):
        ev = list(range(cuts_e[r], cuts_e[r + 1]))
        part = synth.subset_events(cat, ev)
        for k in ("inj_m1", "inj_m2", "inj_dl", "inj_lnpd"):
            part[k] = cat[k][cuts_i[r]:cuts_i[r + 1]]
        o = orc.loglik(part, lam, n_threads=1, neff_min_event=0.0)
        parts.append({"sum_events": o["lnL_event"].sum(axis=1), "ln_xi": o["ln_xi"], "neff_sel": o["neff_sel"],
                      "flags": o["flags"], "n_events": len(ev)})
    merged = shard.merge_parts(parts)
    assert merged["lnL_total"].device.type == "cpu"
    ref = orc.loglik(cat, lam, n_threads=1, neff_min_event=0.0)
    np.testing.assert_allclose(merged["ln_xi"].numpy(), ref["ln_xi"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(merged["neff_sel"].numpy(), ref["neff_sel"], rtol=1e-12)
    np.testing.assert_allclose(merged["lnL_total"].numpy(), ref["lnL_total"], rtol=0, atol=1e-10)
    np.testing.assert_array_equal(merged["flags"].numpy(), ref["flags"])


def test_merge_entry_rejects_bad_shapes():
    import ctypes
    import paper_2605_23538_gb300 as g
    buf = np.zeros(64)
    outs = [np.zeros(4) for _ in range(3)] + [np.zeros(4, np.int32)]
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    assert g.lib().gwc_merge_parts(2, 1, 7, p(buf), 0, *[p(o) for o in outs], None, None) != 0
    assert g.lib().gwc_merge_parts(0, 1, 0, p(buf), 0, *[p(o) for o in outs], None, None) != 0
    assert g.lib().gwc_merge_parts(1, 1, 0, p(buf), 0, None, *[p(o) for o in outs[1:]], None, None) != 0
