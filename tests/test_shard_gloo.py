"""The patch-sharded form of a reconstruction pass, run as CPU ranks over
gloo (world size 2).  Each rank computes its own rows with the oracle (the
forward model and adjoint) and runs the EM E-step on its own pixels; the
exchanges (adjoint sum, the EM statistics before and the M-step sums after
the E-step, the per-patch p-bar gather, slowest-rank time) go through
paper_1611_07289_b300.shard and must reproduce the unsharded oracle's
volumes, EM state, pixel weights and patch potentials."""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import pvr_oracle as O
from paper_1611_07289_b300 import shard
from tests.cases import uneven_case


def test_partition_is_contiguous_balanced_and_rebased():
    geom, desc, npix, poses, rng = uneven_case(7)
    for ws in (1, 2, 3, 5, 200):
        b = shard.partition_by_pixels(desc, ws)
        assert b[0] == 0 and b[-1] == desc.shape[0] and np.all(np.diff(b) >= 0)
        sizes = desc[:, 4].astype(np.int64) * desc[:, 5]
        per = np.array([sizes[b[r]:b[r + 1]].sum() for r in range(ws)])
        assert per.sum() == npix
        if ws <= desc.shape[0]:
            # each cut lands within one patch of the ideal share
            cuts = np.cumsum(per)[:-1]
            ideal = (npix * np.arange(1, ws)) // ws
            assert np.all(np.abs(cuts - ideal) <= sizes.max())
        rows, spans = [], []
        for r in range(ws):
            d, lo, hi = shard.shard_table(desc, b, r)
            if d.shape[0]:
                assert d[0, 6] == 0
                assert hi - lo == int((d[:, 4].astype(np.int64) * d[:, 5]).sum())
            e = d.copy()
            e[:, 6] += lo
            rows.append(e)
            spans.append((lo, hi))
        assert np.array_equal(np.concatenate(rows), desc)
        nz = [s for s in spans if s[1] > s[0]]
        assert all(nz[i][1] == nz[i + 1][0] for i in range(len(nz) - 1))
    bad = desc.copy()
    bad[3, 6] += 1
    with pytest.raises(ValueError):
        shard.shard_table(bad, np.array([0, bad.shape[0]]), 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port):
    os.environ["OMP_NUM_THREADS"] = "2"
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        geom, desc, npix, poses, rng = uneven_case(11)
        G, ps = O.geom(geom), O.psf(1.2, 1, 3, 0.8)
        x = rng.uniform(0, 1000, geom.n_vox).astype(np.float32)
        y = rng.uniform(0, 1000, npix).astype(np.float32)
        r = rng.normal(size=npix)

        # unsharded oracle (every rank computes it, for comparison)
        fix = O.pose_fixed(G, ps, desc, poses)
        s_full, v_full, _ = O.simulate(G, ps, x, desc, fix, npix)
        a_full, c_full = O.adjoint(G, ps, desc, fix, r=r)
        e_full = y - s_full
        st = O.new_state()
        p_full, _, pb_full, _ = O.em_weights(y, s_full, v_full, desc, O.em_params(), st)

        # this rank's rows
        b = shard.partition_by_pixels(desc, ws)
        d, lo, hi = shard.shard_table(desc, b, rank)
        fx = O.pose_fixed(G, ps, d, poses[b[rank]:b[rank + 1]])
        s, v, _ = O.simulate(G, ps, x, d, fx, hi - lo)
        assert np.array_equal(s, s_full[lo:hi]) and np.array_equal(v, v_full[lo:hi])

        # adjoint: one sum over ranks of (addon, conf)
        a, c = O.adjoint(G, ps, d, fx, r=r[lo:hi])
        ta, tc = torch.from_numpy(a), torch.from_numpy(c)
        shard.allreduce_sum_([ta, tc], dist)
        assert np.max(np.abs(ta.numpy() - a_full)) <= 1e-12 * np.max(np.abs(a_full))
        assert np.max(np.abs(tc.numpy() - c_full)) <= 1e-12 * np.max(np.abs(c_full))

        # EM: global residual statistics, m = 1 / range
        n, se2, emin, emax = shard.em_global_stats(y[lo:hi] - s, v, dist)
        ev = e_full[v_full.astype(bool)]
        assert n == ev.size and emin == ev.min() and emax == ev.max()
        assert abs(se2 - float((ev * ev).sum())) <= 1e-12 * se2
        assert abs(1.0 / (emax - emin) - st[O.ST["M"]]) <= 1e-15 * st[O.ST["M"]]

        # the first call's state from the global statistics, the E-step on
        # this rank's pixels, the M-step from the all-reduced sums
        ep = O.em_params()
        rng_e = emax - emin
        sfloor = max((ep.sigma_floor_rel * rng_e) ** 2, 1e-12)
        sigma2, c, m = max(se2 / n, sfloor), ep.c0, 1.0 / rng_e
        e = (y[lo:hi].astype(np.float64) - s)
        G = np.exp(-e * e / (2.0 * sigma2)) / (math.sqrt(2.0 * math.pi) * math.sqrt(sigma2))
        p = np.where(v > 0, G * c / (G * c + m * (1.0 - c)), 0.0)
        assert np.allclose(p, p_full[lo:hi], rtol=1e-12, atol=1e-300)
        sp, spe2 = shard.em_mstep_sums(p, e, v, dist)
        assert abs(max(spe2 / sp, sfloor) - st[O.ST["SIGMA2"]]) <= 1e-12 * st[O.ST["SIGMA2"]]
        assert abs(min(max(sp / n, 1e-3), 1 - 1e-3) - st[O.ST["C"]]) <= 1e-12

        # per-patch potentials from this rank's own E-step, gathered in table order
        pb = []
        for row in d:
            o, k = int(row[6]), int(row[4] * row[5])
            pv, vv = p[o:o + k], v[o:o + k].astype(bool)
            pb.append(np.sqrt(np.sum(pv[vv] ** 2) / vv.sum()) if vv.sum() else 0.0)
        allpb = shard.gather_patch_values(np.array(pb), b, dist)
        keep = np.array([v_full[int(q[6]):int(q[6] + q[4] * q[5])].sum() > 0 for q in desc])
        assert np.allclose(allpb[keep], pb_full[keep], rtol=1e-12, atol=0)

        # the slowest rank's time
        assert shard.max_over_ranks(0.5 + rank, dist) == ws - 0.5
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2])
def test_sharded_pass_matches_unsharded_oracle_over_gloo(ws):
    mp.spawn(_rank_main, args=(ws, _free_port()), nprocs=ws, join=True)


def _uneven_ranks_main(rank, ws, port):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        desc = np.array([[0, 0, 0, 0, 4, 4, 0, 0]], dtype=np.int32)    # one patch, two ranks
        b = shard.partition_by_pixels(desc, ws)
        d, lo, hi = shard.shard_table(desc, b, rank)
        vals = np.full(d.shape[0], 3.0 + rank)
        got = shard.gather_patch_values(vals, b, dist)
        owner = int(np.searchsorted(b, 0, side="right")) - 1
        assert got.shape == (1,) and got[0] == 3.0 + owner
        t = torch.tensor([float(hi - lo)], dtype=torch.float64)
        shard.allreduce_sum_([t], dist)
        assert t.item() == 16.0
    finally:
        dist.destroy_process_group()


def test_rank_without_rows_over_gloo():
    mp.spawn(_uneven_ranks_main, args=(2, _free_port()), nprocs=2, join=True)
