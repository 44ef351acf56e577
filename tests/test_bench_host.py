"""Host logic of bench.py (no GPU): the algorithmic bytes of a restricted-
smoothing pass count the entries of the filtered operator that the pass
needs, i.e. every diagonal and every negative off-diagonal a_ik (the filter
of Eq. 8 zeroes the positive ones) whose rows i and k share a coarse node;
checked against the oracle's support pattern on a 16^3 MPFA-O case. The
multiply-adds of a pass (the FP64 pipe roofline) count the coarse nodes each
such pair of rows shares."""
import numpy as np
import scipy.sparse as sp

import bench
from oracle import msrsb as O
from synth.darcy import darcy_3d_case


def _colour_slot_ids(part):
    # coarse node J sits in slot sum_d (J_d mod 2) 2^d of every row it supports
    pat, nb = part["pat"], part["nb"]
    n = pat.shape[0]
    J = np.arange(part["nc"])
    jc = (J % nb[0], (J // nb[0]) % nb[1], J // (nb[0] * nb[1]))
    slot = (jc[0] % 2) + 2 * (jc[1] % 2) + 4 * (jc[2] % 2)
    rows = np.repeat(np.arange(n), np.diff(pat.indptr))
    assert np.bincount(rows * 8 + slot[pat.indices], minlength=8 * n).max() <= 1  # no two nodes share a slot
    ids = -np.ones((n, 8), dtype=np.int64)
    ids[rows, slot[pat.indices]] = pat.indices
    return ids


def test_kept_entries_match_the_support_pattern():
    c = darcy_3d_case(n=16, H=4)
    part = O.partition(c["dims"], c["H"], 0)
    ids = _colour_slot_ids(part)
    A = sp.csr_matrix((c["data"], c["indices"], c["indptr"])).tocoo()
    n = A.shape[0]
    off = (A.row != A.col) & (A.data < 0)
    shared = (part["pat"] @ part["pat"].T).tocsr()
    common = np.asarray(shared[A.row[off], A.col[off]]).ravel()
    kept, matches = bench.kept_entries(c, ids)
    assert kept == n + int((common > 0).sum())
    # multiply-adds of A_hat P on P's pattern: coarse nodes rows i and k share
    assert matches == int(common.sum())
    # the filter keeps exactly these off-diagonal values nonzero
    Ah = O.mmatrix_filter(sp.csr_matrix((c["data"], c["indices"], c["indptr"]))).tocoo()
    nz_off = (Ah.row != Ah.col) & (Ah.data != 0)
    assert int(nz_off.sum()) == int(off.sum())
    # about half of the rotated anisotropic stencil is positive off-diagonal
    assert 0.3 < 1 - (n + off.sum()) / A.nnz < 0.7


def test_smooth_bytes_per_kept_entry():
    # value + packed column per kept entry; P read and written, scale, slot mask per row
    assert bench.smooth_bytes(10, 100, 8, 4) == 100 * 8 + 10 * (2 * 8 * 4 + 4 + 1)
    assert bench.smooth_bytes(10, 100, 8, 8) == 100 * 12 + 10 * (2 * 8 * 8 + 8 + 1)


def test_clock_summary_reads_clocks_and_throttle_reasons():
    c = bench.ClockSampler()
    c.lines = ["2070, 2070, Not Active, Not Active, Not Active, Not Active",
               "1980, 2070, Not Active, Not Active, Not Active, Active",
               "2070, 2070, Not Active, Active, Not Active, Not Active",
               "[N/A], 2070, Not Active, Not Active, Not Active, Not Active",  # unreadable sample: skipped
               "garbage"]
    s = c.summary()
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    empty = bench.ClockSampler().summary()
    assert empty["samples"] == 0 and empty["reasons"] == ["unsampled"]


def _max_rank(rank, world, port, out):
    import os
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.max_over_ranks([1.0 + rank, 10.0 - rank], "cpu")
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_max_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        assert out[0] == [2.0, 10.0] and out[1] == [2.0, 10.0]


class _FakeTuneLib:
    """Stands in for the binding's msrsb_tune_table (no GPU)."""

    def __init__(self, rows):
        self.rows = rows

    def msrsb_tune_table(self):
        return self.rows


def _tune_row(variant, n_log2, value_bytes=4, W=8):
    lanes, threads, ahead, capped = bench.SMOOTH_SHAPES[variant]
    return {"kernel": 0, "device": 0, "value_bytes": value_bytes, "W": W, "n_log2": n_log2, "width_log2": 4,
            "variant": variant, "lanes": lanes, "threads": threads, "ahead": ahead, "capped": capped,
            "n_variants": len(bench.SMOOTH_SHAPES), "us": [1.0] * len(bench.SMOOTH_SHAPES)}


def test_smooth_shape_names_the_tuned_kernel():
    M = _FakeTuneLib([_tune_row(4, 18), _tune_row(5, 21), _tune_row(2, 17, value_bytes=8)])
    s64 = bench.smooth_shape(M, 64 ** 3, 8, 4)
    assert s64["variant"] == 4 and s64["kernel"] == "smooth_pf_kernel<float,8,2,true>"
    assert (s64["lanes_per_row"], s64["threads"], s64["entries_ahead"], s64["registers_capped"]) == (1, 256, 2, True)
    assert bench.smooth_shape(M, 128 ** 3, 8, 4)["kernel"] == "smooth_pf_kernel<float,8,3,true>"
    assert bench.smooth_shape(M, 117649, 8, 8)["kernel"] == "smooth_lanes_kernel<double,8,2>"
    assert bench.smooth_shape(M, 32 ** 3, 8, 4) is None  # size class never tuned
    assert bench.smooth_shape(_FakeTuneLib([_tune_row(0, 18)]), 64 ** 3, 8, 4)["kernel"] == "smooth_kernel<float,8>"


def test_smooth_traffic_is_reported_only_for_the_captured_source_and_shape(monkeypatch):
    h = bench.source_hash("basis.cu")
    table = {("darcy64", 4): (h, 123), ("darcy128", 5): ("0" * 16, 456)}
    monkeypatch.setattr(bench, "SMOOTH_TRAFFIC", table)
    assert bench.smooth_traffic("darcy64", 4) == 123      # captured on this source, this shape
    assert bench.smooth_traffic("darcy64", 0) is None     # another shape
    assert bench.smooth_traffic("darcy128", 5) is None    # captured on another source
    assert bench.smooth_traffic("elastic48", 0) is None   # never captured


def test_oracle_timing_runs_on_the_host(capsys):
    # the oracle's own timing needs no GPU: best of the runs per phase, per thread count
    import argparse
    import json
    bench.oracle_timing_run(argparse.Namespace(oracle_workloads="darcy2d64", oracle_repeats=1))
    out = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    per = out["workloads"]["darcy2d64"]
    assert "1" in per and str(out["cores"]) in per
    for r in per.values():
        assert r["setup_s"] > 0 and r["solve_s"] > 0 and r["runs"] == 1
        assert r["basis_iters"] <= 100 and r["relres"] <= 1e-8
