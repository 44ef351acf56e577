"""Benchmark: MsRSB set-up (filter + basis + Galerkin + coarse inverse +
smoother factor) plus the Krylov solve to relative residual 1e-8, on the 3D
Darcy workload (64^3 cells, 27-point MPFA-O, ln k Gaussian random field with
correlation length 8 cells and sigma 3, 10:1 anisotropy rotated (20, 35, 0)
degrees, corner well pair, 8^3-cell coarse blocks, GMRES + ILU(0) post
smoothing). One step = one whole set-up + solve; `value` is seconds per step of
the mixed-precision form (FP32 basis, P and smoother, FP64 Krylov and coarse
inverse); the plain FP64 form is timed the same way and reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank solves its own copy (replicas); rank 0
prints one JSON line with the max over ranks.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MsRSB basis build + PCG/GMRES solve s to 1e-8, HBM GB/s; mixed vs FP64 GPU"
WORKLOAD = "3D Darcy 64^3 MPFA-O 27-point, ln k GRF (l=8, sigma=3), 10:1 aniso rot (20,35,0), corner wells, H=8^3"
WORKLOAD_C3 = ("3D linear elasticity, Q1 hexahedra 48^3 (352,947 dofs, 3x3 BSR), ln E GRF (l=6, sigma=1) around "
               "ln 1e10, nu ~ U(0.2, 0.35), bottom fixed, unit traction on top, H=6^3 elements, PCG + block GS")
WORKLOAD_C5 = ("3D Darcy 128^3 MPFA-O 27-point, ln k GRF (l=8, sigma=2), 10:1 aniso rot (20,35,0), corner wells, "
               "H=8^3 (4096 coarse nodes), GMRES + ILU(0)")
CFG_STEPS, CFG_WARMUP = 3, 3
N_GRID, H_BLOCK, SEED = 64, 8, 1002
RTOL, MAXIT = 1e-8, 300
ENS_MAXIT = 2000  # ensemble solves: random right-hand sides may need several GMRES(200) cycles
BASIS = dict(tol=1e-3, n_it=10, max_iter=100)
PHASES = ("partition", "filter_basis", "galerkin", "coarse_inverse", "workspace", "smoother_wait",
          "smoother_setup_side_stream")


def make_problem():
    from synth.darcy import darcy_3d_case
    return darcy_3d_case(n=N_GRID, H=H_BLOCK, seed=SEED)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def max_over_ranks(values, device):
    """Elementwise maximum of `values` over the ranks of the initialised
    process group (every rank gets it): a run is as slow as its slowest rank."""
    import torch
    t = torch.tensor(values, device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t]


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nme, v in zip(names, parts[2:6]):
                if v.lower().startswith("active"):
                    reasons.add(nme)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def smooth_bytes(n, nnz_hat, W, esize):
    """Algorithmic bytes of one restricted-smoothing pass: the entries of the
    filtered operator that the pass needs (value + packed column each), P read
    once and written once, the per-row scale and slot mask."""
    return nnz_hat * (esize + 4) + n * (2 * W * esize + esize + 1)


def kept_entries(c, ids, comp=None):
    """Entries of the filtered operator a restricted-smoothing pass needs
    (Alg. 1 with the filter of Eq. 8): every diagonal, and every negative
    off-diagonal a_ik (the filter zeroes the positive ones) whose row k holds
    one of row i's coarse nodes in the same slot. ids: P's slot ids [n][W].
    comp: component of a 3x3-block operator (its SDC block, Eq. 20).
    Returns (kept entries, coarse-slot matches over the kept off-diagonals =
    the multiply-adds of A_hat P on P's pattern)."""
    ip, ix = np.asarray(c["indptr"]), np.asarray(c["indices"])
    a = np.asarray(c["data"])
    if comp is not None:
        a = a.reshape(-1, 3, 3)[:, comp, comp]
    n = len(ip) - 1
    r = np.repeat(np.arange(n), np.diff(ip))
    off = (ix != r) & (a < 0)
    ri, ki = r[off], ix[off]
    share = np.zeros(len(ri), dtype=bool)
    matches = 0
    for s in range(ids.shape[1]):
        m = (ids[ri, s] >= 0) & (ids[ri, s] == ids[ki, s])
        share |= m
        matches += int(m.sum())
    return n + int(share.sum()), matches


# DRAM bytes (read + write) per launch of the FP32 smoothing pass, per
# workload and launch shape (the autotuner's variant index), from one ncu
# capture of one launch (caches flushed, as ncu does), keyed by a hash of the
# kernels' source file at the time of the capture; once the source changes, or
# the tuner settles on another shape, the figure no longer describes the
# kernel that ran and the bench reports null.
SMOOTH_TRAFFIC = {
    ("darcy64", 0): ("de0b0da3234c1a41", 40152320 + 13824),
    ("darcy64", 4): ("de0b0da3234c1a41", 40152576 + 40704),
    ("darcy64", 5): ("de0b0da3234c1a41", 40155136 + 39424),
    ("darcy128", 4): ("de0b0da3234c1a41", 317593600 + 52034560),
    ("darcy128", 5): ("de0b0da3234c1a41", 317522688 + 51706624),
}
# the autotuner's shapes (lanes per row, threads, entries loaded ahead,
# registers capped)
SMOOTH_SHAPES = [(1, 256, 0, 0), (1, 128, 0, 0), (2, 256, 0, 0), (1, 256, 2, 0), (1, 256, 2, 1), (1, 256, 3, 1)]


def source_hash(name):
    import hashlib
    with open(os.path.join(ROOT, "paper_1912_06934_gb300", "csrc", name), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def smooth_traffic(workload, variant):
    h, traffic = SMOOTH_TRAFFIC.get((workload, variant), (None, None))
    return traffic if traffic is not None and source_hash("basis.cu") == h else None


def smooth_shape(M, n, W, esize):
    """The launch shape the autotuner settled on for this size class (None
    before any tuned loop of it ran)."""
    nl = math.ceil(math.log2(max(n, 1)))
    for t in M.msrsb_tune_table():
        if t["value_bytes"] == esize and t["W"] == W and t["n_log2"] == nl:
            ty = "float" if esize == 4 else "double"
            lanes, thr, ahead, cap = SMOOTH_SHAPES[t["variant"]]
            if lanes > 1:
                kern = "smooth_lanes_kernel<%s,%d,%d>" % (ty, W, lanes)
            elif ahead:
                kern = "smooth_pf_kernel<%s,%d,%d,%s>" % (ty, W, ahead, "true" if cap else "false")
            else:
                kern = "smooth_kernel<%s,%d>" % (ty, W)
            return {"variant": t["variant"], "kernel": kern, "lanes_per_row": lanes, "threads": thr,
                    "entries_ahead": ahead, "registers_capped": bool(cap), "trial_us": t["us"]}
    return None


def apply_bytes(n, nnz, nnz_p, nc, W, coarse_bytes=None):
    """Algorithmic bytes of one mixed-form two-stage apply on a scalar
    operator (Alg. 3 with no pre-smoother, one ILU(0) post-sweep), each array
    counted once: restriction P^T v (P^T pattern row index, P value, v: 4 + 4 +
    4 per entry of P), coarse solve (dense FP64 inverse n_c^2 * 8 unless given),
    prolongation P w_c (ids + values n*W*(4 + 4), z written n*8), residual
    v - A z in FP32 (column + value per nonzero, z read 8, v 4, r written 4
    per row), and the two triangular sweeps of ILU(0) (column + value per
    factor nonzero; the factors fill A's pattern; r, y, reciprocal diagonal
    and z per row 24)."""
    restrict = nnz_p * 12
    coarse = nc * nc * 8 if coarse_bytes is None else coarse_bytes
    prolong = n * W * 8 + n * 8
    resid = nnz * 8 + n * 16
    ilu = nnz * 8 + n * 24
    return restrict + coarse + prolong + resid + ilu


def apply_bytes_elastic(n, nnzb, nnz_p, nC, W, e, coarse_bytes=None):
    """Algorithmic bytes of one two-stage apply on a 3x3-block operator
    (forward block Gauss-Seidel pre-sweep, coarse correction of v - A z,
    backward block Gauss-Seidel post-sweep; Alg. 4), each array counted once
    per stage, smoother values in e bytes (4 mixed, 8 FP64): every Gauss-Seidel
    colour reads each row's whole block row, so each sweep and each residual
    reads A's blocks once (9e + 4 bytes per block); per node the sweeps read
    the inverse diagonal block 9e and r 3e and write e 3e and z 3*8; the
    residuals read z and v (3*8 each) and write r 3e; the restriction reads
    P^T's row index and three values per entry of P's pattern; the coarse
    solve the dense FP64 inverse unless given; the prolongation P's ids and
    three value families and updates z (3*16 per node)."""
    n3 = 3 * n
    blk = nnzb * (9 * e + 4)
    sweep = blk + n * (9 * e + 3 * e + 3 * e + 24)
    resid = blk + n3 * (16 + e)
    restrict = nnz_p * (4 + 3 * e) + n3 * e
    coarse = nC * nC * 8 if coarse_bytes is None else coarse_bytes
    prolong = n * W * (4 + 3 * e) + n3 * 16
    return n3 * (8 + e) + 2 * sweep + 2 * resid + restrict + coarse + prolong


DENSE_COARSE_MAX = 1024  # coarse systems up to this size are applied through an explicit inverse


def coarse_geometry(c):
    """Coarse nodes per axis, block size, nodes per plane and planes of a
    workload's coarse grid (planes along the last axis)."""
    dims, H = c["dims"], c["H"]
    if c["centering"] == 0:
        nb = [-(-d // h) for d, h in zip(dims, H)]
    else:
        nb = [-(-(d - 1) // h) + 1 for d, h in zip(dims, H)]
    bd = c["ncomp"]
    pn = int(np.prod(nb[:-1]))
    return nb, bd, pn * bd, nb[-1]


def coarse_apply_bytes(c):
    """Bytes one coarse solve reads: the dense inverse (n_C <= 1024), or the
    plane factors X_k, G_k of the 2 n_planes - 1 dependent products plus the
    lower couplings of the stencil (9 in-plane offsets x bd^2 per node)."""
    nb, bd, m, npl = coarse_geometry(c)
    nC = int(np.prod(nb)) * bd
    if nC <= DENSE_COARSE_MAX:
        return nC * nC * 8
    return (2 * npl - 1) * m * m * 8 + int(np.prod(nb)) * 9 * bd * bd * 8


def coarse_factor_fmas(c):
    """Multiply-adds of the coarse factorisation over planes: per plane the
    Gauss-Jordan inverse m^3 and the two sparse couplings 2 m^2 9 bd; plus the
    explicit inverse from the factors when n_C <= 1024 (2 n_planes m^2 n_C)."""
    nb, bd, m, npl = coarse_geometry(c)
    nC = int(np.prod(nb)) * bd
    f = npl * (m ** 3 + 2 * m * m * 9 * bd)
    if nC <= DENSE_COARSE_MAX:
        f += 2 * npl * m * m * nC
    return float(f)


def fma_peaks(M):
    """Measured FMA rates (FMAs/s) of the FP64 and FP32 pipes, by the
    library's probe kernel (best of 5 event-timed launches)."""
    f64, _ = M.msrsb_fma_rate(M.msrsb.MSRSB_F64, 8)
    f32, _ = M.msrsb_fma_rate(M.msrsb.MSRSB_F32, 32)
    return {"fp64_fma_per_s": f64, "fp32_fma_per_s": f32, "fp64_gflops": 2 * f64 / 1e9,
            "fp32_gflops": 2 * f32 / 1e9, "how": "msrsb_fma_rate: 8 independent FMA chains x 2048 per thread, "
            "8 (FP64) / 32 (FP32) CTAs of 256 per SM, best of 5, CUDA events"}


class Runner:
    """Set-up + solve steps of one workload in both forms, event-timed on the
    current stream with L2 flushed before every step."""

    def __init__(self, M, c, kind, flush, stream, dev):
        self.M, self.c, self.kind, self.flush, self.stream, self.dev = M, c, kind, flush, stream, dev
        B = M.msrsb
        if kind == "elastic":
            self.A = M.Mat.from_host(c["indptr"], c["indices"], c["data"], bdim=3, device=dev)
            self.g = M.grid(c["dims"], c["H"], centering=1, ncomp=3)
            self.kw = dict(smoother=B.MSRSB_SMOOTH_GS, pre=1, post=1, krylov=B.MSRSB_PCG)
            self.maxit = 500
        else:
            self.A = M.Mat.from_host(c["indptr"], c["indices"], c["data"], device=dev)
            self.g = M.grid(c["dims"], c["H"])
            self.kw = {}
            self.maxit = MAXIT
        self.b = torch_as(c["b"], dev)

    def opts(self, prec, **basis):
        b = dict(BASIS)
        b.update(basis)
        return self.M.opts(prec=prec, **b, **self.kw)

    def step(self, prec):
        import torch
        M = self.M
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(self.stream)
        h = M.msrsb_setup(self.A, self.g, self.opts(prec))
        e[1].record(self.stream)
        r = h.solve(self.b, rtol=RTOL, maxit=self.maxit)
        e[2].record(self.stream)
        info = h.info()
        h.destroy()
        torch.cuda.synchronize()
        info["setup_ms"] = e[0].elapsed_time(e[1])
        info["solve_ms"] = e[1].elapsed_time(e[2])
        return r, info

    def timed(self, prec, k):
        import torch
        ms, last = [], None
        for _ in range(k):
            self.flush.zero_()  # evict L2 between steps (not timed)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            last = self.step(prec)
            e1.record(self.stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms, last

    def form(self, prec, steps):
        """Timed steps of one form with profiling on: per-step times, the last
        step's results, launches and the smoothing loops' time."""
        M = self.M
        M.msrsb_profile(True)
        ms, (r, inf) = self.timed(prec, steps)
        launches, sm_l, sm_ms = M.msrsb_profile_read()
        M.msrsb_profile(False)
        return {"ms": ms, "r": r, "info": inf, "launches": launches, "smooth_launches": sm_l, "smooth_ms": sm_ms}

    def apply_time(self, prec, reps=20):
        """Median time of one preconditioner application with L2 flushed
        before each (CUDA events), and the handle's pattern for byte counts."""
        import torch
        h = self.M.msrsb_setup(self.A, self.g, self.opts(prec))
        p_ids = h.get_setup()[0]
        v = torch.randn(self.b.numel(), dtype=torch.float64, device=self.dev,
                        generator=torch.Generator(device=self.dev).manual_seed(7))
        z = torch.empty_like(v)
        for _ in range(3):
            h.apply(v, z)
        ts = []
        for _ in range(reps):
            self.flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            h.apply(v, z)
            e1.record(self.stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        info = h.info()
        h.destroy()
        return statistics.median(ts), p_ids, info


def torch_as(a, dev):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device=dev)


def form_summary(f, steps):
    r, inf = f["r"], f["info"]
    return {"ms_per_step": sum(f["ms"]) / steps, "ms_steps": [float(x) for x in f["ms"]],
            "basis_iters": inf["basis_iters"], "krylov_iters": r["iters"],
            "relres": r["relres"], "setup_ms": inf["setup_ms"], "solve_ms": inf["solve_ms"],
            "setup_phase_ms": dict(zip(PHASES, inf["phase_ms"])), "launches_per_step": f["launches"] / steps,
            "smooth_us_per_launch": f["smooth_ms"] / f["smooth_launches"] * 1e3 if f["smooth_launches"] else None}


def smooth_roofline(f, n, W, nnz_hat_list, esize, hbm, peak_kind, traffic=None):
    """HBM roofline of the restricted-smoothing kernel from the profiled
    loops: algorithmic bytes per pass (mean over the basis families, which
    run the same number of passes here) / mean event-timed pass; `traffic`
    the captured DRAM bytes per launch (or None)."""
    if not f["smooth_launches"]:
        return None
    per = float(np.mean([smooth_bytes(n, k, W, esize) for k in nnz_hat_list]))
    us = f["smooth_ms"] / f["smooth_launches"] * 1e3
    ach = per / (us * 1e-6) / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "bytes_per_launch": per, "us_per_launch": us, "launches": f["smooth_launches"], "traffic": traffic,
            "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)"}


def run_extra_config(M, name, c, kind, flush, stream, dev, steps, warmup, hbm, peak_kind, peaks_fma):
    """Both forms of one further workload (set-up + solve, then the apply on
    its own), with the smoothing and apply rooflines of each form."""
    R = Runner(M, c, kind, flush, stream, dev)
    B = M.msrsb
    out = {}
    for _ in range(warmup):
        R.step(B.MSRSB_F32)
        R.step(B.MSRSB_F64)
    forms = {}
    for label, pr in (("mixed", B.MSRSB_F32), ("fp64", B.MSRSB_F64)):
        forms[label] = R.form(pr, steps)
    n = len(c["indptr"]) - 1
    nnzb = len(c["indices"])
    for label, pr in (("mixed", B.MSRSB_F32), ("fp64", B.MSRSB_F64)):
        f = forms[label]
        out[label] = form_summary(f, steps)
        ap_ms, p_ids, info = R.apply_time(pr)
        ids = p_ids.cpu().numpy()
        W = ids.shape[1]
        nnz_p = int((ids >= 0).sum())
        e = 4 if pr == B.MSRSB_F32 else 8
        if kind == "elastic":
            kept = [kept_entries(c, ids, comp=l) for l in range(3)]
            ab = apply_bytes_elastic(n, nnzb, nnz_p, info["nc"] * 3, W, e, coarse_apply_bytes(c))
        else:
            kept = [kept_entries(c, ids)]
            ab = apply_bytes(n, nnzb, nnz_p, info["nc"], W, coarse_apply_bytes(c)) if e == 4 else None
        shape = smooth_shape(M, n, W, e)
        out[label]["smooth_roofline"] = smooth_roofline(
            f, n, W, [k[0] for k in kept], e, hbm, peak_kind,
            smooth_traffic(name, shape["variant"]) if label == "mixed" and shape else None)
        if out[label]["smooth_roofline"] is not None:
            out[label]["smooth_roofline"]["launch_shape"] = shape
        if e == 8 and f["smooth_launches"]:
            # the FP64 pass is bound by the FP64 pipe: multiply-adds of A_hat P
            # on the pattern plus the W-wide update per row
            fmas = float(np.mean([k[1] for k in kept])) + n * W
            rate = fmas / (f["smooth_ms"] / f["smooth_launches"] * 1e-3)
            out[label]["smooth_fp64_pipe"] = {"bound": "fp64", "fma_per_launch": fmas, "achieved_fma_per_s": rate,
                                              "peak_fma_per_s": peaks_fma["fp64_fma_per_s"],
                                              "frac": rate / peaks_fma["fp64_fma_per_s"]}
        out[label]["apply_us"] = ap_ms * 1e3
        ci_ms = f["info"]["phase_ms"][3]
        cf = coarse_factor_fmas(c)
        out[label]["coarse_fp64_pipe"] = {"fmas": cf, "ms": ci_ms,
                                          "achieved_fma_per_s": cf / (ci_ms * 1e-3) if ci_ms else None,
                                          "frac": cf / (ci_ms * 1e-3) / peaks_fma["fp64_fma_per_s"] if ci_ms else None}
        if ab is not None:
            out[label]["apply_roofline"] = {"bound": "hbm", "achieved": ab / (ap_ms * 1e-3) / 1e9, "peak": hbm,
                                            "unit": "GB/s", "frac": ab / (ap_ms * 1e-3) / 1e9 / hbm,
                                            "bytes_per_apply": ab, "l2": "flushed before each apply"}
    out["speedup_mixed_vs_fp64"] = out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"]
    out["steps"], out["warmup"] = steps, warmup
    return out


def device_case(M, n, seed, sigma):
    """The 3D Darcy case (27-point MPFA-O, GRF ln k with correlation length 8
    and the given sigma, rotated 10:1 anisotropy, corner wells, 8^3 blocks)
    assembled on the device by msrsb_mpfa_assemble (the same operator as the
    host generator builds, far faster at 128^3), returned as host arrays."""
    import torch
    from synth.darcy import darcy_3d_field, pattern27
    dims = (n, n, n)
    theta, K_hat, wells = darcy_3d_field(dims, seed, sigma=sigma)
    ip, ix = pattern27(dims)
    g = M.grid(dims, (H_BLOCK,) * 3)
    val, b = M.msrsb.msrsb_mpfa_assemble(g, torch.as_tensor(K_hat, device="cuda"), torch.as_tensor(theta, device="cuda"),
                                         wells, torch.as_tensor(ip, device="cuda"), torch.as_tensor(ix, device="cuda"))
    return dict(indptr=ip, indices=ix, data=val.cpu().numpy(), b=b.cpu().numpy(), dims=dims, H=(H_BLOCK,) * 3,
                centering=0, ncomp=1)


def gpu_arm(args, rank, world):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1912_06934_gb300 as M
    B = M.msrsb

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    c = make_problem()
    n, nnz = len(c["indptr"]) - 1, len(c["indices"])
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream()
    R = Runner(M, c, "scalar", flush, stream, dev)
    A, g, b = R.A, R.g, R.b

    for _ in range(args.warmup):
        R.step(B.MSRSB_F32)
        R.step(B.MSRSB_F64)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        f32 = R.form(B.MSRSB_F32, args.steps)
        f64 = R.form(B.MSRSB_F64, args.steps)
    torch.cuda.synchronize()
    t32, t64 = sum(f32["ms"]), sum(f64["ms"])
    if world > 1:
        t32, t64 = max_over_ranks([t32, t64], dev)
    inf32, inf64 = f32["info"], f64["info"]

    # results of both forms on the same input, kept for the error against the
    # FP64 form and against the oracle (not timed): P, A_c, one apply, x
    vprobe_h = np.random.default_rng(11).standard_normal(n)
    vprobe = torch_as(vprobe_h, dev)
    res = {}
    for label, pr in (("fp64", B.MSRSB_F64), ("mixed", B.MSRSB_F32)):
        h = M.msrsb_setup(A, g, R.opts(pr))
        p_ids, P, Ac = h.get_setup()
        z = h.apply(vprobe)
        x = h.solve(b, rtol=RTOL, maxit=MAXIT)["x"]
        res[label] = {"p_ids": p_ids.cpu().numpy(), "P": P[0].double().cpu().numpy(), "Ac": Ac.cpu().numpy(),
                      "z": z.cpu().numpy(), "x": x.cpu().numpy()}
        h.destroy()
    r64, r32 = res["fp64"], res["mixed"]
    mixed_err = {
        "P_max_abs": float(np.abs(r32["P"] - r64["P"]).max()),
        "Ac_rel": float(np.linalg.norm(r32["Ac"] - r64["Ac"]) / np.linalg.norm(r64["Ac"])),
        "apply_rel": float(np.linalg.norm(r32["z"] - r64["z"]) / np.linalg.norm(r64["z"])),
        "x_rel": float(np.linalg.norm(r32["x"] - r64["x"]) / np.linalg.norm(r64["x"])),
        "what": "mixed-form result against the FP64 form on the same input (both GPU)",
    }

    # two-stage apply on its own: L2 flushed before every apply, event-timed
    ap_med, p_ids, _ = R.apply_time(B.MSRSB_F32)
    ids = p_ids.cpu().numpy()
    nnz_p = int((ids >= 0).sum())
    nnz_hat, matches = kept_entries(c, ids)
    ap_bytes = apply_bytes(n, nnz, nnz_p, inf32["nc"], 8, coarse_apply_bytes(c))

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    ip = torch.as_tensor(np.asarray(c["indptr"], dtype=np.int32)).pin_memory()
    ix = torch.as_tensor(np.asarray(c["indices"], dtype=np.int32)).pin_memory()
    dv = torch.as_tensor(np.asarray(c["data"], dtype=np.float64)).pin_memory()
    bh = torch.as_tensor(c["b"]).pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    o32 = R.opts(B.MSRSB_F32)
    e2e_t = []
    for k in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.msrsb_solve_host_ptrs(ip, ix, dv, 1, g, o32, bh, xh, RTOL, MAXIT)
        torch.cuda.synchronize()
        if k >= args.warmup:
            e2e_t.append(time.perf_counter() - t0)
    resid = np.linalg.norm(c["b"] - _spmv(c, xh.numpy())) / np.linalg.norm(c["b"])
    h2d = 4 * (n + 1) + 4 * nnz + 8 * nnz + 8 * n
    d2h = 8 * n

    hbm, peak_kind = peaks()
    pk = fma_peaks(M)
    W = 8
    per_launch32 = smooth_bytes(n, nnz_hat, W, 4)
    sm_l32, sm_ms32 = f32["smooth_launches"], f32["smooth_ms"]
    sm_l64, sm_ms64 = f64["smooth_launches"], f64["smooth_ms"]
    achieved = per_launch32 / (sm_ms32 / sm_l32 * 1e-3) / 1e9 if sm_l32 else None
    per_launch64 = smooth_bytes(n, nnz_hat, W, 8)
    achieved64 = per_launch64 / (sm_ms64 / sm_l64 * 1e-3) / 1e9 if sm_l64 else None
    fma64 = matches + n * W
    coarse_fmas = coarse_factor_fmas(c)
    mixed = form_summary(f32, args.steps)
    fp64 = form_summary(f64, args.steps)
    fp64["smooth_kernel_gbs"] = achieved64
    fp64["smooth_fp64_pipe"] = {
        "bound": "fp64", "fma_per_launch": fma64,
        "achieved_fma_per_s": fma64 / (sm_ms64 / sm_l64 * 1e-3) if sm_l64 else None,
        "peak_fma_per_s": pk["fp64_fma_per_s"],
        "frac": fma64 / (sm_ms64 / sm_l64 * 1e-3) / pk["fp64_fma_per_s"] if sm_l64 else None}
    ci_ms = inf64["phase_ms"][3]
    fp64["coarse_fp64_pipe"] = {"op": "coarse factorisation over planes (+ explicit inverse when n_C <= 1024)",
                                "fmas": coarse_fmas,
                                "achieved_fma_per_s": coarse_fmas / (ci_ms * 1e-3) if ci_ms else None,
                                "frac": coarse_fmas / (ci_ms * 1e-3) / pk["fp64_fma_per_s"] if ci_ms else None}
    shape64 = smooth_shape(M, n, 8, 4)  # the FP32 pass's tuned shape for this size class
    out = {
        "metric": METRIC,
        "value": t32 / args.steps / 1e3,
        "unit": "s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t32 / args.steps,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_cells": n, "nnz": nnz, "coarse_nodes": inf32["nc"],
                   "basis": "omega=2/3 tol=1e-3 n_it=10 max_iter=100", "krylov": "GMRES(200) right, ILU(0) post",
                   "rtol": RTOL, "l2": "flushed between steps (512 MB write)", "parallelism": "replicas"},
        "mixed": mixed,
        "fp64": fp64,
        "speedup_mixed_vs_fp64": t64 / t32,
        "mixed_error_vs_fp64": mixed_err,
        "roofline": {"kernel": (shape64["kernel"] if shape64 else "smooth_kernel<float,8>")
                     + " (restricted smoothing, Alg. 1)", "bound": "hbm", "launch_shape": shape64,
                     "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm if achieved else None,
                     "traffic": smooth_traffic("darcy64", shape64["variant"]) if shape64 else None,
                     "bytes_per_launch": per_launch32, "filtered_entries": nnz_hat, "launches": sm_l32,
                     "us_per_launch": sm_ms32 / sm_l32 * 1e3 if sm_l32 else None,
                     "l2_resident": "the kept operator (28 MB) and both P buffers stay in L2 across the passes "
                                    "at 64^3; the HBM-bound cases are under configs",
                     "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs, burst copy)"},
        "apply_roofline": {"op": "two-stage apply (Alg. 3), mixed form, L2 flushed before each", "bound": "hbm",
                           "achieved": ap_bytes / (ap_med * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                           "frac": ap_bytes / (ap_med * 1e-3) / 1e9 / hbm, "bytes_per_apply": ap_bytes,
                           "us_per_apply": ap_med * 1e3},
        "peaks": dict(pk, hbm_gbs=hbm, hbm_source=peak_kind),
        "e2e": {"value": statistics.median(e2e_t) if e2e_t else None, "unit": "s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "relres": float(resid), "call": "msrsb_solve_host (pinned host buffers)"},
        "gpu_launches": int(f32["launches"] + f64["launches"]),
        "clocks": clk.summary(),
    }
    if not args.no_configs:
        from synth.elastic import elastic_3d_case
        from synth.darcy import darcy_3d_case
        cfg = {}
        c3 = elastic_3d_case(ne=48, H=6)
        cfg["elastic48"] = dict(workload=WORKLOAD_C3, **run_extra_config(
            M, "elastic48", c3, "elastic", flush, stream, dev, CFG_STEPS, CFG_WARMUP, hbm, peak_kind, pk))
        del c3
        c5 = device_case(M, 128, 1005, 2.0)
        cfg["darcy128"] = dict(workload=WORKLOAD_C5, **run_extra_config(
            M, "darcy128", c5, "scalar", flush, stream, dev, CFG_STEPS, CFG_WARMUP, hbm, peak_kind, pk))
        del c5
        # the batched ensemble (64 realisations, edges from {32, ..., 96}, 8
        # right-hand sides each): one warm-up and one timed pass at concurrency 6
        ens_edges = [32, 48, 64, 80, 96]
        probs, sizes, rows, nnz = ensemble_members(M, 64, ens_edges)
        cfg["ensemble_c4"] = dict(workload=ensemble_workload(64, ens_edges, sizes, rows, nnz), concurrency=6,
                                  **ensemble_time(M, probs, 6, 1))
        del probs
        out["configs"] = cfg
    # the launch shapes the smoothing passes settled on, per size class (timed
    # in the warm-up steps; "us" = each shape's best trial pass)
    out["autotune"] = M.msrsb_tune_table()
    if rank == 0 and not args.no_cpu_baseline:
        out["_oracle_inputs"] = (c, vprobe_h, res)
    return out


def _csr(c):
    import scipy.sparse as sp
    return sp.csr_matrix((c["data"], c["indices"], c["indptr"]))


def _spmv(c, x):
    return _csr(c) @ x


def oracle_step(c, vprobe=None):
    """One full run of the FP64 oracle on the workload, timed by phase:
    set-up (partition, filter, Alg. 1 to tol 1e-3 / 100 passes, Galerkin,
    coarse LU, colour-ordered ILU(0)) and the right-preconditioned GMRES solve
    to 1e-8. Returns (seconds by phase, results)."""
    import scipy.sparse as sp
    from oracle import msrsb as O
    A = sp.csr_matrix((c["data"], c["indices"], c["indptr"]))
    A.sort_indices()
    t0 = time.perf_counter()
    s = O.setup_scalar(A, c["dims"], c["H"], **BASIS)
    t1 = time.perf_counter()
    x, its, rr, _ = O.gmres_right(A, c["b"], s["tl"].apply, rtol=RTOL, maxit=MAXIT)
    t2 = time.perf_counter()
    out = {"setup_s": t1 - t0, "solve_s": t2 - t1, "total_s": t2 - t0, "basis_iters": s["iters"],
           "krylov_iters": its, "relres": rr}
    res = None
    if vprobe is not None:
        res = {"s": s, "x": x, "z": s["tl"].apply(vprobe)}
    return out, res


# workloads the oracle can be timed on: the 2D 64^2 case (MPFA-O 9-point,
# seed 1001) and the 64^3 benchmark workload
ORACLE_WORKLOADS = {
    "darcy2d64": lambda: __import__("synth.darcy", fromlist=["darcy_2d_case"]).darcy_2d_case(n=64, H=8, seed=1001),
    "darcy64": lambda: make_problem(),
}


def _oracle_subprocess(threads, workload="darcy64"):
    """The oracle step in a fresh process whose BLAS pools use `threads`
    threads (their size is fixed when numpy loads)."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = str(threads)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--oracle-step",
                        "--oracle-workload", workload], env=env, capture_output=True, text=True, timeout=1200)
    if r.returncode != 0:
        return {"error": r.stderr[-500:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


def _errors(res, ores, nc):
    """Errors of one GPU form's results against the oracle's: P (max-abs on
    the pattern), A_c (relative, Frobenius), one apply on the probe vector
    and the solution (relative, 2-norm)."""
    import scipy.sparse as sp
    ids = res["p_ids"]
    rows, slots = np.nonzero(ids >= 0)
    Pg = sp.csr_matrix((res["P"][rows, slots], (rows, ids[rows, slots])), shape=(ids.shape[0], nc))
    s = ores["s"]
    Ac_o = s["tl"].Ac.toarray()
    return {"P_max_abs": float(abs(Pg - s["P"]).max()),
            "Ac_rel": float(np.linalg.norm(res["Ac"] - Ac_o) / np.linalg.norm(Ac_o)),
            "apply_rel": float(np.linalg.norm(res["z"] - ores["z"]) / np.linalg.norm(ores["z"])),
            "x_rel": float(np.linalg.norm(res["x"] - ores["x"]) / np.linalg.norm(ores["x"]))}


def finish_cpu(out):
    """cpu_baseline leg (rank 0): the FP64 oracle as it stands, one full
    set-up + solve of the workload with 1 BLAS thread (in this process) and
    with every host core (a fresh process); and the error of each GPU form
    against the oracle's results on the same input."""
    inputs = out.pop("_oracle_inputs", None)
    if inputs is None:
        return
    c, vprobe, res = inputs
    t1, ores = oracle_step(c, vprobe)
    ncores = os.cpu_count() or 1
    tall = _oracle_subprocess(ncores)
    best = t1["total_s"]
    cores = 1
    if "total_s" in tall and tall["total_s"] < best:
        best, cores = tall["total_s"], ncores
    out["cpu_baseline"] = {
        "value": best, "unit": "s", "cores": cores, "kind": "oracle",
        "sample": "one full FP64 oracle set-up + GMRES solve of the 64^3 workload per thread count (no "
                  "extrapolation); value = the faster of 1 BLAS thread and %d (scipy's sparse kernels are "
                  "single-threaded either way)" % ncores,
        "one_thread": t1, "all_cores": dict(tall, threads=ncores)}
    nc = out["config"]["coarse_nodes"]
    out["mixed_error_vs_oracle"] = dict(_errors(res["mixed"], ores, nc),
                                        what="mixed-form GPU result against the FP64 oracle on the same input "
                                             "(P max-abs, A_c Frobenius-relative, one apply and the solution "
                                             "2-norm-relative; both solves stop at relative residual 1e-8)")
    out["fp64_error_vs_oracle"] = _errors(res["fp64"], ores, nc)


def reference_arm(args, rank, world):
    """The oracle as the reference implementation: every step is one full
    FP64 oracle set-up + GMRES solve of the workload (1 BLAS thread); the
    median over the timed steps is the value."""
    if rank != 0:
        return None
    c = make_problem()
    vals, last = [], None
    for k in range(args.warmup + args.steps):
        t, _ = oracle_step(c)
        if k >= args.warmup:
            vals.append(t["total_s"])
            last = t
    v = statistics.median(vals)
    sample = ("every step one full FP64 oracle set-up (%d Alg. 1 passes) + GMRES solve (%d iterations) of the "
              "64^3 workload, 1 thread; median of %d steps after %d warm-up steps"
              % (last["basis_iters"], last["krylov_iters"], args.steps, args.warmup))
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "parallelism": "replicas"},
            "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle", "sample": sample},
            "oracle_phases_s": {"setup": last["setup_s"], "solve": last["solve_s"]},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def profile_run(args):
    """Workloads for profilers (no timing output): 'solve' runs the mixed
    set-up + GMRES solve twice; 'basis' runs three restricted smoothing passes
    (FP32) twice; on an N^3 grid (N = --grid; N = 64 is the benchmark's
    operator, N = 128 the 128^3 configuration's, any other N the benchmark's
    generator at that size); --shape forces the smoothing pass's launch shape."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1912_06934_gb300 as M
    from synth.darcy import darcy_3d_case
    if args.grid == N_GRID:
        c = make_problem()
    elif args.grid == 128:
        c = device_case(M, 128, 1005, 2.0)  # the 128^3 configuration's operator
    else:
        c = darcy_3d_case(n=args.grid, H=H_BLOCK, seed=SEED)
    A = M.Mat.from_host(c["indptr"], c["indices"], c["data"])
    g = M.grid(c["dims"], c["H"])
    if args.shape is not None:
        M.msrsb_tune_mode(args.shape)
    if args.profile == "solve":
        b = torch.as_tensor(c["b"], device="cuda")
        o = M.opts(prec=M.msrsb.MSRSB_F32, **BASIS)
        for _ in range(2):
            h = M.msrsb_setup(A, g, o)
            r = h.solve(b, rtol=RTOL, maxit=MAXIT)
            h.destroy()
        torch.cuda.synchronize()
        print("profile solve: iters %d relres %.3e" % (r["iters"], r["relres"]))
    else:
        ahat, _ = M.msrsb_filter(A)
        Ah = M.Mat(A.rowptr, A.colidx, ahat)
        part, cnode, p_ids, skel = M.msrsb_partition(g)
        P0 = ((p_ids >= 0) & (p_ids == part[:, None].to(torch.int32))).to(torch.float32).contiguous()
        for _ in range(2):
            P = P0.clone()
            it, e = M.msrsb_build_basis(Ah, p_ids, skel, p_ids.shape[1], M.basis_opts(tol=0.0, max_iter=3),
                                        M.msrsb.MSRSB_F32, P)
        torch.cuda.synchronize()
        print("profile basis: n %d passes %d e_it %.4f" % (c["indptr"].shape[0] - 1, it, e))


def ensemble_members(M, R, edges):
    """The batched-ensemble workload: R seeded 3D Darcy realisations (field
    and stencil as the main workload: MPFA-O 27-point, ln k Gaussian random
    field l = 8, sigma = 3, 10:1 anisotropy rotated (20, 35, 0), corner wells;
    grid edges drawn uniformly from `edges` with seed 1004; fields seed
    40000 + r; the operators assembled on the device by msrsb_mpfa_assemble),
    8 right-hand sides b = A xi with xi ~ N(0, 1) each (seed 50000 + r).
    Returns (problems, sizes, rows, nnz)."""
    import torch
    from synth.darcy import darcy_3d_field, pattern27
    rng = np.random.default_rng(1004)
    sizes = [int(rng.choice(edges)) for _ in range(R)]
    nrhs = 8
    probs, rows, nnz_tot = [], 0, 0
    for r, e in enumerate(sizes):
        dims = (e, e, e)
        theta, K_hat, wells = darcy_3d_field(dims, 40000 + r)
        ip, ix = pattern27(dims)
        rowptr = torch.as_tensor(ip, device="cuda")
        colidx = torch.as_tensor(ix, device="cuda")
        g = M.grid(dims, (H_BLOCK,) * 3)
        val, _ = M.msrsb.msrsb_mpfa_assemble(g, torch.as_tensor(K_hat, device="cuda"),
                                             torch.as_tensor(theta, device="cuda"), wells, rowptr, colidx)
        A = M.Mat(rowptr, colidx, val)
        n = len(theta)
        # b = A xi: a raw N(0, 1) b on a sigma = 3 field can sit at FP64's
        # attainable-accuracy floor (~1e-8), in the FP64 form as well
        As = torch.sparse_csr_tensor(rowptr.long(), colidx.long(), val, size=(n, n))
        xi = torch.as_tensor(np.random.default_rng(50000 + r).standard_normal((nrhs, n)), device="cuda")
        B = (As @ xi.T).T.contiguous()
        probs.append((A, g, B, torch.zeros_like(B)))
        rows += n
        nnz_tot += len(ix)
    return probs, sizes, rows, nnz_tot


def ensemble_time(M, probs, conc, passes):
    """Median wall time of `passes` whole-ensemble solves (mixed form, GMRES
    to 1e-8) at concurrency `conc`, after one warm-up; with the iteration
    and residual statistics of the last."""
    import torch
    o = M.opts(prec=M.msrsb.MSRSB_F32, **BASIS)
    M.msrsb_solve_ensemble(probs, o, RTOL, ENS_MAXIT, conc)  # warm-up
    ts = []
    for _ in range(passes):
        for P_ in probs:
            P_[3].zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = M.msrsb_solve_ensemble(probs, o, RTOL, ENS_MAXIT, conc)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    t = statistics.median(ts)
    its = [i for r_ in res for i in r_[0]]
    nrhs = probs[0][2].shape[0] if probs else 0
    return {"s": t, "solves_per_s": len(probs) * nrhs / t, "realisations_per_s": len(probs) / t,
            "mean_iters": float(np.mean(its)), "max_relres": float(max(x for r_ in res for x in r_[1]))}


def ensemble_workload(R, edges, sizes, rows, nnz):
    return ("ensemble of %d 3D Darcy realisations (MPFA-O 27-point, GRF l=8 sigma=3), edges drawn from %s: %s "
            "(rows %d, nnz %d), 8 rhs b = A xi each solved together (msrsb_solve_multi), H=8^3"
            % (R, edges, sizes, rows, nnz))


def ensemble_run(args):
    """Ensemble throughput (msrsb_solve_ensemble) on the batched-ensemble
    workload (ensemble_members), the whole ensemble timed at concurrency 1
    and at --ens-conc. Prints one JSON line."""
    import __graft_entry__
    __graft_entry__.build()
    import paper_1912_06934_gb300 as M
    edges = [int(e) for e in args.ens_edges.split(",")]
    probs, sizes, rows, nnz = ensemble_members(M, args.ens_R, edges)
    out = {conc: ensemble_time(M, probs, conc, 3) for conc in (1, args.ens_conc)}
    line = {"metric": "ensemble: MsRSB set-up + 8 GMRES solves per realisation, realisations per second",
            "value": out[args.ens_conc]["realisations_per_s"], "unit": "realisations/s", "higher_is_better": True,
            "n_gpus": 1, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": ensemble_workload(args.ens_R, edges, sizes, rows, nnz),
                       "concurrency": args.ens_conc},
            "sequential": out[1], "concurrent": out[args.ens_conc],
            "speedup_concurrent_vs_sequential": out[1]["s"] / out[args.ens_conc]["s"],
            "autotune": M.msrsb_tune_table()}
    print(json.dumps(line))


def oracle_timing_run(args):
    """The oracle's own timing (no GPU): for each workload of
    --oracle-workloads and for one thread and every host core,
    --oracle-repeats full runs, each in a fresh process; the best time of each
    phase. Prints one JSON line."""
    cores = os.cpu_count() or 1
    out = {"metric": "FP64 oracle: MsRSB set-up + GMRES solve to 1e-8, seconds (best of %d per phase)"
                     % args.oracle_repeats, "unit": "s", "cores": cores, "workloads": {}}
    for wl in args.oracle_workloads.split(","):
        per = {}
        for threads in sorted({1, cores}):
            runs = [_oracle_subprocess(threads, wl) for _ in range(args.oracle_repeats)]
            ok = [r for r in runs if "error" not in r]
            if not ok:
                per[str(threads)] = {"error": runs[-1].get("error")}
                continue
            per[str(threads)] = {"setup_s": min(r["setup_s"] for r in ok), "solve_s": min(r["solve_s"] for r in ok),
                                 "runs": len(ok), "basis_iters": ok[0]["basis_iters"],
                                 "krylov_iters": ok[0]["krylov_iters"], "relres": ok[0]["relres"]}
        out["workloads"][wl] = per
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="time only the 64^3 workload")
    ap.add_argument("--oracle-step", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--oracle-workload", default="darcy64", choices=sorted(ORACLE_WORKLOADS), help=argparse.SUPPRESS)
    ap.add_argument("--oracle-timing", action="store_true",
                    help="time the FP64 oracle alone: best of --oracle-repeats full set-up + solve runs per phase, "
                         "one thread and every host core, on the 2D 64^2 and 3D 64^3 workloads")
    ap.add_argument("--oracle-repeats", type=int, default=3)
    ap.add_argument("--oracle-workloads", default="darcy2d64,darcy64")
    ap.add_argument("--profile", choices=["solve", "basis"], default=None,
                    help="run a workload for a profiler instead of the benchmark")
    ap.add_argument("--grid", type=int, default=N_GRID, help="grid edge for --profile")
    ap.add_argument("--shape", type=int, default=None,
                    help="for --profile: force this smoothing launch shape (autotuner variant index)")
    ap.add_argument("--ensemble", action="store_true", help="ensemble throughput instead of the benchmark")
    ap.add_argument("--ens-R", type=int, default=64)
    ap.add_argument("--ens-edges", default="32,48,64,80,96")
    ap.add_argument("--ens-conc", type=int, default=6)
    args = ap.parse_args()
    if args.oracle_step:  # cpu_baseline leg in a process of its own (thread count from the environment)
        print(json.dumps(oracle_step(ORACLE_WORKLOADS[args.oracle_workload]())[0]))
        return
    if args.oracle_timing:
        oracle_timing_run(args)
        return
    if args.profile:
        profile_run(args)
        return
    if args.ensemble:
        ensemble_run(args)
        return
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        out = reference_arm(args, rank, world)
        if out is not None:
            print(json.dumps(out))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    out = gpu_arm(args, rank, world)
    if rank == 0:
        finish_cpu(out)
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
