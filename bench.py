"""Benchmark: HODLR3D matrix-vector product time at N = 1,000,000 (uniform points
in [-1,1]^3, Laplace 1/(4 pi r), leaf 128, ACA tolerance 1e-7, one RHS), FP32
factors, with the plain FP64 form timed beside it.

One step = one product y = A~ x through the C ABI (permutation, source-side
gather V^T x, per-leaf near field + U t, inverse permutation) with x already in
HBM.  The factors (~tens of GB) are far larger than L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With --impl reference the CPU oracle's dense
direct sum (O1) is timed on a bounded sample of rows on the host cores and
scaled to a full product.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2307_16303_gb300 import inputs as I  # noqa: E402

METRIC = "HODLR3D matvec ms @N=1M rel.err<=1e-6 (FP32 factors; plain FP64 beside it), %HBM peak"
FALLBACK_HBM_GBS = 6800.0

# dram__bytes_read.sum + dram__bytes_write.sum per launch divided by the launch's
# algorithmic bytes, from one ncu capture of the unchanged kernels on the
# N = 125,000 uniform case (same per-leaf shape as N = 1M; FP32, one right-hand
# side): traffic grows with the factor entries, so a launch's traffic is this
# ratio times its algorithmic bytes.  Kernels without a capture report None.
NCU_TRAFFIC_RATIO: dict = {"k_leaf": 1.052, "k_gather": 1.058}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--N", type=int, default=1_000_000)
    p.add_argument("--leaf", type=int, default=128)
    p.add_argument("--tol", type=float, default=1e-7)
    p.add_argument("--nrhs", type=int, default=1)
    p.add_argument("--seed", type=int, default=3)
    p.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison")
    p.add_argument("--no-symmetric", action="store_true",
                   help="skip the symmetric-storage product (each unordered pair stored once) beside the main line")
    p.add_argument("--rows", type=int, default=10_000, help="sampled rows for the error / CPU baseline")
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="CPU work budget of the baseline leg")
    p.add_argument("--o2-N", type=int, default=262_144,
                   help="points of the oracle's HODLR3D (Alg. 1 + Alg. 2 on the host cores) timed beside the "
                        "dense sum; 0 skips it")
    p.add_argument("--batched", action="store_true",
                   help="time --batch-count independent clouds (N log-uniform in [8192, --batch-nmax], half cube / "
                        "half sphere, Laplace / Yukawa alternating, FP32) as one persistent launch or one graph "
                        "(whichever the tuner picks; both reported) against separate products")
    p.add_argument("--batch-nmax", type=int, default=131072)
    p.add_argument("--batch-storage", default="factors", choices=["factors", "symmetric"],
                   help="storage of the members that fit in device memory (the rest take skeleton storage): "
                        "ordered factors, or symmetric storage (each unordered pair once, fewer bytes)")
    p.add_argument("--batch-count", type=int, default=64, help="clouds in the batch (64: the batched workload)")
    p.add_argument("--batch-reserve-gb", type=float, default=24.0,
                   help="device memory kept free while clouds are built with stored factors; larger clouds then "
                        "take the skeleton storage")
    p.add_argument("--skeleton", action="store_true",
                   help="time the skeleton storage (pivots + LU of K(sigma,tau), entries recomputed in FP64) "
                        "on the same workload")
    p.add_argument("--points", default="uniform", choices=["uniform", "jittered"],
                   help="jittered: the cell-centred grid of round(N^(1/3))^3 points with U(-h/4, h/4) jitter")
    p.add_argument("--forces", action="store_true",
                   help="(the default) time the energy and forces (charges ~ U(-1,1) FP32, pivots frozen) and check "
                        "them against the exact dense forces on 4,096 sampled points")
    p.add_argument("--no-forces", action="store_true", help="skip the energy and forces")
    p.add_argument("--no-wide", action="store_true",
                   help="skip the 32-column product (3xTF32 tensor cores) beside the one-column headline")
    return p.parse_args()


def workload(a):
    return {"workload": f"uniform N={a.N} in [-1,1]^3, Laplace 1/(4 pi r), leaf {a.leaf}, tol {a.tol:g}, "
                        f"nrhs {a.nrhs}, seed {a.seed}",
            "N": a.N, "leaf_size": a.leaf, "tol": a.tol, "nrhs": a.nrhs, "kernel": "laplace",
            "points": "uniform", "x": "N(0,1) fp32, seed 2", "l2": "inputs larger than L2 (factors >> 129 MB)"}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """Sample nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if len(r) > 3 + k and r[3 + k] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def replica_seeds(rank: int, seed: int) -> tuple[int, int]:
    """Seeds of one rank's independent replica (points, right-hand sides): the
    product has no exchange step, so ranks run replicas and share nothing."""
    return seed + 1000 * rank, 2 + 1000 * rank


def max_over_ranks(ms: float, dist, device) -> float:
    """The job's time is the slowest rank's (all_reduce MAX; identity on one rank)."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def time_steps(fn, steps, warmup, torch, dist=None):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(steps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    return e0.elapsed_time(e1) / steps


def cpu_baseline(pts, x64, y_ours, a, budget_s):
    """O1 on sampled rows: timed (scaled to a full product) and used for the error."""
    from oracle import oracle as O
    rows = I.sample_rows(a.N, a.rows, 4)
    # size the sample to the CPU budget with a short probe
    probe = rows[:64]
    t0 = time.perf_counter()
    O.direct_rows(pts, x64, probe)
    tp = time.perf_counter() - t0
    per_row = tp / len(probe)
    S = int(min(len(rows), max(256, budget_s / max(per_row, 1e-9))))
    rows = rows[:S]
    t0 = time.perf_counter()
    ref = O.direct_rows(pts, x64, rows)
    t = time.perf_counter() - t0
    ref = ref if ref.ndim == 2 else ref[:, None]
    yr = y_ours[rows] if y_ours.ndim == 2 else y_ours[rows][:, None]
    err = float(np.linalg.norm(yr - ref) / np.linalg.norm(ref))
    full_ms = t * 1e3 * a.N / S
    return {"value": round(full_ms, 3), "unit": "ms", "cores": O.num_threads(), "kind": "oracle",
            "sample": f"O1 FP64 direct sum on {S} seeded rows of the N={a.N} workload "
                      f"({t:.1f} s), scaled by N/rows to one full dense product"}, err, S, (rows, ref)


def cpu_hodlr3d(a):
    """The oracle's HODLR3D on the host cores: Alg. 1 (tree, lists, ACA pivots) and
    one Alg. 2 product (factors re-formed from the pivots, as the paper does), FP64,
    on uniform points with the workload's leaf size and tolerance."""
    from oracle import oracle as O
    n = a.o2_N
    pts = I.uniform(n, 1)
    x = I.rhs_normal(n, 1, 2)[:, 0]
    t0 = time.perf_counter()
    o = O.Oracle(pts, leaf_size=a.leaf, tol=a.tol).compress()
    tb = time.perf_counter() - t0
    t0 = time.perf_counter()
    o.matvec(x)
    tm = time.perf_counter() - t0
    return {"N": n, "leaf_size": a.leaf, "tol": a.tol, "depth": o.L, "build_s": round(tb, 2),
            "matvec_ms": round(tm * 1e3, 1), "cores": O.num_threads(), "kind": "oracle",
            "sample": f"O2: the oracle's HODLR3D build (Alg. 1) and one product (Alg. 2, factors re-formed from "
                      f"the pivots in the product) on N={n} uniform points, FP64, timed whole (not scaled)"}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    pts = I.uniform(a.N, a.seed)
    x = I.rhs_normal(a.N, a.nrhs, 2).astype(np.float32).astype(np.float64)
    per_step_rows = 128
    rng_rows = I.sample_rows(a.N, per_step_rows * (a.steps + a.warmup), 5)
    times = []
    for s in range(a.warmup + a.steps):
        rows = rng_rows[s * per_step_rows:(s + 1) * per_step_rows]
        t0 = time.perf_counter()
        O.direct_rows(pts, x, rows)
        dt = time.perf_counter() - t0
        if s >= a.warmup:
            times.append(dt * 1e3 * a.N / per_step_rows)
    v = float(np.mean(times))
    out = {"metric": METRIC, "value": round(v, 3), "unit": "ms", "n_gpus": a.gpus, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": round(v, 3), "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload(a), "impl": "reference",
           "cpu_baseline": {"value": round(v, 3), "unit": "ms", "cores": O.num_threads(), "kind": "oracle",
                            "sample": f"O1 FP64 direct sum on {per_step_rows} seeded rows per step, "
                                      f"scaled by N/rows to one full dense product"},
           "e2e": {"value": round(v, 3), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_batched(a):
    """Independent clouds: one batched product (persistent kernel or graph) against
    separate products.  Clouds are built smallest first with stored FP32 factors
    (ordered, or symmetric storage with --batch-storage symmetric) while they fit
    in device memory (keeping --batch-reserve-gb free); larger clouds then take
    the skeleton storage (pivots and LU of K(sigma,tau), entries recomputed),
    which only the graph form runs, as it does symmetric storage.  The factor
    members are also timed as a batch of their own."""
    import torch
    from paper_2307_16303_gb300.api import H3DMatrix, H3DBatch, H3DError
    from oracle import oracle as O
    rng = np.random.default_rng(5)
    sizes = np.round(np.exp(rng.uniform(np.log(8192), np.log(a.batch_nmax), a.batch_count))).astype(int)
    nc = len(sizes)
    mats, pts, kerns, xs, store = [None] * nc, [None] * nc, [None] * nc, [None] * nc, [None] * nc
    reserve = a.batch_reserve_gb * 1e9
    per_point = 0.0          # largest device bytes per point of a factor member so far
    skeleton_from = None
    t0 = time.perf_counter()
    for c in np.argsort(sizes, kind="stable"):
        n = int(sizes[c])
        p = I.uniform(n, 500 + c) if c % 2 == 0 else I.sphere(n, 500 + c)
        kern = "laplace" if (c // 2) % 2 == 0 else "yukawa"
        dev = torch.from_numpy(p).cuda()
        kind = a.batch_storage
        if skeleton_from is not None or torch.cuda.mem_get_info()[0] - 1.3 * per_point * n < reserve:
            kind = "skeleton"
        try:
            m = H3DMatrix(dev, leaf_size=a.leaf, tol=a.tol, precision="fp32", kernel=kern, storage=kind)
        except H3DError as e:
            if e.status != 3 or kind == "skeleton":
                raise
            kind = "skeleton"
            m = H3DMatrix(dev, leaf_size=a.leaf, tol=a.tol, precision="fp32", kernel=kern, storage=kind)
        if kind != "skeleton":
            per_point = max(per_point, m.stats()["device_bytes"] / n)
        elif skeleton_from is None:
            skeleton_from = n
        mats[c], pts[c], kerns[c], store[c] = m, p, kern, kind
        xs[c] = torch.from_numpy(I.rhs_normal(n, 1, 600 + c)[:, 0].astype(np.float32)).cuda()
        del dev
    build_s = time.perf_counter() - t0
    ys = [torch.empty_like(x) for x in xs]
    fac = [c for c in range(nc) if store[c] != "skeleton"]
    skel = [c for c in range(nc) if store[c] == "skeleton"]
    peak, src = peaks()

    def batch_forms(idx):
        """Tuned batch of the members idx: (chosen ms, info, forms, branches, groups)."""
        bx, by = [xs[c] for c in idx], [ys[c] for c in idx]
        B = H3DBatch([mats[c] for c in idx])
        forms = {}
        if B.info()["persistent"] == 1:
            B.set_mode(True)
            forms["persistent_untuned_ms"] = round(time_steps(lambda: B.matvec(bx, by), a.steps, a.warmup, torch), 4)
        branches = B.tune(bx, by)
        info = B.info()
        with Clocks(torch.cuda.current_device()) as clk:
            ms = time_steps(lambda: B.matvec(bx, by), a.steps, a.warmup, torch)
        if info["persistent"] == 1:
            B.set_mode(False)
            forms["graph_ms"] = round(time_steps(lambda: B.matvec(bx, by), a.steps, a.warmup, torch), 4)
            forms["persistent_ms"] = round(ms, 4)
        else:
            forms["graph_ms"] = round(ms, 4)
            if info["persistent"] == 0:
                B.set_mode(True)
                forms["persistent_ms"] = round(time_steps(lambda: B.matvec(bx, by), a.steps, a.warmup, torch), 4)
        groups = None
        if info["persistent"] >= 0:
            ng, lg = B.groups()
            groups = sorted({(int(u), int(v)) for u, v in zip(ng, lg)})
        B.set_mode(info["persistent"] == 1)
        B.matvec(bx, by)
        torch.cuda.synchronize()
        B.free()
        return ms, info, forms, branches, groups, clk.summary()

    # separate products, one after another on one stream
    seq = sum(time_steps(lambda m=mats[c], x=xs[c], y=ys[c]: m.matvec(x, out=y), a.steps, a.warmup, torch)
              for c in range(nc))
    ms, info, forms, branches, groups, clk = batch_forms(list(range(nc)))
    errs = {}
    check = sorted(set([0, 1, 2, 3] + ([skel[-1]] if skel else [])))
    for c in check:
        if c >= nc:
            continue
        rows = I.sample_rows(int(sizes[c]), 256, 8 + c)
        ref = O.direct_rows(pts[c], xs[c].double().cpu().numpy(), rows, kernel=kerns[c])
        got = ys[c].double().cpu().numpy()[rows]
        errs[f"cloud{c}_{store[c]}_N{int(sizes[c])}"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    fbytes = sum(mats[c].stats()["factor_bytes"] for c in fac)
    persistent = info["persistent"] == 1
    out = {"metric": f"HODLR3D batched matvec ms, {nc} clouds (one persistent launch)" if persistent else
                     f"HODLR3D batched matvec ms, {nc} clouds (one graph launch)",
           "value": round(ms, 4), "unit": "ms",
           "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(ms, 4),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"{nc} clouds, N log-uniform in [8192, {a.batch_nmax}] seed 5, even: uniform cube, "
                                  f"odd: unit sphere; Laplace / Yukawa by pairs; leaf {a.leaf}, tol {a.tol}",
                      "total_points": int(sizes.sum()), "n_min": int(sizes.min()), "n_max": int(sizes.max()),
                      "l2": "inputs larger than L2 (factors >> 129 MB)"},
           "form": "persistent" if persistent else "graph", "ctas_per_sm": info["ctas_per_sm"],
           "graph_branches": branches if branches else info["branches"], "item_shapes": groups,
           "separate_products_ms": round(seq, 4), "speedup_vs_separate": round(seq / ms, 3), "forms": forms,
           "storage": {"factor_storage": a.batch_storage,
                       "factor_members": len(fac), "factor_points": int(sum(sizes[c] for c in fac)),
                       "skeleton_members": len(skel), "skeleton_points": int(sum(sizes[c] for c in skel)),
                       "skeleton_from_N": skeleton_from, "factor_bytes": fbytes},
           "build_s": round(build_s, 1), "rel_err_sampled_rows": errs, "clocks": clk,
           # kernels per product: ordered 5 (permute, near field, gather, reduce, leaf),
           # symmetric 7 (and the fused pairs' kernel and its addition), skeleton ~6
           "gpu_launches": (1 if persistent else sum(7 if store[c] == "symmetric" else 5 if store[c] == "factors"
                                                     else 6 for c in range(nc))) * a.steps}
    if not skel:
        alg = fbytes + 8 * int(sizes.sum())
        gbs = alg / (ms * 1e-3) / 1e9
        out["roofline"] = {"bound": "hbm", "kernel": "k_batch" if persistent else "graph", "achieved": round(gbs, 1),
                           "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4), "peak_source": src,
                           "traffic": None, "alg_bytes_per_launch": alg}
    else:
        # the factor members alone: the persistent kernel's share of the workload
        fms, finfo, fforms, _, fgroups, _ = batch_forms(fac)
        alg = fbytes + 8 * int(sum(sizes[c] for c in fac))
        gbs = alg / (fms * 1e-3) / 1e9
        out["factor_members_batch"] = {"ms": round(fms, 4), "form": "persistent" if finfo["persistent"] == 1 else "graph",
                                       "forms": fforms, "item_shapes": fgroups}
        out["roofline"] = {"bound": "hbm", "kernel": "k_batch (factor members)" if finfo["persistent"] == 1 else
                           "graph (factor members)", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                           "frac": round(gbs / peak, 4), "peak_source": src, "traffic": None,
                           "alg_bytes_per_launch": alg}
    print(json.dumps(out), flush=True)


def run_skeleton(a):
    import torch
    from paper_2307_16303_gb300.api import H3DMatrix
    from oracle import oracle as O
    if a.points == "jittered":
        g = int(round(a.N ** (1 / 3)))
        pts = I.jittered_grid(g, a.seed)
    else:
        pts = I.uniform(a.N, a.seed)
    N = pts.shape[0]
    t0 = time.perf_counter()
    A = H3DMatrix(torch.from_numpy(pts).cuda(), leaf_size=a.leaf, tol=a.tol, precision="fp32", storage="skeleton")
    build_s = time.perf_counter() - t0
    st = A.stats()
    xh = I.rhs_normal(N, a.nrhs, 2).astype(np.float32)
    x = torch.from_numpy(np.ascontiguousarray(xh.T)).cuda()
    y = torch.empty_like(x)
    with Clocks(torch.cuda.current_device()) as clk:
        ms = time_steps(lambda: A.matvec_raw(x.data_ptr(), y.data_ptr(), a.nrhs), a.steps, a.warmup, torch)
    rows = I.sample_rows(N, min(a.rows, N), 4)
    ref = O.direct_rows(pts, xh.astype(np.float64), rows)
    ref = ref if ref.ndim == 2 else ref[:, None]
    got = y.cpu().numpy().T.reshape(N, a.nrhs)[rows].astype(np.float64)
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    out = {"metric": "HODLR3D matvec ms, skeleton storage (pivots + LU of K(sigma,tau), entries recomputed in "
                     "float-float on the FP32 pipes)",
           "value": round(ms, 3), "unit": "ms", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
           "ms_per_step": round(ms, 3), "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "float-float (f32 pairs); f32 in / out", "data": "synthetic",
           "config": {"workload": f"{a.points} N={N}, Laplace, leaf {a.leaf}, tol {a.tol}, nrhs {a.nrhs}", "N": N},
           "rel_err_sampled_rows": err, "build_s": round(build_s, 1), "stored_bytes": st["factor_bytes"],
           "device_bytes": st["device_bytes"], "factor_entries_equivalent": st["factor_entries"],
           "interactions_per_s": N * N * a.nrhs / (ms * 1e-3), "clocks": clk.summary(),
           "gpu_launches": 4 * a.nrhs * a.steps}
    print(json.dumps(out), flush=True)


def main():
    a = parse()
    if a.skeleton and a.impl != "reference":
        run_skeleton(a)
        return
    if a.impl == "reference":
        run_reference(a)
        return
    if a.batched:
        run_batched(a)
        return
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as td
        td.init_process_group("nccl")
        dist = td
    torch.cuda.set_device(local)
    from paper_2307_16303_gb300.api import H3DMatrix, H3DError

    # independent replica per rank (the product does not need a collective)
    pseed, xseed = replica_seeds(rank, a.seed)
    pts = I.uniform(a.N, pseed)
    xh = I.rhs_normal(a.N, a.nrhs, xseed).astype(np.float32)
    dev_pts = torch.from_numpy(pts).cuda()
    A = H3DMatrix(dev_pts, leaf_size=a.leaf, tol=a.tol, precision="fp32_3xtf32")
    st = A.stats()
    x = torch.from_numpy(np.ascontiguousarray(xh.T)).cuda()      # column-major N x nrhs
    y = torch.empty_like(x)
    nrhs = a.nrhs

    def step():
        A.matvec_raw(x.data_ptr(), y.data_ptr(), nrhs)

    with Clocks(local) as clk:
        ms = time_steps(step, a.steps, a.warmup, torch, dist)
    ms = max_over_ranks(ms, dist, "cuda")

    # per-kernel durations (CUDA events on the launching stream) over K more products
    phases = np.zeros(4)
    for _ in range(a.steps):
        phases += np.array(A.matvec_profile(x.data_ptr(), y.data_ptr(), nrhs))
    phases /= a.steps
    # factors are streamed once per pass; a pass covers up to 8 right-hand sides
    per = 32 if (nrhs > 8 and a.leaf <= 128) else 8
    passes = (nrhs + per - 1) // per
    rhs_per_pass = min(nrhs, per)
    names = ["k_permute_in", "k_gather", "k_reduce_partials", "k_leaf"]
    s = 4
    N = a.N
    # algorithmic bytes per launch (one RHS): factor entries once, x / t / y once,
    # FP32 local coordinates (16 B) and the permutation (4 B) per point
    q = rhs_per_pass
    alg_bytes = {
        "k_gather": s * st["v_entries"] + s * N * q + s * st["sum_rank"] * q,
        "k_leaf": s * st["u_entries"] + s * st["sum_rank"] * q + (2 * s * q + 4) * N,
    }
    dom = max(("k_gather", "k_leaf"), key=lambda k: phases[names.index(k)])
    dom_ms = phases[names.index(dom)] / passes
    peak, peak_kind = peaks()
    achieved = alg_bytes[dom] / (dom_ms * 1e-3) / 1e9
    total_bytes = passes * s * (st["u_entries"] + st["v_entries"]) + (4 * s * nrhs + 20) * N
    roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_source": peak_kind,
            "traffic": (int(NCU_TRAFFIC_RATIO[dom] * alg_bytes[dom]) if nrhs == 1 and dom in NCU_TRAFFIC_RATIO
                        else None),
            "alg_bytes_per_launch": int(alg_bytes[dom]),
            "launch_ms": round(dom_ms, 4)}
    phase_ms = {n: round(v / passes, 4) for n, v in zip(names, phases)}

    # end to end through the host entry point (pinned buffers, copies inside)
    xp = torch.from_numpy(np.asfortranarray(xh)).pin_memory() if nrhs > 1 else torch.from_numpy(xh[:, 0].copy()).pin_memory()
    yp = torch.empty_like(xp).pin_memory()
    def e2e_step():
        A.matvec_host_ptr(xp.data_ptr(), yp.data_ptr(), nrhs)
    for _ in range(max(3, a.warmup)):
        e2e_step()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        e2e_step()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / a.steps

    # 32 right-hand sides in one call (3xTF32 factor products on the tensor cores)
    wide = None
    if not a.no_wide and nrhs == 1 and a.leaf <= 128:
        xw = I.rhs_normal(a.N, 32, xseed + 17).astype(np.float32)
        Xw = torch.from_numpy(np.ascontiguousarray(xw.T)).cuda()
        Yw = torch.empty_like(Xw)
        w_ms = time_steps(lambda: A.matvec_raw(Xw.data_ptr(), Yw.data_ptr(), 32), max(2, a.steps // 4), 2, torch,
                          None)
        wph = np.array(A.matvec_profile(Xw.data_ptr(), Yw.data_ptr(), 32))
        fb = 4 * (st["u_entries"] + st["v_entries"])
        wide = {"nrhs": 32, "ms": round(w_ms, 4), "ms_per_column": round(w_ms / 32, 4),
                "phase_ms": {"k_permute_in_w": round(float(wph[0]), 4), "k_tc_stream_gather": round(float(wph[1]), 4),
                             "k_reduce_partials_w": round(float(wph[2]), 4), "k_tc_stream_far": round(float(wph[3]), 4)},
                "factor_bytes_per_pass": fb,
                "factor_GBps": round(fb / (w_ms * 1e-3) / 1e9, 1),
                "factor_hbm_frac": round(fb / (w_ms * 1e-3) / 1e9 / peaks()[0], 4)}
        if rank == 0:
            from oracle import oracle as O
            wrows = I.sample_rows(a.N, 1000, 9)
            ref = O.direct_rows(pts, xw[:, [0, 31]].astype(np.float64), wrows)
            got = Yw.cpu().numpy().T[wrows][:, [0, 31]].astype(np.float64)
            wide["rel_err_1000_rows_cols_0_31"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        del Xw, Yw

    y_host = y.cpu().numpy().T          # N x nrhs
    if nrhs == 1:
        y_host = y_host.reshape(-1)
    forces = None
    if not a.no_forces:
        qh = I.rhs_uniform(a.N, 1, 6 + 1000 * rank)[:, 0].astype(np.float32)
        qd = torch.from_numpy(qh).cuda()
        Fo = {}
        def force_step():
            Fo["E"], Fo["F"] = A.forces(qd)
        f_ms = time_steps(force_step, max(1, a.steps // 4), 1, torch, None)
        e_ms = time_steps(lambda: A.energy(qd), a.steps, a.warmup, torch, None)
        forces = {"forces_ms": round(f_ms, 3), "energy_grad_q_ms": round(e_ms, 3),
                  "energy": Fo["E"].item()}
        if rank == 0:
            from oracle import oracle as O
            frows = I.sample_rows(a.N, 4096, 7)
            Fx = O.direct_forces_rows(pts, qh.astype(np.float64), frows)
            Fg = Fo["F"].cpu().numpy()[frows]
            forces["rel_err_4096_points"] = float(np.linalg.norm(Fg - Fx) / np.linalg.norm(Fx))
            forces["sum_of_forces_rel"] = float(np.abs(Fo["F"].sum(dim=0).cpu().numpy()).max()
                                                / Fo["F"].abs().sum().item())
    st_ordered = st
    A.free()
    del A
    torch.cuda.empty_cache()

    # symmetric storage on the same points: each unordered pair compressed once;
    # pairs that fit a shared-memory stage are streamed once for both directions
    # (k_sym), the rest in the ordered layout for both orders
    sym, ysym_host = None, None
    if not a.no_symmetric and nrhs == 1:
        try:
            As = H3DMatrix(dev_pts, leaf_size=a.leaf, tol=a.tol, precision="fp32_3xtf32", storage="symmetric")
            ss = As.stats()
            ys = torch.empty_like(x)
            s_ms = time_steps(lambda: As.matvec_raw(x.data_ptr(), ys.data_ptr(), 1), a.steps, a.warmup, torch, None)
            ph = np.zeros(4)
            for _ in range(a.steps):
                ph += np.array(As.matvec_profile(x.data_ptr(), ys.data_ptr(), 1))
            ph /= a.steps
            # the fused pairs' entries: stored twice by the ordered handle, once here
            fused = st_ordered["factor_entries"] - ss["factor_entries"]
            sym = {"ms": round(s_ms, 4), "factor_bytes": ss["factor_bytes"], "factor_entries": ss["factor_entries"],
                   "build_ms": round(ss["build_ms"], 1), "device_bytes": ss["device_bytes"],
                   "fused_pair_entries": int(fused),
                   "phase_ms": {"k_permute_in": round(ph[0], 4), "k_sym": round(ph[1], 4),
                                "gather_reduce_and_fused_add": round(ph[2], 4), "k_leaf": round(ph[3], 4)},
                   "k_sym_GBps": round(4 * fused / (ph[1] * 1e-3) / 1e9, 1),
                   "vs_ordered_ms": round(s_ms / ms, 3)}
            ysym_host = ys.cpu().numpy().reshape(-1)
            As.free()
            del As
            torch.cuda.empty_cache()
        except H3DError as e:
            sym = {"ms": None, "error": str(e)}

    fp64 = None
    y64_host = None
    if not a.no_fp64:
        try:
            A64 = H3DMatrix(dev_pts, leaf_size=a.leaf, tol=a.tol, precision="fp64")
            x64 = x.double()
            y64 = torch.empty_like(x64)
            f64 = time_steps(lambda: A64.matvec_raw(x64.data_ptr(), y64.data_ptr(), nrhs), a.steps, a.warmup,
                             torch, None)
            s64 = A64.stats()
            fp64 = {"ms": round(f64, 4), "build_ms": round(s64["build_ms"], 1),
                    "factor_bytes": s64["factor_bytes"]}
            # what bounds the FP64 comparator: its per-phase times (CUDA events on the
            # launching stream), the factor stream's HBM rate and its FMA rate against
            # GB300's nominal FP64 peak (1.25 TFLOP/s dense, no FP64 tensor path)
            ph = np.zeros(4)
            for _ in range(max(1, a.steps // 4)):
                ph += np.array(A64.matvec_profile(x64.data_ptr(), y64.data_ptr(), nrhs))
            ph /= max(1, a.steps // 4)
            p64 = (nrhs + 7) // 8 if nrhs > 1 else 1
            fac_ms = (ph[1] + ph[3]) / p64
            fmas = s64["factor_entries"] * min(nrhs, 8)
            fp64.update({
                "phase_ms_per_pass": {n: round(v / p64, 4) for n, v in zip(
                    ["k_permute_in", "k_gather", "k_reduce_partials", "k_leaf"], ph)},
                "factor_GBps": round(8 * s64["factor_entries"] / (fac_ms * 1e-3) / 1e9, 1),
                "factor_hbm_frac": round(8 * s64["factor_entries"] / (fac_ms * 1e-3) / 1e9 / peaks()[0], 4),
                "factor_fp64_TFLOPs": round(2 * fmas / (fac_ms * 1e-3) / 1e12, 3),
                "factor_fp64_frac_of_nominal_1.25TF": round(2 * fmas / (fac_ms * 1e-3) / 1.25e12, 4),
                "near_interactions": s64["near_interactions"]})
            y64_host = y64.cpu().numpy().T
            if nrhs == 1:
                y64_host = y64_host.reshape(-1)
            A64.free()
        except H3DError as e:
            fp64 = {"ms": None, "error": str(e)}

    out_cpu, err = None, None
    if rank == 0:
        out_cpu, err, nrows, ref_rows = cpu_baseline(pts, xh.astype(np.float64), y_host.astype(np.float64), a,
                                                     a.cpu_seconds)
        if fp64 is not None and fp64.get("ms") is not None:
            yr = y64_host[ref_rows[0]] if y64_host.ndim == 2 else y64_host[ref_rows[0]][:, None]
            fp64["rel_err_sampled_rows"] = float(np.linalg.norm(yr - ref_rows[1]) / np.linalg.norm(ref_rows[1]))
        if sym is not None and ysym_host is not None:
            yr = ysym_host[ref_rows[0]][:, None].astype(np.float64)
            sym["rel_err_sampled_rows"] = float(np.linalg.norm(yr - ref_rows[1]) / np.linalg.norm(ref_rows[1]))
        if a.o2_N > 0:
            out_cpu["o2"] = cpu_hodlr3d(a)

    launches = 5 * passes * a.steps   # permute, near field, gather, partial reduce, leaf
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    clk_s = clk.summary()
    out = {
        "metric": METRIC, "value": round(ms, 4), "unit": "ms", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": round(ms, 4), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload(a),
        "rel_err_sampled_rows": err, "fp64": fp64, "forces": forces, "symmetric": sym, "nrhs32": wide,
        "speedup_vs_fp64": (round(fp64["ms"] / ms, 3) if fp64 and fp64.get("ms") else None),
        "interactions_per_s": N * N * nrhs / (ms * 1e-3),
        "matvec_alg_GBps": round(total_bytes / (ms * 1e-3) / 1e9, 1),
        "roofline": roof, "phase_ms_per_pass": phase_ms, "passes": passes,
        "cpu_baseline": out_cpu,
        "e2e": {"value": round(e2e_ms, 4), "unit": "ms", "h2d_bytes_per_step": 4 * N * nrhs,
                "d2h_bytes_per_step": 4 * N * nrhs},
        "gpu_launches": int(launches),
        "clocks": clk_s,
        "build": {"build_ms": round(st["build_ms"], 1), "depth": st["depth"], "n_blocks": st["n_blocks"],
                  "max_rank": st["max_rank"], "factor_entries": st["factor_entries"],
                  "factor_bytes": st["factor_bytes"], "device_bytes": st["device_bytes"],
                  "near_interactions": st["near_interactions"]},
    }
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
