#!/usr/bin/env python
"""Benchmark of the Static PageRank hot path on one GB300 (replicas on N GPUs).

Workload (default `rmat24`): the 2^24-vertex R-MAT graph, 2^28 samples with
(a, b, c, d) = (0.57, 0.19, 0.19, 0.05), seed 1, duplicates removed, one
self-loop per vertex; FP64 Static PageRank, alpha = 0.85, uniform 1/n start,
L-inf tolerance 1e-10, at most 500 sweeps. One step = one full solve
(initialisation, in-degree partition, sweeps to tolerance), graph resident.

Prints one JSON line (rank 0). `value` is GTEPS = sweeps x |E| / time to
tolerance, summed over ranks (each rank solves its own replica: weak scaling).
`--impl reference` times the CPU oracle instead on a bounded sample of sweeps.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GTEPS & time-to-tol 1e-10: static vs DF-P, FP32-refined vs FP64, on 1 GB300"

WORKLOADS = {
    # name: (kind, params, description)
    "rmat24": ("rmat", (24, 1 << 28), "R-MAT 2^24 vertices, 2^28 samples (a,b,c,d)=(.57,.19,.19,.05) seed 1, "
                                      "dedup + self-loops; Static FP64, alpha 0.85, tol 1e-10 L-inf"),
    "grid4096": ("grid", (4096, 0.05), "4096x4096 bidirectional 4-neighbour grid, 5% edges dropped, seed 1, "
                                       "self-loops; Static FP64, alpha 0.85, tol 1e-10 L-inf"),
    "rmat16": ("rmat", (16, 1 << 20), "R-MAT 2^16 vertices, 2^20 samples seed 1, dedup + self-loops; "
                                      "Static FP64, alpha 0.85, tol 1e-10 L-inf"),
    "rmat22": ("rmat", (22, 1 << 26), "R-MAT 2^22 vertices, 2^26 samples seed 1, dedup + self-loops; "
                                      "Static FP64, alpha 0.85, tol 1e-10 L-inf (the size profiles are captured on)"),
}


def aggregate_ranks(ms_local, units_local, dist=None):
    """Replicas: every rank solves its own copy. Returns (max time over ranks, units summed over ranks)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms_local, units_local
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms_local], dtype=torch.float64, device=dev)
    u = torch.tensor([units_local], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def make_edges(name):
    import synth
    kind, prm, _ = WORKLOADS[name]
    if kind == "rmat":
        return synth.rmat(prm[0], prm[1], seed=1)
    return synth.grid(prm[0], prm[1], seed=1)


def algorithmic_bytes_per_sweep(n, m):
    """Compulsory bytes of one FP64 Static sweep: in-CSR indices 4m, offsets 4(n+1),
    the gathered vector and the degree read once each (12n), the new ranks written (8n)."""
    return 4 * m + 24 * n


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def sweep_source_hash():
    """sha256 over what the rank-sweep kernels are compiled from: sweep.cu, common.cuh and the SweepArgs
    declaration in internal.cuh (other declarations there do not change the sweep)."""
    csrc = os.path.join(ROOT, "paper_2404_08299_gb300", "csrc")
    h = hashlib.sha256()
    for fn in ("sweep.cu", "common.cuh"):
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(f.read())
    with open(os.path.join(csrc, "internal.cuh")) as f:
        text = f.read()
    i = text.index("struct SweepArgs {")
    h.update(text[i:text.index("};", i) + 2].encode())
    return h.hexdigest()


def recorded_traffic(workload):
    """DRAM bytes per sweep from the committed ncu summary, for the workload it was captured on and only
    while the sweep sources are unchanged (sha256 recorded beside the number)."""
    path = os.path.join(ROOT, "profiles", "sweep_rmat24_traffic.txt")
    try:
        rec = {}
        with open(path) as f:
            for line in f:
                parts = line.split()
                if len(parts) == 2:
                    rec[parts[0]] = parts[1]
        if rec.get("workload") == workload and rec.get("source_sha256") == sweep_source_hash():
            return float(rec["dram_bytes_per_sweep"])
    except Exception:
        pass
    return None


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index, keep_dir=None):
        """Samples nvidia-smi every 200 ms into a temporary CSV; with keep_dir, the CSV is also
        copied there as clocks_rank<index>.csv."""
        self.index = index
        self.proc = None
        self.keep_dir = keep_dir
        self.path = None

    def start(self):
        import tempfile
        fd, self.path = tempfile.mkstemp(prefix="clocks_rank%d_" % self.index, suffix=".csv")
        self.f = os.fdopen(fd, "w")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            self.f.close()
            os.remove(self.path)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            lines = f.readlines()
        try:
            if self.keep_dir:
                import shutil
                os.makedirs(self.keep_dir, exist_ok=True)
                shutil.copyfile(self.path, os.path.join(self.keep_dir, "clocks_rank%d.csv" % self.index))
            os.remove(self.path)
        except OSError:
            pass
        return self.summarise(lines)

    @classmethod
    def summarise(cls, lines):
        """Median SM clock, maximum clock and the throttle reasons seen active, from the CSV lines."""
        sm, mx, reasons = [], [], set()
        for line in lines:
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for k, nm in enumerate(cls.REASONS):
                if p[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measure_mixed(g, R64, m, args):
    """FP32 sweeps with compensated sums to ||dR|| <= 1e-6 ||R|| (relative), then FP64 sweeps to the
    same L-inf 1e-10: time to tolerance beside the FP64 path and the L-inf distance to its result.
    The result tensor is kept under "_R" for the error against the oracle."""
    import torch
    import paper_2404_08299_gb300 as prdf
    for _ in range(2):
        g.pagerank_static(precision=prdf.PRDF_FP32_REFINE)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        R, st = g.pagerank_static(precision=prdf.PRDF_FP32_REFINE)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    return {"time_to_tol_ms": ms, "sweeps_fp32": st.iterations_fp32,
            "sweeps_fp64": st.iterations - st.iterations_fp32, "converged": bool(st.converged),
            "gteps": st.iterations * m / (ms * 1e-3) / 1e9,
            "linf_vs_fp64_path": float((R - R64).abs().max()),
            "note": "FP32 stage stops at ||dR||_inf <= 1e-6 ||R||_inf; FP64 stage to L-inf 1e-10", "_R": R}


def measure_dfp(g, n, m, args):
    """DF-P after random batches (80% uniform insertions, 20% deletions of existing non-self-loop edges)
    of size f*|E|, consecutive batches per size, each starting from the previous DF-P ranks. Reports
    DF-P time (partition + marking + sweeps + expansion, batch application excluded as in the paper),
    Dynamic Traversal, Naive-dynamic and DF times from the same previous ranks, GPU Static time from scratch on the same
    snapshot, and the L1 errors against a GPU Static solve at L-inf 1e-13 (the oracle pins the same
    path on smaller graphs)."""
    import numpy as np
    import torch
    import synth
    import paper_2404_08299_gb300 as prdf
    R_prev, _ = g.pagerank_static()
    out = []
    for fi, f in enumerate(args.dfp_sizes):
        t_dfp, t_static, errs, iters, aff = [], [], [], [], []
        t_dt, errs_dt, aff_dt = [], [], []
        t_nd, t_df, errs_nd, errs_df = [], [], [], []
        t_apply = []
        errs_inf = []
        t_mix, errs_mix, sweeps_mix = [], [], []
        parts = {"partition": [], "mark": [], "iterate": []}
        for b in range(args.dfp_batches):
            off, adj, _ = g.export_csr(prdf.PRDF_OUT)
            size = max(1, int(round(f * m)))
            ds, dd, is_, id_ = synth.batch(n, off.cpu().numpy(), adj.cpu().numpy(), size, seed=1, s1=fi, s2=b)
            t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
            args_b = [t(ds), t(dd), t(is_), t(id_)]
            torch.cuda.synchronize()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record()
            de, ie = g.apply_batch(*args_b)
            a1.record()
            torch.cuda.synchronize()
            t_apply.append(a0.elapsed_time(a1))
            R, st, _ = g.pagerank_dfp(t(ds), t(dd), t(is_), R_prev, del_mask=de, ins_mask=ie)
            Rm, stm, _ = g.pagerank_dfp(t(ds), t(dd), t(is_), R_prev, del_mask=de, ins_mask=ie,
                                        precision=prdf.PRDF_FP32_REFINE)
            Rd, std, _ = g.pagerank_dt(t(ds), t(dd), t(is_), R_prev, del_mask=de, ins_mask=ie)
            Rn, stn = g.pagerank_static(R0=R_prev)  # Naive-dynamic (Alg. naive)
            Rf, stf, _ = g.pagerank_dfp(t(ds), t(dd), t(is_), R_prev, del_mask=de, ins_mask=ie, prune=0)  # DF
            Rs, sts = g.pagerank_static()
            Rt, _ = g.pagerank_static(tol=1e-13)
            t_dt.append(std.ms_total)
            t_nd.append(stn.ms_total)
            t_df.append(stf.ms_total)
            errs_nd.append(float((Rn - Rt).abs().sum()))
            errs_df.append(float((Rf - Rt).abs().sum()))
            errs_dt.append(float((Rd - Rt).abs().sum()))
            aff_dt.append(std.affected_initial)
            t_dfp.append(st.ms_total)
            parts["partition"].append(st.ms_partition)
            parts["mark"].append(st.ms_mark)
            parts["iterate"].append(st.ms_iterate)
            t_static.append(sts.ms_total)
            errs.append(float((R - Rt).abs().sum()))
            errs_inf.append(float((R - Rt).abs().max() / Rt.abs().max()))
            t_mix.append(stm.ms_total)
            errs_mix.append(float((Rm - Rt).abs().sum()))
            sweeps_mix.append((stm.iterations_fp32, stm.iterations - stm.iterations_fp32))
            iters.append(st.iterations)
            aff.append(st.affected_initial)
            R_prev = R
        out.append({"batch_fraction": f, "batch_size": int(round(f * m)), "batches": args.dfp_batches,
                    "dfp_ms": statistics.median(t_dfp), "static_ms": statistics.median(t_static),
                    "speedup_vs_static": statistics.median(t_static) / statistics.median(t_dfp),
                    "dfp_ms_parts": {k: statistics.median(v) for k, v in parts.items()},
                    "dfp_sweeps": statistics.median(iters), "affected_initial": int(statistics.median(aff)),
                    "l1_err_max": max(errs), "linf_err_rel_max": max(errs_inf),
                    "dt_ms": statistics.median(t_dt), "dt_affected": int(statistics.median(aff_dt)),
                    "dt_l1_err_max": max(errs_dt),
                    "dfp_speedup_vs_dt": statistics.median(t_dt) / statistics.median(t_dfp),
                    "nd_ms": statistics.median(t_nd), "nd_l1_err_max": max(errs_nd),
                    "df_ms": statistics.median(t_df), "df_l1_err_max": max(errs_df),
                    "fp32_refined": {"dfp_ms": statistics.median(t_mix), "l1_err_max": max(errs_mix),
                                     "speedup_vs_fp64_dfp": statistics.median(t_dfp) / statistics.median(t_mix),
                                     "sweeps_fp32_fp64": sweeps_mix[len(sweeps_mix) // 2]},
                    "apply_batch_ms": statistics.median(t_apply),
                    "errors_against": "GPU Static at L-inf 1e-13 on the same snapshot (see oracle_errors for the "
                                      "oracle-referenced errors)"})
    return out


def _timed(fn, reps):
    """Median device time (stats.ms_total) of reps calls, and the last call's result."""
    ms, res = [], None
    for _ in range(reps):
        res = fn()
        ms.append(res[1].ms_total)
    return statistics.median(ms), res


def measure_oracle_errors(args, og0, h_src, h_dst, R_gpu, R_mixed):
    """Errors against the FP64 oracle at full size.

    Static: the headline FP64 result and the mixed-precision result against the oracle's own Static solve
    (Alg. static, same tolerance 1e-10, same start). DF-P: for each batch fraction in --oracle-dfp-sizes one
    random batch (80% insertions of uniform pairs, 20% deletions of existing non-self-loop edges, drawn from
    the oracle's CSR) is applied by the oracle (set semantics) and by the GPU to a fresh copy of the base
    graph; the reference is the oracle's Static solve of G^t at L-inf 1e-13. From the GPU Static ranks of
    G^0 (L-inf 1e-10) the GPU runs DF-P with tau_f = tau_p in --tau-p, DF-P in mixed precision, DF,
    Naive-dynamic and Dynamic Traversal, and GPU Static from scratch; each is reported with its device time
    (median of --oracle-reps calls), sweeps, and L1 / relative L-inf error against the oracle reference."""
    import numpy as np
    import torch
    import oracle
    import synth
    import paper_2404_08299_gb300 as prdf
    n = og0.n
    out = {}
    t0 = time.time()
    Ro, sto = oracle.pagerank_static(og0)
    t_static = time.time() - t0

    def errs(R, ref, ref10=None):
        r = R.cpu().numpy() if hasattr(R, "cpu") else R
        d = np.abs(r - ref)
        e = {"l1": float(d.sum()), "linf": float(d.max()), "linf_rel": float(d.max() / ref.max())}
        if ref10 is not None:
            e["l1_vs_oracle_static_1e-10"] = float(np.abs(r - ref10).sum())
        return e

    out["static"] = dict(errs(R_gpu, Ro), oracle_sweeps=sto.iterations, oracle_seconds=round(t_static, 2),
                         reference="oracle Static, L-inf 1e-10 (the same iteration and stop rule)")
    if R_mixed is not None:
        out["fp32_refined"] = dict(errs(R_mixed, Ro), reference="oracle Static, L-inf 1e-10")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    dfp = []
    for fi, f in enumerate(args.oracle_dfp_sizes):
        m0 = og0.m
        size = max(1, int(round(f * m0)))
        ds, dd, is_, id_ = synth.batch(n, og0.out_off, og0.out_adj, size, seed=1, s1=100 + fi, s2=0)
        t0 = time.time()
        og1, _, _ = oracle.apply_batch(og0, ds, dd, is_, id_)
        ref, st_ref = oracle.pagerank_static(og1, tol=1e-13)
        # the oracle's from-scratch Static ranks of G^t with the paper's settings (tau 1e-10)
        ref10, st10 = oracle.pagerank_static(og1)
        t_ref = time.time() - t0
        del og1
        gf = prdf.Graph(n, h_src.cuda(non_blocking=True), h_dst.cuda(non_blocking=True))
        de, ie = gf.apply_batch(t(ds), t(dd), t(is_), t(id_))
        b = (t(ds), t(dd), t(is_))
        rec = {"batch_fraction": f, "batch_size": size, "oracle_reference_sweeps": st_ref.iterations,
               "oracle_seconds": round(t_ref, 1),
               "references": "l1, linf: oracle Static of G^t at L-inf 1e-13 (converged); l1_vs_oracle_static_1e-10: "
                             "the oracle's from-scratch Static of G^t with the paper's tau 1e-10 (%d sweeps)"
                             % st10.iterations}
        ms, (Rs, sts) = _timed(lambda: gf.pagerank_static(), args.oracle_reps)
        rec["static"] = dict(errs(Rs, ref, ref10), ms=ms, sweeps=sts.iterations)
        rec["dfp"] = []
        for tau in args.tau_p:
            ms, (R, st, _) = _timed(lambda: gf.pagerank_dfp(*b, R_gpu, del_mask=de, ins_mask=ie, tau_f=tau, tau_p=tau),
                                    args.oracle_reps)
            rec["dfp"].append(dict(errs(R, ref, ref10), tau_f=tau, tau_p=tau, ms=ms, sweeps=st.iterations,
                                   speedup_vs_static=rec["static"]["ms"] / ms))
        ms, (R, st, _) = _timed(lambda: gf.pagerank_dfp(*b, R_gpu, del_mask=de, ins_mask=ie,
                                                        precision=prdf.PRDF_FP32_REFINE), args.oracle_reps)
        rec["dfp_fp32_refined"] = dict(errs(R, ref, ref10), ms=ms, sweeps_fp32=st.iterations_fp32,
                                       sweeps_fp64=st.iterations - st.iterations_fp32,
                                       speedup_vs_static=rec["static"]["ms"] / ms)
        ms, (R, st, _) = _timed(lambda: gf.pagerank_dfp(*b, R_gpu, del_mask=de, ins_mask=ie, prune=0),
                                args.oracle_reps)
        rec["df"] = dict(errs(R, ref, ref10), ms=ms, sweeps=st.iterations)
        ms, (R, st) = _timed(lambda: gf.pagerank_static(R0=R_gpu), args.oracle_reps)
        rec["naive_dynamic"] = dict(errs(R, ref, ref10), ms=ms, sweeps=st.iterations)
        ms, (R, st, _) = _timed(lambda: gf.pagerank_dt(*b, R_gpu, del_mask=de, ins_mask=ie), args.oracle_reps)
        rec["dt"] = dict(errs(R, ref, ref10), ms=ms, sweeps=st.iterations)
        dfp.append(rec)
        del gf, ref, ref10
        torch.cuda.empty_cache()
    out["dfp"] = dfp
    return out


def measure_temporal(args):
    """Temporal-stream stand-in for the paper's real-world dynamic graphs (Sec. 5.1.4): the sample order of a
    seeded R-MAT edge stream (2^20 vertices, 2^24 samples) is its time order; the first 90% is loaded with
    self-loops, then consecutive insertion-only batches of B = f*|E_T| stream edges are applied, for
    f = 1e-5, 1e-4, 1e-3 (each size starting again from the 90% snapshot). Static runs from scratch on
    every snapshot; Naive-dynamic, Dynamic Traversal, DF and DF-P each continue from their own previous
    ranks. Reports mean time per batch and the worst L1 error against a Static solve at L-inf 1e-13."""
    import numpy as np
    import torch
    import synth
    import paper_2404_08299_gb300 as prdf
    n, s, d = synth.rmat(20, 1 << 24, seed=3)
    E = len(s)
    pre = int(0.9 * E)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    empty = torch.zeros(0, dtype=torch.int32, device="cuda")
    out = {"n": n, "stream_edges": E, "preloaded": pre, "batches": args.temporal_batches, "sizes": []}
    for f in (1e-5, 1e-4, 1e-3):
        g = prdf.Graph(n, t(s[:pre]), t(d[:pre]))
        R0, _ = g.pagerank_static(tol=1e-13)
        prev = {k: R0 for k in ("nd", "dt", "df", "dfp")}
        B = max(1, int(round(f * E)))
        times = {k: [] for k in ("static", "nd", "dt", "df", "dfp")}
        errs = {k: [] for k in ("static", "nd", "dt", "df", "dfp")}
        pos = pre
        for b in range(args.temporal_batches):
            if pos + B > E:
                break
            bs, bd = t(s[pos:pos + B]), t(d[pos:pos + B])
            pos += B
            _, ie = g.apply_batch(empty, empty, bs, bd)
            ref, _ = g.pagerank_static(tol=1e-13)
            Rs, st = g.pagerank_static()
            res = {"static": (Rs, st)}
            res["nd"] = g.pagerank_static(R0=prev["nd"])
            Rdt, st_dt, _ = g.pagerank_dt(empty, empty, bs, prev["dt"], ins_mask=ie)
            res["dt"] = (Rdt, st_dt)
            Rdf, st_df, _ = g.pagerank_dfp(empty, empty, bs, prev["df"], ins_mask=ie, prune=0)
            res["df"] = (Rdf, st_df)
            Rp, st_p, _ = g.pagerank_dfp(empty, empty, bs, prev["dfp"], ins_mask=ie)
            res["dfp"] = (Rp, st_p)
            for k, (R, stk) in res.items():
                times[k].append(stk.ms_total)
                errs[k].append(float((R - ref).abs().sum()))
                if k != "static":
                    prev[k] = R
        mean = {k: sum(v) / len(v) for k, v in times.items()}
        out["sizes"].append({"batch_fraction": f, "batch_size": B, "batches_run": len(times["static"]),
                             "mean_ms": mean, "l1_err_max": {k: max(v) for k, v in errs.items()},
                             "speedup_vs_static": {k: mean["static"] / mean[k] for k in mean}})
        del g
        torch.cuda.empty_cache()
    return out


def measure_ppr(args):
    """Weighted personalised PageRank and its adjoint on the 2^22-vertex R-MAT (2^26 samples, weights
    U[0.5, 1.5) on every edge and self-loop, row-normalised), K = 64 teleport columns each on 16 seed
    vertices with Dirichlet(1) weights, loss sum_c g_c . r_c with g ~ N(0, 1): time to tolerance of the
    mixed-precision and FP64 forms (same 1e-10 L-inf stop rule) and of the backward pass; the same 64
    columns solved one per call (K = 1) against the batched call; and, on a sample of columns, the error
    of every result against the FP64 oracle (forward ranks, dL/dS; dL/dw from the same job restricted to
    the sampled columns, since it sums over columns)."""
    import numpy as np
    import torch
    import synth
    import paper_2404_08299_gb300 as prdf
    n, s, d = synth.rmat(22, 1 << 26, seed=1)
    loops = np.arange(n, dtype=np.int32)
    s2, d2 = np.concatenate([s, loops]), np.concatenate([d, loops])
    w = synth.edge_weights(s2, d2, seed=1)
    g = prdf.Graph(n, torch.from_numpy(s2).cuda(), torch.from_numpy(d2).cuda(), torch.from_numpy(w).cuda())
    m = g.m
    K = 64
    S_h = synth.ppr_seeds(n, K, n_seed=16, seed=2)
    S = torch.from_numpy(S_h).cuda()
    Gw_h = synth.normal((n, K), seed=3)
    Gw = torch.from_numpy(Gw_h).cuda()
    out = {"n": n, "m": m, "K": K}
    res = {}
    for name, prec in (("fp32_refined", prdf.PRDF_FP32_REFINE), ("fp64", prdf.PRDF_FP64)):
        g.pagerank_ppr(S, precision=prec)  # warm-up
        torch.cuda.synchronize()
        t0 = time.time()
        R, st = g.pagerank_ppr(S, precision=prec)
        torch.cuda.synchronize()
        res[name] = R
        out[name] = {"ms": st.ms_total, "wall_ms": (time.time() - t0) * 1e3, "sweeps_fp32": st.iterations_fp32,
                     "steps_fp64": st.iterations - st.iterations_fp32, "converged": bool(st.converged),
                     "column_gteps": st.iterations * m * K / (st.ms_total * 1e-3) / 1e9}
    out["linf_mixed_vs_fp64"] = float((res["fp32_refined"] - res["fp64"]).abs().max())
    out["speedup_mixed_vs_fp64"] = out["fp64"]["ms"] / out["fp32_refined"]["ms"]
    g.pagerank_backward(res["fp32_refined"], Gw, precision=prdf.PRDF_FP32_REFINE)
    gS, gw, stb = g.pagerank_backward(res["fp32_refined"], Gw, precision=prdf.PRDF_FP32_REFINE)
    out["backward"] = {"ms": stb.ms_total, "sweeps_fp32": stb.iterations_fp32,
                       "steps_fp64": stb.iterations - stb.iterations_fp32, "converged": bool(stb.converged)}
    # batching: the same 64 columns one per call (K = 1), mixed precision, same stop rule
    R1 = None
    if args.ppr_single:
        single_ms, single_sweeps = 0.0, 0
        R1 = torch.empty_like(res["fp32_refined"])
        g.pagerank_ppr(S[:, :1].contiguous(), precision=prdf.PRDF_FP32_REFINE)  # warm-up of the K = 1 shapes
        for c in range(K):
            Rc, stc = g.pagerank_ppr(S[:, c:c + 1].contiguous(), precision=prdf.PRDF_FP32_REFINE)
            single_ms += stc.ms_total
            single_sweeps += stc.iterations
            R1[:, c:c + 1] = Rc
        out["single_column_calls"] = {
            "calls": K, "ms_total": single_ms, "sweeps_total": single_sweeps,
            "batched_speedup": single_ms / out["fp32_refined"]["ms"],
            "linf_vs_batched": float((R1 - res["fp32_refined"]).abs().max()),
            "note": "64 calls of prdf_pagerank_ppr with K = 1 (mixed precision) against one call with K = 64"}
    # errors against the FP64 oracle on sampled columns
    if args.ppr_oracle_cols:
        import oracle
        oracle.build()
        cols = args.ppr_oracle_cols
        t0 = time.time()
        og = oracle.graph(n, s2, d2)
        rows, dsts = oracle.csr_to_edges(og.out_off, og.out_adj)
        w_out = synth.edge_weights(rows, dsts, seed=1).astype(np.float64)
        P = oracle.row_normalise(og, w_out)
        Ro, sto = oracle.ppr(og, P, np.ascontiguousarray(S_h[:, cols]), tol=1e-13)
        Gc = np.ascontiguousarray(Gw_h[:, cols])
        _, gSo, gwo, sta = oracle.ppr_adjoint(og, w_out, P, Ro, Gc, tol=1e-13)
        t_or = time.time() - t0
        err = {"columns": cols, "oracle_seconds": round(t_or, 1), "oracle_sweeps": sto.iterations,
               "reference": "oracle K-column PPR and adjoint at L-inf 1e-13 on the sampled columns"}
        for name in ("fp32_refined", "fp64"):
            err[name] = float(np.abs(res[name][:, cols].cpu().numpy() - Ro).max())
        if R1 is not None:
            err["single_column_calls"] = float(np.abs(R1[:, cols].cpu().numpy() - Ro).max())
        err["backward_grad_S"] = float(np.abs(gS[:, cols].cpu().numpy() - gSo).max() / np.abs(gSo).max())
        # dL/dw sums over columns: the GPU runs the same job restricted to the sampled columns
        Sc = torch.from_numpy(np.ascontiguousarray(S_h[:, cols])).cuda()
        Rc, _ = g.pagerank_ppr(Sc, precision=prdf.PRDF_FP32_REFINE)
        _, gwc, _ = g.pagerank_backward(Rc, torch.from_numpy(Gc).cuda(), precision=prdf.PRDF_FP32_REFINE)
        err["backward_grad_w"] = float(np.abs(gwc.cpu().numpy() - gwo).max() / np.abs(gwo).max())
        err["note"] = "forward: max abs error; gradients: max abs error / max abs oracle gradient"
        out["oracle_errors"] = err
    del g, R1
    torch.cuda.empty_cache()
    return out


def cpu_baseline(og, t_build, m, target_s):
    """The FP64 oracle (as it stands) on the host cores: a bounded sample of sweeps
    of the same Static iteration on the same graph (og, built in t_build seconds)."""
    import oracle
    t0 = time.time()
    oracle.pagerank_static(og, tol=0.0, max_iter=1)
    t1 = time.time() - t0
    k = max(1, min(200, int(target_s / max(t1, 1e-6))))
    t0 = time.time()
    oracle.pagerank_static(og, tol=0.0, max_iter=k)
    t = time.time() - t0
    cores = oracle.num_threads()
    # the same sweeps on one thread (bit-identical results), a shorter sample
    oracle.set_threads(1)
    k1 = max(1, min(k, int(0.3 * target_s / max(t1 * cores, 1e-6))))
    t0 = time.time()
    oracle.pagerank_static(og, tol=0.0, max_iter=k1)
    t_one = time.time() - t0
    oracle.set_threads(cores)
    return {"value": k * m / t / 1e9, "unit": "GTEPS", "cores": cores, "kind": "oracle",
            "sample": "%d FP64 Static sweeps of the full graph (oracle CSR build %.1fs untimed)" % (k, t_build),
            "seconds": round(t, 3),
            "one_thread": {"value": k1 * m / t_one / 1e9, "unit": "GTEPS", "cores": 1,
                           "sample": "%d FP64 Static sweeps of the full graph" % k1, "seconds": round(t_one, 3)}}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    n, src, dst = make_edges(args.workload)
    import oracle
    oracle.build()
    og = oracle.graph(n, src, dst)
    m = og.m
    sweeps = args.ref_sweeps
    for _ in range(args.warmup):
        oracle.pagerank_static(og, tol=0.0, max_iter=sweeps)
    ts = []
    for _ in range(args.steps):
        t0 = time.time()
        oracle.pagerank_static(og, tol=0.0, max_iter=sweeps)
        ts.append(time.time() - t0)
    T = sum(ts)
    val = args.steps * sweeps * m / T / 1e9
    kind, prm, desc = WORKLOADS[args.workload]
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GTEPS", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": T / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": desc, "n": n, "m": m,
                       "step": "%d oracle sweeps (bounded sample of the solve)" % sweeps},
            "cpu_baseline": {"value": val, "unit": "GTEPS", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": "%d FP64 Static sweeps per step" % sweeps},
            "e2e": {"value": val, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat24", choices=sorted(WORKLOADS))
    ap.add_argument("--accumulate", default="exact", choices=["exact", "fp64"])
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-sweeps", type=int, default=2)
    ap.add_argument("--no-extras", action="store_true", help="skip the mixed-precision and DF-P side measurements")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default in-degree class thresholds")
    ap.add_argument("--dfp-sizes", type=float, nargs="*", default=[1e-7, 1e-5, 1e-3])
    ap.add_argument("--dfp-batches", type=int, default=3)
    ap.add_argument("--temporal-batches", type=int, default=10)
    ap.add_argument("--profile-build", action="store_true",
                    help="build the workload's graph twice and exit (for a launch list of the build)")
    ap.add_argument("--profile-run", action="store_true",
                    help="build the graph and run one solve capped at --max-iter sweeps (for ncu captures)")
    ap.add_argument("--max-iter", type=int, default=500)
    ap.add_argument("--profile-precision", type=int, default=0,
                    help="with --profile-run: 0 = FP64 sweeps, 1 = FP32 stage then FP64 (mixed precision)")
    ap.add_argument("--tile", type=int, default=0, help="column tile of the K-column calls (0: default)")
    ap.add_argument("--clock-dir", default=None,
                    help="also keep the nvidia-smi clock samples of the timed region in this directory")
    ap.add_argument("--profile-ppr", action="store_true",
                    help="build the 2^22 weighted graph and run a few K=64 PPR sweeps (for ncu captures)")
    ap.add_argument("--no-oracle", action="store_true", help="skip the errors against the oracle at full size")
    ap.add_argument("--oracle-dfp-sizes", type=float, nargs="*", default=[1e-4],
                    help="batch fractions of the DF-P errors against the oracle")
    ap.add_argument("--tau-p", type=float, nargs="*", default=[1e-6, 3e-7, 1e-7],
                    help="tau_f = tau_p values of DF-P in the oracle comparison")
    ap.add_argument("--oracle-reps", type=int, default=3)
    ap.add_argument("--ppr-oracle-cols", type=int, nargs="*", default=[0, 63],
                    help="columns of the K = 64 job checked against the oracle (none: skip)")
    ap.add_argument("--ppr-single", type=int, default=1, help="also solve the 64 columns one per call (K = 1)")
    ap.add_argument("--no-ppr", action="store_true", help="skip the K-column PPR and adjoint side measurement")
    ap.add_argument("--dfp-workload", default="rmat22", choices=sorted(WORKLOADS),
                    help="graph of --profile-dfp")
    ap.add_argument("--profile-dfp", type=float, default=0.0,
                    help="build the 2^22 R-MAT, solve Static, apply one random batch of this fraction of |E| and run "
                         "DF-P once (for ncu captures of the build, batch-update, marking and DF-P sweep kernels)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch
    import paper_2404_08299_gb300 as prdf
    from paper_2404_08299_gb300 import build as pbuild
    import synth

    if args.profile_ppr:
        pbuild.build()
        synth.build()
        n, s, d = synth.rmat(22, 1 << 26, seed=1)
        loops = np.arange(n, dtype=np.int32)
        s2, d2 = np.concatenate([s, loops]), np.concatenate([d, loops])
        w = synth.edge_weights(s2, d2, seed=1)
        g = prdf.Graph(n, torch.from_numpy(s2).cuda(), torch.from_numpy(d2).cuda(), torch.from_numpy(w).cuda())
        S = torch.from_numpy(synth.ppr_seeds(n, 64, n_seed=16, seed=2)).cuda()
        # host-driven loop (time_sweeps=1): a profiler sees every sweep kernel as its own launch
        R, st = g.pagerank_ppr(S, precision=prdf.PRDF_FP32_REFINE, max_iter=args.max_iter, check_every=args.max_iter,
                               tile=args.tile, time_sweeps=1)
        torch.cuda.synchronize()
        print(json.dumps({"profile_ppr": True, "n": n, "m": g.m, "sweeps": st.iterations}), flush=True)
        return 0

    if args.profile_dfp > 0:
        pbuild.build()
        synth.build()
        n, s, d = make_edges(args.dfp_workload)
        g = prdf.Graph(n, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda())
        n_, m = g.size()
        # host-driven loops (time_sweeps=1): a profiler sees every sweep kernel as its own launch
        R0, _ = g.pagerank_static(time_sweeps=1)
        off, adj, _ = g.export_csr(prdf.PRDF_OUT)
        size = max(1, int(round(args.profile_dfp * m)))
        ds, dd, is_, id_ = synth.batch(n, off.cpu().numpy(), adj.cpu().numpy(), size, seed=1, s1=0, s2=0)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        de, ie = g.apply_batch(t(ds), t(dd), t(is_), t(id_))
        R, st, _ = g.pagerank_dfp(t(ds), t(dd), t(is_), R0, del_mask=de, ins_mask=ie, time_sweeps=1)
        torch.cuda.synchronize()
        print(json.dumps({"profile_dfp": args.profile_dfp, "n": n, "m": m, "batch": size, "sweeps": st.iterations,
                          "affected_initial": st.affected_initial, "ms_total": st.ms_total}), flush=True)
        return 0

    if rank == 0:
        pbuild.build()
        synth.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        dist.barrier()

    n, src, dst = make_edges(args.workload)
    m0 = len(src)
    acc = prdf.PRDF_ACC_EXACT if args.accumulate == "exact" else prdf.PRDF_ACC_FP64

    # pinned host inputs (also used by the end-to-end leg)
    h_src = torch.from_numpy(src).pin_memory()
    h_dst = torch.from_numpy(dst).pin_memory()
    d_src = h_src.cuda(non_blocking=True)
    d_dst = h_dst.cuda(non_blocking=True)
    g = prdf.Graph(n, d_src, d_dst)
    n_, m = g.size()
    del d_src, d_dst
    torch.cuda.synchronize()

    if args.profile_build:
        # the graph build again, from the device edge list (a profiler sees the second build's launches apart)
        d_src = h_src.cuda(non_blocking=True)
        d_dst = h_dst.cuda(non_blocking=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g2 = prdf.Graph(n, d_src, d_dst)
        torch.cuda.synchronize()
        print(json.dumps({"profile_build": args.workload, "n": n, "m": g2.m,
                          "ms_second_build": 1e3 * (time.perf_counter() - t0)}), flush=True)
        return 0

    if args.profile_run:
        R, st = g.pagerank_static(accumulate=acc, max_iter=args.max_iter, check_every=args.max_iter, time_sweeps=1,
                                  precision=args.profile_precision)
        torch.cuda.synchronize()
        print(json.dumps({"profile_run": args.workload, "n": n, "m": m, "sweeps": st.iterations,
                          "ms_total": st.ms_total}), flush=True)
        return 0

    tuned = None
    if not args.no_autotune:
        idx, ms = g.autotune(sweeps=8, accumulate=acc)
        tuned = {"candidate": idx, "ms_per_sweep": ms}

    # warm-up solves
    for _ in range(args.warmup):
        g.pagerank_static(accumulate=acc)
    torch.cuda.synchronize()

    # timed region: K full solves, device-timed with CUDA events on the launching stream
    clocks = ClockSampler(local, args.clock_dir)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sts = []
    for _ in range(args.steps):
        R, st = g.pagerank_static(accumulate=acc, time_sweeps=1)
        sts.append(st)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms_total = e0.elapsed_time(e1)
    clk = clocks.stop()
    iters = sts[-1].iterations
    edges_per_step = sum(s.iterations for s in sts) / len(sts) * m
    ms_step, edges_all = aggregate_ranks(ms_total / args.steps, edges_per_step, dist)
    value = edges_all / (ms_step * 1e-3) / 1e9

    # roofline of the dominant kernel: the rank sweep, each sweep bracketed by CUDA events on the
    # launching stream (host-driven loop with a convergence read every 8 sweeps)
    sweep_ms = sum(s.ms_sweep for s in sts) / sum(s.iterations for s in sts)
    B = algorithmic_bytes_per_sweep(n, m)
    achieved = B / (sweep_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    traffic = recorded_traffic(args.workload)

    extras = {}
    # the same solve as one CUDA graph (device-side convergence loop): time to tolerance
    for _ in range(2):
        g.pagerank_static(accumulate=acc)
    torch.cuda.synchronize()
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    for _ in range(args.steps):
        g.pagerank_static(accumulate=acc)
    c1.record(stream)
    torch.cuda.synchronize()
    extras["cuda_graph_time_to_tol_ms"] = c0.elapsed_time(c1) / args.steps
    R_mixed = None
    if not args.no_extras:
        extras["fp32_refined"] = measure_mixed(g, R, m, args)
        R_mixed = extras["fp32_refined"].pop("_R")

    # end to end through the public API with host buffers: H2D edge list, graph build, solve, D2H ranks
    h_R = torch.empty(n, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for k in range(args.e2e_steps + 1):
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        s_d = h_src.cuda(non_blocking=True)
        d_d = h_dst.cuda(non_blocking=True)
        g2 = prdf.Graph(n, s_d, d_d)
        R2, st2 = g2.pagerank_static(accumulate=acc)
        h_R.copy_(R2, non_blocking=True)
        a1.record(stream)
        torch.cuda.synchronize()
        if k > 0:
            e2e_ms.append(a0.elapsed_time(a1))
        del g2, s_d, d_d, R2
    e2e_step, e2e_edges = aggregate_ranks(sum(e2e_ms) / len(e2e_ms), st2.iterations * m, dist)
    e2e_val = e2e_edges / (e2e_step * 1e-3) / 1e9

    # errors against the FP64 oracle at full size (the oracle graph also serves the CPU baseline)
    og0, t_og = None, 0.0
    oracle_errors = None
    if rank == 0 and world == 1 and (not args.no_oracle or not args.no_cpu_baseline):
        import oracle
        oracle.build()
        t0 = time.time()
        og0 = oracle.graph(n, src, dst)
        t_og = time.time() - t0
    if og0 is not None and not args.no_oracle:
        oracle_errors = measure_oracle_errors(args, og0, h_src, h_dst, R, R_mixed)
        extras["oracle_errors"] = oracle_errors
    del R_mixed

    if not args.no_extras and args.dfp_sizes:
        extras["dfp"] = measure_dfp(g, n, m, args)
    if not args.no_extras:
        del g
        torch.cuda.empty_cache()
        if not args.no_ppr:
            extras["ppr_adjoint"] = measure_ppr(args)
        if args.temporal_batches > 0:
            extras["temporal"] = measure_temporal(args)

    cpu = None
    if og0 is not None and not args.no_cpu_baseline:
        cpu = cpu_baseline(og0, t_og, m, args.cpu_seconds)

    if rank == 0:
        kind, prm, desc = WORKLOADS[args.workload]
        line = {
            "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": desc, "n": n, "m": m, "samples": m0,
                       "accumulate": args.accumulate, "parallelism": "replicas" if world > 1 else "single",
                       "autotune": tuned,
                       "l2": "inputs larger than L2 (in-CSR %.2f GB, rank vector %.0f MB)" % (
                           (4 * m + 8 * (n + 1)) / 1e9, 8 * n / 1e6)},
            "time_to_tol_ms": ms_step, "iterations": iters, "converged": bool(sts[-1].converged),
            "linf_vs_oracle": oracle_errors["static"]["linf"] if oracle_errors else None,
            "final_delta": sts[-1].final_delta, "paper_style_geps": m / (ms_step * 1e-3) / 1e9,
            "ms_partition": statistics.median(s.ms_partition for s in sts),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "rank sweep (k_sweep_group / k_sweep_warp / k_sweep_block, one launch per "
                                   "in-degree class); one unit = one sweep",
                         "bytes_per_sweep": B, "ms_per_sweep": sweep_ms, "peak_source": peak_kind},
            "e2e": {"value": e2e_val, "unit": "GTEPS", "h2d_bytes_per_step": 8 * m0, "d2h_bytes_per_step": 8 * n,
                    "ms_per_step": e2e_step},
            "gpu_launches": int(sum(s.kernel_launches for s in sts)),
            "extras": extras,
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
