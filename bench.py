#!/usr/bin/env python
"""Benchmark: Vecchia NLL + gradient evaluations per second at n ~ 1.1M, m = 30.

Workload ("continental"): 3,300 stations drawn from a 40-component Gaussian
mixture in a 58 x 24 degree box, observed daily for 365 days with 8% of the
station-days missing (n = 1,108,140 points), time-stratified random order,
Gneiting covariance with sigma1^2 = 1, spatial range 8% of the box width,
temporal range 3 days, interaction 0.5, nugget 0.05 (alpha 0.4, delta 0.2,
nu 1.5), m = 30 correlation-based neighbours, responses drawn by Vecchia
sampling at the true parameters.

One step = one evaluation of the NLL and its gradient with respect to the 5
covariance parameters (vecchia_nll_grad) in the mixed-precision form, with the
neighbour sets fixed (they are re-selected only at iterations 2^j of an
optimiser, Sect. 4.4.1).  The FP64 form and the neighbour search are timed in
the same run and reported beside it.  Inputs stay resident in HBM and are
larger than L2 (~173 MB), so no L2 flush is needed between steps.

--impl reference times the CPU oracle (oracle/) on the host cores on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Vecchia NLL+grad evals/s at n=1.2M, m=30: mixed vs FP64, |ΔNLL|/n≤1e-6"
# Peaks for the "alu" roofline, from unit counts and the maximum SM clock:
# 152 SMs x 128 FP32 lanes x 2 flop/FMA x 2.070 GHz; FP64: the nominal
# 1.25 TFLOP/s of this part (a probe measured 1.20).
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
FP64_PEAK_TFLOPS = 1.25


def _measured_peak(key, fallback):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key])
    except (OSError, KeyError, ValueError):
        return fallback


# DRAM bytes (read + write) of one launch of the mixed row kernel on the
# continental workload, from one ncu capture of the current kernel
# (dram__bytes_read.sum + dram__bytes_write.sum): the inputs, read once
ROWS_TRAFFIC_BYTES = 173642496 + 4249856

# dense BF16 tensor peak (a cuBLAS GEMM timed alone on this part), for the
# VIF low-rank GEMM
BF16_PEAK = _measured_peak("bf16_tflops", 1900.0)


# Algorithmic work of one NLL + gradient evaluation, the count the roofline
# fraction is reported on: about 80 GFLOP at n ~ 1.1M, m = 30 (per row: 496
# covariance pair evaluations of ~17 operations with exp and sqrt, a
# Cholesky of (m+1)^3/6 FMA and ~1k FMA of solves, ~19-20k operations for the
# NLL, and ~3.8 times that with the gradient)
SURVEY_FLOPS_PER_ROW_M30 = 80e9 / 1.1e6


def flops_per_row(m: int) -> float:
    """FP operations the adjoint kernel itself needs for one row of NLL +
    gradient (p = m + 1): 12 per covariance pair (distance 5, sqrt 1, scale 1,
    exp 1, Matern 3, amplitude 1) over p(p-1)/2 pairs; Cholesky p^3/3; three
    triangular solves 3 p^2; the adjoint pass 38 per pair (covariance
    recomputation 12, weight 6, five derivatives 20).  exp and sqrt count as
    one operation each.  Below the count above: the adjoint form needs about
    half the operations of differentiating each row's factor directly."""
    p = m + 1
    pairs = p * (p - 1) / 2
    return pairs * 12 + p ** 3 / 3 + 3 * p ** 2 + pairs * 38


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="continental", choices=["continental", "box", "tiny"])
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-baseline", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-datasets leg")
    ap.add_argument("--no-vif", action="store_true", help="skip the VIF leg")
    ap.add_argument("--legs", default="main,batched,predict,vif,baseline",
                    help="comma list of legs to run: main, batched, predict, vif, baseline")
    ap.add_argument("--vif-n", type=int, default=30000, help="rows of the exact-search VIF leg")
    ap.add_argument("--vif-full", type=int, default=1, help="1: also time the full-size VIF NLL")
    return ap.parse_args()


def workload(name):
    import synthetic_inputs as si
    if name == "continental":
        return si.continental()
    if name == "box":
        return si.box_uniform(m=30)
    return si.tiny_uniform(m=10)


def describe(w):
    return {
        "workload": f"{w.name}: {w.n} space-time points, m={w.m}, Gneiting nu=1.5, "
                    "time-stratified order, Vecchia-sampled responses",
        "n": w.n, "m": w.m,
        "l2": "inputs resident and larger than L2 (no flush needed)",
        "parallelism": "replicas",
    }


# ---------------------------------------------------------------------------
class Clocks:
    """SM clock and throttle reasons sampled during the timed region: NVML
    (read-only queries through ctypes) polled every 20 ms from a thread, so
    that a timed region of a few tens of ms still gets samples; nvidia-smi
    (-lms 200) if NVML cannot be loaded.  The GPU is found by its UUID."""
    # NVML clock-event reason bits
    REASONS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, uuid=None):
        self.index = index
        self.uuid = uuid
        self.proc = None
        self.nvml = None
        self.lines = []
        self.samples = []
        self.mx = None
        self.stop_ev = threading.Event()

    def _nvml_handle(self):
        import ctypes
        L = ctypes.CDLL("libnvidia-ml.so.1")
        if L.nvmlInit_v2() != 0:
            return None
        h = ctypes.c_void_p()
        if self.uuid:
            rc = L.nvmlDeviceGetHandleByUUID(self.uuid.encode(), ctypes.byref(h))
        else:
            rc = L.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.index), ctypes.byref(h))
        if rc != 0:
            return None
        mx = ctypes.c_uint()
        if L.nvmlDeviceGetMaxClockInfo(h, ctypes.c_int(1), ctypes.byref(mx)) == 0:  # NVML_CLOCK_SM
            self.mx = float(mx.value)
        try:
            reasons = L.nvmlDeviceGetCurrentClocksEventReasons
        except AttributeError:
            reasons = L.nvmlDeviceGetCurrentClocksThrottleReasons
        return L.nvmlDeviceGetClockInfo, reasons, h

    def _poll(self):
        import ctypes
        clock_info, reasons, h = self.nvml
        clk = ctypes.c_uint()
        rs = ctypes.c_ulonglong()
        while not self.stop_ev.is_set():
            if clock_info(h, ctypes.c_int(1), ctypes.byref(clk)) == 0:
                r = rs.value if reasons(h, ctypes.byref(rs)) == 0 else 0
                self.samples.append((float(clk.value), r))
            self.stop_ev.wait(0.02)

    def start(self):
        try:
            self.nvml = self._nvml_handle()
        except (OSError, AttributeError):
            self.nvml = None
        if self.nvml is not None:
            self.th = threading.Thread(target=self._poll, daemon=True)
            self.th.start()
            return
        try:
            gid = self.uuid or str(self.index)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={gid}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.nvml is not None:
            self.stop_ev.set()
            self.th.join(timeout=2)
            if not self.samples:
                return None
            reasons = sorted(nm for nm, bit in self.REASONS.items() if any(r & bit for _, r in self.samples))
            return {"sm_mhz": statistics.median(c for c, _ in self.samples), "sm_max_mhz": self.mx,
                    "reasons": reasons, "samples": len(self.samples), "source": "nvml, 20 ms"}
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm),
                "source": "nvidia-smi, 200 ms"}


def device_uuid(torch, index):
    """'GPU-…' UUID of a CUDA device (for NVML / nvidia-smi), or None."""
    try:
        u = str(torch.cuda.get_device_properties(index).uuid)
    except (AttributeError, RuntimeError):
        return None
    return u if u.startswith("GPU-") else "GPU-" + u


def batched_leg(vst, torch, dev, steps):
    """64 independent datasets (n_d log-uniform in [5e3, 5e4], m = 20, own
    parameters each): neighbours and responses per dataset, then one captured
    CUDA graph of the batched NLL + gradient (one persistent launch), launch
    shape autotuned first.  One step = all datasets evaluated once."""
    import synthetic_inputs as si
    sets = si.batched()
    m = sets[0].m
    xs, ts, ys, nns, cnts, ths = [], [], [], [], [], []
    for w in sets:
        th = vst.vst_theta_from_ranges(*w.theta.astuple())
        xy = torch.from_numpy(w.xy).to(dev)
        t = torch.from_numpy(w.t).to(dev)
        ws = vst.Workspace(w.n, m, device=dev)
        nn, cnt = vst.vif_build_neighbors(xy, t, th, m, ws=ws)
        y = vst.vecchia_sample(xy, t, th, m, nn, cnt, torch.from_numpy(w.z).to(dev), ws=ws)
        vst.vst_workspace_status(ws)
        xs.append(xy); ts.append(t); ys.append(y); nns.append(nn); cnts.append(cnt); ths.append(th)
    offs = torch.tensor(np.concatenate([[0], np.cumsum([w.n for w in sets])]), dtype=torch.int64, device=dev)
    xy, t, y = torch.cat(xs), torch.cat(ts), torch.cat(ys)
    nn, cnt = torch.cat(nns), torch.cat(cnts)
    thetas = torch.tensor(ths, dtype=torch.float64, device=dev)
    ns, n = len(sets), int(t.shape[0])
    ws = vst.BatchedWorkspace(ns, n, m, device=dev)
    shape = vst.vst_autotune_nll_grad_batched(offs, thetas, 1.5, xy, t, m, nn, cnt, y, precision=vst.MIXED, ws=ws)
    nll = torch.empty(ns, dtype=torch.float64, device=dev)
    grad = torch.empty((ns, 5), dtype=torch.float64, device=dev)
    out = {}
    for name, prec in (("mixed", vst.MIXED), ("fp64", vst.FP64)):
        gr = vst.BatchedGraph(offs, thetas, 1.5, xy, t, m, nn, cnt, y, prec, nll, grad, ws)
        k = steps if prec == vst.MIXED else max(2, steps // 5)
        for _ in range(3):
            gr.launch()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(k):
            gr.launch()
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / k
        vst.vst_workspace_status(ws)
        out[name] = {"value": 1e3 / ms, "unit": "batch evals/s", "ms": ms, "nll_sum": float(nll.sum().item())}
        gr.close()
    out["workload"] = f"{ns} datasets, {n} points, m={m}, per-dataset parameters, one graph-captured launch"
    out["autotuned_shape"] = {"blocks_per_sm": shape[0], "row_chunk": shape[1]}
    out["dnll_per_n_mixed_vs_fp64"] = abs(out["mixed"]["nll_sum"] - out["fp64"]["nll_sum"]) / n
    return out


def vif_leg(vst, torch, dev, w, nv=30000, full=True):
    """VIF (Sect. 4.3).  (a) the first 30,000 rows of the bench workload with
    k = 1000 inducing points (seeded space-time kMeans++ with Lloyd steps on
    coordinates scaled by the ranges): the exact residual-correlation
    neighbour search and the Woodbury NLL and gradient in both forms;
    (b) the full 1.108M rows with k = 1000 (inducing points from a 50,000-row
    subsample): the exact residual-correlation neighbour search, the NLL in
    both mixed forms (and FP64 once, for the error per point) and the mixed
    NLL + gradient with those neighbours."""
    import synthetic_inputs as si
    th = vst.vst_theta_from_ranges(*w.theta.astuple())
    out = {}

    def timed(f, reps):
        f()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            f()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    k = 1000
    # space-time separated kMeans++ selection (Algorithm 3) on the full
    # workload, timed on its own (the legs below use the seeded inducing sets
    # of the input generator)
    xyf, tf = torch.from_numpy(w.xy).to(dev), torch.from_numpy(w.t).to(dev)
    vst.sts_kmeanspp(xyf, tf, k, seed=11, lloyd_iters=10)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, _, (ms_c, mt_c) = vst.sts_kmeanspp(xyf, tf, k, seed=11, lloyd_iters=10)
    torch.cuda.synchronize()
    out["sts_kmeanspp"] = {"ms": (time.perf_counter() - t0) * 1e3, "m_s": ms_c, "m_t": mt_c, "k": ms_c * mt_c,
                           "lloyd_iters": 10, "n": w.n}
    del xyf, tf
    sub = type(w)(name="sub", xy=w.xy[:nv], t=w.t[:nv], z=w.z[:nv], theta=w.theta, m=w.m, order=None)
    xyk, tk = si.inducing_points(sub, k, seed=11, lloyd_iters=10)
    ind = (torch.from_numpy(xyk).to(dev), torch.from_numpy(tk).to(dev))
    xy, t = torch.from_numpy(w.xy[:nv].copy()).to(dev), torch.from_numpy(w.t[:nv].copy()).to(dev)
    y = torch.from_numpy(w.z[:nv].copy()).to(dev)
    ws = vst.Workspace(nv, w.m, k, device=dev)
    knn_ms = timed(lambda: vst.vif_build_neighbors(xy, t, th, w.m, ws=ws, inducing=ind), 1)
    nn, cnt = vst.vif_build_neighbors(xy, t, th, w.m, ws=ws, inducing=ind)
    knn_info = vst.vst_workspace_status(ws)
    t64 = timed(lambda: vst.vecchia_nll(xy, t, th, w.m, nn, cnt, y, precision=vst.FP64, ws=ws, inducing=ind), 2)
    v64 = vst.vecchia_nll(xy, t, th, w.m, nn, cnt, y, precision=vst.FP64, ws=ws, inducing=ind).item()
    tmx = timed(lambda: vst.vecchia_nll(xy, t, th, w.m, nn, cnt, y, precision=vst.MIXED, ws=ws, inducing=ind), 3)
    vmx = vst.vecchia_nll(xy, t, th, w.m, nn, cnt, y, precision=vst.MIXED, ws=ws, inducing=ind).item()
    t3 = timed(lambda: vst.vecchia_nll(xy, t, th, w.m, nn, cnt, y, precision=vst.MIXED_BF16X3, ws=ws,
                                       inducing=ind), 3)
    v3 = vst.vecchia_nll(xy, t, th, w.m, nn, cnt, y, precision=vst.MIXED_BF16X3, ws=ws, inducing=ind).item()
    vst.vst_workspace_status(ws)
    # the VIF NLL and gradient (FP64, adjoint pass), its own larger workspace
    del ws
    wsg = vst.Workspace(nv, w.m, k, device=dev, vif_grad=True)
    tg = timed(lambda: vst.vecchia_nll_grad(xy, t, th, w.m, nn, cnt, y, precision=vst.FP64, ws=wsg,
                                            inducing=ind), 2)
    vg, gg = vst.vecchia_nll_grad(xy, t, th, w.m, nn, cnt, y, precision=vst.FP64, ws=wsg, inducing=ind)
    vst.vst_workspace_status(wsg)
    v64g, g64 = vg.item(), gg.cpu().numpy()
    tgm = timed(lambda: vst.vecchia_nll_grad(xy, t, th, w.m, nn, cnt, y, precision=vst.MIXED, ws=wsg,
                                             inducing=ind), 3)
    _, ggm = vst.vecchia_nll_grad(xy, t, th, w.m, nn, cnt, y, precision=vst.MIXED, ws=wsg, inducing=ind)
    vst.vst_workspace_status(wsg)
    gm = ggm.cpu().numpy()
    out["sub"] = {"n": nv, "k": k, "m": w.m, "knn_ms": knn_ms, "knn_queries_per_s": nv / (knn_ms * 1e-3),
                  "knn_brute_force_rows": knn_info["n_fallback"], "knn_tie_rows": knn_info["n_tie"],
                  "nll_fp64_ms": t64, "nll_mixed_ms": tmx, "dnll_per_n": abs(vmx - v64) / nv,
                  "nll_mixed_bf16x3_ms": t3, "dnll_per_n_bf16x3": abs(v3 - v64) / nv,
                  "nll_grad_fp64_ms": tg, "nll_grad_fp64_evals_per_s": 1e3 / tg,
                  "grad_nll_equals_nll": v64g == v64, "grad": [float(v) for v in g64],
                  "nll_grad_mixed_ms": tgm, "grad_mixed_abs_err_per_n": (np.abs(gm - g64) / nv).tolist()}
    del wsg, nn, cnt
    if not full:
        return out
    # full size: the exact residual-correlation neighbour search, then the
    # NLL (mixed, and FP64 once for the accuracy record) and NLL + gradient
    # with those neighbours
    xy, t, y = (torch.from_numpy(a).to(dev) for a in (w.xy, w.t, w.z))
    r = np.random.default_rng(5).choice(w.n, 50000, replace=False)
    r.sort()
    sub = type(w)(name="sub", xy=w.xy[r], t=w.t[r], z=w.z[r], theta=w.theta, m=w.m, order=None)
    xyk, tk = si.inducing_points(sub, k, seed=11, lloyd_iters=10)
    ind = (torch.from_numpy(xyk).to(dev), torch.from_numpy(tk).to(dev))
    ws = vst.Workspace(w.n, w.m, k, device=dev, vif_grad=True)
    full = {"n": w.n, "k": k, "m": w.m}
    nn = torch.empty((w.n, w.m), dtype=torch.int32, device=dev)
    cnt = torch.empty(w.n, dtype=torch.int32, device=dev)
    vst.vif_build_neighbors(xy, t, th, w.m, nn=nn, nn_cnt=cnt, ws=ws, inducing=ind)
    torch.cuda.synchronize()
    vst.vst_profile_enable(1)
    t0 = time.perf_counter()
    vst.vif_build_neighbors(xy, t, th, w.m, nn=nn, nn_cnt=cnt, ws=ws, inducing=ind)
    kinfo = vst.vst_workspace_status(ws)
    knn_ms = (time.perf_counter() - t0) * 1e3  # the call synchronises; wall time
    fl, fms = vst.vst_profile_read(vst.PROF_VIF_FILTER)
    vst.vst_profile_enable(0)
    # the filter's algorithmic work: the lower triangle of U U^T, 2 k flops per
    # pair j < i (the triangle pass; later rounds re-screen overflowing rows)
    ffl = float(w.n) * (w.n - 1) / 2 * 2 * k
    full["residual_knn"] = {"ms": knn_ms, "value": w.n / (knn_ms * 1e-3), "unit": "queries/s",
                            "filter_ms": fms, "filter_launches": fl,
                            "filter_roofline": {"bound": "tensor", "achieved": ffl / (fms * 1e-3) / 1e12,
                                                "peak": BF16_PEAK, "unit": "TFLOP/s",
                                                "frac": ffl / (fms * 1e-3) / 1e12 / BF16_PEAK,
                                                "flops": ffl, "peak_note": "measured cuBLAS bf16 (burst)"},
                            "exhaustive_rows": kinfo["n_fallback"], "tie_rows": kinfo["n_tie"],
                            "what": "exact residual-correlation neighbours (FP64 low rank, tensor-core BF16 "
                                    "candidate filter with a rigorous bound, FP64 re-rank)"}
    v64 = vst.vecchia_nll(xy, t, th, w.m, nn, cnt, y, precision=vst.FP64, ws=ws, inducing=ind).item()
    vst.vst_workspace_status(ws)
    for name, prec, terms in (("mixed", vst.MIXED, 6), ("mixed_bf16x3", vst.MIXED_BF16X3, 3)):
        f = (lambda p=prec: vst.vecchia_nll(xy, t, th, w.m, nn, cnt, y, precision=p, ws=ws, inducing=ind))
        tms = timed(f, 2)
        vst.vst_profile_enable(1)
        f()
        parts = {nm: vst.vst_profile_read(c) for nm, c in (("u_gemm", 4), ("gram", 5), ("syrk", 6), ("rows", 0))}
        vst.vst_profile_enable(0)
        vst.vst_workspace_status(ws)
        gemm_ms = parts["u_gemm"][1]
        # algorithmic work of the triangular product U[i][c] = sum_{p <= c}
        # S[i][p] X[c][p]: 2 (c + 1) flops per entry, n k (k + 1) per launch;
        # the split's `terms` BF16 products are overhead of the precision
        # scheme (reported as the tensor pipe's issued work)
        flops = float(w.n) * k * (k + 1)
        full[name] = {"nll_ms": tms, "value": 1e3 / tms, "unit": "VIF NLL evals/s",
                      "kernel_ms": {nm: v[1] for nm, v in parts.items()},
                      "u_gemm_roofline": {"bound": "tensor", "achieved": flops / (gemm_ms * 1e-3) / 1e12,
                                          "peak": BF16_PEAK, "unit": "TFLOP/s",
                                          "frac": flops / (gemm_ms * 1e-3) / 1e12 / BF16_PEAK,
                                          "flops_per_launch": flops, "split_products": terms,
                                          "issued_frac": terms * flops / (gemm_ms * 1e-3) / 1e12 / BF16_PEAK,
                                          "peak_note": "measured cuBLAS bf16 (burst)"}}
        # the per-row residual Gram (32-position blocks, tensor cores, with the
        # split of U): algorithmic 2 k flops per entry of the 32 x 33 / 2 lower
        # triangle; issued: six part products on 128 x 128 tiles per four rows
        # (the diagonal blocks read are a quarter of each tile)
        gram_ms, syrk_ms = parts["gram"][1], parts["syrk"][1]
        pm = 32
        gfl = float(w.n) * pm * (pm + 1) / 2 * 2 * k
        gissued = 6.0 * 128 * 128 * (-(-k // 256) * 256) * 2 * (-(-w.n // 4))
        # [W e]^T [W e]: algorithmic n kc (kc + 1) flops (symmetric, kc = k + 1);
        # issued: six products on the lower triangle of 128 x 128 tiles
        kc = k + 1
        sfl = float(w.n) * kc * (kc + 1)
        tt = -(-kc // 256) * 256 // 128
        sissued = 6.0 * tt * (tt + 1) / 2 * 128 * 128 * (-(-w.n // 128) * 128) * 2
        for key, fl, iss, ms_ in (("gram_roofline", gfl, gissued, gram_ms), ("syrk_roofline", sfl, sissued, syrk_ms)):
            full[name][key] = {"bound": "tensor", "achieved": fl / (ms_ * 1e-3) / 1e12, "peak": BF16_PEAK,
                               "unit": "TFLOP/s", "frac": fl / (ms_ * 1e-3) / 1e12 / BF16_PEAK,
                               "flops_per_launch": fl, "issued_flops": iss,
                               "issued_frac": iss / (ms_ * 1e-3) / 1e12 / BF16_PEAK,
                               "peak_note": "measured cuBLAS bf16 (burst)"}
        vmix = vst.vecchia_nll(xy, t, th, w.m, nn, cnt, y, precision=prec, ws=ws, inducing=ind).item()
        full[name]["dnll_per_n_vs_fp64"] = abs(vmix - v64) / w.n
    full["nll_fp64"] = v64
    # NLL + gradient, mixed (FP32 low rank and n x k products, FP64 reductions)
    fg = (lambda: vst.vecchia_nll_grad(xy, t, th, w.m, nn, cnt, y, precision=vst.MIXED, ws=ws, inducing=ind))
    full["nll_grad_mixed_ms"] = timed(fg, 2)
    vst.vst_workspace_status(ws)
    full["nll_mixed_ms"] = full["mixed"]["nll_ms"]
    full["value"] = full["mixed"]["value"]
    full["unit"] = "VIF NLL evals/s"
    out["full"] = full
    del ws
    torch.cuda.empty_cache()
    return out


def predict_leg(vst, torch, dev, w):
    """Vecchia prediction (mean and variance) from the bench workload's
    training points: (a) the next day at every station of the last day
    (the forecasting case), (b) one million points of a regular 1000 x 1000
    grid over the domain on the next day.  Each call includes the bucket grid
    over all points, the exact neighbour search of the prediction points among
    the training points, and their factor rows."""
    th = vst.vst_theta_from_ranges(*w.theta.astuple())
    xy, t, y = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (w.xy, w.t, w.z))
    last = float(w.t.max())
    st_xy = np.unique(w.xy[w.t == last], axis=0)
    lo, hi = w.xy.min(0), w.xy.max(0)
    gx, gy = np.meshgrid(np.linspace(lo[0], hi[0], 1000), np.linspace(lo[1], hi[1], 1000))
    cases = {"next_day_stations": st_xy, "grid_1e6": np.stack([gx.ravel(), gy.ravel()], 1)}
    out = {}
    for name, pxy in cases.items():
        xp = torch.from_numpy(np.ascontiguousarray(pxy)).to(dev)
        tp = torch.full((pxy.shape[0],), last + 1.0, dtype=torch.float64, device=dev)
        ws = vst.PredictWorkspace(w.n, pxy.shape[0], w.m, device=dev)
        res = {"n_pred": int(pxy.shape[0])}
        for pname, prec in (("mixed", vst.MIXED), ("fp64", vst.FP64)):
            f = (lambda p=prec: vst.vecchia_predict(xy, t, y, th, w.m, xp, tp, precision=p, ws=ws))
            f()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 3
            a.record()
            for _ in range(reps):
                f()
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / reps
            res[pname] = {"ms": ms, "value": pxy.shape[0] / (ms * 1e-3), "unit": "predictions/s"}
        vst.vst_workspace_status(ws)
        out[name] = res
        del ws
    return out


def cpu_baseline(w, th, seconds_hint=True):
    """The oracle as it stands, on the host cores, on a bounded sample: NLL +
    gradient terms of the first S rows (each with m = 30 neighbours found by
    the oracle's brute-force search).  Per-row cost does not depend on the
    row's position, so evals/s = S / (n * t_sample)."""
    import oracle
    threads = oracle.default_threads()
    S = min(w.n, 2000 * threads)
    rows = np.arange(S, dtype=np.int64)
    xy, t = w.xy[:S], w.t[:S]
    nn, cnt, _, _ = oracle.knn(xy, t, th, w.m, rows=rows, threads=threads)
    y = w.z  # response values do not change the work
    t0 = time.perf_counter()
    oracle.nll_grad_rows(w.xy, w.t, th, w.m, rows, nn, cnt, y, threads=threads)
    dt = time.perf_counter() - t0
    # the neighbour search as the paper runs it (cover tree, Algorithms 1-2) on
    # the first points of the workload: the tree over them, then every query
    Sk = min(w.n, 10000)
    t0 = time.perf_counter()
    with oracle.CoverTree(w.xy[:Sk], w.t[:Sk], th) as T:
        tb = time.perf_counter() - t0
        T.knn(w.m, threads=threads)
    tk = time.perf_counter() - t0
    return {"value": S / (w.n * dt), "unit": "evals/s", "cores": threads, "kind": "oracle",
            "sample": f"NLL+grad terms of the first {S} rows of the {w.n}-point workload "
                      f"({dt:.2f} s on {threads} threads), scaled to one full evaluation",
            "neighbor_search": {"value": Sk / tk, "unit": "queries/s", "n": Sk, "build_s": tb, "total_s": tk,
                                "sample": f"cover tree (Algorithms 1-2) over the first {Sk} points, built on one "
                                          f"thread, then all {Sk} queries on {threads} threads; the per-query "
                                          "cost grows with n"}}


# ---------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    w = workload(args.workload)
    th = oracle.theta_native(w.theta)
    threads = oracle.default_threads()
    S = min(w.n, 2000 * threads)
    rows = np.arange(S, dtype=np.int64)
    nn, cnt, _, _ = oracle.knn(w.xy[:S], w.t[:S], th, w.m, rows=rows, threads=threads)
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.nll_grad_rows(w.xy, w.t, th, w.m, rows, nn, cnt, w.z, threads=threads)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    per_eval = statistics.mean(times) * w.n / S
    value = 1.0 / per_eval
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_eval * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": describe(w),
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": threads, "kind": "oracle",
                         "sample": f"each step: NLL+grad terms of the first {S} of {w.n} rows, scaled to a "
                                   "full evaluation"},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def ranks_barrier(dist):
    """Barrier across the ranks of a torchrun job (nothing for one process)."""
    if dist is not None:
        dist.barrier()


def max_over_ranks(ms, dist, device):
    """The slowest rank's time for the timed region: the whole job's time."""
    if dist is None:
        return ms
    import torch
    tt = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_value(world, steps, ms):
    """Evaluations per second of the whole job.  Every rank evaluates the full
    workload on its own GPU (replicas: the hot path has no exchange step), so
    the job completes world x steps evaluations in the slowest rank's time."""
    return world * steps / (ms * 1e-3)


def run_ours(args):
    import torch
    import paper_2602_03609_gb300 as vst
    from paper_2602_03609_gb300 import build as vbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    vbuild.build()
    dev = torch.device("cuda", local)

    w = workload(args.workload)
    th = vst.vst_theta_from_ranges(*w.theta.astuple())
    legs = set(args.legs.split(","))
    if "main" not in legs:
        out = {"legs": sorted(legs)}
        if "vif" in legs:
            out["vif"] = vif_leg(vst, torch, dev, w, args.vif_n, args.vif_full != 0)
        if "batched" in legs:
            out["batched"] = batched_leg(vst, torch, dev, args.steps)
        if "predict" in legs:
            out["predict"] = predict_leg(vst, torch, dev, w)
        if rank == 0:
            print(json.dumps(out), flush=True)
        return 0
    stream = torch.cuda.current_stream()
    xy = torch.from_numpy(w.xy).to(dev)
    t = torch.from_numpy(w.t).to(dev)
    z = torch.from_numpy(w.z).to(dev)
    ws = vst.Workspace(w.n, w.m, device=dev)

    # neighbour search (a3 + a4)
    vst.vst_profile_enable(True)
    nn, cnt = vst.vif_build_neighbors(xy, t, th, w.m, ws=ws)
    vst.vst_workspace_status(ws)
    reps = 3
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    vst.vst_profile_enable(True)
    e0.record(stream)
    for _ in range(reps):
        vst.vif_build_neighbors(xy, t, th, w.m, nn=nn, nn_cnt=cnt, ws=ws)
    e1.record(stream)
    torch.cuda.synchronize()
    knn_ms = e0.elapsed_time(e1) / reps
    kl, kms = vst.vst_profile_read(vst.PROF_KNN)
    info_knn = vst.vst_workspace_status(ws)

    # responses by Vecchia sampling at the true parameters
    y = vst.vecchia_sample(xy, t, th, w.m, nn, cnt, z, ws=ws)
    vst.vst_workspace_status(ws)
    nll = torch.empty(1, dtype=torch.float64, device=dev)
    grad = torch.empty(5, dtype=torch.float64, device=dev)

    def step(prec):
        vst.vecchia_nll_grad(xy, t, th, w.m, nn, cnt, y, precision=prec, nll=nll, grad=grad, ws=ws)

    # accuracy of the mixed form against the FP64 form on this workload
    step(vst.FP64)
    v64, g64 = nll.item(), grad.cpu().numpy().copy()
    step(vst.MIXED)
    info_mx = vst.vst_workspace_status(ws)
    vmx, gmx = nll.item(), grad.cpu().numpy().copy()

    def timed(prec, warm, steps):
        for _ in range(warm):
            step(prec)
        torch.cuda.synchronize()
        ranks_barrier(dist)
        torch.cuda.synchronize()
        vst.vst_profile_enable(True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            step(prec)
        b.record(stream)
        torch.cuda.synchronize()
        ranks_barrier(dist)
        torch.cuda.synchronize()
        ms = max_over_ranks(a.elapsed_time(b), dist, dev)
        rows_l, rows_ms = vst.vst_profile_read(vst.PROF_ROWS)
        fb_l, fb_ms = vst.vst_profile_read(vst.PROF_FALLBACK)
        return ms, rows_l, rows_ms, fb_l, fb_ms

    fp64_steps = max(1, min(args.fp64_steps, args.steps))
    ms64, l64, k64, _, _ = timed(vst.FP64, 1, fp64_steps)
    clocks = Clocks(local, device_uuid(torch, local))
    clocks.start()
    ms, lrows, krows, lfb, kfb = timed(vst.MIXED, args.warmup, args.steps)
    clk = clocks.stop()

    # end to end through the public API with host buffers: pinned host inputs
    # copied in, result copied out, every step.  Two device input buffers and
    # a copy stream: the host-to-device copy of step s + 1 overlaps the
    # evaluation of step s (the inputs do not depend on the result); the
    # copy into a buffer waits until the evaluation that last read it is done
    h_in = [torch.from_numpy(a).pin_memory() for a in (w.xy, w.t)]
    h_y = y.cpu().pin_memory()
    h_nn, h_cnt = nn.cpu().pin_memory(), cnt.cpu().pin_memory()
    h_out = torch.empty(6, dtype=torch.float64).pin_memory()
    bufs = [tuple(torch.empty_like(x) for x in (xy, t, y, nn, cnt)) for _ in range(2)]
    h2d = sum(x.numel() * x.element_size() for x in (h_in[0], h_in[1], h_y, h_nn, h_cnt))
    d2h = 6 * 8
    out6 = torch.empty(6, dtype=torch.float64, device=dev)
    cstream = torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event() for _ in range(2)]
    freed = [torch.cuda.Event() for _ in range(2)]

    def e2e_step(s):
        bi = s % 2
        d_xy, d_t, d_y, d_nn, d_cnt = bufs[bi]
        with torch.cuda.stream(cstream):
            cstream.wait_event(freed[bi])
            d_xy.copy_(h_in[0], non_blocking=True)
            d_t.copy_(h_in[1], non_blocking=True)
            d_y.copy_(h_y, non_blocking=True)
            d_nn.copy_(h_nn, non_blocking=True)
            d_cnt.copy_(h_cnt, non_blocking=True)
            copied[bi].record(cstream)
        stream.wait_event(copied[bi])
        vst.vecchia_nll_grad(d_xy, d_t, th, w.m, d_nn, d_cnt, d_y, precision=vst.MIXED, nll=out6[:1],
                             grad=out6[1:], ws=ws, stream=stream)
        freed[bi].record(stream)
        h_out.copy_(out6, non_blocking=True)

    for s_ in range(2):
        e2e_step(s_)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(3, args.steps // 2)
    a.record(stream)
    cstream.wait_event(a)
    for s_ in range(e2e_steps):
        e2e_step(s_)
    b.record(stream)
    torch.cuda.synchronize()
    e2e_ms = a.elapsed_time(b) / e2e_steps

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    F = SURVEY_FLOPS_PER_ROW_M30 * (((w.m + 1) / 31.0) ** 3) * w.n  # the m = 30 count, scaled by (m+1)^3
    Fx = flops_per_row(w.m) * w.n
    rows_ms_avg = krows / max(lrows, 1)
    achieved = F / (rows_ms_avg * 1e-3) / 1e12
    rows64_avg = k64 / max(l64, 1)
    achieved64 = F / (rows64_avg * 1e-3) / 1e12
    value = whole_job_value(world, args.steps, ms)
    line = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": dict(describe(w), precision="mixed (FP32 covariance + Cholesky, double-float refinement, "
                                              "FP64 accumulation)"),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP32_PEAK_TFLOPS, "traffic": ROWS_TRAFFIC_BYTES,
                     "kernel": "rows_kernel<float, nu=1.5, 32, nll_grad>",
                     "flops_per_launch": F, "avg_launch_ms": rows_ms_avg,
                     "flops_note": "algorithmic NLL+grad work, ~80 GFLOP per evaluation at n ~ 1.1M, m = 30",
                     "frac_of_adjoint_count": Fx / (rows_ms_avg * 1e-3) / 1e12 / FP32_PEAK_TFLOPS,
                     "adjoint_flops_per_launch": Fx,
                     "peak_note": "FP32 peak from unit counts and clocks (152 x 128 x 2 x 2.07 GHz)"},
        "fp64": {"value": 1e3 * fp64_steps / ms64, "unit": "evals/s", "ms_per_step": ms64 / fp64_steps,
                 "roofline": {"bound": "alu", "achieved": achieved64, "peak": FP64_PEAK_TFLOPS,
                              "unit": "TFLOP/s", "frac": achieved64 / FP64_PEAK_TFLOPS,
                              "kernel": "rows_kernel<double, nu=1.5, 32, nll_grad>",
                              "avg_launch_ms": rows64_avg, "flops_per_launch": F,
                              "frac_of_adjoint_count": Fx / (rows64_avg * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                              "peak_note": "nominal FP64 rate of the part"}},
        "mixed_speedup_vs_fp64": (ms64 / fp64_steps) / (ms / args.steps),
        "accuracy": {"nll_fp64": v64, "nll_mixed": vmx, "dnll_per_n": abs(vmx - v64) / w.n,
                     "grad_fp64": g64.tolist(), "grad_mixed": gmx.tolist(),
                     "grad_rel_err": (np.abs(gmx - g64) / np.maximum(np.abs(g64), 1e-300)).tolist(),
                     # per component against the bar |dg_j| <= 1e-4 |g_j| + 1e-6 n
                     "grad_abs_err": np.abs(gmx - g64).tolist(),
                     "grad_bar": (1e-4 * np.abs(g64) + 1e-6 * w.n).tolist(),
                     "grad_within_bar": bool(np.all(np.abs(gmx - g64) <= 1e-4 * np.abs(g64) + 1e-6 * w.n)),
                     "fallback_rows": info_mx["n_fallback"]},
        "neighbor_search": {"value": w.n / (knn_ms * 1e-3), "unit": "queries/s", "ms": knn_ms,
                            "query_kernel_ms": kms / max(kl, 1), "tie_rows": info_knn["n_tie"]},
        "fallback_kernel_ms": kfb / max(lfb, 1),
        "e2e": {"value": 1e3 / e2e_ms, "unit": "evals/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        # per mixed step: header init, lag table, per-point records, row
        # kernel, FP64 fallback row kernel (exits at once when no row is
        # flagged), reduction of the per-warp partials
        "gpu_launches": 6 * args.steps,
        "clocks": clk,
    }
    if not args.no_batched and "batched" in legs:
        line["batched"] = batched_leg(vst, torch, dev, args.steps)
    if "predict" in legs:
        line["predict"] = predict_leg(vst, torch, dev, w)
    if not args.no_vif and "vif" in legs:
        del ws
        torch.cuda.empty_cache()
        line["vif"] = vif_leg(vst, torch, dev, w, args.vif_n, args.vif_full != 0)
    if not args.no_baseline and "baseline" in legs:
        import oracle  # CPU-baseline leg only
        line["cpu_baseline"] = cpu_baseline(w, oracle.theta_native(w.theta))
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
