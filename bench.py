#!/usr/bin/env python
"""Benchmark: events/s from linear-index EER to COM-DPC + SSB phase images.

Workload: 1024x1024 scan, 576x576 detector binned 6x to 96x96 and cropped to
the bright-field disk (553 pixels), 50 e-/frame (about 5.2e7 uint32 events,
uint64 CSR offsets), seeded synthetic data.  One step = the whole hot path:
ssb_accumulate_com (one pass over the events: offset and index checks,
bin/crop/densify, per-frame COM sums and PACBED totals; then the scan DFT ->
G) -> com_dpc_sums (COM maps + Fourier-integrated DPC) -> ssb_reconstruct
(trotter + aberration phase + inverse transform + variance).
``--separate-passes`` times the same outputs through eer_load_csr ->
com_dpc -> ssb_accumulate (three passes over the events) instead.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload instead.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "events/s to COM+SSB phase"
UNIT = "events/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", type=int, default=5)
    ap.add_argument("--scan", type=int, default=0, help="smaller square scan of the same geometry (profiling)")
    ap.add_argument("--scan-shape", default="", help="NYxNX scan of the same geometry (profiling), e.g. 256x1024")
    ap.add_argument("--crop-px", type=float, default=0.0,
                    help="crop radius in binned pixels (default: the bright-field disk); 48 on the "
                         "1024x1024 workload keeps the disk inscribed in the 96x96 pattern")
    ap.add_argument("--refocus-steps", type=int, default=220)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--separate-passes", action="store_true",
                    help="validate, COM and scatter as three passes over the events")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the built-in launch shapes instead of timing the candidates first")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the comparison of the scan-DFT forms (fused FP32, plain Stockham, split-FP16)")
    ap.add_argument("--batching", action="store_true",
                    help="also time the 16-dataset batching workload: one batched launch vs one call per dataset")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "split"],
                    help="scan DFT form: FP32 FFT or split-FP16 tensor-core DFT along x")
    ap.add_argument("--no-refocus-fit", action="store_true",
                    help="skip the refocus comparison on the 25 mrad optics (adjoint fit from zero vs "
                         "a 64-candidate grid search)")
    return ap.parse_args()


def job_throughput(ms: float, units_per_rank: int, world: int, device=None):
    """Whole-job throughput of replicas: every rank processes units_per_rank
    units; the job takes as long as its slowest rank (max over ranks of the
    per-step time, an all-reduce when world > 1).  Returns (units/s, max ms)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    t_max = float(t.item())
    return world * units_per_rank / (t_max * 1e-3), t_max


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            time.sleep(0.25)
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
                self.out = ""

    def summary(self):
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sms:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sms)}


# --------------------------------------------------------------- oracle arm --
def oracle_pipeline(idx, off, geom):
    """The FP64 oracle's whole path: COM + iDPC + densify + G + SSB phase."""
    import oracle as orc
    W, H = geom["det_w"], geom["det_h"]
    sx, sy, n = orc.com_sums(idx, off, W, H)
    cx, cy = orc.pacbed_centre(sx, sy, n)
    ox, oy = orc.com_maps(sx, sy, n, cx, cy)
    orc.idpc(ox, oy, geom)
    counts = orc.densify(idx, off, geom)
    G = orc.g_function(counts, geom)
    return orc.ssb_phase(G, geom, (0.0, 0.0, 0.0, 0.0, 0.0), "none")


def oracle_sample(scan: int, device: str):
    import synth
    w = synth.workload(5, scan_ny=scan, scan_nx=scan)
    d = synth.generate(w, device)
    idx, off = d.numpy()
    return w, synth.geometry(w), idx, off


def cpu_threads():
    """Threads the oracle runs on: numpy's element-wise operations and its
    FFT (pocketfft) are single-threaded and the oracle makes no BLAS call, so
    one core, whatever the size of the machine's BLAS thread pool."""
    return 1


def time_oracle(scan: int, device: str, reps: int = 1):
    w, geom, idx, off = oracle_sample(scan, device)
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle_pipeline(idx, off, geom)
        ts.append(time.perf_counter() - t0)
    return len(idx), ts, w


def run_reference(args, rank):
    if rank != 0:
        return
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    scan = 128
    w, geom, idx, off = oracle_sample(scan, dev)
    for _ in range(args.warmup):
        oracle_pipeline(idx, off, geom)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_pipeline(idx, off, geom)
        ts.append(time.perf_counter() - t0)
    t = sum(ts) / len(ts)
    v = len(idx) / t
    cores = cpu_threads()
    sample = (f"{scan}x{scan} scan of the same geometry and dose ({len(idx)} events, "
              f"{scan * scan} frames) per step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "scan": [scan, scan], "events_per_step": len(idx)},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                         "affinity_cores": len(os.sched_getaffinity(0))},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ------------------------------------------------------------------ GPU arm --
STAGE_BYTES_DOC = {
    "validate": "4 B/event + 8 B/frame",
    "com": "one pass: 24 B/frame of sums in, 16 B/frame out; three passes: 4 B/event + 8 B/frame in, 40 B/frame out",
    "dpc": "8 B/frame in + 4 B/frame out",
    "scatter": "4 B/event + 8 B/frame in; 2 B x P_pad per frame out (+ 24 B/frame of COM sums in the one-pass step)",
    "dft_x": "2 B x P_pad per frame in; 8 B x P_pad x (Nx/2+1)/Nx per frame out",
    "dft_y": "8 B x P_pad x (Nx/2+1)/Nx per frame in and out (transposed out)",
    "trotter": "8 B per (pixel, K) pair of the trotter sets + 8 B per stored bin out",
    "image": "8 B per stored bin in (x2) + 4 B/frame out",
    "dft_xy": "2 B x P_pad per frame in; 8 B x P_pad x (Nx/2+1)/Nx per frame out (both axes, one launch)",
}


def stage_bytes(C, F, P_pad, Ny, nkx, sigma_k, single_pass=False):
    half = Ny * nkx
    return {
        "validate": 4 * C + 8 * (F + 1),
        # single pass: COM maps from the sums (24 B/frame in, 16 B/frame out)
        "com": 40 * F if single_pass else 4 * C + 8 * (F + 1) + 40 * F,
        "dpc": 12 * F,
        # single pass: the scatter also writes the sums (24 B/frame)
        "scatter": 4 * C + 8 * (F + 1) + 2 * P_pad * F + (24 * F if single_pass else 0),
        "dft_x": 2 * P_pad * F + 8 * P_pad * half,
        "dft_y": 16 * P_pad * half,
        "trotter": 8 * sigma_k + 8 * half,
        "image": 16 * half + 4 * F,
        "dft_xy": 2 * P_pad * F + 8 * P_pad * half,
    }


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2104_06336_gb300 as P
    import synth

    P.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    over = dict(scan_ny=args.scan, scan_nx=args.scan) if args.scan else {}
    if args.scan_shape:
        ny, nx = (int(v) for v in args.scan_shape.lower().split("x"))
        over = dict(scan_ny=ny, scan_nx=nx)
    w = synth.workload(args.workload, seed=synth.workload(args.workload).seed + 1000 * rank, **over)
    geom = synth.geometry(w)
    if args.crop_px:
        geom["crop_px"] = float(args.crop_px)
    d = synth.generate(w, dev)
    idx, off = d.idx.contiguous(), d.off.contiguous()
    C, F = idx.numel(), w.n_frames
    prec = P.SPLIT_FP16 if args.precision == "split" else P.FP32_FFT
    rec = P.Reconstructor(geom, precision=prec, n_cand=64, device=dev)
    tuned = P.tuning.autotune(rec, idx, off) if not args.no_autotune else None
    Ny, nkx, P_pad = w.scan_ny, rec.info["nkx"], rec.info["P_pad"]
    theta = torch.zeros(5, dtype=torch.float64, device=dev)
    sums = torch.empty(3, F, dtype=torch.int64, device=dev)
    com = torch.empty(2, F, dtype=torch.float32, device=dev)
    dpc = torch.empty(Ny, w.scan_nx, dtype=torch.float32, device=dev)
    phase = torch.empty(1, Ny, w.scan_nx, dtype=torch.float32, device=dev)
    var = torch.empty(1, dtype=torch.float64, device=dev)

    def step(ix, of):
        rec.totals.zero_()
        if args.separate_passes:
            P.eer_load_csr(rec.plan, ix, of, totals=rec.totals, status=rec.status)
            P.com_dpc(rec.plan, ix, of, sums, com, dpc, totals=rec.totals, scratch=rec.scratch,
                      status=rec.status)
            P.ssb_accumulate(rec.plan, ix, of, 0, rec.work, rec.G, True, status=rec.status)
        else:
            P.ssb_accumulate_com(rec.plan, ix, of, 0, rec.work, rec.G, True, sums, rec.totals,
                                 status=rec.status)
            P.com_dpc_sums(rec.plan, sums, com, dpc, totals=rec.totals, scratch=rec.scratch,
                           status=rec.status)
        P.ssb_reconstruct(rec.plan, rec.G, theta, rec.scratch, phase, var, status=rec.status)

    nst = len(P._lib.STAGES)
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(nst)] for _ in range(args.steps)]
    for row in ev:  # torch creates CUDA events lazily: record once so the handles exist
        for a, b in row:
            a.record()
            b.record()
    for _ in range(args.warmup):
        step(idx, off)
    torch.cuda.synchronize()
    rec.check()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_start, t_stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = P.eer4d_launch_count()
    with ClockSampler(local_rank) as clk:
        t_start.record()
        for k in range(args.steps):
            P.eer4d_set_stage_events(rec.plan, [e[0] for e in ev[k]], [e[1] for e in ev[k]])
            step(idx, off)
        t_stop.record()
        torch.cuda.synchronize()
    launches = P.eer4d_launch_count() - l0
    P.eer4d_set_stage_events(rec.plan)
    if world > 1:
        dist.barrier()
    ms = t_start.elapsed_time(t_stop) / args.steps
    value, ms = job_throughput(ms, C, world, device=dev)
    # a stage whose events were not recorded inside the timed region did not run
    ran = [t_start.elapsed_time(ev[0][i][0]) >= 0.0 for i in range(nst)]
    stage_ms = {n: statistics.mean(ev[k][i][0].elapsed_time(ev[k][i][1]) for k in range(args.steps))
                for i, n in enumerate(P._lib.STAGES) if ran[i]}
    rec.check()

    # algorithmic bytes of each stage; sigma_k = sum over bins of |K(K)|
    cnt = rec.trotter_counts(0.0)
    sigma_k = int(cnt.sum().item())
    sb = stage_bytes(C, F, P_pad, Ny, nkx, sigma_k, single_pass=not args.separate_passes)
    hbm, hsrc = peaks()
    dom = max(stage_ms, key=stage_ms.get)
    ach = sb[dom] / (stage_ms[dom] * 1e-3) / 1e9
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tr_path):
        try:
            traffic = json.load(open(tr_path)).get(dom)
        except Exception:
            traffic = None
    stages = {n: {"ms": round(stage_ms[n], 4), "bytes": sb[n],
                  "GB_s": round(sb[n] / (stage_ms[n] * 1e-3) / 1e9, 1) if stage_ms[n] > 0 else None,
                  "frac": round(sb[n] / (stage_ms[n] * 1e-3) / 1e9 / hbm, 3) if stage_ms[n] > 0 else None}
              for n in stage_ms}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name + (f"-crop{args.crop_px:g}" if args.crop_px else ""),
                   "scan": [w.scan_ny, w.scan_nx], "detector": [w.det_h, w.det_w],
                   "bin": w.bin, "P": rec.info["P"], "events_per_gpu": C, "e_per_frame": w.e_per_frame,
                   "precision": "FP32 FFT" if args.precision == "fp32" else "split-FP16 tcgen05 DFT (x) + FP32 FFT (y)",
                   "norm": "none", "sigma_K": sigma_k,
                   "event_passes": 3 if args.separate_passes else 1,
                   "l2": "inputs larger than L2 (events 4 B x C = %.0f MB; G %.2f GB); no flush" %
                         (4 * C / 1e6, 8 * P_pad * Ny * nkx / 1e9),
                   "parallelism": f"replicas x{world} (independent datasets, no collective)"},
        "gpu_launches": launches,
        "tuning": tuned,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(ach, 1), "peak": hbm,
                     "unit": "GB/s", "frac": round(ach / hbm, 3), "traffic": traffic,
                     "peak_source": hsrc, "algorithmic_bytes": sb[dom]},
        "stages": stages,
        "clocks": clk.summary(),
    }

    # ---- the scan-DFT forms on the same events ----------------------------
    # fused FP32 register FFT (one persistent launch), the plain FP32 Stockham
    # form (two launches + transpose) and the split-FP16 tcgen05 DFT along x:
    # ssb_accumulate time and the phase against the fused form's
    if not args.no_forms:
        ref_ph = torch.empty(1, Ny, w.scan_nx, dtype=torch.float32, device=dev)
        v1 = torch.empty(1, dtype=torch.float64, device=dev)
        forms = {}
        for name, prec_f in (("fp32_fused", P.FP32_FFT), ("fp32_stockham", P.FP32_STOCKHAM),
                             ("split_fp16_tcgen05", P.SPLIT_FP16)):
            rf = P.Reconstructor(geom, precision=prec_f, device=dev)
            rf.totals.zero_()

            def acc():
                P.ssb_accumulate(rf.plan, idx, off, 0, rf.work, rf.G, True, status=rf.status)

            acc()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(3):
                acc()
            b.record()
            torch.cuda.synchronize()
            # per-stage times of one more call (stage events on the launching stream)
            sev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(nst)]
            for e0, e1 in sev:
                e0.record()
                e1.record()
            torch.cuda.synchronize()
            P.eer4d_set_stage_events(rf.plan, [e[0] for e in sev], [e[1] for e in sev])
            m0 = torch.cuda.Event(enable_timing=True)
            m0.record()
            acc()
            torch.cuda.synchronize()
            P.eer4d_set_stage_events(rf.plan)
            f_stages = {n: round(sev[i][0].elapsed_time(sev[i][1]), 4) for i, n in enumerate(P._lib.STAGES)
                        if m0.elapsed_time(sev[i][0]) >= 0.0}
            ph_f = torch.empty(1, Ny, w.scan_nx, dtype=torch.float32, device=dev)
            P.ssb_reconstruct(rf.plan, rf.G, theta, rf.scratch, ph_f, v1, status=rf.status)
            torch.cuda.synchronize()
            rf.check()
            if name == "fp32_fused":
                ref_ph.copy_(ph_f)
            err = float((ph_f - ref_ph).double().norm() / ref_ph.double().norm())
            forms[name] = {"accumulate_ms": a.elapsed_time(b) / 3, "stages_ms": f_stages,
                           "phase_rel_l2_vs_fused": err}
            del rf
            torch.cuda.empty_cache()
        # vendor library beside the fused form, for comparison only (it is not
        # part of the path): cuFFT's batched 2D R2C (torch.fft.rfft2) of the
        # same counts as fp32 [P_pad][Ny][Nx] (the conversion is not timed),
        # output [P_pad][Ny][Nx/2+1] left in its own layout
        if Ny == w.scan_nx:
            rf = P.Reconstructor(geom, precision=P.FP32_FFT, device=dev)
            P.ssb_accumulate(rf.plan, idx, off, 0, rf.work, rf.G, True, status=rf.status)
            cnt32 = rf.counts.view(P_pad, Ny, w.scan_nx).float()
            Gc = torch.fft.rfft2(cnt32)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(3):
                Gc = torch.fft.rfft2(cnt32)
            b.record()
            torch.cuda.synchronize()
            # the same transform: our G [K_x][p][K_y] against the library's on
            # three pixels, every K
            Gv = torch.view_as_complex(rf.G.view(-1, 2)).view(nkx, P_pad, Ny)
            num = den = 0.0
            for pp in (0, P_pad // 2, rec.info["P"] - 1):
                ours = Gv[:, pp, :].to(torch.complex128)
                lib = Gc[pp].transpose(0, 1).to(torch.complex128)
                num += float((ours - lib).abs().pow(2).sum())
                den += float(lib.abs().pow(2).sum())
            forms["cufft_rfft2_fp32_reference"] = {
                "transform_ms": a.elapsed_time(b) / 3,
                "what": "vendor cuFFT batched 2D R2C of the fp32 counts (comparison only, not the path); "
                        "compare with fp32_fused stages_ms.dft_xy, which also reads fp16 and writes G transposed",
                "G_rel_l2_vs_fused_3_pixels": (num / den) ** 0.5 if den > 0 else None}
            del rf, cnt32, Gc, Gv
            torch.cuda.empty_cache()
        out["dft_forms"] = forms

    # ---- end to end through the public API with host buffers -------------
    # every step uploads its events from pinned host memory and reads its
    # phase image and variance back; StreamedSteps overlaps the upload of
    # step k+1 with the computation of step k (copy engine, second stream)
    if not args.no_e2e:
        h_idx = idx.cpu().pin_memory()
        h_off = off.cpu().pin_memory()
        h_phase = torch.empty_like(phase, device="cpu").pin_memory()
        h_var = torch.empty(1, dtype=torch.float64).pin_memory()
        pipe = P.StreamedSteps(idx.numel(), F, device=dev)

        def body(di, do):
            step(di, do)
            h_phase.copy_(phase, non_blocking=True)
            h_var.copy_(var, non_blocking=True)

        for _ in range(args.warmup):
            pipe.run(h_idx, h_off, body)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        pipe.start(a)  # uploads of the timed steps begin after the start mark
        for _ in range(args.steps):
            pipe.run(h_idx, h_off, body)
        b.record()
        torch.cuda.synchronize()
        e_val, e_max = job_throughput(a.elapsed_time(b) / args.steps, C, world, device=dev)
        out["e2e"] = {"value": e_val, "unit": UNIT,
                      "h2d_bytes_per_step": h_idx.numel() * 4 + h_off.numel() * 8,
                      "d2h_bytes_per_step": h_phase.numel() * 4 + 8,
                      "ms_per_step": e_max,
                      "overlap": "upload of step k+1 on a copy stream during step k (StreamedSteps)"}
        assert torch.isfinite(h_phase).all()

    # ---- refocus: adjoint step (CUDA graph) vs the plain form ----------------
    if args.refocus_steps > 0:
        rg = P.refocus.RefocusGraph(rec, [0.0] * 5, step=[1e-3, 1e-3, 1e-3, 0.0, 0.0])
        lat = []
        for _ in range(args.refocus_steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            rg.graph.replay()
            b.record()
            b.synchronize()
            lat.append(a.elapsed_time(b))
        lat.sort()
        cands = torch.zeros(64, 5, dtype=torch.float64, device=dev)
        cands[:, 0] = torch.linspace(-200.0, 200.0, 64, dtype=torch.float64, device=dev)
        ph64 = torch.empty(64, Ny, w.scan_nx, dtype=torch.float32, device=dev)
        v64 = torch.empty(64, dtype=torch.float64, device=dev)

        def timed(fn, reps=3):
            fn()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                fn()
            b.record()
            torch.cuda.synchronize()
            return a.elapsed_time(b) / reps

        def plain_sweep():  # one unbatched forward (trotter + image + variance) per candidate
            for i in range(64):
                P.ssb_reconstruct(rec.plan, rec.G, cands[i], rec.scratch, phase, var, status=rec.status)

        t_plain1 = timed(lambda: P.ssb_reconstruct(rec.plan, rec.G, theta, rec.scratch, phase, var,
                                                   status=rec.status), reps=10)
        t_plain64 = timed(plain_sweep)
        t_b64v = timed(lambda: P.ssb_reconstruct(rec.plan, rec.G, cands, rec.scratch, None, v64,
                                                 status=rec.status))
        t_b64i = timed(lambda: P.ssb_reconstruct(rec.plan, rec.G, cands, rec.scratch, ph64, v64,
                                                 status=rec.status))
        out["refocus"] = {
            "adjoint_step_ms_p50": lat[len(lat) // 2],
            "adjoint_step_ms_p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
            "replays": len(lat), "graph": True,
            "adjoint_step": "V, dV/dtheta, phase image and ascent update: one pass over G",
            "plain_forward_ms": t_plain1,
            "plain_sweep64_ms": t_plain64,
            "batched_sweep64_var_ms": t_b64v,
            "batched_sweep64_images_ms": t_b64i,
            "phase_images_per_s": 64.0 / (t_b64i * 1e-3),
        }
        # the 64-candidate launch is bound by arithmetic, not by its G bytes:
        # per (pixel, bin, candidate) term the kernel evaluates chi(k - K') and
        # the phase (about 26 FP32-pipe operations: the polynomial, the turn
        # reduction, the rotation by e^{-i chi(k)}, the product with G and the
        # two accumulations) and two MUFU operations (sin, cos)
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        try:
            mhz = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"])
        except Exception:
            mhz = 2070.0
        terms = float(sigma_k) * 64
        fp32_peak = nsm * 128 * mhz * 1e6        # FP32 lanes per SM per clock
        mufu_peak = nsm * 16 * mhz * 1e6         # MUFU lanes per SM per clock
        t_alu = max(terms * 26 / fp32_peak, terms * 2 / mufu_peak)
        # the adjoint step (V and five derivatives per term, FP64 block sums):
        # about 26 forward and 65 derivative FP32-pipe operations per term
        # (the five dpsi/dtheta and their two weighted accumulations each)
        t_adj = lat[len(lat) // 2] * 1e-3
        out["refocus"]["adjoint_step_roofline"] = {
            "bound": "alu", "terms": float(sigma_k), "fp32_ops_per_term": 91,
            "frac": float(sigma_k) * 91 / fp32_peak / t_adj,
            "hbm_frac": (8 * sigma_k + 8 * Ny * nkx) / t_adj / 1e9 / hbm,
        }
        out["refocus"]["batched_sweep64_roofline"] = {
            "bound": "alu", "terms": terms, "fp32_ops_per_term": 26, "mufu_ops_per_term": 2,
            "peak_fp32_ops_s": fp32_peak, "peak_mufu_ops_s": mufu_peak,
            "achieved_fp32_ops_s": terms * 26 / (t_b64v * 1e-3),
            "frac": t_alu / (t_b64v * 1e-3),
            "hbm_frac": (8 * sigma_k + 8 * Ny * nkx * 64) / (t_b64v * 1e-3) / 1e9 / hbm,
            "peak_source": "unit counts (128 FP32, 16 MUFU lanes per SM) x SMs x max SM clock",
        }
        rec.check()

    # ---- refocus accuracy: adjoint fit vs grid search ----------------------------
    # the differentiation workload's optics (25 mrad, 1941 bright-field pixels,
    # true C1 = 8 nm, C12 = 3 nm at 30 deg, C3 = 1 um) on the benchmark's scan:
    # the plain arm is a 64-candidate defocus grid (-20..20 nm, the other
    # aberrations 0) in one batched launch; the adjoint arm takes the grid's
    # best defocus as its seed and replays the captured Adam step
    # (ssb_refocus_step_adam) over C1, C12a, C12b and C3.  The same steps
    # started from all aberrations 0 are reported too (at 1024x1024 they stop
    # at a local maximum of the variance; at 512x512 they converge).
    if args.refocus_steps > 0 and not args.no_refocus_fit and rank == 0:
        del rec
        torch.cuda.empty_cache()
        w3 = synth.workload(3, scan_ny=w.scan_ny, scan_nx=w.scan_nx)
        d3 = synth.generate(w3, dev)
        r3 = P.Reconstructor(synth.geometry(w3), n_cand=64, device=dev)
        r3.load(d3.idx, d3.off)
        del d3
        true = torch.tensor(w3.aberr, dtype=torch.float64)
        grid = torch.zeros(64, 5, dtype=torch.float64, device=dev)
        grid[:, 0] = torch.linspace(-200.0, 200.0, 64, dtype=torch.float64, device=dev)
        vg = torch.empty(64, dtype=torch.float64, device=dev)

        def grid_search():
            P.ssb_reconstruct(r3.plan, r3.G, grid, r3.scratch, None, vg, status=r3.status)

        def timed_ms(fn):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize()
            return a.elapsed_time(b)

        grid_search()
        torch.cuda.synchronize()
        t_grid = timed_ms(grid_search)
        best = grid[int(torch.argmax(vg))].cpu()
        err_grid = (best - true)[:4].abs().tolist()
        n_fit = 200
        arms = {}
        for arm, start in (("seeded", [float(best[0]), 0.0, 0.0, 0.0, 0.0]), ("from_zero", [0.0] * 5)):
            fg = P.refocus.RefocusGraph(r3, start, adam=[0.05, 0.05, 0.05, 0.05, 0.0])
            traj = []
            for k in range(n_fit):
                fg.replay()
                if (k + 1) % 10 == 0:
                    traj.append((k + 1, (fg.theta.cpu() - true)[:4].abs().tolist()))
            fg.reset()
            torch.cuda.synchronize()
            t_fit = timed_ms(lambda: fg.replay(n_fit))
            err_fit = (fg.theta.cpu() - true)[:4].abs().tolist()
            reach = next((k for k, e in traj if e[0] <= err_grid[0]), None)
            arms[arm] = {"start": start[:4], "steps": n_fit, "fit_ms": t_fit, "ms_per_step": t_fit / n_fit,
                         "abs_err": err_fit, "V": float(fg.var.item()),
                         "steps_to_grid_C1_accuracy": reach,
                         "ms_to_grid_C1_accuracy": None if reach is None else reach * t_fit / n_fit}
            del fg
        arms["seeded"]["total_ms"] = t_grid + arms["seeded"]["fit_ms"]
        r3.check()
        out["refocus_fit"] = {
            "workload": w3.name.replace("512x512", f"{w.scan_ny}x{w.scan_nx}"),
            "true": [float(v) for v in w3.aberr[:4]],
            "V_true": float(r3.variance_grad(true)[0]),
            "grid_search": {"candidates": 64, "what": "C1 in -20..20 nm, others 0, one batched launch",
                            "ms": t_grid, "abs_err": err_grid},
            "adjoint_fit": {"what": "graph-replayed Adam steps (ssb_refocus_step_adam) over C1, C12a, "
                                    "C12b, C3; seeded = from the grid's best C1", **arms},
            "abs_err_units": "A (C1, C12a, C12b, C3)",
        }
        del r3
        torch.cuda.empty_cache()

    # ---- uneven batches: 16 datasets in one launch vs one call each ----------
    if args.batching:
        rec = None
        torch.cuda.empty_cache()
        ws = synth.batching_datasets()
        recs = []
        for wb in ws:
            db = synth.generate(wb, dev)
            rb = P.Reconstructor(synth.geometry(wb), device=dev)
            rb.load(db.idx, db.off)
            recs.append(rb)
            del db
        abb = torch.tensor(synth.candidate_aberrations(n=len(ws)), device=dev)
        plans = [r.plan for r in recs]
        bscr = torch.empty(P.batched_scratch_bytes(plans), dtype=torch.uint8, device=dev)
        phs = [torch.empty(r.Ny, r.Nx, dtype=torch.float32, device=dev) for r in recs]
        vb = torch.empty(len(recs), dtype=torch.float64, device=dev)
        v1 = torch.empty(1, dtype=torch.float64, device=dev)

        def batched():
            P.ssb_reconstruct_batched(plans, [r.G for r in recs], abb, bscr, phs, vb, status=recs[0].status)

        def one_by_one():
            for i, r in enumerate(recs):
                P.ssb_reconstruct(r.plan, r.G, abb[i], r.scratch, phs[i], v1, status=r.status)

        def timed_b(fn, reps=5):
            fn()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                fn()
            b.record()
            torch.cuda.synchronize()
            return a.elapsed_time(b) / reps

        tb, ts1 = timed_b(batched), timed_b(one_by_one)
        out["batching"] = {
            "datasets": [r.Ny for r in recs], "batched_ms": tb, "one_call_each_ms": ts1,
            "phase_images_per_s": len(recs) / (tb * 1e-3),
            "what": "SSB phase + variance of 16 uneven square scans (config 4 detector), "
                    "ssb_reconstruct_batched vs one ssb_reconstruct per dataset",
        }
        recs[0].check()

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N = 1) ---------
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n_ev, ts, ws = time_oracle(256, str(dev), reps=1)
        out["cpu_baseline"] = {"value": n_ev / ts[0], "unit": UNIT, "cores": cpu_threads(),
                               "kind": "oracle",
                               "sample": f"256x256 scan of the same detector geometry and dose "
                                         f"({n_ev} events), whole oracle path, one run",
                               "seconds": ts[0], "affinity_cores": len(os.sched_getaffinity(0))}
    if rank == 0:
        print(json.dumps(out))


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
