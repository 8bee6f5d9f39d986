#!/usr/bin/env python3
"""Benchmark: image-series registration (preprocessing + prefix scan of the
registration operator) on a synthetic 400 x 1024^2 series, 5-level pyramid.

One step = one full series registration on a handle whose frames and pyramid
are resident in HBM: all A(f_e, f_{e+1}) applications in one batch, then every
level of the scan schedule as one batch.  value = operator applications per
second (A + B) over the whole job; ms_per_step = series time.

Prints one JSON line on rank 0.  Multi-GPU (torchrun): every rank registers
its own series (independent problems, weak scaling, no collective on the data
path); the timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(name="c3_400x1024", seed=3, n_frames=400, side=1024, spacing=16.0, sigma=2.0, peak=5.0,
                drift_sd=1.0, dist_amp=2.0, n_levels=5, iter_max=50, lam=10.0)
METRIC = "operator applications/s and series scan time at 400x1024^2; % of HBM roofline"
UNIT = "op-apps/s"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--kind", default="sklansky",
                    choices=["serial", "sklansky", "kogge_stone", "brent_kung", "blelloch", "chunked", "chunked_alt",
                             "han_carlson", "ladner_fischer"])
    ap.add_argument("--chunks", type=int, default=None,
                    help="chunk count of the chunked kinds (default 16), k of han_carlson and ladner_fischer (default 1)")
    ap.add_argument("--frames", type=int, default=WORKLOAD["n_frames"])
    ap.add_argument("--side", type=int, default=WORKLOAD["side"])
    ap.add_argument("--levels", type=int, default=WORKLOAD["n_levels"])
    ap.add_argument("--preprocess-only", action="store_true",
                    help="a step is the preprocessing batch only (profiling case)")
    ap.add_argument("--autotune", type=int, default=64,
                    help="pairs in the tile autotuner's sample batch before timing (0: default tiles)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cnn", action="store_true", help="skip the CNN tensor-core roofline entry")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-initialiser leg")
    ap.add_argument("--learned-pairs", type=int, default=4096, help="training pairs of the learned leg")
    ap.add_argument("--no-cpu", action="store_true")
    return ap.parse_args()


# DRAM traffic per launch, estimated from one ncu capture per kernel (a bulk
# launch of 16 operators at the finest level, 1025^2 nodes each; the bench's
# own launches are too many to capture): its dram__bytes_read.sum +
# dram__bytes_write.sum over its library bytes (the kernel statistics' count:
# 36 B per node for a trial pass, 60 B for a gradient pass, FP32 images),
# times a bench launch's library bytes.  Recorded for one kernels.cu source
# (re-keyed after changes elsewhere in the file that leave k_trial and k_grad
# as captured); any other source reports no traffic.
TRAFFIC_CAPTURE = {"kernels_cu_sha1": "e6d63029c90d2dfd1074d5829260f689e608cb95",
                   "trial": (416.283904 + 5.409536) / (16 * 1025 * 1025 * 36 / 1e6),
                   "grad": (505.808128 + 340.208384) / (16 * 1025 * 1025 * 60 / 1e6)}


def _traffic(family, algo_bytes_per_launch):
    import hashlib
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1712_02533_gb300", "csrc", "kernels.cu")
    try:
        sha = hashlib.sha1(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    if sha != TRAFFIC_CAPTURE["kernels_cu_sha1"] or family not in TRAFFIC_CAPTURE:
        return None
    return round(TRAFFIC_CAPTURE[family] * algo_bytes_per_launch)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


FAMILIES = ("prolong", "grad", "trial", "control", "plan", "setup")

# Algorithmic bytes per node of the step kernels in the survey's model of one
# gradient iteration (FP32 storage): the gradient pass reads u and d (16 B), the
# template (4) and M~R~ (4) and writes u and d (16): 40 B; every sequential
# Armijo trial reads u and d, the template and M~R~: 24 B; every per-level
# setup pass 16 B.  With BF16 images the template read is 2 B.
MODEL_BYTES = {"grad": 40.0, "trial_seq": 24.0, "trial_start": 16.0}


def roofline_of(stats, cfg, bf16=False):
    """Roofline of the dominant step kernel from one profiled step: achieved =
    model bytes per launch / mean launch time (CUDA events), against the
    measured HBM peak; the library's own byte count (what the kernels read and
    write per node: the 32-byte node records) is given beside it."""
    peak, peak_kind = _peaks()
    img_save = 2.0 if bf16 else 0.0
    model = {"grad": stats["grad"]["items"] * (MODEL_BYTES["grad"] - img_save),
             "trial": stats["trial_seq_nodes"]["items"] * (MODEL_BYTES["trial_seq"] - img_save)
             + stats["trial_start_nodes"]["items"] * MODEL_BYTES["trial_start"],
             "prolong": None}
    fams = {k: v for k, v in stats.items() if k in ("grad", "trial", "prolong")}
    dom = max(fams, key=lambda k: fams[k]["ms"])
    dk = fams[dom]
    launches = max(1, dk["launches"])
    sec = dk["ms"] * 1e-3
    mb = model[dom] if model[dom] is not None else dk["bytes"]
    achieved = mb / sec / 1e9 if sec > 0 else 0.0
    lib_achieved = dk["bytes"] / sec / 1e9 if sec > 0 else 0.0
    total_ms = sum(v["ms"] for k, v in stats.items() if k in FAMILIES)
    kern = {}
    for k, v in stats.items():
        if k not in FAMILIES:
            continue
        e = {"ms": round(v["ms"], 2), "launches": v["launches"], "share": round(v["ms"] / total_ms, 4) if total_ms else None,
             "GBps_library_bytes": round(v["bytes"] / (v["ms"] * 1e-3) / 1e9, 1) if v["ms"] > 0 and v["bytes"] else None}
        if model.get(k):
            e["GBps_model_bytes"] = round(model[k] / (v["ms"] * 1e-3) / 1e9, 1) if v["ms"] > 0 else None
        kern[k] = e
    seq_per_pass = (stats["trial_seq_nodes"]["items"] / max(1, stats["trial"]["items"] - stats["trial_start_nodes"]["items"]))
    return {"bound": "hbm", "kernel": f"k_{dom}", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_source": peak_kind,
            "bytes_model": "40 B/node per gradient pass + 24 B/node per sequential Armijo trial + 16 B/node per "
                           "level-start pass (FP32 storage)",
            "traffic": _traffic(dom, dk["bytes"] / launches), "traffic_note": "estimated: DRAM/library-byte ratio of one ncu "
                       "capture (a 16-operator launch at the finest level) times this launch's library bytes (null "
                       "if the kernel source changed)",
            "bytes_per_launch": mb / launches, "library_bytes_per_launch": dk["bytes"] / launches,
            "achieved_library_bytes": round(lib_achieved, 1), "frac_library_bytes": round(lib_achieved / peak, 4),
            "ms_per_launch": dk["ms"] / launches, "sequential_trials_per_trial_pass": round(seq_per_pass, 3),
            "kernels": kern}


def cnn_roofline(reg, s, torch, batch=64, reps=20):
    """Tensor-core roofline of the learned initialiser's forward pass: the 64
    network inputs of the series' first neighbour pairs through the 6-layer
    CNN (the four 32->32 layers on the BF16 tensor cores), timed with CUDA
    events; FLOPs = 2 x multiply-adds of all six layers (0.326 GFLOP per pair)."""
    import synth
    peak = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak, src = float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        peak, src = 1900.0, "fallback"
    x = torch.empty((batch, 2, 256, 256), dtype=torch.float32, device="cuda")
    s.cnn_pairs(0, batch, x)
    flop_pair = 0.0
    side = 256
    for (c, o), stride in zip(synth.CNN_SHAPES, (2, 2, 1, 1, 1, 1)):
        side //= stride
        flop_pair += 2.0 * side * side * o * c * 9
    with reg.Cnn(synth.cnn_params(1), side=256, max_batch=batch) as net:
        y = net.forward(x, tensor_cores=True)
        for _ in range(3):
            net.forward(x, y, tensor_cores=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            net.forward(x, y, tensor_cores=True)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
    tflops = flop_pair * batch / (ms * 1e-3) / 1e12
    return {"bound": "tensor", "kernel": "CNN forward (k_conv32_umma_fwd, tcgen05 + TMA, on the four 32->32 layers, BF16 operands, FP32 "
                                        "accumulation; the 2->32 and 32->2 layers on the CUDA cores)",
            "achieved": round(tflops, 2), "peak": peak, "unit": "TFLOP/s", "frac": round(tflops / peak, 5),
            "peak_source": src, "batch": batch, "ms_per_forward": round(ms, 4),
            "gflop_per_pair": round(flop_pair / 1e9, 4), "traffic": None}


def learned_leg(reg, fd, cfg, kind, chunks, plain_d, tiles, n_pairs=4096, epochs=20, init_levels=(1, 3)):
    """The learned form on the benchmark's series: a network trained on the
    tensor cores on n_pairs neighbour pairs of other generator series of the
    same shape (targets: the plain method's displacements), then the series
    registered with the network's start on the finest init_levels levels (the
    plain method judging every start), timed with CUDA events from resident
    frames to all deformations, network inference included, and compared with
    the plain result of the timed steps (distance over the frames' interior,
    32 px margin)."""
    import torch
    import synth
    from paper_1712_02533_gb300 import learned
    gen = {k: v for k, v in synth.CONFIGS["c3_400x1024"].items() if k not in ("seed", "n_frames", "side", "n_levels")}
    t0 = time.time()
    x, t = learned.training_set(n_pairs, seed=4000, frames_per_series=64, n_levels=cfg["n_levels"], side=cfg["side"],
                                series_kw=gen)
    torch.cuda.synchronize()
    t1 = time.time()
    net = reg.Cnn(synth.cnn_params(1), side=256, max_batch=64)
    hist = learned.train(net, x, t, epochs=epochs, batch=32, lr=1e-3, lr_final=1e-4, tensor_cores=True)
    torch.cuda.synchronize()
    t2 = time.time()
    del x, t
    forms = []
    m = 32
    for il in init_levels:
        p = reg.default_params(n_levels=cfg["n_levels"], iter_max=cfg["iter_max"], lam=cfg["lam"], init_levels=il)
        if tiles:
            p.trials_per_pass = tiles["trials_per_pass"]
        with reg.Series([fd], p) as s:
            for lv in (tiles or {}).get("levels", []):
                s.set_tile_rows(lv["level"], lv["grad_rows"], lv["trial_rows"])
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            s.cnn_init(net, tensor_cores=True)
            rep = s.prefix_scan(kind, chunks, reg.KOGGE_STONE)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            d = torch.empty_like(plain_d)
            s.get_deformations(out=d)
        dev = (d[1:] - plain_d[1:]).abs()[:, :, m:-m, m:-m]
        forms.append({"init_levels": il, "series_ms": round(ms, 2), "op_apps_per_s": round(rep["ops"] / (ms * 1e-3), 3),
                      "dev_from_plain_mean_px": float(dev.mean()), "dev_from_plain_max_px": float(dev.max()),
                      "frac_within_0.05px": float((dev <= 0.05).float().mean()), "judged": rep.get("learned"),
                      "iters": rep["iters"]})
        del d, dev
    net.close()
    return {"network": "trained on the tensor cores (BF16 operands, FP32 accumulation)", "train_pairs": n_pairs,
            "epochs": epochs, "loss_first": hist[0], "loss_last": hist[-1], "data_s": round(t1 - t0, 1),
            "train_s": round(t2 - t1, 1), "forms": forms,
            "note": "one timed run per form, first run of its handle (graph capture included)"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if p[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def rank_seed(seed, rank):
    """Seed of the series that rank registers: every rank works on its own series
    (independent problems, no collective on the data path)."""
    return seed + 1000 * rank


def max_over_ranks(x, world, device="cpu"):
    """The largest value of x over all ranks (the job takes as long as its slowest
    rank); x itself when there is one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, seconds):
    """Whole-job throughput: the units all ranks processed over the job's time."""
    return world * units_per_rank / seconds


def cpu_baseline(frames, cfg, n_ops=None, budget_s=30.0):
    """The FP64 oracle as it stands, on a bounded sample: A(f_e, f_{e+1}) ops of
    the same series and parameters, run in parallel over the host cores."""
    import numpy as np
    import oracle
    cores = os.cpu_count() or 1
    n = n_ops or min(cores, 16)
    p = oracle.params(n_levels=cfg["n_levels"], iter_max=cfg["iter_max"], lam=cfg["lam"])
    g = [oracle.embed(frames[e]) for e in range(n + 1)]
    t = time.time()
    oracle.apply_batch([dict(R=g[e], T=g[e + 1]) for e in range(n)], p)
    dt = time.time() - t
    return {"value": n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} A operator applications (frame pairs 0..{n}) of the {cfg['name']} series, "
                      f"{cfg['side']}^2, {cfg['n_levels']} levels, iter_max {cfg['iter_max']}, "
                      f"run in parallel over {cores} host threads; {dt:.1f} s"}


def main():
    a = _args()
    import numpy as np

    cfg = dict(WORKLOAD)
    cfg["n_frames"], cfg["side"], cfg["n_levels"] = a.frames, a.side, a.levels
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if a.impl == "reference":
        if rank != 0:
            return 0
        import synth
        frames = synth.series(cfg["seed"], 17, cfg["side"], spacing=cfg["spacing"], sigma=cfg["sigma"],
                              peak=cfg["peak"], drift_sd=cfg["drift_sd"], dist_amp=cfg["dist_amp"])
        for _ in range(a.warmup):  # untimed, as on the GPU arm
            cpu_baseline(frames, cfg)
        vals = []
        for _ in range(max(1, a.steps)):
            cb = cpu_baseline(frames, cfg)
            vals.append(cb["value"])
        v = float(np.median(vals))
        cb["value"] = v
        # operator applications of one full step of the workload (preprocessing + scan)
        from oracle import schedules as OS
        kind = {name: k for k, name in OS.NAMES.items()}.get(a.kind, OS.SKLANSKY)
        n_data = cfg["n_frames"] - 1
        step_ops = n_data + OS.counts(OS.schedule(kind, n_data, a.chunks if a.chunks is not None else
                                                  (1 if kind in (OS.HAN_CARLSON, OS.LADNER_FISCHER) else 16)))[0]
        out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
               "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(step_ops / v * 1e3, 1),
               "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {"workload": cfg["name"], "frames": cfg["n_frames"], "side": cfg["side"],
                          "levels": cfg["n_levels"], "schedule": a.kind, "ops_per_step": step_ops,
                          "note": "FP64 CPU oracle on a bounded sample of the workload; ms_per_step "
                                  "extrapolated from the sample's rate to the step's operator applications"},
               "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out), flush=True)
        return 0

    import torch
    import synth
    import paper_1712_02533_gb300 as reg

    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    kind = {v: k for k, v in reg.SCAN_NAMES.items()}[a.kind]

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # each rank registers its own series (independent problems)
    t0 = time.time()
    frames = synth.series(rank_seed(cfg["seed"], rank), cfg["n_frames"], cfg["side"], spacing=cfg["spacing"],
                          sigma=cfg["sigma"], peak=cfg["peak"], drift_sd=cfg["drift_sd"], dist_amp=cfg["dist_amp"])
    gen_s = time.time() - t0
    # the product path: the step kernels replayed as captured CUDA graphs (flags 0)
    params = reg.default_params(n_levels=cfg["n_levels"], iter_max=cfg["iter_max"], lam=cfg["lam"], flags=0)
    fd = torch.from_numpy(frames).to(dev)
    torch.cuda.synchronize()
    t0 = time.time()
    s = reg.Series([fd], params)
    torch.cuda.synchronize()
    create_s = time.time() - t0

    n_pre = cfg["n_frames"] - 1
    pre_ops = [(0, -1, -1, e, e, e + 1) for e in range(n_pre)]
    tiles = None
    if a.autotune > 0:
        t0 = time.time()
        tiles = s.autotune(n_pairs=min(a.autotune, n_pre), repeats=1)
        tiles["tune_s"] = round(time.time() - t0, 1)

    def step():
        if a.preprocess_only:
            s.apply_operator_batch(pre_ops)
            return {"ops": n_pre, "preprocessing_ops": n_pre, "scan_ops": 0, "scan_batches": 0, "iters": None}
        return s.prefix_scan(kind, a.chunks, reg.KOGGE_STONE)

    for _ in range(a.warmup):
        step()
    s.reset_kernel_stats()
    sampler = ClockSampler(dev)
    barrier()
    sampler.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    ev0.record(stream)
    reports = []
    for _ in range(a.steps):
        reports.append(step())
    ev1.record(stream)
    barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    timed = s.kernel_stats()  # launches, algorithmic bytes and node counters of the timed steps
    ops_per_step = reports[-1]["ops"]
    ms = max_over_ranks(ms, world, dev)
    ms_step = ms / a.steps
    value = job_rate(world, ops_per_step, ms_step / 1e3)

    # Per-kernel device times: one more step, untimed, with every step kernel
    # launched directly between CUDA events on the library's stream
    # (REG_FLAG_PROFILE); the same work as a timed step.
    s.set_flags(reg.FLAG_PROFILE)
    s.reset_kernel_stats()
    prof_rep = step()
    torch.cuda.synchronize()
    stats = s.kernel_stats()
    s.set_flags(0)
    roofline = roofline_of(stats, cfg, bf16=False)
    roofline["profiled_step_ms"] = round(prof_rep["ms"], 2) if prof_rep.get("ms") else None
    gpu_launches = int(sum(v["launches"] for k, v in timed.items() if k in FAMILIES))
    roofline_cnn = None if a.preprocess_only or a.no_cnn else cnn_roofline(reg, s, torch)
    learned_res = None
    if not (a.preprocess_only or a.no_learned) and world == 1:
        plain_d = torch.empty((cfg["n_frames"], 2, cfg["side"], cfg["side"]), dtype=torch.float32, device=dev)
        s.get_deformations(out=plain_d)
        learned_res = learned_leg(reg, fd, cfg, kind, a.chunks, plain_d, tiles, n_pairs=a.learned_pairs)
        learned_res["plain_series_ms"] = round(ms_step, 2)
        for f in learned_res["forms"]:
            f["speedup_vs_plain"] = round(ms_step / f["series_ms"], 4)

    # end to end through the C-ABI with host buffers (upload, pyramid, scan, download)
    e2e = None
    if not a.no_e2e and not a.preprocess_only:
        host = torch.from_numpy(frames).pin_memory()
        out = torch.empty((cfg["n_frames"], 2, cfg["side"], cfg["side"]), dtype=torch.float32).pin_memory()
        p2 = reg.default_params(n_levels=cfg["n_levels"], iter_max=cfg["iter_max"], lam=cfg["lam"])
        if tiles:
            p2.trials_per_pass = tiles["trials_per_pass"]
        e2e_steps = max(1, a.steps)
        barrier()
        t = time.time()
        phases = []  # per step: wall ms of creation (upload + pyramid), scan, download, release
        for _ in range(e2e_steps):
            t_a = time.time()
            with reg.Series([host], p2) as s2:
                for lv in (tiles or {}).get("levels", []):  # the tuned table, as a user reuses it
                    s2.set_tile_rows(lv["level"], lv["grad_rows"], lv["trial_rows"])
                t_b = time.time()
                r2 = s2.prefix_scan(kind, a.chunks, reg.KOGGE_STONE)
                t_c = time.time()
                s2.get_deformations(out=out)
                t_d = time.time()
            t_e = time.time()
            phases.append([round((y - x) * 1e3, 1) for x, y in ((t_a, t_b), (t_b, t_c), (t_c, t_d), (t_d, t_e))])
        barrier()
        e2e_s = max_over_ranks((time.time() - t) / e2e_steps, world, dev)
        e2e = {"value": job_rate(world, r2["ops"], e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": int(host.numel() * 4), "d2h_bytes_per_step": int(out.numel() * 4),
               "ms_per_step": round(e2e_s * 1e3, 2),
               "phases_ms": {"order": ["create", "scan", "download", "release"], "steps": phases}}
    s.close()

    if rank == 0:
        cb = None
        if not a.no_cpu and world == 1:
            cb = cpu_baseline(frames, cfg)
        rep = reports[-1]
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": round(ms_step, 2), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (f64 global sums)", "data": "synthetic",
            "config": {"workload": cfg["name"], "frames": cfg["n_frames"], "side": cfg["side"],
                       "levels": cfg["n_levels"], "iter_max": cfg["iter_max"], "lambda": cfg["lam"],
                       "schedule": a.kind,
                       "chunks": (a.chunks or 16) if "chunked" in a.kind else None,
                       "hybrid_k": (a.chunks if a.chunks is not None else 1)
                       if a.kind in ("han_carlson", "ladner_fischer") else None,
                       "ops_per_step": ops_per_step, "preprocessing_ops": rep["preprocessing_ops"],
                       "scan_ops": rep["scan_ops"], "scan_batches": rep["scan_batches"],
                       "iters_per_step": rep["iters"], "trials_per_step": rep.get("trials"),
                       "timed_path": "captured CUDA graphs (8 steps per replay); per-kernel times from one "
                                     "more untimed step with per-kernel CUDA events",
                       "l2": "working set (GBs) larger than L2; no flush",
                       "tiles": tiles,
                       "generator_s": round(gen_s, 1), "create_ms": round(create_s * 1e3, 1)},
            "roofline": roofline, "roofline_cnn": roofline_cnn, "learned": learned_res, "cpu_baseline": cb, "e2e": e2e,
            "gpu_launches": gpu_launches,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
