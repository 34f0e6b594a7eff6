"""Benchmark of the mixture-of-media random walk on B300.

One step = one sss_walk over the spectral workload: a 256 x 256 texel
parameter field x 81 bands (380-780 nm), three media per texel and band,
4096 paths per instance, 64 radial bins over 10 mm, semi-infinite slab with
n = 1.4 (Fresnel faces).  The metric is paths/s on the whole job.  Beside it:
the same metric end to end through the public API with host buffers, the
adjoint/forward time ratio on the adjoint workload (64 x 64 x 81 at 2^16
paths), the ALU roofline of the walk kernel and the FP64 oracle timed on the
host cores on a sample of the same workload.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl b300|reference] [--strong]
Under torchrun (N > 1) the batch is sharded by contiguous instance ranges
(instance_offset = the range's first global instance), so every path keeps
its random numbers whatever the rank count:
  * default (weak scaling): rank r walks its own full-size field as
    instances r*n .. r*n + n - 1 of a global batch of N fields; there is no
    collective on the data path;
  * --strong: one field is cut into N ranges and every step ends with one
    all_gather of R and the radial bins (the only exchange the walk has).
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "mixture random-walk paths/s on 1 B300 (81 bands); adjoint/forward time ratio"
UNIT = "paths/s"
WORKLOAD = dict(workload="spectral_field_256x256x81", texels=256 * 256, bands=81,
                paths_per_instance=4096, nbins=64, r_max_mm=10.0, n_rel=1.4,
                slab="semi-infinite", K=3, param_seed=1, walk_seed=1001)
# Algorithmic lane-operations of one walk step: one Philox4x32-10 block
# (10 rounds of two 32x32->64 multiplies, two XORs and the key bump, about
# 60-70 integer lane-operations) plus the step's binary32 work (flight,
# move, face test, weighting, Henyey-Greenstein, rotation, renormalisation,
# about 40-50), about 110 in all; about 6 of the special-function unit.
ALG_ALU_OPS_PER_STEP = 110
ALG_FP32_OPS_PER_STEP = 50
ALG_MUFU_OPS_PER_STEP = 6
SM_LANES_PER_CLK = 128
MUFU_LANES_PER_CLK = 16
# Multiply-adds per texel of the chained decoder (unpadded): Enc 3-256-256-5,
# Dec_R 5-512-512-376, Dec_T 381-768-768-768 and the 121 source bands x 12
# outputs that the 81 visible bands need.
DECODER_MACS_PER_TEXEL = (3 * 256 + 256 * 256 + 256 * 5) + (5 * 512 + 512 * 512 + 512 * 376) \
    + (381 * 768 + 2 * 768 * 768 + 768 * 121 * 12)


# DRAM traffic of the walk kernel from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum) of the 1024-texel case, scaled by 64 to the
# 65536-texel launch (the traffic grows with the instances walked).  Valid
# only while the kernel sources are the ones captured (sha1 below).
WALK_TRAFFIC = {"bytes_per_launch": (61.70496e6 + 11.221504e6) * 64,
                "source_sha1": "99fb3fb6d1fbd7e0e34e140e7182d0b8185e9a87"}


def _walk_source_sha1():
    import hashlib
    h = hashlib.sha1()
    for f in ("walk_core.cuh", "walk_kernels.cu"):
        with open(os.path.join(ROOT, "paper_2606_27604_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _measured_peak(key, fallback):
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            v = float(json.load(f)[key])
        return v, "of measured"
    except (OSError, ValueError, KeyError):
        return fallback, "of fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def spectral_inputs(rank):
    from paper_2606_27604_b300 import inputs
    return inputs.spectral_field(n_texels=WORKLOAD["texels"],
                                 param_seed=WORKLOAD["param_seed"] + rank,
                                 n_paths=WORKLOAD["paths_per_instance"], n_rel=1.4)


def cpu_baseline_sample(n_texels=64, with_other_configs=True):
    """The FP64 oracle on a bounded sample of the workload (host cores); with
    `with_other_configs`, also on bounded samples of the other workloads."""
    import oracle
    from paper_2606_27604_b300 import inputs
    x = inputs.spectral_field(n_texels=n_texels, param_seed=WORKLOAD["param_seed"],
                              n_paths=WORKLOAD["paths_per_instance"], n_rel=1.4)
    o = oracle.OracleOpts(nbins=64, r_max_mm=10.0, seed=WORKLOAD["walk_seed"])
    t0 = time.perf_counter()
    oracle.walk(x.alpha, x.sigma_t, x.g, x.w, x.n_paths, None, x.n_rel, o)
    dt = time.perf_counter() - t0
    paths = int(x.n_paths.sum())
    res = {"value": paths / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"{n_texels} texels x 81 bands x 4096 paths ({paths} paths) of the "
                     f"spectral workload, FP64, {dt:.1f} s"}
    if with_other_configs:
        res["other_configs"] = cpu_other_configs()
    return res


def cpu_other_configs():
    """The FP64 oracle on bounded samples of the other workloads' shapes."""
    import oracle
    from paper_2606_27604_b300 import inputs
    per_config = {}
    x0 = inputs.single_wavelength(param_seed=0, n_paths=1 << 18)
    o0 = oracle.OracleOpts(nbins=32, r_max_mm=10.0, seed=1000)
    t = time.perf_counter()
    r0 = oracle.walk(x0.alpha, x0.sigma_t, x0.g, x0.w, x0.n_paths, None, x0.n_rel, o0)
    d0 = time.perf_counter() - t
    p0 = int(x0.n_paths.sum())
    per_config["single_wavelength_16_sets"] = {
        "paths_per_s": p0 / d0, "sample": f"all 16 sets x 2^18 paths ({p0} paths), {d0:.1f} s",
        "steps_per_path": float(np.mean(r0["steps"]))}
    xu = inputs.uneven_batch(n_inst=4096, param_seed=2).subset(np.arange(0, 4096, 64))
    ou = oracle.OracleOpts(nbins=64, r_max_mm=10.0, seed=1002)
    t = time.perf_counter()
    ru = oracle.walk(xu.alpha, xu.sigma_t, xu.g, xu.w, xu.n_paths, xu.thickness_mm, xu.n_rel, ou)
    du = time.perf_counter() - t
    pu = int(xu.n_paths.astype(np.int64).sum())
    per_config["uneven_batch"] = {
        "paths_per_s": pu / du,
        "sample": f"every 64th of the 4096 uneven instances ({xu.n_inst} instances, {pu} paths), "
                  f"{du:.1f} s",
        "steps_per_path": float(np.average(ru["steps"], weights=xu.n_paths))}
    return per_config


def pipeline_leg(side=1024, oracle_block=32, dev_index=0):
    """RGB texture -> decoder (tensor cores) -> batched walk at 1024 paths per
    texel and band (the full-pipeline workload), timed on the GPU, with the
    error of R against the FP64 oracle pipeline (oracle decoder + oracle
    walk, same Philox streams) on a 32 x 32 texel block and that oracle
    pipeline timed on the host cores."""
    import torch
    import oracle
    from oracle import decoder as dec_ref
    from paper_2606_27604_b300 import api, inputs
    T = side * side
    dev = torch.device("cuda", dev_index)
    rgb_np = inputs.rgb_texture(side=side, seed=4)
    W = inputs.decoder_weights(seed=4)
    rgb = torch.from_numpy(rgb_np).to(dev)
    packed = api.decoder_pack(W, device=dev)
    dws = torch.empty(api.lib.sss_decode_workspace_size(T), dtype=torch.uint8, device=dev)
    prm = {k: torch.empty(3, 81 * T, dtype=torch.float32, device=dev)
           for k in ("alpha", "g", "sigma_t", "w")}
    o = api.WalkOptions(nbins=64, r_max_mm=10.0, seed=1004)
    m = api.Media(prm["alpha"], prm["sigma_t"], prm["g"], prm["w"], None, 1024, None, 1.4)
    wsp = api.alloc_workspace(m, o)
    # only the outputs the comparison reads (the full set would add ~90 GB)
    d = lambda: torch.empty(m.n_inst, dtype=torch.float64, device=dev)
    out = {"R": d(), "stderr_R": d(), "steps": d()}
    stream = torch.cuda.current_stream(dev)
    api.decode(rgb, packed, workspace=dws, out=prm)      # warm-up
    api.walk(m, o, workspace=wsp, out=out)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record(stream)
    api.decode(rgb, packed, workspace=dws, out=prm)
    e[1].record(stream)
    api.walk(m, o, workspace=wsp, out=out)
    e[2].record(stream)
    torch.cuda.synchronize()
    t_dec, t_walk = e[0].elapsed_time(e[1]) / 1e3, e[1].elapsed_time(e[2]) / 1e3
    dcode, _ = api.read_status(dws)
    wcode, _ = api.read_status(wsp)
    # oracle pipeline on a 32 x 32 block of texels (rows 0..31, columns 0..31)
    blk = (np.arange(oracle_block)[:, None] * side + np.arange(oracle_block)[None, :]).ravel()
    sub = len(blk)
    t_or = time.perf_counter()
    ref = dec_ref.decode(rgb_np[blk], W, bf16_activations=True)
    ids = (np.arange(81)[:, None] * T + blk[None, :]).reshape(-1)   # band-major numbers
    refw = oracle.walk(ref["alpha"].astype(np.float32), ref["sigma_t"].astype(np.float32),
                       ref["g"].astype(np.float32), ref["w"].astype(np.float32),
                       np.full(81 * sub, 1024, np.uint32), None, 1.4,
                       oracle.OracleOpts(nbins=64, r_max_mm=10.0, seed=1004), inst_ids=ids)
    t_or = time.perf_counter() - t_or
    ii = torch.from_numpy(ids).to(dev)
    R = out["R"][ii].cpu().numpy()
    se = np.sqrt(refw["se_R"] ** 2 + out["stderr_R"][ii].cpu().numpy() ** 2)
    z = (R - refw["R"]) / np.maximum(se, 1e-12)
    paths = 81.0 * T * 1024
    res = {"workload": f"{side}x{side} RGB -> decoder -> 81 bands x 1024 paths, 64 bins, n=1.4",
           "decode_ms": t_dec * 1e3, "walk_ms": t_walk * 1e3,
           "total_ms": (t_dec + t_walk) * 1e3, "paths_per_s": paths / (t_dec + t_walk),
           "steps_per_path": float(out["steps"].mean().item()),
           "status": [dcode, wcode],
           "subset": f"{oracle_block}x{oracle_block} texel block x 81 bands vs the FP64 oracle "
                     "decoder + oracle walk on the same Philox streams",
           "R_rel_err_median": float(np.median(np.abs(R - refw["R"]) / refw["R"])),
           "R_z_abs_max": float(np.abs(z).max()), "R_z_rms": float(np.sqrt((z ** 2).mean())),
           "frac_within_4sigma": float((np.abs(z) <= 4).mean()),
           "cpu_baseline": {"value": 81.0 * sub * 1024 / t_or, "unit": "paths/s",
                            "cores": oracle.num_threads(), "kind": "oracle",
                            "sample": f"the {oracle_block}x{oracle_block} block: FP64 decoder "
                                      f"and walk, {81 * sub * 1024} paths, {t_or:.1f} s"}}
    del wsp, out, prm, dws
    torch.cuda.empty_cache()
    return res


def run_pipeline(args):
    """The full pipeline alone, as one JSON line."""
    line = dict(metric="full pipeline RGB -> decoder -> walk",
                **pipeline_leg(side=args.pipeline_side))
    print(json.dumps(line), flush=True)
    return 0


def lut_leg(n, n_paths):
    """Scale-independent LUT precompute (one instance per (alpha, g) grid
    point, sigma_t = 1, K = 1), timed on the GPU, with the time the paper's
    800 x 800 x 10^6-path table would take at the same rate."""
    import torch
    from paper_2606_27604_b300 import lut
    alphas = np.linspace(0.0, 0.999, n)
    gs = np.linspace(0.0, 0.95, n)
    lut.build(alphas[:8], gs[:8], n_paths=1024, nbins=128)   # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L = lut.build(alphas, gs, n_paths=n_paths, nbins=128, r_max=32.0)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    paths = float(n * n) * n_paths
    return {"workload": f"{n}x{n} (alpha, g) grid x {n_paths} paths, 128 bins to 32 mfp, n=1.4",
            "seconds": dt, "paths_per_s": paths / dt,
            "full_paper_table_estimate_s": 800 * 800 * 1e6 / (paths / dt),
            "R_range": [float(L.R.min()), float(L.R.max())]}


def run_lut(args):
    line = dict(metric="LUT precompute paths/s (Sec. 4.2 tables R(alpha,g), P_d(r|alpha,g))",
                **lut_leg(args.lut_side, args.lut_paths))
    print(json.dumps(line), flush=True)
    return 0


def fit_leg(n, steps):
    """Batched LUT mixture fit (Sec. 4.2): K = 3, Adam, timed on the GPU and
    extrapolated to the paper's 25,000 tones x 376 bands x 10,000 steps."""
    import torch
    from paper_2606_27604_b300 import api, lut
    dev = torch.device("cuda", 0)
    alphas = np.linspace(0.5, 0.999, 64)
    gs = np.linspace(0.0, 0.95, 32)
    L = lut.build(alphas, gs, n_paths=1 << 14, nbins=64, r_max=32.0)
    dens = torch.from_numpy(L.density().astype(np.float32)).to(dev)
    Rl = torch.from_numpy(L.R.astype(np.float32)).to(dev)
    K = 3
    rng = np.random.default_rng(0)
    r = torch.from_numpy(np.linspace(0.05, 4.0, 64).astype(np.float32)).to(dev)
    lam = rng.uniform(0.5, 3.0, size=(n, 1))
    P_mc = torch.from_numpy((lam ** 2 / (2 * np.pi) * np.exp(-lam * np.linspace(0.05, 4.0, 64)[None, :]))
                            .astype(np.float32)).to(dev)
    R_mc = torch.from_numpy(rng.uniform(0.2, 0.7, size=n).astype(np.float32)).to(dev)
    raw0 = torch.zeros(n, 4 * K, dtype=torch.float32, device=dev)
    args_ = (Rl, dens, float(alphas[0]), float(alphas[1] - alphas[0]), float(gs[0]),
             float(gs[1] - gs[0]), L.r_max / 64, r, P_mc, R_mc)
    api.lut_fit(*args_, raw0.clone(), K=K, steps=10, a_rng=(0.5, 0.999))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    raw = raw0.clone()
    e0.record()
    loss, _ = api.lut_fit(*args_, raw, K=K, steps=steps, a_rng=(0.5, 0.999))
    e1.record()
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    rate = n * steps / sec
    return {"workload": f"{n} problems x {steps} steps, 64x32x64 table", "seconds": sec,
            "problem_steps_per_s": rate,
            "paper_workload_estimate_s": 25000 * 376 * 10000 / rate,
            "paper_workload_paper_time_s": 46 * 3600,
            "median_final_loss": float(loss.median().item())}


def run_fit(args):
    line = dict(metric="LUT mixture fit problem-steps/s (K=3, 64 radii, Adam)",
                **fit_leg(args.fit_problems, args.fit_steps))
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    per_step = []
    for _ in range(args.warmup):
        cpu_baseline_sample(args.ref_texels, with_other_configs=False)
    res = None
    for _ in range(args.steps):
        res = cpu_baseline_sample(args.ref_texels, with_other_configs=False)
        per_step.append(res["value"])
    res["other_configs"] = cpu_other_configs()
    v = float(np.mean(per_step))
    paths_per_step = args.ref_texels * 81 * 4096
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": paths_per_step / v * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(WORKLOAD, sample_texels=args.ref_texels),
            "cpu_baseline": dict(res, value=v),
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--ref-texels", type=int, default=16)
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-baselines", action="store_true",
                    help="skip the uneven-batch and plain one-launch-per-instance timings")
    ap.add_argument("--no-decoder", action="store_true")
    ap.add_argument("--decoder-side", type=int, default=1024,
                    help="texture side of the decoder line (default 1024; smaller for profiling)")
    ap.add_argument("--no-hero", action="store_true",
                    help="skip the hero-wavelength comparison")
    ap.add_argument("--no-probe", action="store_true",
                    help="skip the issue-rate probes")
    ap.add_argument("--pipeline", action="store_true",
                    help="run the full RGB -> decoder -> walk pipeline alone")
    ap.add_argument("--no-pipeline", action="store_true",
                    help="skip the full-pipeline leg of the default line")
    ap.add_argument("--pipeline-side", type=int, default=1024)
    ap.add_argument("--lut", action="store_true", help="time the LUT precompute instead")
    ap.add_argument("--no-lut", action="store_true",
                    help="skip the LUT precompute and LUT fit legs of the default line")
    ap.add_argument("--lut-side", type=int, default=128)
    ap.add_argument("--lut-paths", type=int, default=1 << 20)
    ap.add_argument("--fit", action="store_true", help="time the batched LUT fit instead")
    ap.add_argument("--fit-problems", type=int, default=1 << 16)
    ap.add_argument("--fit-steps", type=int, default=1000)
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the built-in launch shape instead of the autotuner's")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the walk directly instead of replaying a CUDA graph")
    ap.add_argument("--texels", type=int, default=WORKLOAD["texels"],
                    help="texels of the spectral field (smaller values: profiling cases)")
    ap.add_argument("--strong", action="store_true",
                    help="N > 1: shard one field across the ranks and gather R and the bins "
                         "every step (strong scaling) instead of one field per rank")
    args = ap.parse_args()
    if args.texels != WORKLOAD["texels"]:
        WORKLOAD["texels"] = args.texels
        WORKLOAD["workload"] = f"spectral_field_{args.texels}texels_x81"
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.pipeline:
        return run_pipeline(args)
    if args.lut:
        return run_lut(args)
    if args.fit:
        return run_fit(args)

    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_2606_27604_b300 import api, shard

    strong = ws > 1 and args.strong
    if strong:
        # one field, contiguous instance ranges, one gather per step
        x_all = spectral_inputs(0)
        x, begin = shard.shard_batch(x_all, rank, ws)
        n_total = x_all.n_inst
        del x_all
    else:
        # rank r's field is instances r*n .. r*n + n - 1 of the global batch
        x = spectral_inputs(rank)
        begin = rank * x.n_inst
        n_total = x.n_inst * ws
    m = api.Media.from_inputs(x, device=dev)
    o = api.WalkOptions(nbins=64, r_max_mm=10.0, seed=WORKLOAD["walk_seed"],
                        instance_offset=begin)
    # launch shape from the autotuner (a sweep on a sample of this field),
    # and the call replayed from a cached CUDA graph
    if not args.no_autotune:
        from paper_2606_27604_b300 import autotune
        o = autotune.tune(m, o)
    o_plain = o
    if not args.no_graph:
        from dataclasses import replace as _rep
        o = _rep(o, use_graph=1)
    wsp = api.alloc_workspace(m, o)
    wsp_bytes = wsp.numel()
    out = api.alloc_tallies(m, o)
    stream = torch.cuda.current_stream(dev)
    paths_per_step = int(x.n_paths.astype(np.int64).sum())

    def barrier():
        if dist is not None:
            dist.barrier()

    def gpu_walk(_x, _begin):
        api.walk(m, o, workspace=wsp, out=out)
        return out["R"], out["bins"]

    def step():
        # the walk, then (strong sharding) the one exchange: R and the bins
        shard.walk_and_gather(gpu_walk, x, begin, n_total, gather=strong)

    for _ in range(args.warmup):
        api.walk(m, o, workspace=wsp, out=out)
    torch.cuda.synchronize()
    code, flags = api.read_status(wsp)
    if code != 0:
        raise RuntimeError(f"walk status {code} flags {flags}")

    # ---- device-timed region: inputs resident in HBM ----------------------
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(dev.index)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    t0.record(stream)
    for i in range(args.steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    # the walk kernel alone (a graph replay cannot bracket one of its kernels):
    # three launches of the same shape outside the graph, events around the
    # kernel on its stream, while the clock sampler still runs
    n_k = 3
    k_start = [torch.cuda.Event(enable_timing=True) for _ in range(n_k)]
    k_stop = [torch.cuda.Event(enable_timing=True) for _ in range(n_k)]
    for e in k_start + k_stop:
        e.record(stream)   # creates the CUDA events
    torch.cuda.synchronize()
    for i in range(n_k):
        api.profile_events(k_start[i], k_stop[i])
        api.walk(m, o_plain, workspace=wsp, out=out)
    api.profile_events(None, None)
    torch.cuda.synchronize()
    clk = clocks.stop()
    elapsed = t0.elapsed_time(t1) / 1e3
    kern = [a.elapsed_time(b) / 1e3 for a, b in zip(k_start, k_stop)]
    if dist is not None:
        tt = torch.tensor([elapsed], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        elapsed = float(tt.item())
    # units all ranks processed: each rank's paths (equal shares up to one instance)
    total_paths = (n_total * WORKLOAD["paths_per_instance"] if strong
                   else paths_per_step * ws) * args.steps
    value = total_paths / elapsed
    steps_mean = float(out["steps"].mean().item())
    total_draws = float(out["steps"].double().sum().item()) * WORKLOAD["paths_per_instance"]
    code, flags = api.read_status(wsp)
    se_per_band = out["stderr_R"].clone()

    # ---- end to end through the API with host buffers ---------------------
    e2e = None
    if not args.no_e2e:
        host = {k: torch.from_numpy(np.ascontiguousarray(getattr(x, k))).pin_memory()
                for k in ("alpha", "sigma_t", "g", "w")}
        res_host = {k: torch.empty(out[k].shape, dtype=out[k].dtype).pin_memory()
                    for k in ("R", "bins")}
        h2d = sum(v.numel() * v.element_size() for v in host.values())
        d2h = sum(v.numel() * v.element_size() for v in res_host.values())
        dm = api.Media(*(torch.empty_like(getattr(m, k)) for k in ("alpha", "sigma_t", "g", "w")),
                       n_paths=None, uniform_paths=m.uniform_paths, n_rel=m.n_rel)
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            for k in ("alpha", "sigma_t", "g", "w"):
                getattr(dm, k).copy_(host[k], non_blocking=True)
            api.walk(dm, o, workspace=wsp, out=out)
            for k in res_host:
                res_host[k].copy_(out[k], non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        et = e0.elapsed_time(e1) / 1e3
        if dist is not None:
            tt = torch.tensor([et], device=dev, dtype=torch.float64)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            et = float(tt.item())
        e2e = {"value": total_paths / et, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}
        del dm

    # ---- adjoint / forward ratio on the adjoint workload ------------------
    ratio = None
    if not args.no_adjoint:
        del wsp, out
        torch.cuda.empty_cache()
        from paper_2606_27604_b300 import inputs
        xa = inputs.spectral_field(n_texels=64 * 64, param_seed=3 + rank, n_paths=1 << 16)
        ma = api.Media.from_inputs(xa, device=dev)
        oa = api.WalkOptions(nbins=64, r_max_mm=10.0, seed=1003)
        wa = api.alloc_workspace(ma, oa)
        wb = api.alloc_workspace(ma, oa, adjoint=True)
        oa_out = api.alloc_tallies(ma, oa)
        gen = torch.Generator(device=dev).manual_seed(3)
        gR = torch.randn(ma.n_inst, device=dev, dtype=torch.float64, generator=gen)
        gB = torch.randn(ma.n_inst, 64, device=dev, dtype=torch.float64, generator=gen)
        grads = None
        api.walk(ma, oa, workspace=wa, out=oa_out)
        grads = api.walk_bwd(ma, oa, grad_R=gR, grad_bins=gB, workspace=wb)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        api.walk(ma, oa, workspace=wa, out=oa_out)
        ev[1].record(stream)
        ev[2].record(stream)
        api.walk_bwd(ma, oa, grad_R=gR, grad_bins=gB, workspace=wb, out=grads)
        ev[3].record(stream)
        torch.cuda.synchronize()
        tf, tb = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])
        ratio = {"value": tb / tf, "fwd_ms": tf, "bwd_ms": tb,
                 "workload": "spectral_field_64x64x81 at 65536 paths, grads w.r.t. "
                             "(alpha, sigma_t, g, w) x 3 from upstream on R and 64 bins"}

    # ---- batched uneven instances vs one launch per instance ---------------
    baselines = None
    if not args.no_baselines:
        from paper_2606_27604_b300 import inputs

        def timed(fn):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            fn()
            torch.cuda.synchronize()
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b) / 1e3

        xu = inputs.uneven_batch(n_inst=4096, param_seed=2)
        mu_ = api.Media.from_inputs(xu, device=dev)
        ou = api.WalkOptions(nbins=64, r_max_mm=10.0, seed=1002, use_graph=1)
        wu = api.alloc_workspace(mu_, ou)
        tu = api.alloc_tallies(mu_, ou)
        t_graph = timed(lambda: api.walk(mu_, ou, workspace=wu, out=tu))
        op = api.WalkOptions(nbins=64, r_max_mm=10.0, seed=1002, schedule=1)
        t_plain = timed(lambda: api.walk(mu_, op, workspace=wu, out=tu))
        pu = float(xu.n_paths.astype(np.float64).sum())
        # plain baseline on a slice of the spectral workload (5.3 M launches
        # for the whole field would be impractical): 2048 instances
        xs = x.subset(np.arange(2048))
        ms_ = api.Media.from_inputs(xs, device=dev)
        wsb = api.alloc_workspace(ms_, o_plain)
        tsb = api.alloc_tallies(ms_, o_plain)
        from dataclasses import replace as _rep
        t_sub_plain = timed(lambda: api.walk(ms_, _rep(o_plain, schedule=1), workspace=wsb,
                                             out=tsb))
        t_sub_pers = timed(lambda: api.walk(ms_, o_plain, workspace=wsb, out=tsb))
        ps = 2048.0 * WORKLOAD["paths_per_instance"]
        baselines = {
            "uneven_batch": {"workload": "4096 instances, budgets floor(2^U[10,20]) "
                                         f"({pu:.3g} paths), finite and semi-infinite slabs",
                             "persistent_graph_paths_per_s": pu / t_graph,
                             "one_launch_per_instance_paths_per_s": pu / t_plain,
                             "speedup": t_plain / t_graph},
            "plain_on_spectral_slice": {"sample": "first 2048 instances of the spectral "
                                                  "workload at 4096 paths",
                                        "plain_paths_per_s": ps / t_sub_plain,
                                        "persistent_paths_per_s_same_slice": ps / t_sub_pers},
        }
        api.release_plans()
        del wu, tu, wsb, tsb

    # ---- hero-wavelength sharing: one path per group of 3 adjacent bands ---
    hero = None
    if not args.no_hero:
        from dataclasses import replace as _rep
        oh = _rep(o_plain, hero_bands=3, hero_texel_bands=81)
        wh = api.alloc_workspace(m, oh)
        th_ = api.alloc_tallies(m, oh)
        api.walk(m, oh, workspace=wh, out=th_)
        torch.cuda.synchronize()
        hts = []
        for _ in range(2):
            ha, hb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ha.record(stream)   # creates the CUDA events
            hb.record(stream)
            api.profile_events(ha, hb)
            api.walk(m, oh, workspace=wh, out=th_)
            api.profile_events(None, None)
            torch.cuda.synchronize()
            hts.append(ha.elapsed_time(hb) / 1e3)
        hcode, hflags = api.read_status(wh)
        t_h = float(np.mean(hts))
        t_b = float(np.mean(kern))
        se_ratio = float(torch.median(th_["stderr_R"] / se_per_band).item())
        n_inst = x.n_inst
        N = WORKLOAD["paths_per_instance"]
        hero = {"C": 3, "grouping": "blocks of 3 adjacent bands of a texel",
                "workload": f"{WORKLOAD['workload']}, {N} paths per group",
                "kernel_ms": t_h * 1e3, "per_band_kernel_ms": t_b * 1e3,
                "paths_per_s": n_inst / 3 * N / t_h,
                "band_samples_per_s": n_inst * N / t_h,
                "stderr_R_ratio_median": se_ratio,
                "speedup_at_equal_error": (t_b / t_h) / se_ratio ** 2,
                "status": hcode}
        del wh, th_

    # ---- decoder (RGB -> per-band mixture parameters, tensor cores) --------
    decoder = None
    if not args.no_decoder and ws == 1:
        from paper_2606_27604_b300 import inputs
        side = args.decoder_side
        rgb = torch.from_numpy(inputs.rgb_texture(side=side, seed=4)).to(dev)
        packed = api.decoder_pack(inputs.decoder_weights(seed=4), device=dev)
        dws = torch.empty(api.lib.sss_decode_workspace_size(side * side), dtype=torch.uint8,
                          device=dev)
        dout = {k: torch.empty(3, 81 * side * side, dtype=torch.float32, device=dev)
                for k in ("alpha", "g", "sigma_t", "w")}
        for _ in range(3):
            api.decode(rgb, packed, workspace=dws, out=dout)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record(stream)
        for _ in range(reps):
            api.decode(rgb, packed, workspace=dws, out=dout)
        e1.record(stream)
        torch.cuda.synchronize()
        dms = e0.elapsed_time(e1) / reps
        flops = 2.0 * DECODER_MACS_PER_TEXEL * side * side
        dcode, dflags = api.read_status(dws)
        peak_bf16 = _measured_peak("bf16_tflops", 1792.8)
        decoder = {"workload": f"{side}x{side} RGB texels -> 3 media x 81 bands",
                   "ms": dms, "texels_per_s": side * side / (dms / 1e3),
                   "achieved_tflops": flops / (dms / 1e3) / 1e12,
                   "peak_tflops": peak_bf16[0], "peak_basis": peak_bf16[1],
                   "frac": flops / (dms / 1e3) / 1e12 / peak_bf16[0],
                   "flops_per_texel": 2 * DECODER_MACS_PER_TEXEL, "status": dcode}
        del dws, dout

    # ---- full pipeline: RGB -> decoder -> walk (one GPU) -------------------
    pipeline = None
    if not args.no_pipeline and ws == 1:
        pipeline = pipeline_leg(side=args.pipeline_side)

    # ---- LUT precompute and LUT mixture fit (Sec. 4.2), bounded sizes -------
    lut_res = fit_res = None
    if not args.no_lut and ws == 1:
        lut_res = lut_leg(128, 1 << 16)
        fit_res = fit_leg(1 << 16, 1000)

    # ---- roofline of the walk kernel --------------------------------------
    kmean = float(np.mean(kern))
    f_mhz = clk["sm_mhz"] if clk else 2032.0
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * SM_LANES_PER_CLK * f_mhz * 1e6 / 1e12
    achieved = total_draws * ALG_ALU_OPS_PER_STEP / kmean / 1e12
    mufu = total_draws * ALG_MUFU_OPS_PER_STEP / kmean / (sms * MUFU_LANES_PER_CLK * f_mhz * 1e6)
    traffic = WALK_TRAFFIC["bytes_per_launch"] \
        if _walk_source_sha1() == WALK_TRAFFIC["source_sha1"] and \
        WORKLOAD["texels"] == 256 * 256 else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "walk_persistent_kernel<false, false, 0, true, 0> (semi-infinite slabs, "
                          "albedo weighting)",
                "peak_basis": f"{sms} SMs x {SM_LANES_PER_CLK} FP32/INT32 lanes/clk x "
                              f"{f_mhz:.0f} MHz (median SM clock sampled in the timed region)",
                "ops_per_step": ALG_ALU_OPS_PER_STEP, "steps_per_launch": total_draws,
                "mufu_frac": mufu, "kernel_ms": kmean * 1e3}

    # ---- issue-rate probes: the measured per-SM lane throughputs -----------
    probe = None
    if not args.no_probe:
        blocks = sms * 8          # 2048 threads per SM
        sink = torch.empty(blocks * 256, dtype=torch.float32, device=dev)
        probe = {"clock_mhz": f_mhz, "unit": "lane operations per clock per SM",
                 "method": "8 independent chains per thread, 2048 threads per SM, "
                           "iteration loop unrolled 8x (loop control < 5% of issue)"}
        for kind, iters in (("ffma", 1 << 19), ("ffma2", 1 << 18), ("imad", 1 << 19),
                            ("lop3", 1 << 19), ("mufu_lg2", 1 << 16), ("philox", 1 << 14)):
            api.probe(kind, 64, blocks, sink, stream)   # warm-up
            pa, pb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            pa.record(stream)
            ops = api.probe(kind, iters, blocks, sink, stream)
            pb.record(stream)
            torch.cuda.synchronize()
            dt = pa.elapsed_time(pb) / 1e3
            probe[kind] = ops / dt / (sms * f_mhz * 1e6)
        del sink
        roofline["peak_measured_ffma"] = sms * probe["ffma"] * f_mhz * 1e6 / 1e12
        roofline["frac_of_measured_ffma"] = achieved / roofline["peak_measured_ffma"]
        # Philox-aware peak: a draw needs one Philox block (at the measured
        # block rate, probe "philox" in blocks per clock per SM) plus its
        # ~50 binary32 operations (at the measured FFMA rate), issued one
        # after the other on the SM's schedulers
        per_draw_clk = 1.0 / probe["philox"] + ALG_FP32_OPS_PER_STEP / probe["ffma"]
        peak_draws = sms * f_mhz * 1e6 / per_draw_clk
        roofline["peak_philox_aware_draws_per_s"] = peak_draws
        roofline["draws_per_s"] = total_draws / kmean
        roofline["frac_philox_aware"] = total_draws / kmean / peak_draws

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample()

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3,
            "higher_is_better": True, "scaling": "strong" if strong else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(WORKLOAD,
                           parallelism=(f"instance-shard x{ws}, one field, all_gather per step"
                                        if strong else
                                        f"instance-shard x{ws}, one field per rank"),
                           l2=f"inputs ({x.alpha.nbytes * 4 / 1e6:.0f} MB) and tally workspace "
                              f"({wsp_bytes / 1e9:.1f} GB) vs the 126 MB L2",
                           steps_per_path=steps_mean),
            "clocks": clk, "e2e": e2e, "gpu_launches": 3 * args.steps,
            "roofline": roofline, "cpu_baseline": cpu,
            "adjoint_forward_ratio": ratio, "baselines": baselines, "hero_wavelength": hero,
            "probe": probe,
            "decoder": decoder, "pipeline": pipeline, "lut": lut_res, "lut_fit": fit_res,
            "launch_shape": dict({k: getattr(o, k) for k in ("block_threads", "unit_paths",
                                                             "regroup")},
                                 autotuned=not args.no_autotune, cuda_graph=bool(o.use_graph)),
            "status_flags": flags}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
