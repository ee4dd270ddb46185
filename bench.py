"""Throughput bench for the batched Voice render.

Workload: the Voice, batch 128 x 4 s at 44.1 kHz, FP32 out; consecutive
batches with seed = batch index (synth1B1-style generation), K batches per
timed region captured in one CUDA graph. A step is one batch through the
whole render path. Metric: audio MHz = samples rendered per second / 1e6.

Our arm (default) times the fused persistent kernel (and, beside it, the
plain unfused module-by-module form on the same GPU). ``--impl reference``
times the FP64 CPU oracle as it stands on the host cores.

The timed loop renders up to 20 consecutive batches per launch
(synth_render_batches, each batch with seed = its index); the same render
with one launch per batch is reported beside it.

Under torchrun (N > 1) every rank renders its own batches (batch indices
rank * K .. rank * K + K - 1): voices are independent, so there is no
collective on the data path; the timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BATCH = 128
GROUP = 20  # at most this many consecutive batches per launch of the timed loop
SECONDS = 4.0
SR = 44100.0
N_SAMPLES = int(SECONDS * SR)
METRIC = "audio MHz (samples/s) at batch 128×4 s: fused vs plain GPU form; % roofline"
PAPER_MHZ = 714.0  # Abstract: 714 MHz on a single V100 (context only)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1024)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-normalized", action="store_true")
    ap.add_argument("--no-generator", action="store_true")
    ap.add_argument("--no-rates", action="store_true")
    ap.add_argument("--no-fm", action="store_true")
    ap.add_argument("--no-proposal", action="store_true")
    ap.add_argument("--no-sfu", action="store_true")
    ap.add_argument("--no-mmd", action="store_true")
    ap.add_argument("--no-cfg5", action="store_true")
    ap.add_argument("--cfg5-train-steps", type=int, default=78125)  # 10 M voices
    ap.add_argument("--cfg5-voices", type=int, default=4096)
    ap.add_argument("--cfg5-refine", type=int, default=50)
    ap.add_argument("--cfg5-judge", type=int, default=256)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--load-seconds", type=float, default=1.0,
                    help="untimed load before and after the timed region (clock sampling)")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
        return False

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in getattr(self, "lines", []):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax or None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_batch_index(step: int, ws: int, rank: int, steps: int) -> int:
    """Replicas: step s of rank r renders batch index r * steps + s, so each
    rank's batches are consecutive (several go into one launch), the ranks'
    batches are disjoint and together they cover 0 .. steps * ws - 1."""
    return rank * steps + step


def max_over_ranks(value: float, dist, device) -> float:
    """The slowest rank's time (an all-reduce MAX, then a barrier)."""
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


FUSED_SOURCES = ["render_fused.cu", "render_common.cuh", "control_ff.cuh", "ff.cuh", "philox_noise.cuh",
                 "voice_device.cuh", "internal.h"]
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "render_fused_batch128x4s.md")


def fused_source_digest():
    h = hashlib.sha256()
    for f in FUSED_SOURCES:
        with open(os.path.join(ROOT, "paper_2104_12922_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic():
    """DRAM bytes per launch of the fused kernel from the committed ncu summary,
    or None when that capture was taken on other kernel sources."""
    try:
        lines = open(PROFILE_SUMMARY).read().splitlines()
    except OSError:
        return None
    kv = {}
    for ln in lines:
        if ln.startswith("- ") and ": " in ln:
            k, v = ln[2:].split(": ", 1)
            kv[k.strip("`")] = v.strip().strip("`")
    if kv.get("kernel_sources_sha256") != fused_source_digest():
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def profiled_instructions():
    """Warp instructions per launch of the fused kernel (GROUP batches) from the
    committed ncu summary, or None when it was taken on other sources."""
    try:
        text = open(PROFILE_SUMMARY).read()
    except OSError:
        return None
    if f"kernel_sources_sha256: `{fused_source_digest()}`" not in text:
        return None
    for ln in text.splitlines():
        if ln.startswith("| `smsp__inst_executed.sum` |"):
            try:
                return float(ln.split("|")[2].split()[0])
            except (IndexError, ValueError):
                return None
    return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def oracle_judge(finals, judge_voices: int, cores: int):
    """Oracle re-synthesis of the proposal evaluation's fitted parameters:
    for the first judge_voices evaluated voices, the FP64 oracle renders the
    target (its drawn parameters, seed 0) and both fits (the refinement's
    noise seed 1), and measures the FP64 MR-STFT distance of each fit."""
    import numpy as np

    import oracle
    from oracle import spectral as osp
    cfg = oracle.default_config(seconds=SECONDS)
    t0 = time.perf_counter()
    d = {"proposal": [], "random": []}
    done = 0
    for i, bi in enumerate(finals["target_batch"]):
        if done >= judge_voices:
            break
        n = min(len(finals["proposal"][i]), judge_voices - done)
        rows = list(range(n))
        target, _ = oracle.render_batch(cfg, 0, bi, BATCH, threads=cores, voices=rows)
        for arm in ("proposal", "random"):
            u = np.zeros((BATCH, 78))
            u[:n] = np.clip(finals[arm][i][:n].numpy().astype(np.float64), 0.0, 1.0)
            fit, _ = oracle.render_batch(cfg, 1, bi, BATCH, u_in=u, threads=cores, voices=rows)
            d[arm].extend(osp.mrstft_loss(fit[:n], target[:n], per_voice=True).numpy().tolist())
        done += n
    return {"voices": done, "seconds": time.perf_counter() - t0,
            "oracle_distance_mean": {k: float(np.mean(v)) for k, v in d.items()},
            "proposal_better_fraction": float(np.mean(np.array(d["proposal"]) <
                                                      np.array(d["random"])))}


def cpu_oracle_baseline(budget_s: float, gpu, cfg5_finals=None, judge_voices: int = 256):
    """The FP64 oracle as it stands on this host's cores: batches of 128 x 4 s
    voices (seed = batch index) until about budget_s of wall time is spent;
    one thread on the small configuration (16 voices x 4 s); and the
    precision configuration (32 voices x 60 s, sine-only patch, constant
    pitch and linear glide). The GPU renders the same voices beside it, so the
    same oracle runs also give the GPU's max-abs error per configuration.
    ``gpu(kind, ...)`` renders them through the library."""
    import math

    import numpy as np

    import oracle
    import seeded_inputs as si
    cfg = oracle.default_config(seconds=SECONDS)
    cores = oracle.hardware_threads()
    t0 = time.perf_counter()
    done = 0
    b = 0
    first = None
    while True:
        audio, params = oracle.render_batch(cfg, b, b, BATCH, threads=cores)
        if first is None:
            first = (audio, params)
        done += 1
        b += 1
        el = time.perf_counter() - t0
        if el >= budget_s or el / done * (done + 1) > 1.5 * budget_s:
            break
    el = time.perf_counter() - t0
    mhz = done * BATCH * N_SAMPLES / el / 1e6
    # one thread on the small configuration: 16 voices x 4 s, seed 0, batch index 0
    t1 = time.perf_counter()
    small, small_p = oracle.render_batch(cfg, 0, 0, 16, threads=1)
    el1 = time.perf_counter() - t1
    errors = {}
    ga, gp = gpu("render", 0, 0, 16)
    errors["batch16x4s_all_voices"] = {"max_abs": float(np.abs(ga - small).max()),
                                       "params_bit_exact": bool(np.array_equal(gp, small_p))}
    ga, gp = gpu("render", 0, 0, BATCH)
    errors["batch128x4s_batch0_all_voices"] = {
        "max_abs": float(np.abs(ga - first[0]).max()),
        "params_bit_exact": bool(np.array_equal(gp, first[1]))}
    # precision configuration: 32 x 60 s, sine only, fixed-point carries
    secs, nb32 = 60.0, 32
    lo = 69.0 + 12.0 * math.log2(20.0 / 440.0)
    hi = 69.0 + 12.0 * math.log2(8000.0 / 440.0)
    nb = si.precision_patch_nebula(oracle.default_nebula(), secs, lo, hi, hi - lo)
    pcfg = oracle.default_config(seconds=secs, nebula=nb)
    prec = {}
    t2 = time.perf_counter()
    for glide in (False, True):
        u, _ = si.precision_patch_params(31 if glide else 30, nb32, lo, hi, hi - lo, glide)
        u = u.astype(np.float32).astype(np.float64)
        ref, _ = oracle.render_batch(pcfg, 0, 0, nb32, u_in=u, threads=cores)
        ga = gpu("precision", nb, u)
        err = np.abs(ga - ref)
        prec["glide" if glide else "constant"] = {
            "max_abs": float(err.max()),
            "drift_cycles_last_1s": float(err[:, -44100:].max() / (2 * math.pi))}
    el2 = time.perf_counter() - t2
    errors["precision_32x60s"] = prec
    judge = oracle_judge(cfg5_finals, judge_voices, cores) if cfg5_finals else None
    return {"value": mhz, "unit": "MHz", "cores": cores, "kind": "oracle",
            "proposal_judge": judge,
            "sample": f"{done} batch(es) of {BATCH} voices x {SECONDS:g} s (seed = batch index), "
                      f"{el:.1f} s wall on {cores} threads",
            "single_thread": {"value": 16 * N_SAMPLES / el1 / 1e6, "unit": "MHz", "cores": 1,
                              "sample": f"16 voices x {SECONDS:g} s, seed 0, {el1:.2f} s wall"},
            "precision_config": {"value": 2 * nb32 * int(secs * SR) / el2 / 1e6, "unit": "MHz",
                                 "cores": cores,
                                 "sample": "32 voices x 60 s, constant pitch and glide"},
            "gpu_vs_oracle": errors}


def adjoint_leg(pkg, torch, dev, steps: int = 20):
    """Inverse-synthesis step of batch 64 x 1 s voices: render from the current
    parameters, multi-resolution STFT distance to target voices of another
    seed and its gradient, the adjoint render, one Adam step. Device time per
    step (CUDA events over `steps` steps after 3 untimed ones)."""
    B, seconds = 64, 1.0
    syn = pkg.Synth(seconds=seconds, max_batch=B)
    n = syn.num_samples
    target, _ = syn.render(1_000_000, 0, B)
    gen = torch.Generator(device=dev).manual_seed(0)
    u = torch.rand((B, 78), device=dev, generator=gen)
    m, v = torch.zeros_like(u), torch.zeros_like(u)
    audio = torch.empty((B, n), device=dev)
    pout = torch.empty_like(u)
    mr = pkg.MRSTFT(syn, B)

    def step(s):
        syn.render(0, 0, B, params_in=u, out=audio, params_out=pout)
        _, g_audio = mr(audio, target, grad=True, target_ready=s > 0)
        g_u = syn.backward(0, 0, u, g_audio)
        pkg.param_adam(syn, u, g_u, m, v, s + 1, 0.01)

    for s in range(3):
        step(s)
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record()
    for s in range(3, 3 + steps):
        step(s)
    end.record()
    end.synchronize()
    ms = start.elapsed_time(end) / steps
    syn.sync()
    syn.close()
    return {"ms_per_step": ms, "value": B * n / (ms / 1e3) / 1e6, "unit": "MHz",
            "config": "batch 64 x 1 s; per step: render, MR-STFT distance (n_fft 512/1024/2048, "
                      "hop n_fft/4) and its gradient, adjoint render, Adam on the 78 parameters",
            "steps": steps}


def _events_ms(torch, fn, reps: int) -> float:
    """Device milliseconds per call of fn (CUDA events on the current stream,
    after one untimed call)."""
    fn(0)
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record()
    for r in range(reps):
        fn(r)
    end.record()
    end.synchronize()
    return start.elapsed_time(end) / reps


def proposal_leg(pkg, torch, dev, peaks, steps: int = 20):
    """The learned proposal's training step at batch 128 x 4 s (render on the
    fly, log-mel features, the 4-layer network's forward, backward and Adam),
    its parts, and the two large contractions alone on the tensor cores: the
    first layer's forward product 128 x 1024 x 44160 (split-K) and its weight
    gradient 1024 x 44160 x 128 (1,384 output tiles). Weights rotate over 3
    copies (270 MB > L2) so that the timed products read them from HBM."""
    B = 128
    syn = pkg.Synth(seconds=SECONDS, max_batch=B)
    model = pkg.ProposalModel(syn, max_batch=B, seed=0)
    loss = torch.zeros(1, device=dev)
    audio = torch.empty((B, N_SAMPLES), device=dev)
    params = torch.empty((B, 78), device=dev)
    feats = torch.empty((B, model.feature_dim), dtype=torch.bfloat16, device=dev)
    for s in range(3):
        model.train_step(0, s, B, 1e-4, loss=loss)
    step_ms = _events_ms(torch, lambda r: model.train_step(0, 10 + r, B, 1e-4, loss=loss), steps)
    render_ms = _events_ms(torch, lambda r: syn.render(r, r, B, out=audio, params_out=params), steps)
    st0 = torch.cuda.current_stream().cuda_stream
    feat_ms = _events_ms(torch, lambda r: pkg.lib().synth_model_features(
        model.handle, audio.data_ptr(), B, feats.data_ptr(), st0), steps)
    mlp_ms = _events_ms(torch, lambda r: model.train_features(feats, params, 1e-4, loss=loss), steps)
    syn.sync()
    L = pkg.lib()
    import ctypes
    k_in = model.feature_dim
    w = [torch.randn(1024, k_in, device=dev).to(torch.bfloat16) for _ in range(3)]
    x = torch.randn(B, k_in, device=dev).to(torch.bfloat16)
    xt = x.t().contiguous()
    dzt = torch.randn(1024, B, device=dev).to(torch.bfloat16)
    c1 = torch.empty(B, 1024, device=dev)
    c2 = torch.empty(1024, k_in, device=dev)
    nb = ctypes.c_size_t()
    L.synth_gemm_bf16_workspace_size(syn.handle, B, 1024, ctypes.byref(nb))
    ws = torch.empty(nb.value // 4 + 1, device=dev)
    st = torch.cuda.current_stream().cuda_stream
    fwd_ms = _events_ms(torch, lambda r: L.synth_gemm_bf16_splitk(
        syn.handle, x.data_ptr(), k_in, w[r % 3].data_ptr(), k_in, c1.data_ptr(), 1024, B, 1024,
        k_in, 1.0, ws.data_ptr(), nb.value, st), 30)
    dw_ms = _events_ms(torch, lambda r: L.synth_gemm_bf16(
        syn.handle, dzt.data_ptr(), B, xt.data_ptr(), B, c2.data_ptr(), k_in, 1024, k_in, B, 1.0,
        st), 30)
    syn.sync()
    model.close()
    syn.close()
    flop = 2.0 * B * 1024 * k_in
    tf = peaks.get("bf16_tflops", 1900.0)
    hbm = peaks["hbm_gbs"]
    return {"ms_per_step": step_ms, "voices_per_s": B / (step_ms / 1e3),
            "parts_ms": {"render": render_ms, "features": feat_ms, "network_train": mlp_ms},
            "config": "batch 128 x 4 s voices rendered on the fly, log-mel 345 x 128, "
                      "MLP 44160-1024-1024-1024-78 (bf16 tcgen05 GEMMs, FP32 Adam)",
            "gemm_first_layer_forward": {
                "shape": [B, 1024, k_in], "ms": fwd_ms, "tflops": flop / fwd_ms / 1e9,
                "frac_tensor": flop / fwd_ms / 1e9 / tf,
                "hbm_gbs": 2.0 * 1024 * k_in / fwd_ms / 1e6,
                "frac_hbm": 2.0 * 1024 * k_in / fwd_ms / 1e6 / hbm,
                "bound": "hbm (the bf16 weights, 90 MB, read once: 128 FLOP per weight byte "
                         "is below the tensor/HBM ratio)"},
            "gemm_first_layer_weight_grad": {
                "shape": [1024, k_in, B], "ms": dw_ms, "tflops": flop / dw_ms / 1e9,
                "frac_tensor": flop / dw_ms / 1e9 / tf,
                "hbm_gbs": 4.0 * 1024 * k_in / dw_ms / 1e6,
                "frac_hbm": 4.0 * 1024 * k_in / dw_ms / 1e6 / hbm,
                "bound": "hbm (the FP32 gradient, 181 MB, written once)"},
            "peaks": {"bf16_tflops": tf, "hbm_gbs": hbm}}


def sfu_leg(pkg, torch, dev, num_sms: int):
    """Measured special-function-unit rate: each probe (sin, cos, ex2, rcp,
    tanh: the .approx forms the render issues) runs ~0.25 s of launches of
    8 independent chains per thread on a full grid; CUDA events give the
    time, nvidia-smi samples taken meanwhile the SM clock."""
    L = pkg.lib()
    import ctypes
    sink = torch.zeros(256, device=dev)
    st = torch.cuda.current_stream().cuda_stream
    blocks, iters = num_sms * 8, 4096
    ops = ctypes.c_int64()
    out = {}
    for name, op in (("sin", pkg.SFU_SIN), ("cos", pkg.SFU_COS), ("ex2", pkg.SFU_EX2),
                     ("rcp", pkg.SFU_RCP), ("tanh", pkg.SFU_TANH)):
        L.synth_sfu_probe(op, blocks, iters, sink.data_ptr(), ctypes.byref(ops), st)
        torch.cuda.synchronize()
        t1 = torch.cuda.Event(enable_timing=True)
        t0 = torch.cuda.Event(enable_timing=True)
        t0.record()
        L.synth_sfu_probe(op, blocks, iters, sink.data_ptr(), None, st)
        t1.record()
        t1.synchronize()
        reps = max(4, int(250.0 / max(t0.elapsed_time(t1), 1e-3)))
        with ClockSampler(dev.index if dev.index is not None else 0) as cs:
            time.sleep(0.05)
            t0.record()
            for _ in range(reps):
                L.synth_sfu_probe(op, blocks, iters, sink.data_ptr(), None, st)
            t1.record()
            t1.synchronize()
        ms = t0.elapsed_time(t1)
        clk = cs.summary()
        mhz = clk["sm_mhz"] or 0.0
        rate = ops.value * reps / (ms / 1e3)
        out[name] = {"gops_per_s": rate / 1e9, "sm_mhz": mhz,
                     "per_clk_per_sm": rate / (num_sms * mhz * 1e6) if mhz else None}
    return out


def mmd_leg(pkg, torch, dev, num_sms: int, sm_mhz: float, per_corpus: int = 1024, n: int = 512,
            trials: int = 100):
    """Corpus similarity (Sec. 5): log-mel embeddings (44160 bf16 values per
    4 s sound) of three corpora -- Voice sounds, 4-operator FM sounds, and
    white noise (the Voice with only its noise oscillator sounding) -- the
    pooled l1 distance matrix on the GPU, and MMD trials: within each corpus
    (random n / n splits) and between each pair (n sounds from each)."""
    import numpy as np

    import seeded_inputs as si
    B = 128
    syn = pkg.Synth(seconds=SECONDS, max_batch=B)
    model = pkg.ProposalModel(syn, max_batch=B, seed=0)
    m = 3 * per_corpus
    emb = torch.empty((m, model.feature_dim), dtype=torch.bfloat16, device=dev)
    noise_u = np.full((B, 78), 0.5)
    noise_u[:, si.MIX], noise_u[:, si.MIX + 1], noise_u[:, si.MIX + 2] = 0.0, 0.0, 1.0
    noise_u[:, si.DURATION] = 1.0
    noise_u[:, si.ADSR:si.ADSR + 5] = [0.0, 0.0, 1.0, 1.0, 1.0]
    for src in range(4):
        noise_u[:, si.mod_slot(src, 4)] = 0.0
    noise_u[:, si.mod_slot(0, 4)] = 1.0
    pin = torch.tensor(noise_u, dtype=torch.float32, device=dev)
    for c in range(3):
        for b in range(per_corpus // B):
            if c == 0:
                audio, _ = syn.render(7, b, B)
            elif c == 1:
                audio, _ = syn.fm_render(7, b, B)
            else:
                audio, _ = syn.render(7, b, B, params_in=pin)
            lo = c * per_corpus + b * B
            emb[lo:lo + B] = model.features(audio)
    dist = torch.empty((m, m), dtype=torch.float32, device=dev)
    pkg.l1_distances(syn, emb, out=dist)
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record()
    for _ in range(3):
        pkg.l1_distances(syn, emb, out=dist)
    end.record()
    end.synchronize()
    dist_ms = start.elapsed_time(end) / 3
    names = ("voice", "fm", "noise")
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    labels = np.concatenate([si.mmd_labels(100 + i, trials, [per_corpus] * 3, p, n)
                             for i, p in enumerate(pairs)])
    lab = torch.tensor(labels, device=dev)
    start.record()
    mm = pkg.mmd_trials(syn, dist, lab)
    end.record()
    end.synchronize()
    trials_ms = start.elapsed_time(end)
    mm = mm.cpu().numpy().reshape(len(pairs), trials)
    syn.sync()
    model.close()
    syn.close()
    dim = emb.shape[1]
    pair_elems = m * (m + 1) / 2 * dim  # upper triangle incl. the diagonal tiles' halves
    # FP32 pipe: 128 lanes per SM per clock, 2 instructions per element pair
    peak = num_sms * 128 * sm_mhz * 1e6 / 2
    return {"corpora": {nm: per_corpus for nm in names}, "n_per_set": n, "trials_per_pair": trials,
            "embedding": "log-mel features (345 frames x 128 bands, bf16), l1 distance",
            "mmd": {f"{names[a]}/{names[b]}": {"mean": float(mm[i].mean()),
                                                "std": float(mm[i].std())}
                    for i, (a, b) in enumerate(pairs)},
            "distance_matrix": {"m": m, "ms": dist_ms,
                                "g_pair_elements_per_s": pair_elems / (dist_ms / 1e3) / 1e9,
                                "roofline": {"bound": "alu", "peak_g_per_s": peak / 1e9,
                                             "frac": pair_elems / (dist_ms / 1e3) / peak,
                                             "peak_source": f"{num_sms} SMs x 128 FP32 lanes x "
                                                            f"{sm_mhz:.0f} MHz / 2 instructions "
                                                            "per element pair"}},
            "trials_ms": trials_ms}


def proposal_eval_leg(pkg, torch, train_steps: int, voices: int, refine_steps: int):
    """The learned proposal's evaluation (inverse synthesis): the network is
    trained on train_steps batches of 128 voices (4 s) rendered on the fly,
    then `voices` held-out test-split voices are fitted by refine_steps
    adjoint refinement steps on the MR-STFT distance, once from the
    network's proposal and once from random parameters. Reported: GPU time
    of the training, the mean distance per step and GPU seconds (CUDA
    events, the proposal's inference included) until each arm first
    reaches a stated distance (the random-start arm's final one). The fitted
    parameters go to the oracle leg, whose re-synthesis judges them."""
    from paper_2104_12922_gb300 import proposal as pr
    syn = pkg.Synth(seconds=SECONDS, max_batch=BATCH)
    model = pkg.ProposalModel(syn, max_batch=BATCH, seed=0)
    tr = pr.train(model, train_steps, BATCH, log_every=max(1, train_steps // 10))
    res, finals = pr.evaluate(model, voices, refine_steps, batch=BATCH)
    summ = pr.summarize(res)
    model.close()
    syn.close()
    keep = [0, refine_steps // 10, refine_steps // 2, refine_steps]
    arms = {}
    for k in ("proposal", "random"):
        a = summ[k]
        arms[k] = {"distance_at_steps": {str(i): a["distance"][i] for i in keep},
                   "steps_to_goal": a["steps_to_goal"],
                   "gpu_s_to_goal": a["gpu_ms_to_goal"] / 1e3 if a["gpu_ms_to_goal"] else None,
                   "gpu_s_all_steps": a["gpu_ms"][-1] / 1e3}
    g_p, g_r = arms["proposal"]["gpu_s_to_goal"], arms["random"]["gpu_s_to_goal"]
    return ({"train": {"voices": train_steps * BATCH, "steps": train_steps,
                       "gpu_s": tr["gpu_ms"] / 1e3, "wall_s": tr["seconds"],
                       "ms_per_step": tr["gpu_ms"] / train_steps,
                       "loss_first_last": [tr["loss"][0][1], tr["loss"][-1][1]]},
             "eval": {"voices": voices, "refine_steps": refine_steps,
                      "goal_distance": summ["goal_distance"],
                      "goal": "the random-start arm's mean MR-STFT distance after all steps",
                      "arms": arms,
                      "gpu_time_ratio_random_over_proposal": (g_r / g_p) if g_p and g_r else None}},
            finals)


def rates_leg(pkg, torch, stream, steps: int = 64):
    """The fused render at a fractional samples-per-interval ratio: batch 128 x
    4 s at 16 kHz with the 441 Hz control rate (R = 36.28..), outputs rotated
    over 4 buffers; CUDA events around `steps` renders captured in a graph."""
    sr, B, seconds = 16000.0, 128, 4.0
    syn = pkg.Synth(seconds=seconds, max_batch=B, sample_rate=sr, control_rate=441.0)
    n = syn.num_samples
    outs = [torch.empty((B, n), dtype=torch.float32, device=syn.device) for _ in range(4)]
    pouts = [torch.empty((B, 78), dtype=torch.float32, device=syn.device) for _ in range(4)]

    def record(k):
        for s in range(k):
            syn.render(s, s, B, out=outs[s % 4], params_out=pouts[s % 4], stream=stream)
    with torch.cuda.stream(stream):
        record(3)
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        record(steps)
    with torch.cuda.stream(stream):
        g.replay()
    stream.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        start.record(stream)
        g.replay()
        end.record(stream)
    end.synchronize()
    ms = start.elapsed_time(end) / steps
    del g
    syn.sync(stream)
    syn.close()
    return {"value": B * n / (ms / 1e3) / 1e6, "unit": "MHz", "ms_per_step": ms, "steps": steps,
            "config": "batch 128 x 4 s at 16 kHz, control rate 441 Hz (R = 16000/441)"}


def fm_leg(pkg, torch, syn, stream, steps: int = 64):
    """The 4-operator FM voice at the bench workload (batch 128 x 4 s,
    44.1 kHz), outputs rotated over 4 buffers; CUDA events around `steps`
    renders captured in a graph."""
    B, n = BATCH, N_SAMPLES
    outs = [torch.empty((B, n), dtype=torch.float32, device=syn.device) for _ in range(4)]
    pout = torch.empty((B, 30), dtype=torch.float32, device=syn.device)

    def record(k):
        for s in range(k):
            syn.fm_render(s, s, B, out=outs[s % 4], params_out=pout, stream=stream)
    with torch.cuda.stream(stream):
        record(3)
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        record(steps)
    with torch.cuda.stream(stream):
        g.replay()
    stream.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        start.record(stream)
        g.replay()
        end.record(stream)
    end.synchronize()
    ms = start.elapsed_time(end) / steps
    del g
    return {"value": B * n / (ms / 1e3) / 1e6, "unit": "MHz", "ms_per_step": ms, "steps": steps,
            "config": "4-operator FM voice, batch 128 x 4 s at 44.1 kHz"}


def generator_leg(pkg, torch, syn, stream, count: int = 8192):
    """Streaming synth1B1 generator: log-mel features and parameters of
    `count` train-split voices (4 s), rendered and transformed chunk by
    chunk; CUDA events around one call per chunk size. Larger chunks fill
    the GPU's last wave of render tiles better; smaller ones keep the chunk's
    audio in L2 between the two kernels."""
    model = pkg.ProposalModel(syn, max_batch=min(512, syn.max_batch), seed=0)
    dev = syn.device
    feats = torch.empty((count, model.feature_dim), dtype=torch.bfloat16, device=dev)
    params = torch.empty((count, 78), dtype=torch.float32, device=dev)
    out = {}
    for chunk in (c for c in (512, 256, 128, 64) if c <= model.max_batch):
        with torch.cuda.stream(stream):
            model.stream_features(0, pkg.SPLIT_TRAIN, 0, 4 * chunk, chunk=chunk,
                                  features=feats[:4 * chunk], params=params[:4 * chunk],
                                  stream=stream)
        stream.synchronize()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            start.record(stream)
            model.stream_features(0, pkg.SPLIT_TRAIN, 10**9, count, chunk=chunk, features=feats,
                                  params=params, stream=stream)
            end.record(stream)
        end.synchronize()
        ms = start.elapsed_time(end)
        out[f"chunk{chunk}"] = {"voices_per_s": count / (ms / 1e3),
                                "msamples_per_s": count * N_SAMPLES / (ms / 1e3) / 1e6,
                                "ms_per_128_voices": ms / count * 128}
    syn.sync(stream)
    model.close()
    best = max(out.values(), key=lambda r: r["voices_per_s"])
    return {"value": best["voices_per_s"], "unit": "voices/s", "voices": count,
            "config": "train split from voice index 1e9, 4 s voices, features 345 x 128 bf16 "
                      "+ 78 params per voice", **out}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    cfg = oracle.default_config(seconds=SECONDS)
    cores = oracle.hardware_threads()
    # each step is a bounded sample of the workload: 16 voices of one batch
    voices = list(range(16))
    for s in range(args.warmup):
        oracle.render_batch(cfg, s, s, BATCH, threads=cores, voices=voices)
    t0 = time.perf_counter()
    for s in range(args.steps):
        oracle.render_batch(cfg, s, s, BATCH, threads=cores, voices=voices)
    el = time.perf_counter() - t0
    samples = args.steps * len(voices) * N_SAMPLES
    mhz = samples / el / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": mhz, "unit": "MHz", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (parameters drawn per voice from seed and voice index)",
            "config": {"workload": "Voice batch 128 x 4 s @ 44.1 kHz, seed = batch index; "
                                   "reference step = 16 voices of the batch", "global_batch": BATCH,
                       "seconds": SECONDS, "sample_rate": SR},
            "cpu_baseline": {"value": mhz, "unit": "MHz", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} steps x 16 voices x 4 s"},
            "e2e": {"value": mhz, "unit": "MHz", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2104_12922_gb300 as pkg
    from paper_2104_12922_gb300 import build as b

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or ws == 1:
        b.build()
    if ws > 1:
        dist.barrier()
    dev = torch.device("cuda", local)
    K, W = args.steps, max(3, args.warmup)
    syn = pkg.Synth(seconds=SECONDS, max_batch=BATCH * GROUP)
    n_buf = 4  # 4 x 90.3 MB rotating outputs: > L2 (129 MB), writes reach HBM
    outs = [torch.empty((BATCH, N_SAMPLES), dtype=torch.float32, device=dev) for _ in range(n_buf)]
    pouts = [torch.empty((BATCH, 78), dtype=torch.float32, device=dev) for _ in range(n_buf)]
    # GROUP consecutive batches per launch into 2 rotating outputs of GROUP x 90.3 MB
    outs_g = [torch.empty((BATCH * GROUP, N_SAMPLES), dtype=torch.float32, device=dev)
              for _ in range(2)]
    pouts_g = [torch.empty((BATCH * GROUP, 78), dtype=torch.float32, device=dev) for _ in range(2)]
    stream = torch.cuda.Stream(device=dev)

    def batch_index(step):
        return rank_batch_index(step, ws, rank, K)

    def record(g_steps):
        """g_steps batches in launches of at most GROUP, as even as possible
        (24 steps: two of 12, not 20 + 4; seed = batch index)"""
        n_launch = (g_steps + GROUP - 1) // GROUP
        s0 = 0
        for l in range(n_launch):
            c = g_steps // n_launch + (1 if l < g_steps % n_launch else 0)
            bi = batch_index(s0)
            i = l % 2
            syn.render_batches(bi, 1, bi, BATCH, c, out=outs_g[i][:c * BATCH],
                               params_out=pouts_g[i][:c * BATCH], stream=stream)
            s0 += c

    def record_single(g_steps, plain=False):
        """one launch per batch"""
        for s in range(g_steps):
            bi = batch_index(s)
            syn.render(bi, bi, BATCH, out=outs[s % n_buf], params_out=pouts[s % n_buf],
                       stream=stream, plain=plain)

    # warm-up (untimed), then capture K steps in one graph
    with torch.cuda.stream(stream):
        record(W * GROUP)
    stream.synchronize()
    syn.sync(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        record(K)
    with torch.cuda.stream(stream):
        graph.replay()  # untimed replay primes the graph
    stream.synchronize()

    def timed(fn, clocks=False, preload=None, postload=None):
        # graph replays and eager renders both go to `stream`, where the
        # events are recorded
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sampler = ClockSampler(local) if clocks else None
        if sampler:
            sampler.__enter__()
            time.sleep(0.05)
        with torch.cuda.stream(stream):
            if preload is not None:  # untimed load so the clock samples see a busy GPU
                preload()
            start.record(stream)
            fn()
            end.record(stream)
            if postload is not None:
                postload()
        end.synchronize()
        torch.cuda.synchronize()
        if sampler:
            sampler.__exit__(None, None, None)
        ms = start.elapsed_time(end)
        if ws > 1:
            ms = max_over_ranks(ms, dist, dev)
        return ms, (sampler.summary() if sampler else None)

    # exactly K timed steps (one replay of the K-step graph), inside at least
    # 1 s of identical untimed load before and after it, so that the clock
    # samples taken meanwhile see the GPU as busy as the timed region does
    ms1, _ = timed(lambda: graph.replay())
    n_load = max(1, int(1000.0 * args.load_seconds / max(ms1, 1e-3)) + 1)

    def load():
        for _ in range(n_load):
            graph.replay()

    ms, clocks = timed(lambda: graph.replay(), clocks=True, preload=load, postload=load)
    # the same replays for at least 1 s, timed as a whole (a steady figure
    # beside the exact-K one)
    ms_long, clocks_long = timed(load, clocks=True)
    sustained = {"value": n_load * K * BATCH * N_SAMPLES * ws / (ms_long / 1e3) / 1e6,
                 "unit": "MHz", "ms_per_step": ms_long / (n_load * K), "steps": n_load * K,
                 "seconds": ms_long / 1e3, "clocks": clocks_long}
    syn.sync(stream)
    steps = K
    samples_total = steps * BATCH * N_SAMPLES * ws
    value = samples_total / (ms / 1e3) / 1e6
    ms_per_step = ms / steps

    # the same fused render with one launch per batch
    Ks = min(K, 256)
    with torch.cuda.stream(stream):
        record_single(2)
    stream.synchronize()
    gs = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gs, stream=stream):
        record_single(Ks)
    with torch.cuda.stream(stream):
        gs.replay()
    stream.synchronize()
    mss, _ = timed(lambda: gs.replay())
    single = {"value": Ks * BATCH * N_SAMPLES * ws / (mss / 1e3) / 1e6, "unit": "MHz",
              "ms_per_step": mss / Ks, "steps": Ks, "launches_per_step": 1}
    del gs

    # plain unfused form on the same GPU (same workload)
    plain = None
    if not args.no_plain:
        Kp = min(K, 64)
        with torch.cuda.stream(stream):
            record_single(2, plain=True)
        stream.synchronize()
        gp = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gp, stream=stream):
            record_single(Kp, plain=True)
        with torch.cuda.stream(stream):
            gp.replay()
        stream.synchronize()
        msp, _ = timed(lambda: gp.replay())
        plain = {"value": Kp * BATCH * N_SAMPLES * ws / (msp / 1e3) / 1e6, "unit": "MHz",
                 "ms_per_step": msp / Kp, "steps": Kp,
                 "kernels_per_step": 15}
        del gp

    # the same workload with per-voice peak normalisation and silence
    # rejection (the render records each voice's peak; the scaling runs as
    # extra work items of the same persistent kernel)
    normalized = None
    if not args.no_normalized:
        Kn = min(K, 64)
        # every buffer rotates, so consecutive launches share none and overlap
        peak_b = [torch.empty(BATCH, dtype=torch.float32, device=dev) for _ in range(n_buf)]
        silent_b = [torch.empty(BATCH, dtype=torch.int32, device=dev) for _ in range(n_buf)]

        def record_norm(g_steps):
            for s in range(g_steps):
                bi = batch_index(s)
                syn.render_normalized(bi, bi, BATCH, threshold=1e-3, out=outs[s % n_buf],
                                      params_out=pouts[s % n_buf], peak=peak_b[s % n_buf],
                                      silent=silent_b[s % n_buf], stream=stream)
        with torch.cuda.stream(stream):
            record_norm(2)
        stream.synchronize()
        gn = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gn, stream=stream):
            record_norm(Kn)
        with torch.cuda.stream(stream):
            gn.replay()
        stream.synchronize()
        msn, _ = timed(lambda: gn.replay())
        normalized = {"value": Kn * BATCH * N_SAMPLES * ws / (msn / 1e3) / 1e6, "unit": "MHz",
                      "ms_per_step": msn / Kn, "steps": Kn, "threshold": 1e-3,
                      "overhead_ms_per_step": msn / Kn - ms_per_step,
                      "kernels_per_step": 1}
        del gn

    # end to end through the public API with host buffers: per step the render
    # and a device->host read of the step's audio and parameters into pinned
    # memory (the only inputs are the seed and the batch index: 0 H2D bytes).
    # The copy of step s runs on a second stream while step s + 1 renders;
    # events keep a device buffer from being rewritten before its copy ends.
    Ke = min(K, 64)
    host_a = torch.empty((BATCH, N_SAMPLES), dtype=torch.float32, pin_memory=True)
    host_p = torch.empty((BATCH, 78), dtype=torch.float32, pin_memory=True)
    copy_stream = torch.cuda.Stream(device=dev)
    rendered = [torch.cuda.Event() for _ in range(n_buf)]
    copied = [torch.cuda.Event() for _ in range(n_buf)]

    def e2e_steps():
        for s in range(Ke):
            i = s % n_buf
            bi = batch_index(s)
            if s >= n_buf:
                stream.wait_event(copied[i])
            with torch.cuda.stream(stream):
                a, p = syn.render(bi, bi, BATCH, out=outs[i], params_out=pouts[i], stream=stream)
            rendered[i].record(stream)
            copy_stream.wait_event(rendered[i])
            with torch.cuda.stream(copy_stream):
                host_a.copy_(a, non_blocking=True)
                host_p.copy_(p, non_blocking=True)
            copied[i].record(copy_stream)
        stream.wait_event(copied[(Ke - 1) % n_buf])  # the end event follows the last copy
    e2e_steps()
    torch.cuda.synchronize()
    mse, _ = timed(e2e_steps)
    e2e = {"value": Ke * BATCH * N_SAMPLES * ws / (mse / 1e3) / 1e6, "unit": "MHz",
           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": BATCH * N_SAMPLES * 4 + BATCH * 78 * 4,
           "overlap": "device->host copy of step s on a second stream during the render of s + 1"}

    if rank != 0:
        if ws > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    peaks, peak_src = measured_peaks()
    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = (clocks or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    # transcendental bound: 4 per sample (sine sin; square-saw sin, cos, tanh)
    # at the MUFU rate measured by the probe (sin.approx per clock per SM),
    # at the maximum SM clock
    sfu = None if args.no_sfu else sfu_leg(pkg, torch, dev, num_sms)
    sfu_rate = (sfu or {}).get("sin", {}).get("per_clk_per_sm") or 16.0
    alu_peak = num_sms * sfu_rate * sm_max * 1e6 / 4
    per_gpu_rate = BATCH * N_SAMPLES / (ms_per_step / 1e3)
    hbm_peak_samples = peaks["hbm_gbs"] * 1e9 / 4
    roofline = {"bound": "alu", "achieved": per_gpu_rate / 1e9, "peak": alu_peak / 1e9,
                "unit": "Gsample/s", "frac": per_gpu_rate / alu_peak, "traffic": profiled_traffic(),
                "peak_source": f"{num_sms} SMs x {sfu_rate:.2f} sin.approx/clk/SM "
                               f"({'measured by the SFU probe' if sfu else 'assumed'}) x "
                               f"{sm_max:.0f} MHz / 4 per sample",
                "hbm": {"achieved": per_gpu_rate * 4 / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": per_gpu_rate / hbm_peak_samples, "peak_source": peak_src},
                # the same bound counting 6 transcendentals per sample (tanh as
                # exp2 + reciprocal, plus an exp2 of the pitch per sample)
                "t6": {"peak": alu_peak * 4 / 6 / 1e9, "frac": per_gpu_rate / (alu_peak * 4 / 6)}}
    inst = profiled_instructions()
    if inst is not None:
        # instruction issue: one warp instruction per clock per scheduler, 4 per SM
        issue_peak = num_sms * 4 * sm_max * 1e6
        per_batch = inst / GROUP
        roofline["issue"] = {"warp_instructions_per_batch": per_batch,
                             "achieved": per_batch / (ms_per_step / 1e3) / 1e9,
                             "peak": issue_peak / 1e9, "unit": "G warp instructions/s",
                             "frac": per_batch / (ms_per_step / 1e3) / issue_peak,
                             "source": "smsp__inst_executed.sum of the committed ncu summary"}
    def gpu_render(kind, *a):
        """Renders through the library for the oracle leg's comparisons."""
        import numpy as np
        if kind == "render":
            seed, bi, nb = a
            audio, params = syn.render(seed, bi, nb)
            syn.sync()
            return audio.cpu().numpy(), params.cpu().numpy()
        nebula, u = a
        ps = pkg.Synth(seconds=60.0, max_batch=u.shape[0], nebula=nebula)
        audio, _ = ps.render(0, 0, u.shape[0],
                             params_in=torch.tensor(u, dtype=torch.float32, device=dev))
        ps.sync()
        out = audio.cpu().numpy()
        ps.close()
        return out

    cfg5, finals = (None, None)
    if not args.no_cfg5:
        cfg5, finals = proposal_eval_leg(pkg, torch, args.cfg5_train_steps, args.cfg5_voices,
                                         args.cfg5_refine)
    cpu = None
    if not args.no_cpu:
        cpu = cpu_oracle_baseline(args.cpu_seconds, gpu_render, finals, args.cfg5_judge)
    adjoint = None if args.no_adjoint else adjoint_leg(pkg, torch, dev)
    generator = None if args.no_generator else generator_leg(pkg, torch, syn, stream)
    rates = None if args.no_rates else rates_leg(pkg, torch, stream)
    fm = None if args.no_fm else fm_leg(pkg, torch, syn, stream)
    proposal = None if args.no_proposal else proposal_leg(pkg, torch, dev, peaks)
    mmd = None if args.no_mmd else mmd_leg(pkg, torch, dev, num_sms, sm_max)
    line = {"metric": METRIC, "value": value, "unit": "MHz", "n_gpus": ws, "steps": steps,
            "warmup": W, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (synth1B1 workload: parameters drawn per voice from seed and voice index)",
            "config": {"workload": "Voice batch 128 x 4 s @ 44.1 kHz, FP32 out, seed = batch index, "
                                   f"{K} batches per CUDA graph in {(K + GROUP - 1) // GROUP} launches "
                                   f"of at most {GROUP} (synth_render_batches)",
                       "global_batch": BATCH * ws,
                       "seconds": SECONDS, "sample_rate": SR,
                       "l2": f"2 rotating {GROUP * BATCH * N_SAMPLES * 4 / 1e6:.0f} MB outputs of "
                             f"{GROUP} batches (> 129 MB L2)",
                       "parallelism": f"replicas x{ws} (disjoint batch indices)"},
            "x_realtime": value * 1e6 / SR,
            "paper_context": {"value": PAPER_MHZ, "unit": "MHz", "hardware": "single V100 (Sec. 2.2)"},
            "one_launch_per_batch": single,
            "plain": plain, "fused_over_plain": (value / plain["value"]) if plain else None,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "sustained": sustained, "sfu_probe": sfu,
            "adjoint": adjoint, "normalized": normalized, "generator": generator,
            "fractional_rate": rates, "fm_voice": fm, "proposal_step": proposal,
            "mmd_diversity": mmd, "proposal_eval": cfg5,
            "gpu_launches": (steps + GROUP - 1) // GROUP}
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
