"""Learned proposal + adjoint refinement (inverse synthesis, Sec. 2 of the paper).

Training: the network sees voices the synth renders on the fly from training
batch indices (Sec. 2.2 split: of every 10 blocks of 1024 voices the last is
test), batch 128, Adam. Evaluation: for held-out target voices, parameters
are refined by gradient descent on the multi-resolution STFT distance
(render -> distance -> adjoint -> Adam in [0,1]^78), starting either from the
network's proposal or from random parameters; the distance reached and the
GPU time spent are recorded per step. Everything runs in libsynth.so kernels.

    python -m paper_2104_12922_gb300.proposal --train-steps 2000 --eval-voices 256
"""
from __future__ import annotations

import argparse
import json
import time

import paper_2104_12922_gb300 as pkg


def is_train_batch(batch_index: int, batch: int) -> bool:
    """True if none of the batch's voices fall in a test block (Sec. 2.2)."""
    g0, g1 = batch_index * batch, batch_index * batch + batch - 1
    return not any(pkg.synth_is_test(g) for g in (g0, g1))


def train_batches(batch: int):
    b = 0
    while True:
        if is_train_batch(b, batch):
            yield b
        b += 1


def test_batches(batch: int):
    b = 0
    while True:
        if all(pkg.synth_is_test(g) for g in (b * batch, b * batch + batch - 1)):
            yield b
        b += 1


def train(model: pkg.ProposalModel, steps: int, batch: int = 128, seed: int = 0,
          lr: float = 3e-4, log_every: int = 100, pipeline: bool = True):
    """On-the-fly training over consecutive training-split batches; returns
    the loss history, wall seconds and GPU milliseconds (CUDA events around
    the whole loop).

    pipeline: the next batch is rendered and turned into features on a
    second stream while the network trains on this one (two sets of
    buffers, events between the streams); the same calls on the same
    inputs as the one-stream loop (synth_model_train_step), so the model
    ends bit-identical to it."""
    import torch
    syn = model.synth
    loss = torch.zeros(1, device=syn.device)
    hist = []
    it = train_batches(batch)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def lr_at(s):
        return lr * min(1.0, (s + 1) / 200) * (0.1 ** (s / max(1, steps)))

    t0 = time.perf_counter()
    main = torch.cuda.current_stream()
    start.record(main)
    if not pipeline:
        for s in range(steps):
            model.train_step(seed, next(it), batch, lr_at(s), loss=loss)
            if s % log_every == 0 or s == steps - 1:
                hist.append((s, loss.clone()))
    else:
        dev = syn.device
        side = torch.cuda.Stream(device=dev)
        audio = [torch.empty((batch, syn.num_samples), device=dev) for _ in range(2)]
        params = [torch.empty((batch, pkg.NUM_PARAMS), device=dev) for _ in range(2)]
        feats = [torch.empty((batch, model.feature_dim), dtype=torch.bfloat16, device=dev)
                 for _ in range(2)]
        ready = [torch.cuda.Event(), torch.cuda.Event()]  # batch in buffer i is prepared
        done = [torch.cuda.Event(), torch.cuda.Event()]   # buffer i has been trained on

        def prepare(i, b):
            syn.render(seed, b, batch, out=audio[i], params_out=params[i], stream=side)
            model.features(audio[i], stream=side, out=feats[i])
            ready[i].record(side)

        side.wait_stream(main)
        if steps > 0:
            prepare(0, next(it))
        for s in range(steps):
            i, j = s % 2, 1 - s % 2
            if s + 1 < steps:
                if s >= 1:
                    side.wait_event(done[j])
                prepare(j, next(it))
            main.wait_event(ready[i])
            model.train_features(feats[i], params[i], lr_at(s), loss=loss, stream=main)
            done[i].record(main)
            if s % log_every == 0 or s == steps - 1:
                hist.append((s, loss.clone()))
        main.wait_stream(side)
    end.record(main)
    end.synchronize()
    syn.sync()
    hist = [(s, float(l.item())) for s, l in hist]
    return {"steps": steps, "batch": batch, "seconds": time.perf_counter() - t0,
            "gpu_ms": start.elapsed_time(end), "loss": hist}


def refine(syn: pkg.Synth, target, u0, steps: int, lr: float, seed: int, batch_index: int):
    """Adam on u against the MR-STFT distance to target; returns per-step
    mean distance and cumulative GPU milliseconds (CUDA events)."""
    import torch
    batch = target.shape[0]
    mr = pkg.MRSTFT(syn, batch)
    u = u0.clone().contiguous()
    m = torch.zeros_like(u)
    v = torch.zeros_like(u)
    audio = torch.empty_like(target)
    pout = torch.empty_like(u)
    curve = []
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total_ms = 0.0
    for s in range(steps + 1):
        start.record()
        syn.render(seed, batch_index, batch, params_in=u, out=audio, params_out=pout)
        loss, g_audio = mr(audio, target, grad=s < steps, target_ready=s > 0)
        if s < steps:
            g_u = syn.backward(seed, batch_index, u, g_audio)
            pkg.param_adam(syn, u, g_u, m, v, s + 1, lr)
        end.record()
        end.synchronize()
        total_ms += start.elapsed_time(end)
        curve.append((s, float(loss.mean().item()), total_ms))
    syn.sync()
    return u, curve


def evaluate(model: pkg.ProposalModel, voices: int, steps: int, lr: float = 0.02, seed: int = 0,
             batch: int = 128):
    import torch
    syn = model.synth
    results = {"proposal": [], "random": []}
    finals = {"proposal": [], "random": [], "true_u": [], "target_batch": []}
    it = test_batches(batch)
    done = 0
    gen = torch.Generator(device=syn.device).manual_seed(seed + 12345)
    while done < voices:
        b = next(it)
        n = min(batch, voices - done)
        target, true_u = syn.render(seed, b, batch)
        target, true_u = target[:n].contiguous(), true_u[:n].contiguous()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record()
        u_prop = model.propose(target)
        end.record()
        end.synchronize()
        prop_ms = start.elapsed_time(end)
        u_rand = torch.rand((n, 78), device=syn.device, generator=gen)
        up, cp = refine(syn, target, u_prop, steps, lr, seed + 1, b)
        ur, cr = refine(syn, target, u_rand, steps, lr, seed + 1, b)
        results["proposal"].append([(s, d, t + prop_ms) for (s, d, t) in cp])
        results["random"].append(cr)
        finals["proposal"].append(up.cpu())
        finals["random"].append(ur.cpu())
        finals["true_u"].append(true_u.cpu())
        finals["target_batch"].append(b)
        done += n
    return results, finals


def summarize(results, goal: float | None = None):
    """Mean distance per refinement step over all evaluated voices, the GPU
    milliseconds spent up to each step (summed over batches; the proposal
    arm includes the network's own inference), and for each arm the step
    and GPU time at which the mean distance first reaches ``goal`` (default:
    the random-start arm's final distance)."""
    out = {}
    for k, runs in results.items():
        steps = len(runs[0])
        dist = [sum(r[s][1] for r in runs) / len(runs) for s in range(steps)]
        ms = [sum(r[s][2] for r in runs) for s in range(steps)]
        out[k] = {"distance": dist, "gpu_ms": ms}
    if goal is None:
        goal = out["random"]["distance"][-1]
    for k in list(out):
        hit = next((i for i, d in enumerate(out[k]["distance"]) if d <= goal), None)
        out[k]["steps_to_goal"] = hit
        out[k]["gpu_ms_to_goal"] = out[k]["gpu_ms"][hit] if hit is not None else None
    out["goal_distance"] = goal
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seconds", type=float, default=4.0)
    ap.add_argument("--train-steps", type=int, default=2000)
    ap.add_argument("--batch", type=int, default=128)
    ap.add_argument("--eval-voices", type=int, default=256)
    ap.add_argument("--refine-steps", type=int, default=50)
    ap.add_argument("--lr", type=float, default=3e-4)
    ap.add_argument("--save", default=None)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    from paper_2104_12922_gb300 import build as b
    b.build()
    syn = pkg.Synth(seconds=args.seconds, max_batch=args.batch)
    model = pkg.ProposalModel(syn, max_batch=args.batch, seed=0)
    tr = train(model, args.train_steps, args.batch, lr=args.lr)
    if args.save:
        model.save(args.save)
    res, _ = evaluate(model, args.eval_voices, args.refine_steps, batch=args.batch)
    summary = {"train": tr, "eval": summarize(res), "config": vars(args)}
    text = json.dumps(summary)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)
    print(text)


if __name__ == "__main__":
    main()
