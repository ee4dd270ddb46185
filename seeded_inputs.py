"""Seeded synthetic inputs shared by the tests, the oracle runs and bench.py.

This module holds input construction only -- seeds, batch indices, normalized
parameter vectors, custom nebula tables, upstream gradients -- and none of the
Voice's arithmetic. Both the CUDA path and the oracle receive what it returns
as plain arrays.

Workload recipe (synth1B1, Sec. 2.1 / 3.3 of the paper): parameters drawn
uniformly in [0,1) per voice by the render itself from (seed, global voice
index); 4 s voices at 44.1 kHz; batch 128 by default (Sec. 2.2).
"""
from __future__ import annotations

import math

import numpy as np

NUM_PARAMS = 78

# Parameter slots (Voice layout): keyboard, 6 ADSRs, 2 LFOs, modulation
# weights, sine VCO, square-saw VCO, mixer levels.
MIDI, DURATION, ADSR, LFO, MOD, SINE, SQR, MIX = 0, 1, 2, 32, 48, 68, 71, 75


def mod_slot(src: int, dest: int) -> int:
    return MOD + 5 * src + dest


def uniform_params(seed: int, batch: int) -> np.ndarray:
    """Normalized parameters [batch][78], uniform in [0,1), float32-exact."""
    rng = np.random.default_rng(seed)
    return (rng.integers(0, 1 << 24, size=(batch, NUM_PARAMS)) / float(1 << 24)).astype(np.float64)


def edge_params(batch: int) -> np.ndarray:
    """Degenerate corners of the normalized cube: all zeros, all ones, and
    alternating 0/1 patterns (zero-length envelope sections, zero weights,
    extreme pitch), cycled over the batch."""
    rows = [np.zeros(NUM_PARAMS), np.ones(NUM_PARAMS),
            np.tile([0.0, 1.0], NUM_PARAMS // 2), np.tile([1.0, 0.0], NUM_PARAMS // 2),
            np.full(NUM_PARAMS, 0.5)]
    return np.stack([rows[i % len(rows)] for i in range(batch)])


def fixed_patch(base: np.ndarray | None = None, **slots: float) -> np.ndarray:
    """A normalized parameter vector with chosen slots set (default 0.5)."""
    u = np.full(NUM_PARAMS, 0.5) if base is None else np.array(base, dtype=np.float64)
    for k, v in slots.items():
        u[int(k.lstrip("p"))] = v
    return u


def pinned_nebula(base: dict, pins: dict[int, float]) -> dict:
    """Copy of a nebula with some parameters pinned to a constant (lo = hi)."""
    nb = {k: np.array(v, copy=True) for k, v in base.items()}
    for p, val in pins.items():
        nb["lo"][p] = val
        nb["hi"][p] = val
        nb["curve"][p] = 1.0
        nb["symmetric"][p] = 0
    return nb


def precision_patch_nebula(base: dict, seconds: float, midi_lo: float, midi_hi: float,
                           depth_max: float) -> dict:
    """Sine-only test patch for the long-note precision study.

    Sine level 1, square-saw and noise levels 0; ADSR0 is a linear ramp over
    the whole voice (attack = seconds, alpha = 1, note held past the end) routed with weight 1
    to the sine pitch and ADSR1 a constant 1 routed to the sine amplitude.
    The base pitch is linear in [midi_lo, midi_hi] and the glide depth linear
    in [-depth_max, depth_max] (both parameters stay free, symmetric = linear).
    """
    pins = {DURATION: seconds + 1.0, SINE + 2: 0.0, MIX: 1.0, MIX + 1: 0.0, MIX + 2: 0.0, SINE: 0.0}
    a0 = ADSR
    pins.update({a0 + 0: seconds, a0 + 1: 0.0, a0 + 2: 1.0, a0 + 3: 0.0, a0 + 4: 1.0})
    a1 = ADSR + 5
    pins.update({a1 + 0: 0.0, a1 + 1: 0.0, a1 + 2: 1.0, a1 + 3: 0.0, a1 + 4: 1.0})
    for src in range(4):
        for dest in range(5):
            pins[mod_slot(src, dest)] = 0.0
    pins[mod_slot(0, 0)] = 1.0
    pins[mod_slot(1, 1)] = 1.0
    nb = pinned_nebula(base, pins)
    nb["lo"][MIDI], nb["hi"][MIDI] = midi_lo, midi_hi
    nb["curve"][MIDI], nb["symmetric"][MIDI] = 1.0, 0
    nb["lo"][SINE + 1], nb["hi"][SINE + 1] = -depth_max, depth_max
    nb["curve"][SINE + 1], nb["symmetric"][SINE + 1] = 1.0, 1
    return nb


def precision_patch_params(seed: int, batch: int, midi_lo: float, midi_hi: float,
                           depth_max: float, glide: bool) -> tuple[np.ndarray, np.ndarray]:
    """Normalized params for the precision patch: start pitch m0 and end pitch
    m1 uniform in [midi_lo, midi_hi] (m1 = m0 for constant pitch). Returns
    (u[batch][78], m0m1[batch][2])."""
    rng = np.random.default_rng(seed)
    m0 = rng.uniform(midi_lo, midi_hi, size=batch)
    m1 = rng.uniform(midi_lo, midi_hi, size=batch) if glide else m0.copy()
    u = np.full((batch, NUM_PARAMS), 0.5)
    u[:, MIDI] = (m0 - midi_lo) / (midi_hi - midi_lo)
    u[:, SINE + 1] = ((m1 - m0) + depth_max) / (2.0 * depth_max)
    return u, np.stack([m0, m1], axis=1)


def upstream_grad(seed: int, shape) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape)


def sample_voices(seed: int, batch: int, count: int) -> np.ndarray:
    """Distinct voice slots of a batch, sorted, including the first and last."""
    rng = np.random.default_rng(seed)
    if count >= batch:
        return np.arange(batch, dtype=np.int32)
    mid = rng.choice(np.arange(1, batch - 1), size=max(0, count - 2), replace=False)
    return np.sort(np.concatenate([[0, batch - 1], mid]).astype(np.int32))


def mmd_labels(seed: int, trials: int, sizes, pair, n: int) -> np.ndarray:
    """Trial labels over a pool of corpora laid end to end (corpus c holds
    sizes[c] sounds): [trials][sum(sizes)] int8, 0 for X, 1 for Y, -1 left
    out. pair = (a, b): with a == b, X and Y are a random split of n + n
    sounds of corpus a (the paper's within-corpus diversity); otherwise n
    sounds drawn from each corpus. Each trial draws afresh."""
    rng = np.random.default_rng(seed)
    starts = np.concatenate([[0], np.cumsum(sizes)])
    out = np.full((trials, int(starts[-1])), -1, dtype=np.int8)
    a, b = pair
    for t in range(trials):
        if a == b:
            pick = rng.choice(sizes[a], size=2 * n, replace=False) + starts[a]
            out[t, pick[:n]], out[t, pick[n:]] = 0, 1
        else:
            out[t, rng.choice(sizes[a], size=n, replace=False) + starts[a]] = 0
            out[t, rng.choice(sizes[b], size=n, replace=False) + starts[b]] = 1
    return out


TWO_PI = 2.0 * math.pi
