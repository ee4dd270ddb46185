"""Precision study: batch 32 x 60 s sine-only voices, constant pitch and a
linear midi glide with endpoints uniform in midi over 20 Hz .. 8 kHz; the
VCO phase running sums in 64-bit fixed point (the library's mode, finer than
FP64) and in FP32 (study mode), each against the FP64 oracle. Max-abs error and the phase drift it implies
(|error| / 2 pi cycles, over the last second) are printed as a JSON line."""
import json
import math

import numpy as np
import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu

SECONDS, BATCH = 60.0, 32
MIDI_LO = 69.0 + 12.0 * math.log2(20.0 / 440.0)
MIDI_HI = 69.0 + 12.0 * math.log2(8000.0 / 440.0)
DEPTH = MIDI_HI - MIDI_LO


@pytest.mark.parametrize("glide", [False, True])
def test_precision_study_60s(oracle_mod, glide):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_12922_gb300 as pkg
    from paper_2104_12922_gb300 import build as b
    b.build()
    nb = si.precision_patch_nebula(oracle_mod.default_nebula(), SECONDS, MIDI_LO, MIDI_HI, DEPTH)
    u, m01 = si.precision_patch_params(31 if glide else 30, BATCH, MIDI_LO, MIDI_HI, DEPTH, glide)
    u = u.astype(np.float32).astype(np.float64)  # both sides see the same float32 inputs
    cfg = oracle_mod.default_config(seconds=SECONDS, nebula=nb)
    ref, _ = oracle_mod.render_batch(cfg, 0, 0, BATCH, u_in=u)
    pin = torch.tensor(u, dtype=torch.float32, device="cuda")
    report = {"glide": glide, "batch": BATCH, "seconds": SECONDS}
    last = int(SECONDS * 44100) - 44100
    for name, carry in (("fixed64_carry", pkg.SYNTH_CARRY_FIXED64), ("fp32_carry", pkg.SYNTH_CARRY_FP32)):
        syn = pkg.Synth(seconds=SECONDS, max_batch=BATCH, carry=carry, nebula=nb)
        audio, params = syn.render(0, 0, BATCH, params_in=pin)
        syn.sync()
        a = audio.cpu().numpy()
        err = np.abs(a - ref)
        report[name] = {"max_abs": float(err.max()),
                        "max_abs_first_4s": float(err[:, :176400].max()),
                        "drift_cycles_last_1s": float(err[:, last:].max() / (2 * math.pi))}
        syn.close()
    print("PRECISION " + json.dumps(report))
    assert report["fixed64_carry"]["max_abs"] <= 2e-4
    assert report["fp32_carry"]["max_abs"] > report["fixed64_carry"]["max_abs"]
