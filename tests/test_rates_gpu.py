"""Renders at sample rates whose ratio R = SR / CR to the control rate is not
an integer multiple of 4 (the paper renders at any sample rate, Sec. 2.2):
a fractional R from integer rates (16 kHz, 8 kHz, 48 kHz, 96 kHz at the
default 441 Hz control rate) and integer R = 50, 98. The fused render is
checked against the FP64 oracle with the same bar as at 44.1 kHz: parameter
draws bit-exact, audio max-abs error <= 2e-4; the lengths include voices
shorter than two intervals and one tile (255 intervals) plus a few samples."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 2e-4


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_12922_gb300 as p
    from paper_2104_12922_gb300 import build as b
    b.build()
    return p


@pytest.mark.parametrize("sr,cr,n", [
    (16000.0, 441.0, 64000),   # R = 36.28..
    (22050.0, 441.0, 88200),   # R = 50
    (8000.0, 441.0, 8000),     # R = 18.14..
    (48000.0, 441.0, 96000),   # R = 108.84..
    (44100.0, 450.0, 44100),   # R = 98
    (96000.0, 441.0, 48000),   # R = 217.68..
    (16000.0, 441.0, 50),      # two intervals
    (16000.0, 441.0, 9253),    # one tile of 255 intervals (9251.7 samples) and a bit
])
def test_fused_matches_oracle_at_other_rates(pkg, oracle_mod, sr, cr, n):
    seconds = n / sr
    syn = pkg.Synth(seconds=seconds, max_batch=6, sample_rate=sr, control_rate=cr)
    assert syn.num_samples == n
    audio, params = syn.render(3, 11, 6)
    syn.sync()
    cfg = oracle_mod.default_config(seconds=seconds, sample_rate=sr, control_rate=cr)
    ref_a, ref_p = oracle_mod.render_batch(cfg, 3, 11, 6)
    assert np.array_equal(params.cpu().numpy(), ref_p)
    a = audio.cpu().numpy()
    assert np.all(np.isfinite(a))
    err = float(np.max(np.abs(a - ref_a)))
    assert err <= TOL, f"max-abs error {err:.3e} at SR {sr}, CR {cr}"
    syn.close()


def test_normalized_and_unsupported_paths_at_fractional_rate(pkg):
    import torch
    syn = pkg.Synth(seconds=1.0, max_batch=8, sample_rate=16000.0, control_rate=441.0)
    raw, _ = syn.render(4, 2, 8)
    a, _, peak, silent = syn.render_normalized(4, 2, 8, threshold=1e-3)
    syn.sync()
    want = raw.abs().amax(dim=1)
    assert torch.equal(peak, want)
    loud = want >= 1e-3
    assert torch.equal(a, torch.where(loud[:, None], raw * (1.0 / want)[:, None], raw))
    # the plain and adjoint renders keep R an integer multiple of 4
    L = pkg.lib()
    b = ctypes.c_size_t()
    assert L.synth_render_plain_workspace_size(syn.handle, 8, ctypes.byref(b)) == pkg.SYNTH_ERR_UNSUPPORTED
    assert L.synth_render_backward_workspace_size(syn.handle, 8, ctypes.byref(b)) == pkg.SYNTH_ERR_UNSUPPORTED
    syn.close()


def test_fractional_rate_full_size_sampled(pkg, oracle_mod):
    """The fractional-rate throughput workload: batch 128 x 4 s at 16 kHz with
    the 441 Hz control rate, seed = batch index; sampled voices vs the oracle."""
    import seeded_inputs as si
    syn = pkg.Synth(seconds=4.0, max_batch=128, sample_rate=16000.0, control_rate=441.0)
    audio, params = syn.render(9, 9, 128)
    syn.sync()
    rows = si.sample_voices(9, 128, 6)
    cfg = oracle_mod.default_config(seconds=4.0, sample_rate=16000.0, control_rate=441.0)
    ref_a, ref_p = oracle_mod.render_batch(cfg, 9, 9, 128, voices=rows)
    assert np.array_equal(params.cpu().numpy()[rows], ref_p[rows])
    a = audio.cpu().numpy()[rows]
    assert np.all(np.isfinite(a))
    err = float(np.max(np.abs(a - ref_a[rows])))
    assert err <= TOL, f"max-abs error {err:.3e}"
    syn.close()
