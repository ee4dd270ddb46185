"""The 4-operator FM voice (synth_fm_render) against the FP64 oracle.

Parameters: bit-exact (Philox stream 2, float32 normalized values).
Audio bar, derived per voice from the FP32 arithmetic: each operator's
sine argument carries about 2e-6 (radians, relative to a unit amplitude)
of rounding -- the 24-bit phase, the float sum of phase and modulation,
the sine itself and the envelope -- and a modulator's error reaches the
output through the levels of every operator below it (d sin / d arg <= 1):
|error| <= 2e-6 l0 (1 + l1 + l1 l2 + l1 l2 l3) + 1e-6, with l_i the mapped
levels (l0 <= 1, modulators up to 8 rad)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_12922_gb300 as p
    from paper_2104_12922_gb300 import build as b
    b.build()
    return p


def _levels(u):
    """mapped levels of the four operators (carrier amplitude, three indices)"""
    return [u[3], 8.0 * u[10] ** 2, 8.0 * u[17] ** 2, 8.0 * u[24] ** 2]


def _bar(u):
    l0, l1, l2, l3 = _levels(u)
    return 2e-6 * l0 * (1 + l1 + l1 * l2 + l1 * l2 * l3) + 1e-6


@pytest.mark.parametrize("sr,cr,n", [(44100.0, 441.0, 44100), (44100.0, 441.0, 10243),
                                     (16000.0, 441.0, 16000), (48000.0, 480.0, 9001)])
def test_fm_matches_oracle(pkg, oracle_mod, sr, cr, n):
    """Drawn voices; N = 10243 and 9001 end in a ragged chunk and quad."""
    seconds = n / sr
    syn = pkg.Synth(seconds=seconds, max_batch=8, sample_rate=sr, control_rate=cr)
    audio, params = syn.fm_render(12, 5, 8)
    syn.sync()
    cfg = oracle_mod.default_config(seconds=seconds, sample_rate=sr, control_rate=cr)
    ref_a, ref_p = oracle_mod.fm_render_batch(cfg, 12, 5, 8)
    p = params.cpu().numpy()
    assert np.array_equal(p, ref_p)
    a = audio.cpu().numpy()
    assert np.all(np.isfinite(a))
    for v in range(8):
        err = float(np.max(np.abs(a[v] - ref_a[v])))
        assert err <= _bar(p[v].astype(np.float64)), (v, err, _levels(p[v]))
    syn.close()


def test_fm_given_params_and_edges(pkg, oracle_mod):
    """Caller parameters: all zeros (silent carrier), all ones (the largest
    indices and ratios: aliasing operators), halves, and values outside
    [0, 1] (clamped)."""
    import torch
    syn = pkg.Synth(seconds=0.5, max_batch=4)
    u = np.stack([np.zeros(30), np.ones(30), np.full(30, 0.5),
                  np.linspace(-0.5, 1.5, 30)]).astype(np.float32)
    audio, params = syn.fm_render(0, 0, 4, params_in=torch.tensor(u, device="cuda"))
    syn.sync()
    uc = np.clip(u, 0.0, 1.0).astype(np.float64)
    assert np.array_equal(params.cpu().numpy(), uc.astype(np.float32))
    cfg = oracle_mod.default_config(seconds=0.5)
    ref_a, _ = oracle_mod.fm_render_batch(cfg, 0, 0, 4, u_in=uc)
    a = audio.cpu().numpy()
    for v in range(4):
        err = float(np.max(np.abs(a[v] - ref_a[v])))
        assert err <= _bar(uc[v]), (v, err)
    assert np.all(a[0] == 0.0)
    syn.close()


def test_fm_argument_errors(pkg):
    import torch
    syn = pkg.Synth(seconds=0.1, max_batch=2)
    L = pkg.lib()
    out = torch.empty((2, syn.num_samples), device="cuda")
    assert L.synth_fm_render(syn.handle, 0, 0, 3, None, out.data_ptr(), None, None) == pkg.SYNTH_ERR_ARG
    assert L.synth_fm_render(syn.handle, 0, 0, 2, None, None, None, None) == pkg.SYNTH_ERR_ARG
    assert L.synth_fm_render(syn.handle, 0, 0, 0, None, None, None, None) == pkg.SYNTH_OK
    syn.close()


def test_fm_index_rule_across_batch_sizes(pkg):
    """Voice g = batch_index * batch + v depends on (seed, g) only: voices
    16..23 of one batch of 32 equal batch index 2 of batches of 8."""
    import torch
    syn = pkg.Synth(seconds=0.5, max_batch=32)
    a32, p32 = syn.fm_render(9, 0, 32)
    a8, p8 = syn.fm_render(9, 2, 8)
    syn.sync()
    assert torch.equal(p32[16:24], p8) and torch.equal(a32[16:24], a8)
    syn.close()


def test_fm_full_size_sampled(pkg, oracle_mod):
    """The FM throughput workload: batch 128 x 4 s at 44.1 kHz, seed = batch
    index = 5, voices g = 5 * 128 + v; sampled voices vs the oracle."""
    import seeded_inputs as si
    syn = pkg.Synth(seconds=4.0, max_batch=128)
    audio, params = syn.fm_render(5, 5, 128)
    syn.sync()
    cfg = oracle_mod.default_config(seconds=4.0)
    a = audio.cpu().numpy()
    p = params.cpu().numpy()
    assert np.all(np.isfinite(a))
    for v in si.sample_voices(5, 128, 5):
        u = oracle_mod.fm_draw_params(5, 5 * 128 + int(v))
        assert np.array_equal(p[v], u.astype(np.float32)), v
        ref = oracle_mod.fm_render_voice(cfg, u)
        err = float(np.max(np.abs(a[v] - ref)))
        assert err <= _bar(u), (int(v), err, _levels(u))
    syn.close()
