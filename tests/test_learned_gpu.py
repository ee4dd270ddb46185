"""GPU spectral front ends and the learned proposal against the FP64 oracle.

Tolerances follow from the arithmetic of each path: the MR-STFT distance
and its gradient run on FP32 FFTs, the log-mel features on an FP32 FFT with
a bf16 output. The MLP's element-wise parity (bf16 operands, FP32
accumulation) is in test_fullsize_gpu.py.
"""
import numpy as np
import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_12922_gb300 as pkg
    from paper_2104_12922_gb300 import build as b
    b.build()
    return torch, pkg


def test_mrstft_loss_matches_oracle_on_voices(env):
    from oracle import spectral as sp
    torch, pkg = env
    syn = pkg.Synth(seconds=0.1, max_batch=2)
    x, _ = syn.render(1, 0, 2)
    y, _ = syn.render(2, 0, 2)
    mr = pkg.MRSTFT(syn, 2)
    loss, _ = mr(x, y)
    syn.sync()
    ref_voice = sp.mrstft_loss(x.cpu().numpy(), y.cpu().numpy(), per_voice=True).numpy()
    # FP32 spectra: |X| carries an absolute error of about 1e-7 of the frame's
    # norm, which moves log(|X| + 1e-7) by O(1) only in bins near silence;
    # averaged over ~1e5 bins that stays below 1e-4 relative (measured 2e-7)
    assert np.allclose(loss.cpu().numpy(), ref_voice, rtol=1e-4)
    syn.close()


def test_mrstft_gradient_matches_oracle(env):
    """Gradient on broadband signals: d log(|X| + eps) / d|X| = 1 / (|X| + eps)
    weights near-silent bins by up to 1/eps, so the gradient is compared where
    every bin carries energy (seeded Gaussian noise). FP32 FFTs: the loss
    within 1e-5 relative, the gradient within 1e-3 in relative norm (the
    small-|X| bins, weighted by 1/|X|, carry most of the rounding; measured
    2.5e-7 and 2.7e-5)."""
    from oracle import spectral as sp
    torch, pkg = env
    syn = pkg.Synth(seconds=0.1, max_batch=2)
    x = torch.tensor(si.upstream_grad(1, (2, syn.num_samples)) * 0.3, dtype=torch.float32,
                     device="cuda")
    y = torch.tensor(si.upstream_grad(2, (2, syn.num_samples)) * 0.3, dtype=torch.float32,
                     device="cuda")
    mr = pkg.MRSTFT(syn, 2)
    loss, gx = mr(x, y)
    syn.sync()
    ref_loss, ref_g = sp.mrstft_loss_and_grad(x.cpu().numpy(), y.cpu().numpy())
    g = gx.cpu().numpy().astype(np.float64)
    assert float(loss.sum()) == pytest.approx(ref_loss, rel=1e-5)
    assert np.linalg.norm(g - ref_g) <= 1e-3 * np.linalg.norm(ref_g)
    # the target spectra kept in the workspace give the same result
    loss2, gx2 = mr(x, y, target_ready=True)
    syn.sync()
    assert torch.equal(loss, loss2) and torch.equal(gx, gx2)
    syn.close()


@pytest.mark.parametrize("seconds,batch", [(1.0, 8), (0.05, 3), (4.0, 2)])
def test_logmel_features_fft_bar(env, seconds, batch):
    """The FFT front end computes the spectrum in FP32, so the bf16 rounding
    of the output feature f = (logmel + 2.5) / 6 dominates: |f| < 2 gives a
    half-ulp of at most 2^-8 in f, 6 x 2^-8 = 0.0234 in log units. Bands
    within 60 dB of the voice's loudest band (FP32 spectrum error far below
    their energy) meet that bar plus 2e-3; every band, including those at
    the 1e-6 floor, stays within 0.1. Sizes: 87 frames (a ragged group of 7),
    5 frames (one group; reflect padding on both sides of every frame),
    345 frames; 0.05 s and 4 s voices have N % 512 != 0."""
    from oracle import spectral as sp
    torch, pkg = env
    syn = pkg.Synth(seconds=seconds, max_batch=8)
    model = pkg.ProposalModel(syn, max_batch=8, seed=0)
    audio, _ = syn.render(6, 1, batch)
    feats = model.features(audio)
    syn.sync()
    got = feats.float().cpu().numpy().reshape(batch, -1, 128)
    ref = sp.log_mel(audio.cpu().numpy()).numpy()
    ref_f = (ref - pkg.FEATURE_SHIFT) / pkg.FEATURE_SCALE
    assert got.shape == ref.shape
    err = np.abs(got - ref_f) * pkg.FEATURE_SCALE
    near = ref > (ref.max(axis=(1, 2), keepdims=True) - np.log(1e6))
    print(f"FFT log-mel: max err {err.max():.4f}, within 60 dB {err[near].max():.4f}, "
          f"median {np.median(err):.5f}")
    assert np.max(err[near]) <= 6 * 2.0 ** -8 + 2e-3
    assert np.max(err) <= 0.1
    model.close()
    syn.close()


def test_training_learns_pitch_and_checkpoint_roundtrip(env, tmp_path):
    """On-the-fly training (1 s voices, batch 64, training split) makes the
    proposal's midi-f0 estimate on held-out test voices clearly better than
    the best constant guess (MSE 1/12 for a uniform parameter); a saved and
    reloaded model proposes identical parameters."""
    torch, pkg = env
    from paper_2104_12922_gb300 import proposal as pr
    syn = pkg.Synth(seconds=1.0, max_batch=64)
    model = pkg.ProposalModel(syn, max_batch=64, seed=1)
    pr.train(model, 1500, batch=64, lr=1e-3, log_every=500)
    it = pr.test_batches(64)
    errs = []
    for _ in range(4):
        b = next(it)
        audio, u = syn.render(0, b, 64)
        prop = model.propose(audio)
        errs.append(((prop - u) ** 2).mean(dim=0).cpu().numpy())
    syn.sync()
    mse = np.mean(errs, axis=0)
    assert np.all(np.isfinite(mse))
    assert mse[si.MIDI] < 0.5 / 12.0, mse[si.MIDI]
    audio, _ = syn.render(9, 3, 8)
    p1 = model.propose(audio)
    path = str(tmp_path / "model.bin")
    model.save(path)
    other = pkg.ProposalModel(syn, max_batch=64, seed=99)
    other.load(path)
    p2 = other.propose(audio)
    syn.sync()
    assert torch.equal(p1, p2)
    other.close()
    model.close()
    syn.close()


def test_param_adam_descends_and_stays_in_range(env):
    torch, pkg = env
    syn = pkg.Synth(seconds=0.01, max_batch=1)
    u = torch.full((78,), 0.5, device="cuda")
    m = torch.zeros_like(u)
    v = torch.zeros_like(u)
    g = torch.linspace(-1, 1, 78, device="cuda")
    for step in range(1, 200):
        pkg.param_adam(syn, u, g, m, v, step, 0.01)
    syn.sync()
    assert float(u.min()) >= 0.0 and float(u.max()) <= 1.0
    assert float(u[0]) > 0.99 and float(u[-1]) < 0.01
    syn.close()


def test_pipelined_training_equals_one_stream_training(env):
    """proposal.train renders and transforms the next batch on a second
    stream while the network trains on this one; the model it leaves is the
    one the one-stream loop of synth_model_train_step leaves, bit for bit."""
    torch, pkg = env
    from paper_2104_12922_gb300 import proposal as pr
    syn = pkg.Synth(seconds=0.25, max_batch=16)
    one = pkg.ProposalModel(syn, max_batch=16, seed=4)
    two = pkg.ProposalModel(syn, max_batch=16, seed=4)
    r1 = pr.train(one, 7, batch=16, lr=1e-3, log_every=3, pipeline=False)
    r2 = pr.train(two, 7, batch=16, lr=1e-3, log_every=3, pipeline=True)
    assert r1["loss"] == r2["loss"]
    for l in range(4):
        assert torch.equal(one.tensor(0, l), two.tensor(0, l)), l
        assert torch.equal(one.tensor(1, l), two.tensor(1, l)), l
    one.close()
    two.close()
    syn.close()
