"""Pins of the spectral oracle (no GPU): STFT against a brute-force DFT with
explicit reflect padding and periodic Hann window, Parseval, a pure tone's
peak bin, the multi-resolution distance's zero/symmetry and gradient, the
Slaney mel scale's fixed points and the filterbank's band placement, and
the MLP gradient against finite differences."""
import math

import numpy as np
import pytest

from oracle import spectral as sp


def _brute_stft(x, n_fft):
    hop = n_fft // 4
    pad = n_fft // 2
    N = len(x)
    idx = np.arange(-pad, N + pad)
    idx = np.where(idx < 0, -idx, idx)
    idx = np.where(idx >= N, 2 * (N - 1) - idx, idx)
    xp = x[idx]
    w = 0.5 - 0.5 * np.cos(2 * math.pi * np.arange(n_fft) / n_fft)
    n_frames = 1 + N // hop
    out = np.zeros((n_fft // 2 + 1, n_frames), dtype=complex)
    for f in range(n_frames):
        seg = xp[f * hop: f * hop + n_fft] * w
        for k in range(n_fft // 2 + 1):
            out[k, f] = sum(seg[t] * complex(math.cos(2 * math.pi * k * t / n_fft),
                                             -math.sin(2 * math.pi * k * t / n_fft))
                            for t in range(n_fft))
    return out


def test_stft_matches_brute_force_dft():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(64)
    got = sp.stft(x[None, :], 16)[0].numpy()
    want = _brute_stft(x, 16)
    assert got.shape == want.shape
    assert np.max(np.abs(got - want)) < 1e-12


def test_stft_parseval_per_frame():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(256)
    n = 32
    X = sp.stft(x[None, :], n)[0].numpy()
    w = 0.5 - 0.5 * np.cos(2 * math.pi * np.arange(n) / n)
    xp = np.pad(x, n // 2, mode="reflect")
    for f in [0, 3, X.shape[1] - 1]:
        seg = xp[f * n // 4: f * n // 4 + n] * w
        e = np.abs(X[0, f]) ** 2 + np.abs(X[-1, f]) ** 2 + 2 * np.sum(np.abs(X[1:-1, f]) ** 2)
        assert e == pytest.approx(n * np.sum(seg ** 2), rel=1e-12)


def test_pure_tone_peaks_at_its_bin():
    n, k0 = 512, 37
    t = np.arange(44100 // 10)
    x = np.sin(2 * math.pi * k0 * t / n)
    mag = sp.stft(x[None, :], n)[0].abs().numpy()
    assert np.all(np.argmax(mag[:, 4:-4], axis=0) == k0)


def test_mrstft_zero_symmetric_and_gradient():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 2048))
    y = rng.standard_normal((2, 2048))
    assert float(sp.mrstft_loss(x, x)) == 0.0
    assert float(sp.mrstft_loss(x, y)) == pytest.approx(float(sp.mrstft_loss(y, x)), rel=1e-14)
    loss, g = sp.mrstft_loss_and_grad(x, y, n_ffts=(64, 128))
    for (b, i) in [(0, 5), (1, 1000), (0, 2047)]:
        h = 1e-6
        xp, xm = x.copy(), x.copy()
        xp[b, i] += h
        xm[b, i] -= h
        fd = (float(sp.mrstft_loss(xp, y, (64, 128), per_voice=True).sum()) -
              float(sp.mrstft_loss(xm, y, (64, 128), per_voice=True).sum())) / (2 * h)
        assert g[b, i] == pytest.approx(fd, rel=1e-5, abs=1e-8)


def test_slaney_mel_scale_points():
    assert float(sp.hz_to_mel(1000.0)) == pytest.approx(15.0)
    assert float(sp.hz_to_mel(6400.0)) == pytest.approx(42.0)
    assert float(sp.hz_to_mel(200.0)) == pytest.approx(3.0)
    f = np.array([0.0, 100.0, 999.0, 1000.0, 5000.0, 22050.0])
    assert np.allclose(sp.mel_to_hz(sp.hz_to_mel(f)), f, rtol=1e-12, atol=1e-9)


def test_mel_filterbank_band_placement():
    fb = sp.mel_filterbank(2048, 128, 44100.0)
    assert fb.shape == (128, 1025) and fb.min() >= 0.0
    assert np.all(fb.sum(axis=1) > 0)
    edges = sp.mel_to_hz(np.linspace(0.0, float(sp.hz_to_mel(22050.0)), 130))
    bins = np.arange(1025) * 44100.0 / 2048
    for i in [5, 40, 100, 127]:
        # the band's peak sits at the FFT bin nearest its centre edge
        assert abs(bins[np.argmax(fb[i])] - edges[i + 1]) <= 44100.0 / 2048
        # unit area in Hz (triangles several bins wide)
        if edges[i + 2] - edges[i] > 10 * 44100.0 / 2048:
            assert np.sum(fb[i]) * 44100.0 / 2048 == pytest.approx(1.0, rel=0.02)


def test_log_mel_shape_and_tone_band():
    sr = 44100.0
    t = np.arange(int(sr)) / sr
    x = np.sin(2 * math.pi * 3000.0 * t)
    feats = sp.log_mel(x[None, :]).numpy()[0]
    assert feats.shape == (1 + 44100 // 512, 128)
    fb = sp.mel_filterbank()
    k = int(round(3000.0 * 2048 / sr))
    assert np.argmax(feats[40]) in np.argsort(fb[:, k])[-2:]


def test_mlp_gradients_match_finite_differences():
    rng = np.random.default_rng(3)
    dims = [6, 5, 4, 3]
    ws = [rng.standard_normal((dims[i + 1], dims[i])) * 0.5 for i in range(3)]
    bs = [rng.standard_normal(dims[i + 1]) * 0.1 for i in range(3)]
    x = rng.standard_normal((4, 6))
    tgt = rng.uniform(size=(4, 3))
    loss, gw, gb = sp.mlp_loss_and_grads(x, tgt, ws, bs)
    h = 1e-6
    for l, (i, j) in [(0, (1, 2)), (1, (3, 0)), (2, (2, 3))]:
        wp = [w.copy() for w in ws]
        wm = [w.copy() for w in ws]
        wp[l][i, j] += h
        wm[l][i, j] -= h
        fd = (sp.mlp_loss_and_grads(x, tgt, wp, bs)[0] - sp.mlp_loss_and_grads(x, tgt, wm, bs)[0]) / (2 * h)
        assert gw[l][i, j] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_mrstft_loss_of_a_scaled_copy():
    """L(c x, x) = sum over the three resolutions of the mean over (bins,
    frames) of |ln(c|X| + eps) - ln(|X| + eps)|, which is 3 |ln c| wherever
    |X| >> eps. Broadband noise keeps every bin far above eps = 1e-7 (the
    smallest |X| is ~1e-2, so the eps terms move the value by < 1e-4 of it).
    Per voice, each voice's own factor; over the batch, the voices' mean.
    Summing instead of averaging, a dropped resolution, |X|^2 instead of |X|
    or a base-10 log all miss this value."""
    rng = np.random.default_rng(5)
    x = rng.standard_normal((3, 8192)) * 0.3
    c = np.array([2.0, 0.25, 1.5])
    per = sp.mrstft_loss(c[:, None] * x, x, per_voice=True).numpy()
    assert np.allclose(per, 3 * np.abs(np.log(c)), rtol=1e-4)
    whole = float(sp.mrstft_loss(c[:, None] * x, x))
    assert whole == pytest.approx(3 * np.mean(np.abs(np.log(c))), rel=1e-4)
    # one resolution alone: |ln c|
    one = sp.mrstft_loss(2.0 * x, x, n_ffts=(1024,), per_voice=True).numpy()
    assert np.allclose(one, math.log(2.0), rtol=1e-4)
    # both silent: every bin at the floor, distance 0; one silent: the
    # distance is the mean of ln((|X| + eps) / eps) over the other's bins
    z = np.zeros((1, 4096))
    assert float(sp.mrstft_loss(z, z)) == 0.0
    y = x[:1, :4096]
    want = 0.0
    for n in (512, 1024, 2048):
        mag = sp.stft(y, n).abs().numpy()
        want += np.mean(np.log((mag + sp.MR_EPS) / sp.MR_EPS))
    assert float(sp.mrstft_loss(y, z)) == pytest.approx(want, rel=1e-12)


def test_mlp_forward_hand_set_two_layer_net():
    """x = (1, -2); W1 = [[1, 0], [0, 1], [1, 1]], b1 = (0, 0, 0.5):
    z1 = (1, -2, -0.5), ReLU zeroes the last two; W2 = [[2, 3, 4]], b2 = -1:
    z2 = 1, sigmoid(1) = 1 / (1 + e^-1) = 0.7310585786300049. A ReLU on the
    output (1.0), a sigmoid on the hidden layer, or a transposed W all give
    other values. The MSE against a target t is (y - t)^2 averaged."""
    w1 = np.array([[1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
    b1 = np.array([0.0, 0.0, 0.5])
    w2 = np.array([[2.0, 3.0, 4.0]])
    b2 = np.array([-1.0])
    y = sp.mlp_forward(np.array([[1.0, -2.0]]), [w1, w2], [b1, b2]).numpy()
    assert y.shape == (1, 1)
    assert y[0, 0] == pytest.approx(0.7310585786300049, abs=1e-15)
    # a row with every hidden unit active: z1 = (0.5, 0.25, 1.25),
    # z2 = 1 + 0.75 + 5 - 1 = 5.75
    y2 = sp.mlp_forward(np.array([[0.5, 0.25]]), [w1, w2], [b1, b2]).numpy()[0, 0]
    assert y2 == pytest.approx(1.0 / (1.0 + math.exp(-5.75)), abs=1e-15)
    loss, _, _ = sp.mlp_loss_and_grads(np.array([[1.0, -2.0], [0.5, 0.25]]),
                                       np.array([[0.5], [1.0]]), [w1, w2], [b1, b2])
    want = ((0.7310585786300049 - 0.5) ** 2 + (y2 - 1.0) ** 2) / 2
    assert loss == pytest.approx(want, rel=1e-12)


def test_log_mel_floor_and_power_scale():
    """Silence gives ln(1e-6) in every band and frame. A tone's mel energies
    are a power spectrum: doubling the amplitude adds ln 4 in the bands that
    hold it (far above the floor). Its absolute value follows from the DFT of
    a bin-centred tone under the periodic Hann window (|X| = A n / 4 at its
    bin, A n / 8 at the two neighbours, 0 elsewhere) weighted by the
    filterbank, in frames clear of the reflect padding."""
    silent = sp.log_mel(np.zeros((2, 8192))).numpy()
    assert silent.shape == (2, 17, 128)
    assert np.all(silent == math.log(1e-6))
    sr, n = 44100.0, 2048
    kbin, A = 139, 0.5                      # 2993 Hz, exactly on bin 139
    t = np.arange(22050)
    x = A * np.cos(2 * math.pi * kbin * t / n)
    m1 = sp.log_mel(x[None, :]).numpy()[0]
    m2 = sp.log_mel(2 * x[None, :]).numpy()[0]
    fb = sp.mel_filterbank(n, 128, sr)
    loud = fb[:, kbin] > 0
    assert np.allclose(m2[10:30][:, loud] - m1[10:30][:, loud], math.log(4.0), atol=1e-9)
    power = np.zeros(n // 2 + 1)
    power[kbin] = (A * n / 4) ** 2
    power[kbin - 1] = power[kbin + 1] = (A * n / 8) ** 2
    want = np.log(fb @ power + 1e-6)
    assert np.allclose(m1[10:30][:, loud], want[loud], atol=1e-9)


def test_mlp_trace_matches_autograd():
    """The written-out chain rule of mlp_trace gives autograd's loss and
    gradients (which the finite-difference test pins), and its Y is
    mlp_forward's output."""
    rng = np.random.default_rng(8)
    dims = [7, 6, 5, 4, 3]
    ws = [rng.standard_normal((dims[i + 1], dims[i])) * 0.6 for i in range(4)]
    bs = [rng.standard_normal(dims[i + 1]) * 0.2 for i in range(4)]
    x = rng.standard_normal((5, 7))
    tgt = rng.uniform(size=(5, 3))
    tr = sp.mlp_trace(x, tgt, ws, bs)
    loss, gw, gb = sp.mlp_loss_and_grads(x, tgt, ws, bs)
    assert tr["loss"] == pytest.approx(loss, rel=1e-14)
    assert np.allclose(tr["Y"], sp.mlp_forward(x, ws, bs).numpy(), rtol=1e-14, atol=0)
    for l in range(4):
        assert np.allclose(tr["gW"][l], gw[l], rtol=1e-12, atol=1e-15)
        assert np.allclose(tr["gb"][l], gb[l], rtol=1e-12, atol=1e-15)
    assert np.any(tr["Z"][1] < 0)  # the ReLU masks something in this case
    # given ReLU decisions: the oracle's own reproduce the trace; flipping one
    # entry moves the gradients below it by exactly that entry's dH term
    own = [tr["Z"][l] > 0 for l in range(3)]
    same = sp.mlp_trace(x, tgt, ws, bs, masks=own)
    assert np.array_equal(same["gW"][0], tr["gW"][0])
    flipped = [m.copy() for m in own]
    b, j = np.argwhere(~own[1])[0]
    flipped[1][b, j] = True
    alt = sp.mlp_trace(x, tgt, ws, bs, masks=flipped)
    extra = np.zeros_like(tr["dZ"][1])
    extra[b, j] = tr["dH"][2][b, j]
    assert np.allclose(alt["gW"][1] - tr["gW"][1], extra.T @ tr["H"][1], atol=1e-15)
    assert np.array_equal(alt["gW"][2], tr["gW"][2])
