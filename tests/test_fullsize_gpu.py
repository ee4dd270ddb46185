"""Full-size parity of the learned proposal's network and the spectral
distance, at the shapes the proposal training and the adjoint refinement run:

* the MLP (44160 -> 1024 -> 1024 -> 1024 -> 78) at batch 128 on the features
  of 4 s voices: outputs and every weight and bias gradient element by
  element against the FP64 oracle, each within an error bar propagated from
  the GPU's own roundings (below);
* the MR-STFT distance and its gradient at batch 64 x 1 s, element by
  element (every persistent CTA takes several work items here, so the
  next-item prefetch and the per-item segment sums run).

Error bars of the MLP. The GPU and the oracle share the bf16 weights and
the bf16 input features; what differs is that the GPU rounds every hidden
activation and every backward operand dZ to bf16 (round to nearest: a
relative error within +-u_b = +-2^-8 (8 significant bits), modelled as uniform, variance
u_b^2 / 3) and accumulates in FP32. These independent roundings are
propagated as variances through each linear map (var(e M) = var(e) M^2),
through the ReLU (1-Lipschitz) and the sigmoid (its derivative y (1 - y));
the bar is 7 standard deviations. The ReLU's derivative is a decision,
not a rounding: where a pre-activation Z lies within 7 sigma of 0 either
choice is correct, so there the oracle's backward takes the GPU's choice
(read back from the GPU's hidden activations), and everywhere else the two
must agree.
"""
import numpy as np
import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu

U_B = 2.0 ** -8     # bf16 unit roundoff (8 significant bits), relative
VAR_B = U_B ** 2 / 3.0
NSIG = 7.0


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_12922_gb300 as pkg
    from paper_2104_12922_gb300 import build as b
    b.build()
    return torch, pkg


def _bf16_values(t):
    import torch
    return t.to(dtype=torch.bfloat16).float().cpu().numpy().astype(np.float64)


def _acc_var(a, w, k):
    """FP32 accumulation of k terms: the tensor cores round once per 16-term
    chunk, at most 2^-24 of the running sum (bounded by sum |terms|)."""
    return (k / 16.0) * (2.0 ** -24 * (np.abs(a) @ np.abs(w))) ** 2 / 3.0


def _forward_var(tr, ws):
    """Variances of the GPU's pre-activations Z_l and hidden activations H_l."""
    vH = [np.zeros_like(tr["H"][0])]
    vZ = []
    for l in range(len(ws)):
        vz = vH[l] @ (ws[l] ** 2).T + _acc_var(tr["H"][l], ws[l].T, ws[l].shape[1])
        vZ.append(vz)
        if l < len(ws) - 1:
            vH.append(vz + VAR_B * tr["H"][l + 1] ** 2)
    return vZ, vH


def _mlp_bars(tr, ws, t, vZ, vH):
    """Element-wise bars of the GPU's outputs and gradients (see the module
    docstring) from the oracle's trace ``tr`` (taken with the GPU's ReLU
    decisions where they are uncertain), the bf16 weights ``ws``, the
    training target ``t`` and the forward variances."""
    L = len(ws)
    W2 = [w * w for w in ws]
    Y = tr["Y"]
    e32 = 2.0 ** -23                                      # FP32 evaluation, relative
    vY = (Y * (1 - Y)) ** 2 * vZ[L - 1] + (e32 * Y) ** 2
    B, P = Y.shape
    s = 2.0 / (B * P)
    fp = np.abs(Y * (1 - Y) + (Y - t) * (1 - 2 * Y))      # |d/dy (y - t) y (1 - y)|
    vdzf = (s * fp) ** 2 * vY + (e32 * tr["dZ"][L - 1]) ** 2
    bars_w, bars_b = [None] * L, [None] * L
    for l in range(L - 1, -1, -1):
        dz = tr["dZ"][l]
        vdzb = vdzf + VAR_B * dz * dz
        H = tr["H"][l]
        bv = vdzb.T @ (H * H) + (dz * dz).T @ vH[l] + _acc_var(dz.T, H, B)
        bars_w[l] = NSIG * np.sqrt(bv)
        bars_b[l] = NSIG * np.sqrt(vdzf.sum(axis=0) + _acc_var(np.ones((1, B)), dz, B)[0])
        if l == 0:
            break
        vdh = vdzb @ W2[l] + _acc_var(dz, ws[l], ws[l].shape[0])
        vdzf = np.where(tr["dZ"][l - 1] != 0, vdh, 0.0) + (e32 * tr["dZ"][l - 1]) ** 2
    return NSIG * np.sqrt(vY), bars_w, bars_b


@pytest.mark.parametrize("seconds,B", [(4.0, 128), (0.25, 16), (0.05, 4864)])
def test_mlp_elementwise(env, seconds, B):
    """Batch 128, 4 s voices (345 frames x 128 bands = 44160 inputs): the
    first layer's forward GEMM is 128 x 1024 x 44160 (split into 37 K-slices
    over the SMs), its weight gradient 1024 x 44160 x 128 (1,384 output
    tiles: every persistent CTA takes many). Batch 16 x 0.25 s (2816 inputs):
    a batch that fills only part of a 128-row tile. Batch 4864 x 0.05 s (640
    inputs): the hidden layers' products have 38 x 4 = 152 output tiles, as
    many as the GPU has SMs, so they are not split and their bias, ReLU, bf16
    and transposed bf16 outputs come from the GEMM's own epilogue."""
    from oracle import spectral as sp
    torch, pkg = env
    syn = pkg.Synth(seconds=seconds, max_batch=B)
    model = pkg.ProposalModel(syn, max_batch=B, seed=11)
    audio, params = syn.render(21, 3, B)
    feats = model.features(audio)
    ws = [_bf16_values(model.tensor(0, l)) for l in range(4)]
    bs = [model.tensor(1, l).cpu().numpy().astype(np.float64) for l in range(4)]
    out = model.forward(feats)
    syn.sync()
    x = feats.float().cpu().numpy().astype(np.float64)
    assert x.shape == (B, model.feature_dim)
    tgt = params.cpu().numpy().astype(np.float64)
    tr = sp.mlp_trace(x, tgt, ws, bs)
    vZ, vH = _forward_var(tr, ws)
    got = out.cpu().numpy().astype(np.float64)
    model.train_features(feats, params, lr=1e-4)
    hidden = [model.tensor(4, l, B).cpu().numpy() for l in (1, 2, 3)]
    syn.sync()
    # the GPU's ReLU decisions: taken where |Z| <= 7 sigma, checked elsewhere
    masks = []
    for l in range(3):
        z, gpu = tr["Z"][l], hidden[l] > 0
        unsure = np.abs(z) <= NSIG * np.sqrt(vZ[l])
        assert np.array_equal(gpu[~unsure], (z > 0)[~unsure]), l
        print(f"hidden layer {l + 1}: {unsure.sum()} of {z.size} ReLU decisions within 7 sigma "
              f"of 0, {np.count_nonzero(gpu != (z > 0))} taken the other way")
        masks.append(np.where(unsure, gpu, z > 0))
    tr = sp.mlp_trace(x, tgt, ws, bs, masks=masks)
    bar_y, bars_w, bars_b = _mlp_bars(tr, ws, tgt, vZ, vH)
    r = np.abs(got - tr["Y"]) / bar_y
    print(f"MLP forward: max |err| {np.abs(got - tr['Y']).max():.3e}, max err/bar {r.max():.3f}, "
          f"median bar {np.median(bar_y):.2e}")
    assert np.all(np.abs(got - tr["Y"]) <= bar_y)
    for l in range(4):
        gw = model.tensor(2, l).cpu().numpy().astype(np.float64)
        gb = model.tensor(3, l).cpu().numpy().astype(np.float64)
        ew = np.abs(gw - tr["gW"][l])
        eb = np.abs(gb - tr["gb"][l])
        print(f"layer {l}: dW max err {ew.max():.3e} (max |dW| {np.abs(tr['gW'][l]).max():.3e}), "
              f"err/bar {np.max(ew / (bars_w[l] + 1e-30)):.3f}, median bar/|dW| "
              f"{np.median(bars_w[l] / (np.abs(tr['gW'][l]) + 1e-30)):.2e}; db err/bar "
              f"{np.max(eb / (bars_b[l] + 1e-30)):.3f}")
        assert np.all(ew <= bars_w[l] + 1e-12 * np.abs(tr["gW"][l]).max()), l
        assert np.all(eb <= bars_b[l] + 1e-12 * np.abs(tr["gb"][l]).max()), l
    model.close()
    syn.close()


def _mrstft_grad_bar(x, y, n_ffts=(512, 1024, 2048), eps=1e-7, c=4.0):
    """Per-sample bar for the FP32 gradient of the MR-STFT distance.

    The distance's gradient weights each bin by 1 / (|X| + eps): a bin where
    |X| is small amplifies any error of X, and the GPU computes X by an FP32
    FFT whose absolute error is about 2^-24 log2(n) times the frame's norm
    (here taken c times that, eps_f). Per bin the gradient term
    scale sign(d) X / (|X| (|X| + eps)) then moves by at most
    scale / (|X| + eps) min(2, 2 eps_f / |X|), plus a sign flip of d where
    |d| is within the two spectra's errors (2 scale / (|X| + eps)), plus the
    SFU's few-ulp relative errors (4e-6 of the term). A frame's bins reach a
    sample m of the frame through the inverse transform with weight at most
    w[m] each, so the bar of the frame at m is w[m] times the sum of its bins'
    bounds; frames add by overlap and the reflect padding folds back, as in
    the gradient itself. Computed from the FP64 spectra of the oracle."""
    from oracle import spectral as sp
    from numpy.lib.stride_tricks import sliding_window_view
    B, N = x.shape
    bar = np.zeros((B, N))
    for n in n_ffts:
        h, pad = n // 4, n // 2
        w = np.hanning(n + 1)[:-1]  # periodic Hann
        X = sp.stft(x, n).numpy()   # [B][bins][F]
        Y = sp.stft(y, n).numpy()
        F = X.shape[2]
        scale = 1.0 / (F * (n // 2 + 1))
        ax, ay = np.abs(X), np.abs(Y)
        norms = []
        for sig in (x, y):
            sp_ = np.pad(sig, ((0, 0), (pad, pad)), mode="reflect")
            fr = sliding_window_view(sp_, n, axis=1)[:, ::h][:, :F]  # [B][F][n]
            norms.append(np.sqrt(((fr * w) ** 2).sum(axis=2)))       # [B][F]
        ex = c * 2.0 ** -24 * np.log2(n) * norms[0][:, None, :]
        ey = c * 2.0 ** -24 * np.log2(n) * norms[1][:, None, :]
        d = np.log(ax + eps) - np.log(ay + eps)
        flip = np.abs(d) <= ex / (ax + eps) + ey / (ay + eps)
        e = scale / (ax + eps) * (np.minimum(2.0, 2.0 * ex / np.maximum(ax, 1e-300))
                                  + 2.0 * flip + 4e-6)
        S = e.sum(axis=1)  # [B][F]
        padded = np.zeros((B, N + 2 * pad))
        for f in range(F):
            padded[:, f * h:f * h + n] += S[:, f:f + 1] * w
        bar += padded[:, pad:pad + N]
        bar[:, 1:pad + 1] += padded[:, pad - 1::-1][:, :pad]            # p = pad - s
        bar[:, N - 1 - pad:N - 1] += padded[:, N + pad:][:, ::-1][:, :pad]  # p = 2(N-1) - s + pad
    return bar


def test_mrstft_full_size_elementwise(env):
    """Batch 64 x 1 s (the adjoint refinement's shape): the loss per voice
    for two batches of rendered voices within 1e-4 relative (FP32 FFTs: |X|
    is off by ~1e-7 of the frame norm, which moves log(|X| + eps) only in
    bins near silence); on seeded broadband noise, against a scaled copy
    (y = x / 2) and an independent target, the loss within 1e-5 and the
    gradient element by element within the per-sample bar of
    _mrstft_grad_bar (the gradient is ill-conditioned where a bin is near
    silence: an FP32 FFT on the CPU misses the FP64 gradient there by as
    much, at the same samples)."""
    from oracle import spectral as sp
    torch, pkg = env
    B = 64
    syn = pkg.Synth(seconds=1.0, max_batch=B)
    mr = pkg.MRSTFT(syn, B)
    x, _ = syn.render(31, 0, B)
    y, _ = syn.render(1000031, 0, B)
    loss, _ = mr(x, y, grad=False)
    syn.sync()
    ref = sp.mrstft_loss(x.cpu().numpy(), y.cpu().numpy(), per_voice=True).numpy()
    rel = np.abs(loss.cpu().numpy() - ref) / ref
    print(f"MR-STFT voices: max relative loss error {rel.max():.2e}")
    assert np.all(rel <= 1e-4)
    xn = torch.tensor(si.upstream_grad(41, (B, syn.num_samples)) * 0.3, dtype=torch.float32,
                      device="cuda")
    for yn, name in ((xn * 0.5, "scaled copy"),
                     (torch.tensor(si.upstream_grad(42, (B, syn.num_samples)) * 0.3,
                                   dtype=torch.float32, device="cuda"), "independent")):
        loss, gx = mr(xn, yn)
        syn.sync()
        xs, ys = xn.cpu().numpy().astype(np.float64), yn.cpu().numpy().astype(np.float64)
        ref_l = sp.mrstft_loss(xs, ys, per_voice=True).numpy()
        _, ref_g = sp.mrstft_loss_and_grad(xs, ys)
        g = gx.cpu().numpy().astype(np.float64)
        rel = np.abs(loss.cpu().numpy() - ref_l) / ref_l
        bar = _mrstft_grad_bar(xs, ys) + 1e-6 * np.abs(ref_g).max(axis=1, keepdims=True)
        err = np.abs(g - ref_g)
        print(f"MR-STFT noise ({name}): max relative loss error {rel.max():.2e}, "
              f"max gradient err/bar {np.max(err / bar):.3f}, median bar / max|g| "
              f"{np.median(bar / np.abs(ref_g).max(axis=1, keepdims=True)):.2e}, relative norm "
              f"{np.linalg.norm(g - ref_g) / np.linalg.norm(ref_g):.2e}")
        assert np.all(rel <= 1e-5)
        assert np.all(err <= bar)
        if name == "scaled copy":
            assert np.allclose(ref_l, 3 * np.log(2.0), rtol=1e-4)
    syn.close()
