"""Spectral parts of the oracle -- TEST INFRASTRUCTURE (plain PyTorch CPU ops, FP64).

* Multi-resolution log-magnitude STFT distance (Sec. 4, Table 2 "multi-scale
  spectrogram" of the paper, after Engel et al. DDSP): periodic Hann window,
  hop n_fft/4, centred frames (reflect padding by n_fft/2),
  L = sum over n_fft of mean over (bins, frames) |log(|X| + eps) - log(|Y| + eps)|.
* Log-mel features for the learned proposal: power spectrum |X|^2 (n_fft
  2048, hop 512, centred), 128 triangular mel bands on the Slaney mel scale
  (linear below 1 kHz, logarithmic above) with area normalisation,
  log(mel + 1e-6).
* The proposal MLP (ReLU hidden layers, sigmoid output) and its MSE loss,
  forward and backward via autograd.

torch.stft (an FFT) serves as the DFT primitive.
"""
from __future__ import annotations

import math

import numpy as np
import torch

MR_EPS = 1e-7
MEL_EPS = 1e-6


def _as64(x):
    return torch.as_tensor(np.asarray(x), dtype=torch.float64) if not torch.is_tensor(x) else x.double()


def stft(x, n_fft: int):
    """Complex STFT [batch][bins][frames] of real signals [batch][N]."""
    x = _as64(x)
    win = torch.hann_window(n_fft, periodic=True, dtype=torch.float64)
    return torch.stft(x, n_fft, hop_length=n_fft // 4, win_length=n_fft, window=win, center=True,
                      pad_mode="reflect", return_complex=True)


def mrstft_loss(x, y, n_ffts=(512, 1024, 2048), eps: float = MR_EPS, per_voice: bool = False):
    x = _as64(x)
    y = _as64(y)
    total = 0.0
    for n in n_ffts:
        lx = torch.log(stft(x, n).abs() + eps)
        ly = torch.log(stft(y, n).abs() + eps)
        d = (lx - ly).abs()
        total = total + (d.mean(dim=(1, 2)) if per_voice else d.mean())
    return total


def mrstft_loss_and_grad(x, y, n_ffts=(512, 1024, 2048), eps: float = MR_EPS):
    """Loss (mean over the batch of per-voice losses summed over voices, i.e.
    the sum of per-voice losses) and d loss / d x."""
    xt = _as64(x).clone().requires_grad_(True)
    loss = mrstft_loss(xt, y, n_ffts, eps, per_voice=True).sum()
    loss.backward()
    return float(loss.detach()), xt.grad.numpy()


def hz_to_mel(f):
    """Slaney mel scale: 3 f / 200 below 1 kHz, 15 + 27 ln(f/1000) / ln 6.4 above."""
    f = np.asarray(f, dtype=np.float64)
    lin = 3.0 * f / 200.0
    log = 15.0 + 27.0 * np.log(np.maximum(f, 1e-12) / 1000.0) / math.log(6.4)
    return np.where(f < 1000.0, lin, log)


def mel_to_hz(m):
    m = np.asarray(m, dtype=np.float64)
    lin = 200.0 * m / 3.0
    log = 1000.0 * np.exp((m - 15.0) * math.log(6.4) / 27.0)
    return np.where(m < 15.0, lin, log)


def mel_filterbank(n_fft: int = 2048, n_mels: int = 128, sample_rate: float = 44100.0) -> np.ndarray:
    """[n_mels][n_fft/2 + 1]: triangle i rises from edge i to edge i+1 and
    falls to edge i+2 (edges equally spaced in mel from 0 to SR/2), scaled by
    2 / (f_{i+2} - f_i) so each triangle has unit area in Hz."""
    bins = np.arange(n_fft // 2 + 1) * sample_rate / n_fft
    edges = mel_to_hz(np.linspace(hz_to_mel(0.0), hz_to_mel(sample_rate / 2.0), n_mels + 2))
    fb = np.zeros((n_mels, len(bins)))
    for i in range(n_mels):
        lo, c, hi = edges[i], edges[i + 1], edges[i + 2]
        up = (bins - lo) / (c - lo)
        down = (hi - bins) / (hi - c)
        fb[i] = np.maximum(0.0, np.minimum(up, down)) * (2.0 / (hi - lo))
    return fb


def log_mel(audio, n_fft: int = 2048, n_mels: int = 128, sample_rate: float = 44100.0):
    """[batch][frames][n_mels] = log(mel filterbank @ |STFT|^2 + 1e-6)."""
    power = stft(audio, n_fft).abs() ** 2                      # [B][bins][frames]
    fb = torch.as_tensor(mel_filterbank(n_fft, n_mels, sample_rate))
    mel = torch.einsum("mk,bkf->bfm", fb, power)
    return torch.log(mel + MEL_EPS)


def mlp_forward(x, weights, biases):
    """ReLU hidden layers, sigmoid output. weights[l]: [out][in]."""
    h = _as64(x)
    for l, (w, b) in enumerate(zip(weights, biases)):
        z = h @ _as64(w).T + _as64(b)
        h = torch.sigmoid(z) if l == len(weights) - 1 else torch.relu(z)
    return h


def mlp_loss_and_grads(x, target, weights, biases):
    """MSE(mean over all outputs) of the MLP output against target, and its
    gradients with respect to every weight and bias."""
    ws = [_as64(w).clone().requires_grad_(True) for w in weights]
    bs = [_as64(b).clone().requires_grad_(True) for b in biases]
    y = mlp_forward(x, ws, bs)
    loss = ((y - _as64(target)) ** 2).mean()
    loss.backward()
    return float(loss.detach()), [w.grad.numpy() for w in ws], [b.grad.numpy() for b in bs]


def mlp_trace(x, target, weights, biases, masks=None):
    """The same network and MSE loss with every intermediate kept, the
    backward written out by the chain rule (FP64):
      Z_l = H_(l-1) W_l^T + b_l, H_l = relu(Z_l) (hidden), Y = sigmoid(Z_L);
      dZ_L = 2 (Y - target) / (B P) * Y (1 - Y);
      dW_l = dZ_l^T H_(l-1), db_l = sum over the batch of dZ_l;
      dH_(l-1) = dZ_l W_l, dZ_(l-1) = dH_(l-1) * [Z_(l-1) > 0].
    ``masks`` (optional, one boolean array per hidden layer) replaces the
    ReLU decisions [Z_l > 0] of the backward by given ones: at Z = 0 the
    derivative is a choice, and near it a rounding of Z may take it either
    way. Returns a dict of lists indexed by layer: Z, H (H[l] is the input of
    layer l, H[0] = x), dZ, dH (dH[l] is the gradient of H[l], l >= 1), gW,
    gb, and Y and the loss."""
    x = _as64(x).numpy()
    t = _as64(target).numpy()
    ws = [_as64(w).numpy() for w in weights]
    bs = [_as64(b).numpy() for b in biases]
    L = len(ws)
    H, Z = [x], []
    for l in range(L):
        z = H[l] @ ws[l].T + bs[l]
        Z.append(z)
        if l < L - 1:
            H.append(np.maximum(z, 0.0))
    Y = 1.0 / (1.0 + np.exp(-Z[-1]))
    B, P = Y.shape
    loss = float(np.mean((Y - t) ** 2))
    dZ = [None] * L
    dH = [None] * L
    gW = [None] * L
    gb = [None] * L
    dZ[L - 1] = 2.0 * (Y - t) / (B * P) * Y * (1.0 - Y)
    for l in range(L - 1, -1, -1):
        gW[l] = dZ[l].T @ H[l]
        gb[l] = dZ[l].sum(axis=0)
        if l > 0:
            dH[l] = dZ[l] @ ws[l]
            mask = (Z[l - 1] > 0.0) if masks is None else masks[l - 1]
            dZ[l - 1] = dH[l] * mask
    return {"Z": Z, "H": H, "Y": Y, "dZ": dZ, "dH": dH, "gW": gW, "gb": gb, "loss": loss}
