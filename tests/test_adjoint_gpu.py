"""GPU adjoint (synth_render_backward) against the oracle's forward-mode
(dual-number) gradient and FP64 central differences of the oracle render.

Workload: batch 2 x 0.1 s voices at 44.1 kHz (4410 samples: a ragged last
control interval), seeded parameters and a seeded Gaussian upstream gradient.
"""
import numpy as np
import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu

SECONDS = 0.1


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_12922_gb300 import build as b
    b.build()
    return torch


def _voice_params(oracle_mod, seed, count):
    """Drawn parameters moved off the boundaries u = 0 and u = 1 (where the
    range map's derivative convention and clamps sit)."""
    u = np.stack([oracle_mod.draw_params(seed, g) for g in range(count)])
    return np.clip(u, 0.02, 0.98).astype(np.float32).astype(np.float64)


def _gpu_grad(torch, syn, u, w, seed, batch_index):
    pin = torch.tensor(u, dtype=torch.float32, device="cuda")
    gout = torch.tensor(w, dtype=torch.float32, device="cuda")
    g = syn.backward(seed, batch_index, pin, gout)
    syn.sync()
    return g.cpu().numpy().astype(np.float64)


def _fd(oracle_mod, cfg, u, seed, g, w, p, h):
    up, um = u.copy(), u.copy()
    up[p] += h
    um[p] -= h
    return float(np.dot(w, oracle_mod.render_voice(cfg, up, seed, g) -
                        oracle_mod.render_voice(cfg, um, seed, g))) / (2 * h)


@pytest.mark.parametrize("seed", [3, 11])
def test_adjoint_matches_oracle_gradient(torch_cuda, oracle_mod, seed):
    import paper_2104_12922_gb300 as pkg
    torch = torch_cuda
    B = 2
    syn = pkg.Synth(seconds=SECONDS, max_batch=B)
    u = _voice_params(oracle_mod, seed, B)
    N = syn.num_samples
    w = si.upstream_grad(seed, (B, N))
    got = _gpu_grad(torch, syn, u, w, seed, 0)
    cfg = oracle_mod.default_config(seconds=SECONDS)
    for v in range(B):
        ref = oracle_mod.render_vjp(cfg, u[v], seed, v, w[v])
        scale = np.max(np.abs(ref))
        err = np.abs(got[v] - ref)
        assert np.all(np.isfinite(got[v]))
        assert np.max(err) <= 2e-3 * scale + 1e-6, (v, np.argmax(err), got[v][np.argmax(err)],
                                                     ref[np.argmax(err)])
    syn.close()


def test_adjoint_matches_fp64_finite_differences(torch_cuda, oracle_mod):
    """Central differences (h = 1e-6 in u) of the FP64 oracle render, on the
    parameters where the render is smooth at that scale."""
    import paper_2104_12922_gb300 as pkg
    torch = torch_cuda
    seed = 5
    syn = pkg.Synth(seconds=SECONDS, max_batch=1)
    u = _voice_params(oracle_mod, seed, 1)
    w = si.upstream_grad(seed + 1, (1, syn.num_samples))
    got = _gpu_grad(torch, syn, u, w, seed, 0)[0]
    cfg = oracle_mod.default_config(seconds=SECONDS)
    checked = 0
    for p in range(78):
        a = _fd(oracle_mod, cfg, u[0], seed, 0, w[0], p, 1e-6)
        b = _fd(oracle_mod, cfg, u[0], seed, 0, w[0], p, 2.5e-7)
        if abs(a - b) > 1e-4 * (abs(a) + 1e-3):
            continue  # a kink within h of u: not smooth at this scale
        checked += 1
        assert abs(got[p] - a) <= 2e-3 * (abs(a) + 1.0), (p, got[p], a)
    assert checked >= 60
    syn.close()


def test_autograd_function_matches_backward(torch_cuda):
    import paper_2104_12922_gb300 as pkg
    torch = torch_cuda
    syn = pkg.Synth(seconds=SECONDS, max_batch=3)
    u = torch.tensor(si.uniform_params(7, 3), dtype=torch.float32, device="cuda").clamp(0.02, 0.98)
    u.requires_grad_(True)
    audio = pkg.render_autograd(syn, 4, 2, u)
    w = torch.tensor(si.upstream_grad(8, tuple(audio.shape)), dtype=torch.float32, device="cuda")
    (audio * w).sum().backward()
    direct = syn.backward(4, 2, u.detach().contiguous(), w)
    syn.sync()
    assert torch.allclose(u.grad, direct, rtol=1e-6, atol=1e-6)
    syn.close()


def test_adjoint_one_second_matches_oracle_gradient(torch_cuda, oracle_mod):
    """2 x 1 s voices (K = 441 control intervals): both chunked reverse scans
    of the adjoint (over intervals and over control points, 256 per chunk)
    carry across a chunk boundary. Element-wise against the oracle's
    dual-number gradient at the same 2e-3 x max|g| bar as the 0.1 s cases."""
    import paper_2104_12922_gb300 as pkg
    torch = torch_cuda
    B, seconds, seed = 2, 1.0, 19
    syn = pkg.Synth(seconds=seconds, max_batch=B)
    u = _voice_params(oracle_mod, seed, B)
    w = si.upstream_grad(seed, (B, syn.num_samples))
    got = _gpu_grad(torch, syn, u, w, seed, 0)
    cfg = oracle_mod.default_config(seconds=seconds)
    for v in range(B):
        ref = oracle_mod.render_vjp(cfg, u[v], seed, v, w[v])
        scale = np.max(np.abs(ref))
        err = np.abs(got[v] - ref)
        print(f"voice {v}: max |g| {scale:.3e}, max err {err.max():.3e} "
              f"({err.max() / scale:.2e} of max|g|)")
        assert np.all(np.isfinite(got[v]))
        assert np.max(err) <= 2e-3 * scale + 1e-6, (v, np.argmax(err))
    syn.close()


def test_adjoint_and_distance_are_bitwise_reproducible(torch_cuda):
    """The adjoint's per-voice sums and the MR-STFT distance's per-voice
    losses are added in a fixed order (no floating-point atomics), so
    repeated calls on the refinement's shape (batch 64 x 1 s) give
    bit-identical gradients and losses."""
    import paper_2104_12922_gb300 as pkg
    torch = torch_cuda
    B = 64
    syn = pkg.Synth(seconds=1.0, max_batch=B)
    u = torch.tensor(si.uniform_params(23, B), dtype=torch.float32, device="cuda")
    audio, _ = syn.render(4, 0, B, params_in=u)
    target, _ = syn.render(1_000_004, 0, B)
    mr = pkg.MRSTFT(syn, B)
    runs = []
    for _ in range(3):
        loss, gx = mr(audio, target)
        gu = syn.backward(4, 0, u, gx)
        runs.append((loss.clone(), gx.clone(), gu.clone()))
    syn.sync()
    for loss, gx, gu in runs[1:]:
        assert torch.equal(loss, runs[0][0])
        assert torch.equal(gx, runs[0][1])
        assert torch.equal(gu, runs[0][2])
    assert torch.isfinite(runs[0][2]).all()
    syn.close()
