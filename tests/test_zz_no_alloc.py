"""synth_render_noalloc -- the fused render for callers that cannot allocate
device memory -- against synth_render through the C ABI.

The allocation-free entry point keeps its scratch in a fixed device array
inside the library, shared by every call; two calls in a row (and a third
with different voices in between) must each give synth_render's audio and
parameters. This file is collected last so that a failure here comes after
every other test has run.

Both entry points run the same kernel on the same inputs with the same
fixed-order look-back carries (64-bit fixed-point phases: exact sums), so
their audio must agree bit for bit; a stale look-back record left in the
shared array by an earlier call would show up as a difference."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_12922_gb300 as pkg
    from paper_2104_12922_gb300 import build as b
    b.build()
    L = pkg.lib()
    vp = ctypes.c_void_p
    L.synth_render_noalloc.argtypes = [ctypes.POINTER(pkg.synth_config), ctypes.c_uint64,
                                       ctypes.c_uint64, ctypes.c_int32, vp, vp, vp, vp]
    L.synth_render_noalloc.restype = ctypes.c_int
    L.synth_noalloc_status.argtypes = [vp]
    L.synth_noalloc_status.restype = ctypes.c_int
    return torch, pkg, L


def _noalloc(torch, pkg, L, cfg, seed, batch_index, batch, n):
    out = torch.full((batch, n), float("nan"), device="cuda")
    pout = torch.full((batch, 78), float("nan"), device="cuda")
    st = L.synth_render_noalloc(ctypes.byref(cfg), seed, batch_index, batch, None, out.data_ptr(),
                                pout.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == pkg.SYNTH_OK, pkg.synth_status_string(st)
    torch.cuda.synchronize()
    return out, pout


def test_noalloc_matches_synth_render_on_consecutive_calls(env):
    torch, pkg, L = env
    batch, seconds = 32, 4.0
    syn = pkg.Synth(seconds=seconds, max_batch=batch)
    ref_a, ref_p = syn.render(17, 3, batch)
    other_a, other_p = syn.render(5, 9, 8)
    syn.sync()
    cfg = pkg.synth_default_config()
    cfg.seconds = seconds
    n = syn.num_samples
    for seed, bi, b, ra, rp in [(17, 3, batch, ref_a, ref_p), (17, 3, batch, ref_a, ref_p),
                                (5, 9, 8, other_a, other_p), (17, 3, batch, ref_a, ref_p)]:
        a, p = _noalloc(torch, pkg, L, cfg, seed, bi, b, n)
        assert L.synth_noalloc_status(None) == pkg.SYNTH_OK
        assert torch.equal(p, rp)
        assert torch.equal(a, ra), float((a - ra).abs().max())
    syn.close()


def test_noalloc_rejects_batches_beyond_its_scratch(env):
    torch, pkg, L = env
    cfg = pkg.synth_default_config()
    out = torch.empty(1, device="cuda")
    # 4 s voices: 256 + 48 * 7 * batch bytes must fit in 256 KiB (batch <= 779)
    st = L.synth_render_noalloc(ctypes.byref(cfg), 0, 0, 780, None, out.data_ptr(), None, None)
    assert st == pkg.SYNTH_ERR_ARG
    assert L.synth_render_noalloc(None, 0, 0, 1, None, out.data_ptr(), None, None) == pkg.SYNTH_ERR_ARG
    assert L.synth_render_noalloc(ctypes.byref(cfg), 0, 0, 0, None, None, None, None) == pkg.SYNTH_OK


def test_noalloc_at_a_fractional_rate(env):
    """16 kHz at the 441 Hz control rate (R = 16000/441): the handle-free
    entry takes the same general-R kernel as synth_render."""
    torch, pkg, L = env
    batch, seconds = 8, 1.0
    syn = pkg.Synth(seconds=seconds, max_batch=batch, sample_rate=16000.0)
    ref_a, ref_p = syn.render(2, 6, batch)
    syn.sync()
    cfg = pkg.synth_default_config()
    cfg.seconds, cfg.sample_rate = seconds, 16000.0
    a, p = _noalloc(torch, pkg, L, cfg, 2, 6, batch, syn.num_samples)
    assert L.synth_noalloc_status(None) == pkg.SYNTH_OK
    assert torch.equal(p, ref_p)
    assert torch.equal(a, ref_a), float((a - ref_a).abs().max())
    syn.close()
