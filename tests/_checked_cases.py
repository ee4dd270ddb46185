"""Render cases run once through the bounds-checked library (a child process
with SYNTH_CHECKED=1, which selects libsynth_checked.so) and once through the
release library: every path of the fused render -- several windows per
voice, a ragged length (scalar stores), several batches in one launch, peak
normalisation, a fractional rate, FP32 carries, caller parameters at the
corners, the allocation-free entry point -- and the adjoint, with the device
status read after each. Used by tests/test_checked_gpu.py."""
import ctypes

import numpy as np

import seeded_inputs as si


def _noalloc(pkg, torch, seconds, seed, batch_index, batch):
    L = pkg.lib()
    vp = ctypes.c_void_p
    L.synth_render_noalloc.argtypes = [ctypes.POINTER(pkg.synth_config), ctypes.c_uint64,
                                       ctypes.c_uint64, ctypes.c_int32, vp, vp, vp, vp]
    L.synth_render_noalloc.restype = ctypes.c_int
    L.synth_noalloc_status.argtypes = [vp]
    L.synth_noalloc_status.restype = ctypes.c_int
    cfg = pkg.synth_default_config()
    cfg.seconds = seconds
    n = int(round(seconds * cfg.sample_rate))
    out = torch.zeros((batch, n), device="cuda")
    pout = torch.zeros((batch, 78), device="cuda")
    st = L.synth_render_noalloc(ctypes.byref(cfg), seed, batch_index, batch, None, out.data_ptr(),
                                pout.data_ptr(), None)
    if st != pkg.SYNTH_OK:
        raise RuntimeError(f"synth_render_noalloc: {pkg.synth_status_string(st)}")
    st = L.synth_noalloc_status(None)
    if st != pkg.SYNTH_OK:
        raise RuntimeError(f"synth_noalloc_status: {pkg.synth_status_string(st)}")
    return out, pout


def run_cases(pkg, torch):
    """name -> numpy array of every output; raises if a render or its
    status check fails."""
    res = {}

    def keep(name, *ts):
        for i, t in enumerate(ts):
            res[f"{name}_{i}"] = t.cpu().numpy()

    s = pkg.Synth(seconds=4.0, max_batch=16)
    keep("four_seconds", *s.render(3, 2, 16))
    s.sync()
    s.close()
    s = pkg.Synth(seconds=0.29, max_batch=5)  # 12789 samples: scalar stores at the end
    keep("ragged", *s.render(5, 1, 5))
    s.sync()
    s.close()
    s = pkg.Synth(seconds=0.6, max_batch=12)
    keep("batches", *s.render_batches(7, 1, 4, 4, 3))
    s.sync()
    s.close()
    s = pkg.Synth(seconds=0.5, max_batch=4)
    keep("normalized", *s.render_normalized(9, 0, 4))
    s.sync()
    s.close()
    s = pkg.Synth(seconds=0.3, sample_rate=16000.0, max_batch=3)
    keep("rate_16k", *s.render(11, 0, 3))
    s.sync()
    s.close()
    s = pkg.Synth(seconds=1.0, max_batch=2, carry=pkg.SYNTH_CARRY_FP32)
    keep("fp32_carry", *s.render(13, 0, 2))
    s.sync()
    s.close()
    s = pkg.Synth(seconds=0.2, max_batch=4)
    u = torch.tensor(si.edge_params(4), dtype=torch.float32, device="cuda")
    keep("params_in", *s.render(0, 0, 4, params_in=u))
    s.sync()
    s.close()
    keep("noalloc", *_noalloc(pkg, torch, 0.3, 17, 5, 2))
    s = pkg.Synth(seconds=1.0, max_batch=8)  # the adjoint: 441 intervals, both scans chunked
    u = torch.tensor(si.uniform_params(19, 8), dtype=torch.float32, device="cuda")
    ga = torch.tensor(si.upstream_grad(20, (8, s.num_samples)), dtype=torch.float32, device="cuda")
    keep("adjoint", s.backward(19, 0, u, ga))
    s.sync()
    s.close()
    return res


def child_main(path):
    """In the bounds-checked library: the cases, then the bounds self-test."""
    import torch

    import paper_2104_12922_gb300 as pkg
    L = pkg.lib()
    assert L.synth_checked_build() == 1, "SYNTH_CHECKED=1 did not load the checked library"
    res = run_cases(pkg, torch)
    s = pkg.Synth(seconds=0.1, max_batch=1)
    before = s.render(1, 0, 1)[0].cpu().numpy()
    stat = [L.synth_selftest_bounds(s.handle, None), L.synth_sync(s.handle, None),
            L.synth_sync(s.handle, None)]
    after = s.render(1, 0, 1)[0].cpu().numpy()
    stat.append(L.synth_sync(s.handle, None))
    s.close()
    res["selftest_status"] = np.array(stat, dtype=np.int32)
    res["selftest_render_unchanged"] = np.array([np.array_equal(before, after)])
    np.savez(path, **res)
