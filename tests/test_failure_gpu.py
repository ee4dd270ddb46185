"""Failure detection on the device without a fault: a bounded wait that runs
out. synth_selftest_wait_timeout runs the fused render's look-back wait
against a window record that nothing publishes; the wait gives up, the
handle records a timeout, synth_sync reports SYNTH_ERR_TIMEOUT once and
clears it, and the handle keeps rendering bit-exactly."""
import time

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
    return torch, pkg


def test_bounded_wait_times_out_and_handle_stays_usable(env):
    torch, pkg = env
    L = pkg.lib()
    syn = pkg.Synth(seconds=0.5, max_batch=8)
    ref, ref_p = syn.render(3, 2, 8)
    syn.sync()
    ref = ref.clone()
    t0 = time.perf_counter()
    assert L.synth_selftest_wait_timeout(syn.handle, None) == pkg.SYNTH_OK
    waited = time.perf_counter() - t0
    assert waited < 10.0, f"the bounded wait took {waited:.1f} s"
    assert L.synth_sync(syn.handle, None) == pkg.SYNTH_ERR_TIMEOUT
    assert L.synth_sync(syn.handle, None) == pkg.SYNTH_OK  # reported once, then cleared
    # the context and the handle are intact: the same render, bit for bit
    again, again_p = syn.render(3, 2, 8)
    syn.sync()
    assert torch.equal(again, ref) and torch.equal(again_p, ref_p)
    syn.close()
