"""Per-voice peak normalisation and silence rejection (synth_render_normalized)
against the FP64 oracle's render followed by its peak_normalize, and against
synth_render's output divided by its own peak. 0.5 s voices (N % 4 != 0)
take the scalar path of the scaling items, 4 s voices the 16-byte one; both
end in a ragged chunk.

Error bar: the render is within 2e-4 of the oracle (max-abs), so the peaks
differ by at most 2e-4 and a normalised sample x/p by at most
(2e-4 + 2e-4 |x|/p) / p <= 4e-4 / p."""
import numpy as np
import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu

TAU = 1e-3


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_12922_gb300 as pkg
    from paper_2104_12922_gb300 import build as b
    b.build()
    return torch, pkg


def test_normalized_matches_oracle(env, oracle_mod):
    torch, pkg = env
    seconds, batch = 0.5, 12
    syn = pkg.Synth(seconds=seconds, max_batch=batch)
    # drawn voices, plus voices whose mixer levels are all 0 (silent)
    u = si.uniform_params(11, batch)
    u[-3:, si.MIX:si.MIX + 3] = 0.0
    u = u.astype(np.float32).astype(np.float64)
    pin = torch.tensor(u, dtype=torch.float32, device="cuda")
    a, p, peak, silent = syn.render_normalized(4, 2, batch, threshold=TAU, params_in=pin)
    syn.sync()
    cfg = oracle_mod.default_config(seconds=seconds)
    ref_a, _ = oracle_mod.render_batch(cfg, 4, 2, batch, u_in=u)
    ref_n, ref_peak, ref_silent = oracle_mod.peak_normalize(ref_a, TAU)
    peak, silent, a = peak.cpu().numpy(), silent.cpu().numpy(), a.cpu().numpy()
    assert np.max(np.abs(peak - ref_peak)) <= 2e-4
    clear = np.abs(ref_peak - TAU) > 2e-4  # flags compared away from the threshold tie
    assert np.array_equal(silent[clear].astype(bool), ref_silent[clear])
    assert ref_silent[-3:].all() and silent[-3:].all()
    for v in range(batch):
        if ref_silent[v]:
            assert np.max(np.abs(a[v] - ref_a[v])) <= 2e-4  # left as rendered
        else:
            err = np.max(np.abs(a[v] - ref_n[v]))
            assert err <= 4e-4 / ref_peak[v] + 1e-6, (v, err, ref_peak[v])
            assert np.max(np.abs(a[v])) == pytest.approx(1.0, abs=1e-6)
    syn.close()


def test_normalized_is_render_divided_by_its_peak(env):
    torch, pkg = env
    syn = pkg.Synth(seconds=4.0, max_batch=32)
    raw, params = syn.render(9, 3, 32)
    # successive launches of both kinds: the work items' flags are tagged
    # with the launch, so none may see a flag of an earlier one
    syn.render_normalized(8, 3, 32, threshold=TAU)
    syn.render(9, 2, 32)
    a, p, peak, silent = syn.render_normalized(9, 3, 32, threshold=TAU)
    syn.sync()
    assert torch.equal(p, params)
    want_peak = raw.abs().amax(dim=1)
    assert torch.equal(peak, want_peak)
    loud = want_peak >= TAU
    assert torch.equal(silent.bool(), ~loud)
    want = torch.where(loud[:, None], raw * (1.0 / want_peak)[:, None], raw)
    assert torch.equal(a, want)
    syn.close()


def test_normalized_argument_errors(env):
    torch, pkg = env
    syn = pkg.Synth(seconds=0.1, max_batch=2)
    out = torch.empty((2, syn.num_samples), device="cuda")
    L = pkg.lib()
    assert L.synth_render_normalized(syn.handle, 0, 0, 3, None, out.data_ptr(), None, 1e-3, None,
                                     None, None) == pkg.SYNTH_ERR_ARG
    assert L.synth_render_normalized(syn.handle, 0, 0, 2, None, out.data_ptr(), None, -1.0, None,
                                     None, None) == pkg.SYNTH_ERR_ARG
    assert L.synth_render_normalized(syn.handle, 0, 0, 0, None, None, None, 1e-3, None, None,
                                     None) == pkg.SYNTH_OK
    syn.close()


def test_normalized_full_size_sampled(env, oracle_mod):
    """The normalised throughput workload: batch 128 x 4 s drawn voices, seed =
    batch index = 21, threshold 1e-3; peaks and flags of all voices are
    checked through the unnormalised render, sampled voices against the
    oracle's render + peak_normalize."""
    torch, pkg = env
    syn = pkg.Synth(seconds=4.0, max_batch=128)
    a, p, peak, silent = syn.render_normalized(21, 21, 128, threshold=TAU)
    raw, _ = syn.render(21, 21, 128)
    syn.sync()
    raw_peak = raw.abs().amax(dim=1)
    assert torch.equal(peak, raw_peak)
    assert torch.equal(silent.bool(), ~((raw_peak >= TAU) & (raw_peak > 0)))
    rows = si.sample_voices(21, 128, 6)
    cfg = oracle_mod.default_config(seconds=4.0)
    ref_a, ref_p = oracle_mod.render_batch(cfg, 21, 21, 128, voices=rows)
    ref_n, ref_peak, ref_silent = oracle_mod.peak_normalize(ref_a[rows], TAU)
    assert np.array_equal(p.cpu().numpy()[rows], ref_p[rows])
    peak_r = peak.cpu().numpy()[rows]
    a_r = a.cpu().numpy()[rows]
    assert np.max(np.abs(peak_r - ref_peak)) <= 2e-4
    for i in range(len(rows)):
        if ref_silent[i]:
            assert np.max(np.abs(a_r[i] - ref_a[rows[i]])) <= 2e-4
        else:
            err = np.max(np.abs(a_r[i] - ref_n[i]))
            assert err <= 4e-4 / ref_peak[i] + 1e-6, (int(rows[i]), err, ref_peak[i])
    syn.close()
