"""Streaming synth1B1 generator (synth_stream_features): voices of a split
rendered and turned into log-mel features chunk by chunk, with no audio
materialised beyond one chunk.

Checks: the parameters are the oracle's draw for exactly the split's voice
indices (bit-exact, Philox); the features equal those of the same voice
rendered alone and passed through synth_model_features (bit-exact: a voice's
render and features do not depend on the chunk it is in); on bands within
30 dB of the voice's loudest band the features are within 0.06 (log units)
of the oracle's log-mel of the oracle's own rendering (the render's 2e-4
audio bar and the bf16 output rounding, 0.0234, both fit well inside)."""
import numpy as np
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


def test_stream_train_range_across_a_test_block(env, oracle_mod):
    from oracle import spectral as sp
    torch, pkg = env
    seed, seconds = 5, 0.5
    syn = pkg.Synth(seconds=seconds, max_batch=8)
    model = pkg.ProposalModel(syn, max_batch=8, seed=0)
    first, count = 9210, 12  # train voices 9210..9215, then 10240..10245
    feats, params = model.stream_features(seed, pkg.SPLIT_TRAIN, first, count, chunk=5)
    syn.sync()
    gs = [g for g in range(9000, 11000) if not pkg.synth_is_test(g)][first - 9000:first - 9000 + count]
    assert gs[:6] == list(range(9210, 9216)) and gs[6:] == list(range(10240, 10246))
    cfg = oracle_mod.default_config(seconds=seconds)
    feats_np, params_np = feats.float().cpu().numpy(), params.cpu().numpy()
    for i, g in enumerate(gs):
        ref_a, ref_p = oracle_mod.render_batch(cfg, seed, g, 1)
        assert np.array_equal(params_np[i], ref_p[0]), g
        a1, _ = syn.render(seed, g, 1)
        f1 = model.features(a1)
        assert torch.equal(f1[0], feats[i]), g
        ref = sp.log_mel(ref_a).numpy()[0]
        got = feats_np[i].reshape(-1, 128) * pkg.FEATURE_SCALE + pkg.FEATURE_SHIFT
        loud = ref > ref.max() - np.log(1e3)
        assert np.max(np.abs(got - ref)[loud]) < 0.06, g
    model.close()
    syn.close()


def test_stream_chunking_and_test_split(env):
    torch, pkg = env
    syn = pkg.Synth(seconds=0.25, max_batch=16)
    model = pkg.ProposalModel(syn, max_batch=16, seed=0)
    f0, p0 = model.stream_features(3, pkg.SPLIT_TEST, 1020, 9)  # test voices 10236..10239, 19456..
    f1, p1 = model.stream_features(3, pkg.SPLIT_TEST, 1020, 9, chunk=2)
    syn.sync()
    assert torch.equal(f0, f1) and torch.equal(p0, p1)
    # voice g of the test split through the plain render path of one voice
    g = pkg.synth_split_voice(pkg.SPLIT_TEST, 1024)
    assert g == 19456
    a, p = syn.render(3, g, 1)
    assert torch.equal(p[0], p0[4]) and torch.equal(model.features(a)[0], f0[4])
    model.close()
    syn.close()


def test_stream_argument_errors(env):
    torch, pkg = env
    syn = pkg.Synth(seconds=0.25, max_batch=8)
    model = pkg.ProposalModel(syn, max_batch=8, seed=0)
    f = torch.empty((2, model.feature_dim), dtype=torch.bfloat16, device="cuda")
    L = pkg.lib()
    assert L.synth_stream_features(model.handle, 0, 3, 0, 2, 0, f.data_ptr(), None, None) == pkg.SYNTH_ERR_ARG
    assert L.synth_stream_features(model.handle, 0, 1, 0, 2, 9, f.data_ptr(), None, None) == pkg.SYNTH_ERR_ARG
    assert L.synth_stream_features(model.handle, 0, 1, 0, -1, 0, f.data_ptr(), None, None) == pkg.SYNTH_ERR_ARG
    assert L.synth_stream_features(model.handle, 0, 1, 0, 2, 0, None, None, None) == pkg.SYNTH_ERR_ARG
    assert L.synth_stream_features(model.handle, 0, 1, 0, 0, 0, None, None, None) == pkg.SYNTH_OK
    assert L.synth_stream_features(model.handle, 0, 1, 0, 2, 0, f.data_ptr(), None, None) == pkg.SYNTH_OK
    syn.sync()
    model.close()
    syn.close()
