"""Corpus similarity by MMD (paper Sec. 5, the MMD equation) on the GPU
against the FP64 oracle (oracle/mmd.py), through the C ABI.

Embeddings are the library's log-mel feature vectors (bf16), shared by both
sides. Bars: the l1 distance of two bf16 vectors is a sum of dim exact FP32
differences |a - b|, accumulated in FP32; the partial sums grow to d, so the
accumulated rounding has a standard deviation of about 2^-24 d sqrt(dim) / 3
and the bar 7 2^-24 sqrt(dim) d (a margin of 3 over 7 sigma). The MMD
statistic combines 4 n^2 distances with weights 1 / n^2, so its bar is that
relative bar times (2 S_xy + S_xx + S_yy) / n^2 (the statistic itself can be
much smaller than its terms: within-corpus MMDs cancel)."""
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


def _rel_bar(dim):
    return 7.0 * 2.0 ** -24 * np.sqrt(dim)


def _features(torch, pkg, seconds, n_voice, n_fm):
    syn = pkg.Synth(seconds=seconds, max_batch=128)
    model = pkg.ProposalModel(syn, max_batch=128, seed=0)
    parts = []
    for kind, count in (("voice", n_voice), ("fm", n_fm)):
        done = 0
        while done < count:
            b = min(128, count - done)
            if kind == "voice":
                audio, _ = syn.render(3, done // 128, b)
            else:
                audio, _ = syn.fm_render(3, done // 128, b)
            parts.append(model.features(audio))
            done += b
    syn.sync()
    feats = torch.cat(parts)
    return syn, model, feats


def test_l1_distances_and_mmd_match_oracle(env):
    """200 sounds (100 Voice, 100 FM voices) of 4 s: 44160-value embeddings,
    a 200 x 200 distance matrix (one full and one ragged tile row), and MMD
    trials within each corpus and between them (n = 40)."""
    from oracle import mmd as om
    torch, pkg = env
    syn, model, feats = _features(torch, pkg, 4.0, 100, 100)
    m, dim = feats.shape
    assert dim == 44160
    dist = pkg.l1_distances(syn, feats)
    labels = np.concatenate([si.mmd_labels(7, 4, [100, 100], pair, 40)
                             for pair in ((0, 0), (1, 1), (0, 1))])
    lab = torch.tensor(labels, device="cuda")
    got_mmd = pkg.mmd_trials(syn, dist, lab).cpu().numpy()
    again = pkg.mmd_trials(syn, dist, lab).cpu().numpy()
    syn.sync()
    e = feats.float().cpu().numpy().astype(np.float64)
    ref = om.l1_distances(e)
    d = dist.cpu().numpy().astype(np.float64)
    assert np.all(np.diag(d) == 0) and np.array_equal(d, d.T)
    rel = np.abs(d - ref) / np.maximum(ref, 1e-300)
    np.fill_diagonal(rel, 0)
    print(f"l1 distances: max relative error {rel.max():.2e} (bar {_rel_bar(dim):.2e}), "
          f"median distance {np.median(ref):.1f}")
    assert np.all(rel <= _rel_bar(dim))
    ref_mmd = om.mmd_trials(ref, labels)
    for t in range(len(labels)):
        x, y = np.where(labels[t] == 0)[0], np.where(labels[t] == 1)[0]
        n = len(x)
        scale = (2 * ref[np.ix_(x, y)].sum() + ref[np.ix_(x, x)].sum()
                 + ref[np.ix_(y, y)].sum()) / (n * n)
        assert abs(got_mmd[t] - ref_mmd[t]) <= _rel_bar(dim) * scale, t
    # the trials kernel alone: the oracle's statistic on the GPU's distances;
    # the kernel adds each row in FP32 (m terms: at most m 2^-24 of the
    # row's sum) and the rows in FP64
    on_gpu_d = om.mmd_trials(d, labels)
    for t in range(len(labels)):
        x, y = np.where(labels[t] == 0)[0], np.where(labels[t] == 1)[0]
        n = len(x)
        scale = (2 * d[np.ix_(x, y)].sum() + d[np.ix_(x, x)].sum() + d[np.ix_(y, y)].sum()) / (n * n)
        assert abs(got_mmd[t] - on_gpu_d[t]) <= m * 2.0 ** -24 * scale, t
    assert np.array_equal(got_mmd, again)
    within_v, within_fm, between = got_mmd[:4].mean(), got_mmd[4:8].mean(), got_mmd[8:].mean()
    print(f"MMD (log-mel l1, n = 40): Voice/Voice {within_v:.1f}, FM/FM {within_fm:.1f}, "
          f"Voice/FM {between:.1f}")
    assert between > max(within_v, within_fm)
    model.close()
    syn.close()


def test_l1_distances_ragged_and_degenerate(env):
    """A dimension that is not a multiple of the 32-value chunk (1000, row
    stride 1000) over 300 rows (3 tile rows, the last ragged); a pool of
    two point masses (10 copies of a, 10 of b) whose MMD is 2 d(a, b); one
    sound; empty sets."""
    from oracle import mmd as om
    torch, pkg = env
    syn = pkg.Synth(seconds=0.01, max_batch=1)
    g = torch.Generator(device="cuda").manual_seed(3)
    emb = (torch.randn(300, 1000, device="cuda", generator=g) * 0.5).to(torch.bfloat16)
    dist = pkg.l1_distances(syn, emb)
    syn.sync()
    ref = om.l1_distances(emb.float().cpu().numpy().astype(np.float64))
    d = dist.cpu().numpy().astype(np.float64)
    rel = np.abs(d - ref) / np.maximum(ref, 1e-300)
    np.fill_diagonal(rel, 0)
    assert np.all(rel <= _rel_bar(1000)) and np.all(np.diag(d) == 0)
    # point masses
    a, b = emb[0], emb[1]
    pool = torch.stack([a] * 10 + [b] * 10).contiguous()
    dp = pkg.l1_distances(syn, pool)
    lab = torch.tensor(np.array([[0] * 10 + [1] * 10, [0] * 10 + [-1] * 10], dtype=np.int8),
                       device="cuda")
    mm = pkg.mmd_trials(syn, dp, lab).cpu().numpy()
    one = pkg.l1_distances(syn, emb[:1].contiguous()).cpu().numpy()
    syn.sync()
    dab = float(dp[0, 10])
    assert float(dp[0, 1]) == 0.0 and dab == pytest.approx(ref[0, 1], rel=_rel_bar(1000))
    assert mm[0] == pytest.approx(2.0 * dab, rel=20 * 2.0 ** -24)  # FP32 row sums of 20
    assert mm[1] == 0.0  # Y empty
    assert one.shape == (1, 1) and one[0, 0] == 0.0
    syn.close()
