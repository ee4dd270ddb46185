"""GPU parity of the fused and plain renders against the FP64 oracle.

Bar: parameter draws bit-exact; audio max-abs error <= 2e-4 per
sample over 4 s voices. Inputs are the synth1B1 workload itself: parameters
drawn from (seed, global voice index), 44.1 kHz, 4 s.
"""
import numpy as np
import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu

TOL = 2e-4


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_12922_gb300 import build as b
    b.build()
    return torch


@pytest.fixture(scope="module")
def synth4(torch_cuda):
    import paper_2104_12922_gb300 as pkg
    s = pkg.Synth(seconds=4.0, max_batch=128)
    yield s
    s.close()


def _oracle_batch(oracle_mod, seconds, seed, batch_index, batch, u_in=None, voices=None, nebula=None):
    cfg = oracle_mod.default_config(seconds=seconds, nebula=nebula)
    return oracle_mod.render_batch(cfg, seed, batch_index, batch, u_in=u_in, voices=voices)


def _check(audio, params, ref_audio, ref_params, rows=None, tol=TOL):
    a = audio.cpu().numpy()
    p = params.cpu().numpy()
    if rows is not None:
        a, p, ref_audio, ref_params = a[rows], p[rows], ref_audio[rows], ref_params[rows]
    assert np.array_equal(p, ref_params), "parameter draw must be bit-exact"
    assert np.all(np.isfinite(a))
    err = float(np.max(np.abs(a - ref_audio)))
    assert err <= tol, f"max-abs error {err:.3e}"
    return err


@pytest.mark.parametrize("plain", [False, True])
def test_batch16_4s_matches_oracle(synth4, oracle_mod, plain):
    """Plain Voice, batch 16 x 4 s, seed 0, batch index 0."""
    audio, params = synth4.render(0, 0, 16, plain=plain)
    synth4.sync()
    ref_a, ref_p = _oracle_batch(oracle_mod, 4.0, 0, 0, 16)
    _check(audio, params, ref_a, ref_p)


@pytest.mark.parametrize("batch_index", [1, 1023])
def test_batch128_sampled_voices(synth4, oracle_mod, batch_index):
    """Full-size batch 128 x 4 s, seed = batch index, as the throughput run
    launches it; a sample of voices is checked against the oracle."""
    audio, params = synth4.render(batch_index, batch_index, 128)
    synth4.sync()
    rows = si.sample_voices(batch_index, 128, 8)
    ref_a, ref_p = _oracle_batch(oracle_mod, 4.0, batch_index, batch_index, 128, voices=rows)
    _check(audio, params, ref_a, ref_p, rows=rows)
    assert np.all(np.abs(audio.cpu().numpy()) <= 1.0)


def test_fused_equals_plain(synth4):
    """The two forms share the control-rate arithmetic but not the parameter
    map (float-float vs FP64) nor the running phase sums (fixed point vs
    FP64), so an interval's starting phase may differ in its last float bit;
    phase0 + local phase (|local| < 64 cycles) then rounds to a neighbouring
    float, 2^-18 cycles apart: 2 pi 2^-18 = 2.4e-5 per oscillator at unit
    gain. The bar is twice that."""
    a1, p1 = synth4.render(3, 2, 64)
    a2, p2 = synth4.render(3, 2, 64, plain=True)
    synth4.sync()
    assert np.array_equal(p1.cpu().numpy(), p2.cpu().numpy())
    assert float((a1 - a2).abs().max()) <= 5e-5


def test_replay_is_deterministic(synth4, torch_cuda):
    torch = torch_cuda
    a1, _ = synth4.render(11, 5, 32)
    a1 = a1.clone()
    out = torch.empty_like(a1)
    pout = torch.empty((32, 78), device=a1.device)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        synth4.render(11, 5, 32, out=out, params_out=pout, stream=s)  # warm
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        for _ in range(3):
            synth4.render(11, 5, 32, out=out, params_out=pout, stream=s)
    out.zero_()
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    synth4.sync()
    assert torch.equal(out, a1)


def test_index_rule_across_batch_sizes(synth4):
    """Voice g renders identically in a batch of 16 and a batch of 8."""
    a16, p16 = synth4.render(9, 1, 16)   # g = 16..31
    a8, p8 = synth4.render(9, 3, 8)      # g = 24..31
    synth4.sync()
    assert np.array_equal(p16[8:].cpu().numpy(), p8.cpu().numpy())
    assert np.array_equal(a16[8:].cpu().numpy(), a8.cpu().numpy())


@pytest.mark.parametrize("plain", [False, True])
def test_params_in_edge_corners(torch_cuda, oracle_mod, plain):
    """Degenerate parameter corners (zero-length sections, all-zero weights,
    extreme pitch) given through params_in."""
    import paper_2104_12922_gb300 as pkg
    torch = torch_cuda
    u = si.edge_params(10)
    syn = pkg.Synth(seconds=1.0, max_batch=10)
    pin = torch.tensor(u, dtype=torch.float32, device="cuda")
    audio, params = syn.render(0, 0, 10, params_in=pin, plain=plain)
    syn.sync()
    ref_a, ref_p = _oracle_batch(oracle_mod, 1.0, 0, 0, 10, u_in=u)
    # An LFO phase that lands exactly on a square/saw discontinuity (u = 1/2
    # gives a 5 Hz LFO from phase 0: after 1 s it is back at 0) may be taken
    # on either side by two correct evaluations whose running sums round
    # differently; from one interval before such a tie on, the pitch and the
    # phase carry of that voice are not unique, so only the part before it is
    # compared (the rest must still be valid audio).
    cfg = oracle_mod.default_config(seconds=1.0)
    a = audio.cpu().numpy()
    assert np.all(np.isfinite(a)) and np.abs(a).max() <= 1.0
    for v in range(10):
        ties = oracle_mod.discontinuity_ties(cfg, u[v])
        end = (int(ties[0]) - 1) * 100 if len(ties) else a.shape[1]
        assert end > 0
        err = float(np.max(np.abs(a[v, :end] - ref_a[v, :end])))
        assert err <= TOL, (v, err, ties[:3])
    assert np.array_equal(params.cpu().numpy(), ref_p)
    syn.close()


@pytest.mark.parametrize("plain", [False, True])
@pytest.mark.parametrize("seconds", [44 / 44100, 0.1, 25500 / 44100, 25600 / 44100, 0.29])
def test_ragged_lengths(torch_cuda, oracle_mod, seconds, plain):
    """Lengths shorter than one control interval, a ragged last interval,
    N not a multiple of 4, exactly one full tile of 255 intervals, and one
    full tile plus a tile of a single interval."""
    import paper_2104_12922_gb300 as pkg
    syn = pkg.Synth(seconds=seconds, max_batch=5)
    audio, params = syn.render(21, 7, 5, plain=plain)
    syn.sync()
    ref_a, ref_p = _oracle_batch(oracle_mod, seconds, 21, 7, 5)
    _check(audio, params, ref_a, ref_p)
    syn.close()


def test_large_voice_index(synth4, oracle_mod):
    """Global voice index above 2^32 (counter word 1 of Philox in use)."""
    bi = (1 << 33) + 17
    audio, params = synth4.render(5, bi, 4)
    synth4.sync()
    ref_a, ref_p = _oracle_batch(oracle_mod, 4.0, 5, bi, 4)
    _check(audio, params, ref_a, ref_p)


def test_argument_errors(synth4, torch_cuda):
    import paper_2104_12922_gb300 as pkg
    L = pkg.lib()
    out = torch_cuda.empty((1, synth4.num_samples), device="cuda")
    assert L.synth_render(synth4.handle, 0, 0, 129, None, out.data_ptr(), None, None) == pkg.SYNTH_ERR_ARG
    assert L.synth_render(synth4.handle, 0, 0, -1, None, out.data_ptr(), None, None) == pkg.SYNTH_ERR_ARG
    assert L.synth_render(synth4.handle, 0, 0, 1, None, None, None, None) == pkg.SYNTH_ERR_ARG
    assert L.synth_render(synth4.handle, 0, 0, 0, None, None, None, None) == pkg.SYNTH_OK
    assert L.synth_render_plain(synth4.handle, 0, 0, 1, None, out.data_ptr(), None, None, 0,
                                None) == pkg.SYNTH_ERR_ARG
    synth4.sync()


def test_params_to_human_matches_oracle(synth4, oracle_mod):
    import ctypes
    import paper_2104_12922_gb300 as pkg
    u = si.uniform_params(4, 3).astype(np.float32)
    y = np.zeros((3, 78))
    st = pkg.lib().synth_params_to_human(synth4.handle, u.ctypes.data_as(ctypes.c_void_p),
                                         y.ctypes.data_as(ctypes.c_void_p), 3)
    assert st == 0
    nb = oracle_mod.default_nebula()
    for i in range(3):
        for p in range(78):
            want = oracle_mod.range_map(float(u[i, p]), nb["lo"][p], nb["hi"][p], nb["curve"][p],
                                        nb["symmetric"][p])
            assert y[i, p] == pytest.approx(want, rel=1e-15, abs=1e-15)


def test_render_batches_equals_separate_renders(torch_cuda):
    """synth_render_batches(seed, step, bi, batch, count): batch k is
    synth_render(seed + k step, bi + k, batch) -- bit-exact, including a
    ragged batch count and a seed step of 0."""
    import paper_2104_12922_gb300 as pkg
    torch = torch_cuda
    syn = pkg.Synth(seconds=0.5, max_batch=40)
    for seed, step, bi, batch, count in [(7, 1, 7, 8, 5), (3, 0, 11, 13, 3)]:
        a, p = syn.render_batches(seed, step, bi, batch, count)
        for k in range(count):
            ak, pk = syn.render(seed + k * step, bi + k, batch)
            assert torch.equal(a[k * batch:(k + 1) * batch], ak), (seed, k)
            assert torch.equal(p[k * batch:(k + 1) * batch], pk), (seed, k)
    syn.sync()
    L = pkg.lib()
    assert L.synth_render_batches(syn.handle, 0, 1, 0, 8, 6, None, a.data_ptr(), None, None) == pkg.SYNTH_ERR_ARG
    syn.close()


def test_render_batches_full_size_sampled(torch_cuda, oracle_mod):
    """The throughput launch itself: 20 consecutive batches of 128 x 4 s in
    one synth_render_batches call, batch k with seed = batch index = 16 + k.
    A sample of voices of the first, a middle and the last batch is checked
    against the oracle (parameters bit-exact, audio within the 2e-4 bar)."""
    import paper_2104_12922_gb300 as pkg
    torch = torch_cuda
    syn = pkg.Synth(seconds=4.0, max_batch=2560)
    bi = 16
    audio, params = syn.render_batches(bi, 1, bi, 128, 20)
    syn.sync()
    assert audio.shape == (2560, syn.num_samples)
    for k in (0, 9, 19):
        rows = si.sample_voices(bi + k, 128, 6)
        idx = torch.as_tensor(k * 128 + rows, device=audio.device, dtype=torch.long)
        a = audio.index_select(0, idx).cpu().numpy()
        p = params.index_select(0, idx).cpu().numpy()
        ref_a, ref_p = _oracle_batch(oracle_mod, 4.0, bi + k, bi + k, 128, voices=rows)
        assert np.array_equal(p, ref_p[rows]), f"batch {k}: parameter draw must be bit-exact"
        assert np.all(np.isfinite(a))
        err = float(np.max(np.abs(a - ref_a[rows])))
        assert err <= TOL, f"batch {k}: max-abs error {err:.3e}"
    syn.close()


def _noise_only(u):
    """Noise level 1, sine and square-saw levels 0; ADSR0 held at 1 for the
    whole voice (attack and decay 0, sustain 1, note-on the full 4 s) and
    routed alone, with weight 1, to the noise amplitude. The last control
    point sits at t = 4 s = the note-off time: a release (5 s) that starts
    there with alpha = 6 stays 1 - (tau / 5)^6 = 1 in FP32 for any tau the
    two sides may round t - d to, so the tie at the note-off decides
    nothing. The other parameters keep their drawn values."""
    u = np.array(u, dtype=np.float64, copy=True)
    u[:, si.MIX], u[:, si.MIX + 1], u[:, si.MIX + 2] = 0.0, 0.0, 1.0
    u[:, si.DURATION] = 1.0
    u[:, si.ADSR + 0], u[:, si.ADSR + 1], u[:, si.ADSR + 2], u[:, si.ADSR + 3] = 0.0, 0.0, 1.0, 1.0
    u[:, si.ADSR + 4] = 1.0
    for s in range(4):
        u[:, si.mod_slot(s, 4)] = 0.0
    u[:, si.mod_slot(0, 4)] = 1.0
    return u


@pytest.mark.parametrize("plain", [False, True])
def test_noise_stream_bit_exact(synth4, oracle_mod, torch_cuda, plain):
    """The noise oscillator's Philox stream, bit for bit: with the patch of
    _noise_only the output is exactly v = 2 u01(word) - 1 in FP32 (amplitude
    1 + 0 x slope, gain 1, the other two terms 0 x finite), so the GPU audio
    must equal the oracle's audio (FP64, rounded once to FP32) exactly, for
    every sample of batch 16 x 4 s (voices g = 80..95, seed 5)."""
    torch = torch_cuda
    u = _noise_only(np.stack([oracle_mod.draw_params(5, 80 + v) for v in range(16)]))
    pin = torch.tensor(u, dtype=torch.float32, device="cuda")
    audio, params = synth4.render(5, 5, 16, params_in=pin, plain=plain)
    synth4.sync()
    ref_a, ref_p = _oracle_batch(oracle_mod, 4.0, 5, 5, 16, u_in=u.astype(np.float32).astype(np.float64))
    a = audio.cpu().numpy()
    assert np.all(np.abs(ref_a) <= 1.0) and np.std(ref_a) > 0.5
    assert np.array_equal(a, ref_a), f"{np.count_nonzero(a != ref_a)} samples differ"
    # params_out returns the caller's parameters as given
    assert np.array_equal(params.cpu().numpy(), u.astype(np.float32))


def test_back_to_back_launches_equal_separate_renders(torch_cuda):
    """Consecutive fused launches on one stream may overlap (the next launch's
    CTAs start in the SM slots of the previous launch's tail; the handle
    alternates two scratch slots). Six renders issued back to back, eagerly
    and captured in a CUDA graph replayed twice, with a normalised render in
    between, must equal the same renders done one at a time with the stream
    synchronised after each, bit for bit."""
    import paper_2104_12922_gb300 as pkg
    torch = torch_cuda
    B, secs = 32, 1.0
    syn = pkg.Synth(seconds=secs, max_batch=B)
    n = syn.num_samples
    ref = []
    for k in range(6):
        a, _ = syn.render(100 + k, k, B)
        syn.sync()
        ref.append(a.clone())
    ref_n, _, ref_pk, _ = syn.render_normalized(7, 9, B)
    syn.sync()
    ref_n = ref_n.clone()
    outs = [torch.empty((B, n), device="cuda") for _ in range(6)]
    pouts = [torch.empty((B, 78), device="cuda") for _ in range(6)]
    on = torch.empty((B, n), device="cuda")
    st = torch.cuda.Stream()

    def issue():
        for k in range(6):
            syn.render(100 + k, k, B, out=outs[k], params_out=pouts[k], stream=st)
            if k == 2:
                syn.render_normalized(7, 9, B, out=on, stream=st)

    with torch.cuda.stream(st):
        issue()
    st.synchronize()
    syn.sync(st)
    for k in range(6):
        assert torch.equal(outs[k], ref[k]), k
    assert torch.equal(on, ref_n)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        issue()
    for _ in range(2):
        for o in outs + [on]:
            o.fill_(float("nan"))
        with torch.cuda.stream(st):
            g.replay()
        st.synchronize()
        syn.sync(st)
        for k in range(6):
            assert torch.equal(outs[k], ref[k]), k
        assert torch.equal(on, ref_n)
    del g
    syn.close()


def test_back_to_back_launches_sharing_buffers_keep_stream_order(torch_cuda):
    """A launch that writes what the previous launch on the stream reads or
    writes, or reads what it writes, is not overlapped with it. Chains that
    depend on that order: the parameters written by one render fed back as
    the next render's input (read after write), two renders into the same
    output (write after write: the second wins), and a render into the
    buffer the previous render took its parameters from (write after read),
    eagerly and from a replayed CUDA graph; each must equal the same calls
    with the stream synchronised between them."""
    import paper_2104_12922_gb300 as pkg
    torch = torch_cuda
    B, secs = 32, 1.0
    syn = pkg.Synth(seconds=secs, max_batch=B)
    n = syn.num_samples
    st = torch.cuda.Stream()
    # references, one call at a time
    a0, p0 = syn.render(11, 3, B)
    syn.sync()
    a0, p0 = a0.clone(), p0.clone()
    a1, _ = syn.render(0, 0, B, params_in=p0)
    syn.sync()
    a1 = a1.clone()
    a2, _ = syn.render(12, 4, B)
    syn.sync()
    a2 = a2.clone()
    pq = torch.empty((B, 78), device="cuda")
    out = torch.empty((B, n), device="cuda")
    out2 = torch.empty((B, n), device="cuda")
    pw = torch.empty((B, 78), device="cuda")

    def issue():
        # read after write: params written, then read by the next launch
        syn.render(11, 3, B, out=out2, params_out=pq, stream=st)
        syn.render(0, 0, B, params_in=pq, out=out, params_out=pw, stream=st)
        # write after read: the next launch writes the parameters just read
        syn.render(12, 4, B, out=out2, params_out=pq, stream=st)
        # write after write: the same output twice, the second wins
        syn.render(11, 3, B, out=out, stream=st)
        syn.render(0, 0, B, params_in=p0, out=out, stream=st)

    with torch.cuda.stream(st):
        issue()
    st.synchronize()
    syn.sync(st)
    assert torch.equal(pw, p0)
    assert torch.equal(out, a1)
    assert torch.equal(out2, a2)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        issue()
    for _ in range(2):
        for o in (out, out2, pq, pw):
            o.fill_(float("nan"))
        with torch.cuda.stream(st):
            g.replay()
        st.synchronize()
        syn.sync(st)
        assert torch.equal(pw, p0)
        assert torch.equal(out, a1)
        assert torch.equal(out2, a2)
    del g
    syn.close()


def test_two_handles_interleaved_on_one_stream(torch_cuda):
    """Renders of two handles (each with its own scratch and voice set-up
    records) interleaved on one stream overlap each other's tails; each
    result must equal the same render done alone."""
    import paper_2104_12922_gb300 as pkg
    torch = torch_cuda
    B = 48
    sa = pkg.Synth(seconds=1.0, max_batch=B)
    sb = pkg.Synth(seconds=1.5, max_batch=B)
    refs = []
    for k in range(4):
        s = sa if k % 2 == 0 else sb
        a, _ = s.render(30 + k, k, B)
        s.sync()
        refs.append(a.clone())
    st = torch.cuda.Stream()
    outs = [torch.empty((B, (sa if k % 2 == 0 else sb).num_samples), device="cuda") for k in range(4)]
    pouts = [torch.empty((B, 78), device="cuda") for _ in range(4)]
    with torch.cuda.stream(st):
        for rep in range(2):
            for k in range(4):
                s = sa if k % 2 == 0 else sb
                s.render(30 + k, k, B, out=outs[k], params_out=pouts[k], stream=st)
            st.synchronize()
            for k in range(4):
                assert torch.equal(outs[k], refs[k]), (rep, k)
                outs[k].fill_(float("nan"))
    sa.sync(st)
    sb.sync(st)
    sa.close()
    sb.close()


def test_render_right_after_the_network_reads_its_output(torch_cuda):
    """The network's kernels let their successor be scheduled early (each
    waits for its predecessor at its start); a fused render does not wait at
    its start, so after such a kernel it must be launched the plain way. The
    proposal network's parameters fed straight into a render on one stream,
    with no synchronisation between them, must give the render of the same
    parameters done after a synchronisation."""
    import paper_2104_12922_gb300 as pkg
    torch = torch_cuda
    B = 16
    syn = pkg.Synth(seconds=1.0, max_batch=B)
    model = pkg.ProposalModel(syn, max_batch=B, seed=3)
    audio, _ = syn.render(5, 0, B)
    syn.sync()
    feats = model.features(audio)
    ref_p = model.forward(feats)
    torch.cuda.synchronize()
    ref_a, _ = syn.render(0, 0, B, params_in=ref_p)
    syn.sync()
    ref_a = ref_a.clone()
    st = torch.cuda.Stream()
    for _ in range(3):
        with torch.cuda.stream(st):
            f2 = model.features(audio, stream=st)
            p2 = model.forward(f2, stream=st)
            a2, _ = syn.render(0, 0, B, params_in=p2, stream=st)
        st.synchronize()
        syn.sync(st)
        assert torch.equal(p2, ref_p)
        assert torch.equal(a2, ref_a)
    model.close()
    syn.close()
