"""Pins of the FP64 oracle to facts outside itself (no GPU).

Each test checks the oracle against something the paper or mathematics fixes:
a library implementation of the published generator, closed forms of the
module readings at exact points, whole-voice closed forms (constant pitch,
linear glide), invariants, and the index rule of Sec. 2.1/2.2. A plausible
slip in the oracle -- a dropped term, a wrong sign, an inclusive instead of
exclusive phase sum, a transposed modulation matrix -- fails at least one.
"""
import math

import numpy as np
import pytest

import seeded_inputs as si
from tests._philox_lib import triton_philox


# --------------------------------------------------------------------- Philox
def test_philox_matches_triton_library(oracle_mod):
    """Philox4x32-10 (Salmon et al., SC'11) equals Triton's implementation."""
    rng = np.random.default_rng(1)
    reqs = []
    for seed in [0, 1, 0xFFFFFFFF, (0x12345678 << 32) | 0x9ABCDEF0, 2**64 - 1]:
        ctrs = rng.integers(0, 2**32, size=(6, 4), dtype=np.uint64).astype(np.uint32)
        ctrs[0] = 0
        ctrs[1] = 0xFFFFFFFF
        reqs.append({"seed": int(seed), "ctrs": ctrs.tolist()})
    ref = triton_philox(reqs)
    for req, blocks in zip(reqs, ref):
        key = [req["seed"] & 0xFFFFFFFF, req["seed"] >> 32]
        for ctr, want in zip(req["ctrs"], blocks):
            got = oracle_mod.philox4x32_10(ctr, key)
            assert got.tolist() == want, (req["seed"], ctr)


def test_param_draw_uses_param_stream(oracle_mod):
    """Sec. 2.1 deterministic draw: param p of voice g is word p%4 of the block
    at counter (g lo, g hi, p/4, 0); u = top 24 bits * 2^-24."""
    seed, g = (3 << 32) | 11, (2 << 32) | 5
    ctrs = [[g & 0xFFFFFFFF, g >> 32, b, 0] for b in range(20)]
    words = np.array(triton_philox([{"seed": seed, "ctrs": ctrs}])[0], dtype=np.uint64).reshape(-1)
    want = (words[:78] >> 8).astype(np.float64) / 2**24
    got = oracle_mod.draw_params(seed, g)
    assert np.array_equal(got, want)
    assert got.min() >= 0.0 and got.max() < 1.0


def test_noise_stream_bit_exact(oracle_mod):
    """Noise-only voice: out(n) = 2 u(n) - 1 with u from counter (g, n/4, 1)."""
    nb = si.pinned_nebula(oracle_mod.default_nebula(), {
        si.MIX: 0.0, si.MIX + 1: 0.0, si.MIX + 2: 1.0,
        si.DURATION: 2.0,
        si.ADSR + 0: 0.0, si.ADSR + 1: 0.0, si.ADSR + 2: 1.0, si.ADSR + 3: 0.0,
        **{si.mod_slot(s, d): 0.0 for s in range(4) for d in range(5)},
        si.mod_slot(0, 4): 1.0})
    cfg = oracle_mod.default_config(seconds=1.0, nebula=nb)
    seed, g = 77, (1 << 33) + 9
    out = oracle_mod.render_voice(cfg, np.full(78, 0.5), seed, g)
    n_blocks = len(out) // 4
    ctrs = [[g & 0xFFFFFFFF, g >> 32, q, 1] for q in range(n_blocks)]
    words = np.array(triton_philox([{"seed": seed, "ctrs": ctrs}])[0], dtype=np.uint64).reshape(-1)
    want = 2.0 * ((words >> 8).astype(np.float64) / 2**24) - 1.0
    assert np.array_equal(out, want)
    assert abs(out.mean()) < 0.01 and abs(out.var() - 1.0 / 3.0) < 0.01


# ------------------------------------------------------------------ range map
@pytest.mark.parametrize("sym", [0, 1])
@pytest.mark.parametrize("curve", [0.3, 1.0, 2.0, 5.0])
def test_range_map_endpoints_monotone(oracle_mod, curve, sym):
    """Sec. 3.3: u=0 -> min, u=1 -> max, monotone; symmetric centre -> midpoint."""
    lo, hi = (-127.0, 127.0) if sym else (0.0, 127.0)
    rm = lambda u: oracle_mod.range_map(u, lo, hi, curve, sym)
    assert rm(0.0) == lo and rm(1.0) == hi
    us = np.linspace(0, 1, 257)
    ys = np.array([rm(u) for u in us])
    assert np.all(np.diff(ys) >= 0)
    if sym:
        assert rm(0.5) == pytest.approx(0.0, abs=1e-12)
        # symmetric about the centre: y(1-u) = -y(u) for a range centred at 0
        assert np.allclose(ys[::-1], -ys, atol=1e-12)
    if curve == 1.0:
        assert np.allclose(ys, lo + (hi - lo) * us, atol=1e-12)


def test_range_map_curve_points(oracle_mod):
    """Closed points: u^2 at u=1/2 is 1/4; symmetric |s|^2 at u=3/4 is 1/4."""
    assert oracle_mod.range_map(0.5, 0.0, 8.0, 2.0, 0) == 2.0
    assert oracle_mod.range_map(0.75, -8.0, 8.0, 2.0, 1) == pytest.approx(2.0)
    assert oracle_mod.range_map(0.25, -8.0, 8.0, 2.0, 1) == pytest.approx(-2.0)


# ---------------------------------------------------------------------- ADSR
def test_adsr_section_values(oracle_mod):
    """Sec. 3.1 ADSR sections at exact times (alpha = 2 so values are squares)."""
    a, dc, s, r, al, d = 0.5, 0.4, 0.6, 1.0, 2.0, 2.0
    f = lambda t: oracle_mod.adsr(t, a, dc, s, r, al, d)
    assert f(0.0) == 0.0
    assert f(0.25) == pytest.approx(0.25)             # (t/a)^2 at half attack
    assert f(0.5) == pytest.approx(1.0)               # peak at end of attack
    assert f(0.7) == pytest.approx(1 - 0.4 * 0.25)    # half-way through decay
    assert f(0.9) == pytest.approx(s)                 # sustain
    assert f(1.9) == pytest.approx(s)
    assert f(2.0) == pytest.approx(s)                 # release starts from g(d)
    assert f(2.5) == pytest.approx(s * (1 - 0.25))
    assert f(3.0) == 0.0 and f(3.5) == 0.0


def test_adsr_release_during_attack_is_continuous(oracle_mod):
    """Note-off inside the attack: release starts from the level reached."""
    a, dc, s, r, al, d = 2.0, 0.5, 0.3, 1.0, 1.0, 1.0
    f = lambda t: oracle_mod.adsr(t, a, dc, s, r, al, d)
    assert f(1.0) == pytest.approx(0.5)
    assert f(1.0 - 1e-9) == pytest.approx(0.5, abs=1e-8)
    assert f(1.5) == pytest.approx(0.25)


def test_adsr_degenerate_sections(oracle_mod):
    f = lambda t, **k: oracle_mod.adsr(t, k.get("a", 0.0), k.get("dc", 0.0), k.get("s", 0.7),
                                       k.get("r", 0.0), 1.5, k.get("d", 1.0))
    assert f(0.0) == 0.7              # a = dc = 0: straight to sustain
    assert f(0.0, dc=0.5) == 1.0      # a = 0: decay starts at the peak
    assert f(1.0) == 0.0              # r = 0: zero at note-off
    assert f(0.0, a=0.3, d=0.0) == 0.0  # d = 0: never leaves zero


def test_adsr_bounds_and_continuity(oracle_mod):
    rng = np.random.default_rng(0)
    for _ in range(200):
        a, dc, r = rng.uniform(0, 2, 3)
        s, al, d = rng.uniform(0, 1), rng.uniform(0.1, 6), rng.uniform(0, 4)
        ts = np.linspace(0, 6, 601)
        v = np.array([oracle_mod.adsr(t, a, dc, s, r, al, d) for t in ts])
        assert v.min() >= 0.0 and v.max() <= 1.0
        # a section of length L with curvature alpha moves by at most
        # (eps / L)^alpha within eps of its start (infinite slope for alpha < 1)
        step = (2e-10 / min(a, dc, r)) ** al + 1e-6
        for tb in [a, a + dc, d, d + r]:
            if tb > d and tb != d + r:
                continue  # sections after note-off are cut by the release
            lo = oracle_mod.adsr(tb - 1e-10, a, dc, s, r, al, d)
            hi = oracle_mod.adsr(tb + 1e-10, a, dc, s, r, al, d)
            assert abs(lo - hi) <= step


# ----------------------------------------------------------------------- LFO
def test_lfo_shapes_at_quarter_points(oracle_mod):
    want = {0: [0, 1, 0, -1], 1: [-1, 0, 1, 0], 2: [-1, -0.5, 0, 0.5],
            3: [1, 0.5, 0, -0.5], 4: [1, 1, -1, -1]}
    for shape, vals in want.items():
        got = [oracle_mod.lfo_shape(shape, p) for p in (0.0, 0.25, 0.5, 0.75)]
        assert np.allclose(got, vals, atol=1e-15), shape


def test_midi_to_hz(oracle_mod):
    assert oracle_mod.midi_to_hz(69) == 440.0
    assert oracle_mod.midi_to_hz(81) == 880.0
    assert oracle_mod.midi_to_hz(57) == 220.0
    assert oracle_mod.midi_to_hz(60) == pytest.approx(261.6255653005986, rel=1e-15)


def _base_nebula(oracle_mod, pins):
    return si.pinned_nebula(oracle_mod.default_nebula(), pins)


def _const_source_pins(amp_dest, extra=None):
    """ADSR0 = constant 1 (a = dc = 0, s = 1, note held past the end),
    routed only to ``amp_dest``; all other weights 0."""
    pins = {si.DURATION: 10.0, si.ADSR + 0: 0.0, si.ADSR + 1: 0.0, si.ADSR + 2: 1.0,
            si.ADSR + 3: 0.0, si.ADSR + 4: 1.0}
    pins.update({si.mod_slot(s, d): 0.0 for s in range(4) for d in range(5)})
    pins[si.mod_slot(0, amp_dest)] = 1.0
    if extra:
        pins.update(extra)
    return pins


def test_lfo_constant_rate_phase_is_exclusive_sum(oracle_mod):
    """Saw LFO at constant rate F: lfo_k = 2 frac(phase0/2pi + k F / CR) - 1."""
    F, ph0 = 7.3, 1.1
    pins = {si.DURATION: 10.0}
    # ADSR2 (LFO0 rate) constant 0, ADSR3 (LFO0 amplitude) constant 1
    pins.update({si.ADSR + 10 + 0: 0.0, si.ADSR + 10 + 1: 0.0, si.ADSR + 10 + 2: 0.0,
                 si.ADSR + 10 + 3: 0.0, si.ADSR + 10 + 4: 1.0,
                 si.ADSR + 15 + 0: 0.0, si.ADSR + 15 + 1: 0.0, si.ADSR + 15 + 2: 1.0,
                 si.ADSR + 15 + 3: 0.0, si.ADSR + 15 + 4: 1.0,
                 si.LFO + 0: F, si.LFO + 1: 0.0, si.LFO + 2: ph0,
                 si.LFO + 3: 0.0, si.LFO + 4: 0.0, si.LFO + 5: 1.0, si.LFO + 6: 0.0, si.LFO + 7: 0.0})
    cfg = oracle_mod.default_config(seconds=1.0, nebula=_base_nebula(oracle_mod, pins))
    env, lfo, dest = oracle_mod.control(cfg, np.full(78, 0.5))
    k = np.arange(lfo.shape[1])
    theta = np.mod(ph0 / (2 * math.pi) + k * F / 441.0, 1.0)
    assert np.allclose(lfo[0], 2 * theta - 1, atol=1e-12)


def _lfo_pins(l, F, D, ph0, weights, rate_env, amp_level=1.0):
    """Pins for LFO ``l`` (0 or 1): frequency F, rate depth D, initial phase
    ph0, shape weights (sin, tri, saw, rsaw, sqr); its rate ADSR is either a
    constant 1 (``rate_env = "one"``) or the linear ramp t / 2 over the voice
    (``"ramp"``: attack 2 s, alpha 1, note held); its amplitude ADSR is the
    constant ``amp_level`` (zero attack and decay, sustain = amp_level)."""
    rate_adsr = si.ADSR + 5 * (2 + 2 * l)
    amp_adsr = si.ADSR + 5 * (3 + 2 * l)
    pins = {si.DURATION: 10.0}
    if rate_env == "one":
        pins.update({rate_adsr + 0: 0.0, rate_adsr + 1: 0.0, rate_adsr + 2: 1.0})
    else:
        pins.update({rate_adsr + 0: 2.0, rate_adsr + 1: 0.0, rate_adsr + 2: 1.0})
    pins.update({rate_adsr + 3: 0.0, rate_adsr + 4: 1.0,
                 amp_adsr + 0: 0.0, amp_adsr + 1: 0.0, amp_adsr + 2: amp_level,
                 amp_adsr + 3: 0.0, amp_adsr + 4: 1.0})
    b = si.LFO + 8 * l
    pins.update({b + 0: F, b + 1: D, b + 2: ph0})
    pins.update({b + 3 + s: w for s, w in enumerate(weights)})
    return pins


def _circ(a, b):
    d = np.abs(np.mod(a - b, 1.0))
    return np.minimum(d, 1.0 - d)


@pytest.mark.parametrize("lfo", [0, 1])
def test_lfo_rate_modulation_by_its_rate_adsr(oracle_mod, lfo):
    """rate_k = F + D ADSR_rate(t_k): with the rate ADSR a linear ramp
    t_k / 2 the exclusive phase sum has the closed form
    theta_k = ph0 / 2pi + k F / CR + D k (k - 1) / (4 CR^2), read back from
    a saw LFO (lfo = 2 theta - 1). A wrong sign of D, the amplitude ADSR in
    place of the rate ADSR, or the other LFO's ADSR fails it."""
    F, D, ph0, CR = 3.25, 9.5, -1.3, 441.0
    pins = _lfo_pins(lfo, F, D, ph0, (0, 0, 1, 0, 0), "ramp")
    cfg = oracle_mod.default_config(seconds=1.0, nebula=_base_nebula(oracle_mod, pins))
    _, out, _ = oracle_mod.control(cfg, np.full(78, 0.5))
    k = np.arange(out.shape[1], dtype=np.float64)
    theta = ph0 / (2 * math.pi) + k * F / CR + D * k * (k - 1) / (4 * CR * CR)
    assert np.max(_circ((out[lfo] + 1) / 2, theta)) < 1e-10


@pytest.mark.parametrize("lfo", [0, 1])
@pytest.mark.parametrize("F,D,rate", [(6.0, 5.5, 11.5), (15.0, 12.0, 20.0), (5.0, -12.0, 0.0),
                                      (20.0, -20.0, 0.0), (0.0, 20.0, 20.0)])
def test_lfo_rate_is_clamped_to_0_20_hz(oracle_mod, lfo, F, D, rate):
    """Constant rate ADSR 1: rate = clamp(F + D, 0, 20 Hz), so the saw's phase
    is ph0/2pi + k rate / CR; above 20 Hz it runs at exactly 20 Hz, below 0
    it stands still (no negative rates)."""
    ph0, CR = 0.9, 441.0
    pins = _lfo_pins(lfo, F, D, ph0, (0, 0, 1, 0, 0), "one")
    cfg = oracle_mod.default_config(seconds=0.5, nebula=_base_nebula(oracle_mod, pins))
    _, out, _ = oracle_mod.control(cfg, np.full(78, 0.5))
    k = np.arange(out.shape[1], dtype=np.float64)
    theta = ph0 / (2 * math.pi) + k * rate / CR
    assert np.max(_circ((out[lfo] + 1) / 2, theta)) < 1e-11


@pytest.mark.parametrize("lfo", [0, 1])
def test_lfo_shape_mix_divides_by_weight_sum(oracle_mod, lfo):
    """A standing LFO (rate 0) at phase p gives amp * sum_s w_s shape_s(p) /
    sum_s w_s, with the shapes' own values at the quarter points: sin 1, 0,
    -1; tri 0, 1, 0 (p = 1/4, 1/2, 3/4); saw 2p - 1; rsaw 1 - 2p; square +1
    for p < 1/2 else -1. Weights summing to less than 1 are normalised too
    (a lone weight of 0.1 gives the full shape), and the amplitude ADSR
    scales the mix."""
    shapes = {0.25: (1.0, 0.0, -0.5, 0.5, 1.0), 0.5: (0.0, 1.0, 0.0, 0.0, -1.0),
              0.75: (-1.0, 0.0, 0.5, -0.5, -1.0)}
    ph0_of = {0.25: math.pi / 2, 0.5: math.pi, 0.75: -math.pi / 2}
    for weights in [(0.2, 0.5, 0.3, 0.7, 0.1), (0.1, 0.0, 0.0, 0.0, 0.0),
                    (0.0, 0.05, 0.0, 0.0, 0.15), (1.0, 1.0, 1.0, 1.0, 1.0)]:
        for p, vals in shapes.items():
            pins = _lfo_pins(lfo, 0.0, 0.0, ph0_of[p], weights, "one", amp_level=0.6)
            cfg = oracle_mod.default_config(seconds=0.05, nebula=_base_nebula(oracle_mod, pins))
            _, out, _ = oracle_mod.control(cfg, np.full(78, 0.5))
            want = 0.6 * sum(w * v for w, v in zip(weights, vals)) / sum(weights)
            assert np.allclose(out[lfo], want, atol=1e-12), (weights, p)
    # all weights 0: the LFO is silent
    pins = _lfo_pins(lfo, 3.0, 0.0, 0.3, (0, 0, 0, 0, 0), "one")
    cfg = oracle_mod.default_config(seconds=0.05, nebula=_base_nebula(oracle_mod, pins))
    _, out, _ = oracle_mod.control(cfg, np.full(78, 0.5))
    assert np.all(out[lfo] == 0.0)


def test_mod_matrix_one_hot_routes_source(oracle_mod):
    """dest_j = sum_i W[i][j] src_i / max(1, sum_i W[i][j]): one-hot W[i][j]
    copies source i to destination j and leaves the others at 0; the
    normaliser divides by the column sum, not the row sum."""
    cfg = oracle_mod.default_config(seconds=0.5)
    u = si.uniform_params(3, 1)[0]
    for i, j in [(0, 3), (1, 0), (2, 4), (3, 1)]:
        ui = u.copy()
        for s in range(4):
            for d in range(5):
                ui[si.mod_slot(s, d)] = 0.0
        ui[si.mod_slot(i, j)] = 1.0
        env, lfo, dest = oracle_mod.control(cfg, ui)
        src = [env[0], env[1], lfo[0], lfo[1]][i]
        assert np.allclose(dest[j], src, atol=1e-15)
        for d in range(5):
            if d != j:
                assert np.all(dest[d] == 0)
    # column normalisation: two weights of 1 into one destination average them
    ui = u.copy()
    for s in range(4):
        for d in range(5):
            ui[si.mod_slot(s, d)] = 0.0
    ui[si.mod_slot(0, 2)] = 1.0
    ui[si.mod_slot(1, 2)] = 1.0
    env, lfo, dest = oracle_mod.control(cfg, ui)
    assert np.allclose(dest[2], 0.5 * (env[0] + env[1]), atol=1e-15)


def test_control_env_matches_adsr_at_control_times(oracle_mod):
    cfg = oracle_mod.default_config()
    u = oracle_mod.draw_params(5, 17)
    env, _, _ = oracle_mod.control(cfg, u)
    nb = oracle_mod.default_nebula()
    y = [oracle_mod.range_map(u[p], nb["lo"][p], nb["hi"][p], nb["curve"][p], nb["symmetric"][p])
         for p in range(78)]
    for a in range(6):
        q = y[2 + 5 * a: 7 + 5 * a]
        for k in [0, 1, 57, 441, 1000, 1764]:
            assert env[a, k] == oracle_mod.adsr(k / 441.0, *q, y[1])


# ---------------------------------------------------------- whole-voice forms
def _sine_patch(oracle_mod, seconds, extra_pins):
    pins = _const_source_pins(1, {si.MIX: 1.0, si.MIX + 1: 0.0, si.MIX + 2: 0.0,
                                  si.SINE + 1: 0.0})
    pins.update(extra_pins)
    return oracle_mod.default_config(seconds=seconds, nebula=_base_nebula(oracle_mod, pins))


def test_constant_pitch_sine_closed_form(oracle_mod):
    """Closed form: constant pitch gives sin(2 pi f n / SR + phase0)
    exactly (exclusive phase sum: sample 0 carries the initial phase)."""
    for midi, tune, ph0 in [(69.0, 0.0, 0.0), (60.0, 3.5, 0.7), (100.0, -24.0, -2.9)]:
        cfg = _sine_patch(oracle_mod, 4.0, {si.MIDI: midi, si.SINE: tune, si.SINE + 2: ph0})
        out = oracle_mod.render_voice(cfg, np.full(78, 0.5), 0, 0)
        f = 440.0 * 2 ** ((midi + tune - 69.0) / 12.0)
        n = np.arange(len(out))
        want = np.sin(2 * math.pi * np.mod(f * n / 44100.0 + ph0 / (2 * math.pi), 1.0))
        assert np.max(np.abs(out - want)) < 1e-9


@pytest.mark.parametrize("sr,cr", [(44100.0, 441.0), (16000.0, 441.0), (22050.0, 441.0),
                                   (8000.0, 441.0), (48000.0, 400.0)])
def test_linear_glide_sine_closed_form(oracle_mod, sr, cr):
    """Linear midi glide m(n) = m0 + D n / (a SR): the phase is the geometric
    sum phi(n) = phi0 + (f0/SR) (r^n - 1)/(r - 1), r = 2^(D/(12 a SR)). The
    pitch is linear in time at the control points (an attack ramp), and
    linear interpolation between control points keeps it linear at every
    sample only if each sample takes its own fraction of its interval: so
    the closed form holds for any R = SR / CR, integer (100, 50, 120) or not
    (36.28..., 18.14...)."""
    secs, m0, D = 2.0, 50.0, 30.0
    extra = {si.MIDI: m0, si.SINE + 1: D, si.SINE + 2: 0.0,
             si.ADSR + 0: secs, si.ADSR + 4: 1.0,
             si.ADSR + 5: 0.0, si.ADSR + 6: 0.0, si.ADSR + 7: 1.0, si.ADSR + 8: 0.0, si.ADSR + 9: 1.0}
    pins = _const_source_pins(1, {si.MIX: 1.0, si.MIX + 1: 0.0, si.MIX + 2: 0.0})
    pins.update(extra)
    pins[si.mod_slot(0, 1)] = 0.0
    pins[si.mod_slot(1, 1)] = 1.0   # ADSR1 = constant 1 drives the amplitude
    pins[si.mod_slot(0, 0)] = 1.0   # ADSR0 = linear ramp drives the pitch
    cfg = oracle_mod.default_config(seconds=secs, sample_rate=sr, control_rate=cr,
                                    nebula=_base_nebula(oracle_mod, pins))
    out = oracle_mod.render_voice(cfg, np.full(78, 0.5), 0, 0)
    assert len(out) == int(secs * sr)
    f0 = 440.0 * 2 ** ((m0 - 69.0) / 12.0)
    n = np.arange(len(out), dtype=np.float64)
    lr = D / (12.0 * secs * sr) * math.log(2.0)
    phi = f0 / sr * np.expm1(n * lr) / math.expm1(lr)
    want = np.sin(2 * math.pi * np.mod(phi, 1.0))
    assert np.max(np.abs(out - want)) < 1e-8


@pytest.mark.parametrize("sr,cr", [(16000.0, 441.0), (44100.0, 441.0), (11025.0, 400.0)])
def test_amplitude_ramp_is_linear_at_every_sample(oracle_mod, sr, cr):
    """A linear attack ramp routed to the sine's amplitude, at constant
    pitch: out(n) = (t_n / a) sin(2 pi f n / SR) with t_n = n / SR, for any
    R = SR / CR (the upsampling fraction of sample n is n B / A - k)."""
    secs, a = 1.0, 1.0
    f = 440.0
    pins = _const_source_pins(1, {si.MIX: 1.0, si.MIX + 1: 0.0, si.MIX + 2: 0.0,
                                  si.SINE + 1: 0.0, si.MIDI: 69.0, si.SINE: 0.0,
                                  si.SINE + 2: 0.0, si.ADSR + 0: a, si.ADSR + 4: 1.0})
    cfg = oracle_mod.default_config(seconds=secs, sample_rate=sr, control_rate=cr,
                                    nebula=_base_nebula(oracle_mod, pins))
    out = oracle_mod.render_voice(cfg, np.full(78, 0.5), 0, 0)
    n = np.arange(len(out), dtype=np.float64)
    want = np.minimum(n / sr / a, 1.0) * np.sin(2 * math.pi * np.mod(f * n / sr, 1.0))
    assert np.max(np.abs(out - want)) < 1e-9


def test_fractional_rate_geometry(oracle_mod):
    """R = 16000 / 441: K = floor((N - 1) B / A) + 1 intervals, each of
    floor(R) or ceil(R) samples (counted by brute force over n); an
    unsupported non-integer pair of non-integer rates is refused."""
    a, b = oracle_mod.rate_ratio(16000.0, 441.0)
    assert (a, b) == (16000, 441)
    assert oracle_mod.rate_ratio(44100.0, 441.0) == (100, 1)
    N = 16000
    k = np.arange(N, dtype=np.int64) * b // a
    counts = np.bincount(k)
    assert len(counts) == (N - 1) * b // a + 1
    assert set(counts[:-1].tolist()) <= {36, 37} and 1 <= counts[-1] <= 37
    cfg = oracle_mod.default_config(seconds=1.0, sample_rate=16000.0, control_rate=441.0)
    assert oracle_mod.num_control_points(cfg) == len(counts) + 1
    bad = oracle_mod.default_config(seconds=2.0, sample_rate=16000.5, control_rate=441.3)
    with pytest.raises(ValueError):
        oracle_mod.render_voice(bad, np.full(78, 0.5), 0, 0)


def test_square_saw_spot_values(oracle_mod):
    """Square-saw at constant pitch: theta = 2 pi f n/SR; out = tanh(k sin)/tanh k
    * (1 + s cos)/(1 + s). Spot checks at theta = 0, pi/2, pi, 3pi/2 and the
    square-wave symmetry out(theta + pi) = -out(theta) at shape 0."""
    f = 44100.0 / 8.0  # 8 samples per cycle, theta lands on multiples of pi/4
    midi = 69.0 + 12.0 * math.log2(f / 440.0)
    kappa = min(50.0, 1.0 + 44100.0 / (8.0 * f))
    for shape in (0.0, 0.5, 1.0):
        pins = _const_source_pins(3, {si.MIX: 0.0, si.MIX + 1: 1.0, si.MIX + 2: 0.0,
                                      si.MIDI: midi, si.SQR: 0.0, si.SQR + 1: 0.0,
                                      si.SQR + 2: 0.0, si.SQR + 3: shape})
        cfg = oracle_mod.default_config(seconds=0.1, nebula=_base_nebula(oracle_mod, pins))
        out = oracle_mod.render_voice(cfg, np.full(78, 0.5), 0, 0)
        assert abs(out[0]) < 1e-12 and abs(out[4]) < 1e-9
        assert out[2] == pytest.approx(1.0 / (1.0 + shape), abs=1e-9)
        assert out[6] == pytest.approx(-1.0 / (1.0 + shape), abs=1e-9)
        s1 = math.sin(math.pi / 4)
        want1 = math.tanh(kappa * s1) / math.tanh(kappa) * (1 + shape * s1) / (1 + shape)
        assert out[1] == pytest.approx(want1, abs=1e-9)
        if shape == 0.0:
            assert np.allclose(out[4:400], -out[0:396], atol=1e-9)


def _square_saw_patch(oracle_mod, seconds, midi, tune, depth, ph0, shape, pitch_dest):
    """Square-saw alone (levels 0, 1, 0; amplitude from ADSR0 = 1 through
    destination 3); ADSR0 also routed with weight 1 to ``pitch_dest``."""
    pins = _const_source_pins(3, {si.MIX: 0.0, si.MIX + 1: 1.0, si.MIX + 2: 0.0,
                                  si.MIDI: midi, si.SQR: tune, si.SQR + 1: depth,
                                  si.SQR + 2: ph0, si.SQR + 3: shape, si.SINE + 1: 0.0})
    if pitch_dest is not None:
        pins[si.mod_slot(0, pitch_dest)] = 1.0
    return oracle_mod.default_config(seconds=seconds, nebula=_base_nebula(oracle_mod, pins))


def _square_saw_closed_form(f, ph0, shape, n, sr=44100.0, kappa=None):
    th = 2 * math.pi * np.mod(f * n / sr + ph0 / (2 * math.pi), 1.0)
    if kappa is None:
        kappa = min(50.0, 1.0 + sr / (8.0 * f))
    return (np.tanh(kappa * np.sin(th)) / math.tanh(kappa)
            * (1.0 + shape * np.cos(th)) / (1.0 + shape))


@pytest.mark.parametrize("f,kappa", [(44100.0 / 16, 3.0), (44100.0 / 32, 5.0), (44100.0 / 64, 9.0),
                                     (55.0, 50.0), (20.0, 50.0)])
def test_square_saw_drive_follows_pitch_and_is_capped(oracle_mod, f, kappa):
    """kappa = min(50, 1 + SR / (8 f)): 3, 5 and 9 at 16, 32 and 64 samples
    per cycle, and the cap 50 at low pitch (55 Hz would give 101.2 and 20 Hz
    276.6 without it). Checked against the closed form at constant pitch with
    kappa stated numerically, over the first 2000 samples."""
    midi = 69.0 + 12.0 * math.log2(f / 440.0)
    for shape in (0.0, 0.4):
        cfg = _square_saw_patch(oracle_mod, 0.05, midi, 0.0, 0.0, 0.0, shape, None)
        out = oracle_mod.render_voice(cfg, np.full(78, 0.5), 0, 0)
        n = np.arange(2000)
        want = _square_saw_closed_form(f, 0.0, shape, n, kappa=kappa)
        assert np.max(np.abs(out[:2000] - want)) < 1e-9, (f, shape)


def test_square_saw_pitch_comes_from_destination_2(oracle_mod):
    """The square-saw's pitch is midi + tune + depth * dest_2: with ADSR0 = 1
    routed to destination 2 it sounds at 440 * 2^((midi + tune + depth - 69)/12)
    (drive kappa from that pitch); routed to destination 0 (the sine's pitch)
    instead it stays at midi + tune."""
    n = np.arange(4410)
    for midi, tune, depth, ph0 in [(60.0, 2.0, 7.0, 0.4), (81.0, -5.0, -13.5, -2.2)]:
        for dest, m in [(2, midi + tune + depth), (0, midi + tune)]:
            cfg = _square_saw_patch(oracle_mod, 0.1, midi, tune, depth, ph0, 0.3, dest)
            out = oracle_mod.render_voice(cfg, np.full(78, 0.5), 0, 0)
            f = 440.0 * 2 ** ((m - 69.0) / 12.0)
            want = _square_saw_closed_form(f, ph0, 0.3, n)
            assert np.max(np.abs(out - want)) < 1e-8, (midi, dest)


def test_nyquist_cap(oracle_mod):
    """Pitch above Nyquist is capped at SR/2: phase advances 1/2 cycle per
    sample, so the sine sits at sin(phase0 + n pi)."""
    cfg = _sine_patch(oracle_mod, 0.1, {si.MIDI: 127.0, si.SINE: 24.0, si.SINE + 2: 1.0})
    out = oracle_mod.render_voice(cfg, np.full(78, 0.5), 0, 0)
    n = np.arange(len(out))
    want = np.sin(1.0 + math.pi * n)
    assert np.max(np.abs(out - want)) < 1e-9


def test_mixer_normalises_by_level_sum(oracle_mod):
    """out = sum l_i A_i x_i / max(1, sum l_i): the normaliser is the sum of the
    levels (not of the audible sources) and never amplifies (max with 1)."""
    base = {si.MIDI: 69.0, si.SINE: 0.0, si.SINE + 2: 0.0, si.SINE + 1: 0.0, si.MIX + 2: 0.0}
    n = np.arange(2205)
    sine = np.sin(2 * math.pi * np.mod(440.0 * n / 44100.0, 1.0))
    for l0, l1, scale in [(1.0, 0.0, 1.0), (0.25, 0.0, 0.25), (1.0, 1.0, 0.5), (0.5, 0.25, 0.5)]:
        pins = _const_source_pins(1, {**base, si.MIX: l0, si.MIX + 1: l1})
        cfg = oracle_mod.default_config(seconds=0.05, nebula=_base_nebula(oracle_mod, pins))
        out = oracle_mod.render_voice(cfg, np.full(78, 0.5), 0, 0)  # square-saw amplitude is 0
        assert np.allclose(out, scale * sine, atol=1e-9), (l0, l1)


# ------------------------------------------------------------- invariants
def test_invariants_random_voices(oracle_mod):
    """Envelopes in [0,1], |LFO|, |dest| <= 1, |audio| <= 1 for drawn voices."""
    cfg = oracle_mod.default_config()
    for g in range(12):
        u = oracle_mod.draw_params(123, g)
        env, lfo, dest = oracle_mod.control(cfg, u)
        assert env.min() >= 0 and env.max() <= 1
        assert np.abs(lfo).max() <= 1 + 1e-15 and np.abs(dest).max() <= 1 + 1e-15
    audio, params = oracle_mod.render_batch(cfg, 123, 0, 8)
    assert np.abs(audio).max() <= 1.0
    assert np.all(np.isfinite(audio))


def test_edge_params_finite(oracle_mod):
    cfg = oracle_mod.default_config(seconds=1.0)
    u = si.edge_params(5)
    audio, _ = oracle_mod.render_batch(cfg, 0, 0, 5, u_in=u)
    assert np.all(np.isfinite(audio)) and np.abs(audio).max() <= 1.0


def test_index_rule_same_voice_any_batch(oracle_mod):
    """Sec. 2.2 replicability: voice g = batch_index * B + v is the same sound
    whatever the batch size it is rendered in."""
    cfg = oracle_mod.default_config(seconds=0.5)
    a16, p16 = oracle_mod.render_batch(cfg, 9, 1, 16)   # g = 16..31
    a8, p8 = oracle_mod.render_batch(cfg, 9, 3, 8)      # g = 24..31
    assert np.array_equal(a16[8:], a8) and np.array_equal(p16[8:], p8)


def test_fp32_pitch_chain_error_is_measured(oracle_mod):
    """Rounding the control-rate pitch chain and per-sample frequency to FP32
    moves drawn 4 s voices by a measurable, nonzero amount (a study of the
    precision split; constant-pitch stretches make the drift systematic)."""
    cfg = oracle_mod.default_config()
    worst = 0.0
    for g in range(8):
        u = oracle_mod.draw_params(0, g)
        a = oracle_mod.render_voice(cfg, u, 0, g)
        b = oracle_mod.render_voice(cfg, u, 0, g, flags=oracle_mod.ROUND_PITCH_CHAIN_F32)
        worst = max(worst, float(np.max(np.abs(a - b))))
    assert 1e-7 < worst < 1e-2


def test_dual_number_gradient_matches_finite_differences(oracle_mod):
    """The oracle's forward-mode gradient equals FP64 central differences on
    every parameter where the render is smooth at the step size."""
    cfg = oracle_mod.default_config(seconds=0.05)
    u = np.clip(oracle_mod.draw_params(2, 1), 0.02, 0.98)
    w = si.upstream_grad(9, (oracle_mod.num_samples(cfg),))
    grad = oracle_mod.render_vjp(cfg, u, 2, 1, w)
    checked = 0
    for p in range(78):
        fd = []
        for h in (1e-6, 2.5e-7):
            up, um = u.copy(), u.copy()
            up[p] += h
            um[p] -= h
            fd.append(float(np.dot(w, oracle_mod.render_voice(cfg, up, 2, 1) -
                                   oracle_mod.render_voice(cfg, um, 2, 1))) / (2 * h))
        if abs(fd[0] - fd[1]) > 1e-5 * (abs(fd[0]) + 1e-3):
            continue
        checked += 1
        assert grad[p] == pytest.approx(fd[0], rel=1e-5, abs=1e-6), p
    assert checked >= 60


def test_peak_normalize_pins(oracle_mod):
    """Peak normalisation: known peaks, a silent voice, the threshold tie."""
    n = 1000
    t = np.arange(n)
    x = np.stack([0.5 * np.sin(2 * np.pi * t / 40.0),    # peak 0.5 (t = 10)
                  -0.25 * np.ones(n),                      # peak 0.25, negative
                  np.zeros(n),                             # silent
                  1e-3 * np.cos(2 * np.pi * t / 40.0)])    # peak exactly 1e-3 (t = 0)
    out, peak, silent = oracle_mod.peak_normalize(x.astype(np.float32), 1e-3)
    assert peak[0] == pytest.approx(0.5, abs=1e-7)
    assert peak[1] == pytest.approx(0.25, abs=1e-7) and peak[2] == 0.0
    assert list(silent) == [False, False, True, False]  # p == threshold is kept
    assert np.max(np.abs(out[0])) == pytest.approx(1.0, abs=1e-12)
    assert np.allclose(out[1], -1.0)
    assert np.array_equal(out[2], np.zeros(n))
    # scale invariance: normalising 3 x gives the same voice
    out3, peak3, _ = oracle_mod.peak_normalize(3.0 * x[:2], 1e-3)
    assert np.allclose(out3, out[:2]) and np.allclose(peak3, 3.0 * peak[:2])
    # a voice below the threshold is returned unchanged
    out_q, _, sil_q = oracle_mod.peak_normalize(x[3:] * 0.5, 1e-3)
    assert sil_q[0] and np.array_equal(out_q[0], (x[3] * 0.5).astype(np.float64))


# ---- 4-operator FM voice -----------------------------------------------------
def _fm_u(midi, ops, duration=4.0):
    """Normalized FM parameters from human values: ops[i] = (ratio, level,
    attack, decay, sustain, release, alpha), inverted through y = lo +
    (hi - lo) u^c with the FM ranges."""
    def inv(y, lo, hi, c):
        return ((y - lo) / (hi - lo)) ** (1.0 / c)
    u = [inv(midi, 0.0, 127.0, 1.0), inv(duration, 0.0, 4.0, 1.0)]
    for i, (ratio, level, a, dc, s, r, alpha) in enumerate(ops):
        u += [inv(ratio, 0.5, 8.0, 2.0),
              inv(level, 0.0, 1.0, 1.0) if i == 0 else inv(level, 0.0, 8.0, 2.0),
              inv(a, 0.0, 2.0, 2.0), inv(dc, 0.0, 2.0, 2.0), inv(s, 0.0, 1.0, 1.0),
              inv(r, 0.0, 5.0, 2.0), inv(alpha, 0.1, 6.0, 2.0)]
    return np.array(u)


def _fm_y(u, p):
    """The mapped value of parameter p (same map, for closed forms)."""
    lo, hi, c = ((0.0, 127.0, 1.0) if p == 0 else (0.0, 4.0, 1.0) if p == 1 else
                 [(0.5, 8.0, 2.0), (0.0, 1.0, 1.0) if (p - 2) // 7 == 0 else (0.0, 8.0, 2.0),
                  (0.0, 2.0, 2.0), (0.0, 2.0, 2.0), (0.0, 1.0, 1.0), (0.0, 5.0, 2.0),
                  (0.1, 6.0, 2.0)][(p - 2) % 7])
    return lo + (hi - lo) * u[p] ** c


FLAT = (0.0, 0.0, 1.0, 0.0, 1.0)  # attack, decay, sustain, release, alpha: E = 1 while held


def test_fm_two_operators_match_jacobi_anger(oracle_mod):
    """Carrier at f0, one modulator at 2 f0 with index b, flat envelopes:
    sin(2 pi fc t + b sin(2 pi fm t)) = sum_k J_k(b) sin(2 pi (fc + k fm) t)
    (Jacobi-Anger; Chowning 1973). Pins the phase-modulation structure."""
    special = pytest.importorskip("scipy.special")
    cfg = oracle_mod.default_config(seconds=0.25)
    for b in (0.5, 2.0, 5.0):
        u = _fm_u(57.0, [(1.0, 1.0) + FLAT, (2.0, b) + FLAT, (1.0, 0.0) + FLAT, (1.0, 0.0) + FLAT])
        out = oracle_mod.fm_render_voice(cfg, u)
        f0 = 440.0 * 2 ** ((_fm_y(u, 0) - 69.0) / 12.0)
        fc, fm, idx = f0 * _fm_y(u, 2), f0 * _fm_y(u, 9), _fm_y(u, 10)
        t = np.arange(len(out)) / 44100.0
        want = sum(special.jv(k, idx) * np.sin(2 * math.pi * (fc + k * fm) * t)
                   for k in range(-30, 31))
        assert np.max(np.abs(out - want)) < 1e-9, b


def test_fm_carrier_alone_and_chain_order(oracle_mod):
    """Modulator levels 0 give the carrier's sine; a zero-level op1 cuts
    op2 and op3 off from the carrier (modulation flows only down the
    serial chain); the carrier's attack ramp scales it linearly."""
    cfg = oracle_mod.default_config(seconds=0.5)
    base = [(3.0, 0.75) + FLAT, (1.0, 0.0) + FLAT, (1.5, 7.0) + FLAT, (4.0, 6.0) + FLAT]
    out = oracle_mod.fm_render_voice(cfg, _fm_u(60.0, base))
    u = _fm_u(60.0, base)
    f = 440.0 * 2 ** ((_fm_y(u, 0) - 69.0) / 12.0) * _fm_y(u, 2)
    n = np.arange(len(out))
    assert np.max(np.abs(out - _fm_y(u, 3) * np.sin(2 * math.pi * np.mod(f * n / 44100.0, 1.0)))) < 1e-9
    ramp = [(3.0, 0.75, 1.0, 0.0, 1.0, 0.0, 1.0)] + base[1:]  # a 1 s attack: no kink in 0.5 s
    u2 = _fm_u(60.0, ramp)
    out2 = oracle_mod.fm_render_voice(cfg, u2)
    a = _fm_y(u2, 4)
    env = np.minimum(n / 44100.0 / a, 1.0)
    assert np.max(np.abs(out2 - env * _fm_y(u2, 3) * np.sin(2 * math.pi * np.mod(f * n / 44100.0, 1.0)))) < 1e-9


def test_fm_param_draw_stream(oracle_mod):
    """FM parameters are Philox stream 2 words: u = (w >> 8) / 2^24."""
    u = oracle_mod.fm_draw_params(7, 123)
    words = np.concatenate([oracle_mod.philox4x32_10([123, 0, b, 2], [7, 0]) for b in range(8)])
    assert np.array_equal(u, (words[:30] >> 8) / 2.0 ** 24)
