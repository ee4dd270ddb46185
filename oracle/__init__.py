"""FP64 CPU oracle for the batched Voice render -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference leg may import this package. It is the plain, slow reference that
the CUDA library is checked against; it shares no code with the library and
the library never imports it.

The C++ part (``voice.cpp``) renders voices in FP64 sample by sample. The
spectral parts (``spectral.py``) are plain PyTorch CPU ops in FP64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = [os.path.join(_HERE, "voice.cpp")]

NUM_PARAMS = 78
ROUND_PITCH_CHAIN_F32 = 1


def build(force: bool = False) -> str:
    """Compile liboracle.so with g++ (IEEE FP64: no fast-math, no FMA contraction)."""
    newest = max(os.path.getmtime(p) for p in _SRC + [os.path.join(_HERE, "oracle.h")])
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
           "-o", tmp] + _SRC + ["-lpthread"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _SO)
    return _SO


class Nebula(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * NUM_PARAMS), ("hi", ctypes.c_double * NUM_PARAMS),
                ("curve", ctypes.c_double * NUM_PARAMS), ("symmetric", ctypes.c_int32 * NUM_PARAMS)]


class Config(ctypes.Structure):
    _fields_ = [("sample_rate", ctypes.c_double), ("control_rate", ctypes.c_double),
                ("seconds", ctypes.c_double), ("nebula", Nebula)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.POINTER
        d, i32, u64 = ctypes.c_double, ctypes.c_int32, ctypes.c_uint64
        L.oracle_philox4x32_10.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
        L.oracle_default_nebula.argtypes = [P(Nebula)]
        L.oracle_default_config.argtypes = [P(Config)]
        L.oracle_draw_params.argtypes = [u64, u64, P(d)]
        L.oracle_range_map.argtypes = [d, d, d, d, i32]
        L.oracle_range_map.restype = d
        L.oracle_adsr.argtypes = [d] * 7
        L.oracle_adsr.restype = d
        L.oracle_lfo_shape.argtypes = [i32, d]
        L.oracle_lfo_shape.restype = d
        L.oracle_midi_to_hz.argtypes = [d]
        L.oracle_midi_to_hz.restype = d
        L.oracle_control.argtypes = [P(Config), P(d), P(d), P(d), P(d)]
        L.oracle_control.restype = i32
        L.oracle_lfo_phase.argtypes = [P(Config), P(d), P(d)]
        L.oracle_lfo_phase.restype = i32
        L.oracle_render_voice.argtypes = [P(Config), P(d), u64, u64, P(d)]
        L.oracle_render_voice.restype = i32
        L.oracle_render_voice_ex.argtypes = [P(Config), P(d), u64, u64, P(d), i32]
        L.oracle_render_voice_ex.restype = i32
        L.oracle_vco_phase.argtypes = [P(Config), P(d), i32, P(d)]
        L.oracle_vco_phase.restype = i32
        L.oracle_render_batch.argtypes = [P(Config), u64, u64, i32, P(d), P(ctypes.c_float),
                                          P(ctypes.c_float), i32, P(i32), i32]
        L.oracle_render_batch.restype = i32
        L.oracle_render_vjp.argtypes = [P(Config), P(d), u64, u64, P(d), P(d), i32]
        L.oracle_render_vjp.restype = i32
        L.oracle_hardware_threads.restype = i32
        L.oracle_fm_draw_params.argtypes = [u64, u64, P(d)]
        L.oracle_fm_render_voice.argtypes = [P(Config), P(d), P(d)]
        L.oracle_fm_render_voice.restype = i32
        L.oracle_fm_render_batch.argtypes = [P(Config), u64, u64, i32, P(d), P(ctypes.c_float),
                                             P(ctypes.c_float), i32]
        L.oracle_fm_render_batch.restype = i32
        _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def default_config(seconds: float = 4.0, sample_rate: float = 44100.0,
                   control_rate: float = 441.0, nebula: dict | None = None) -> Config:
    cfg = Config()
    lib().oracle_default_config(ctypes.byref(cfg))
    cfg.seconds, cfg.sample_rate, cfg.control_rate = seconds, sample_rate, control_rate
    if nebula is not None:
        set_nebula(cfg, nebula)
    return cfg


def set_nebula(cfg: Config, nebula: dict) -> None:
    for p in range(NUM_PARAMS):
        cfg.nebula.lo[p] = float(nebula["lo"][p])
        cfg.nebula.hi[p] = float(nebula["hi"][p])
        cfg.nebula.curve[p] = float(nebula["curve"][p])
        cfg.nebula.symmetric[p] = int(nebula["symmetric"][p])


def default_nebula() -> dict:
    nb = Nebula()
    lib().oracle_default_nebula(ctypes.byref(nb))
    return {"lo": np.array(nb.lo[:]), "hi": np.array(nb.hi[:]),
            "curve": np.array(nb.curve[:]), "symmetric": np.array(nb.symmetric[:], dtype=np.int32)}


def num_samples(cfg: Config) -> int:
    return int(round(cfg.seconds * cfg.sample_rate))


def rate_ratio(sample_rate: float, control_rate: float) -> tuple[int, int]:
    """R = SR / CR as A / B in lowest terms: an integer R, or, for a
    fractional R, integer rates in Hz (the only fractional ratios rendered)."""
    from fractions import Fraction
    r = sample_rate / control_rate
    if round(r) >= 1 and abs(r - round(r)) <= 1e-9:
        return int(round(r)), 1
    f = Fraction(int(round(sample_rate)), int(round(control_rate)))
    return f.numerator, f.denominator


def num_control_points(cfg: Config) -> int:
    """K + 1 points: K = floor((N - 1) B / A) + 1 intervals hold the samples."""
    a, b = rate_ratio(cfg.sample_rate, cfg.control_rate)
    return (num_samples(cfg) - 1) * b // a + 2


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32), _p(out, ctypes.c_uint32))
    return out


def draw_params(seed: int, g: int) -> np.ndarray:
    u = np.zeros(NUM_PARAMS)
    lib().oracle_draw_params(seed, g, _p(u, ctypes.c_double))
    return u


def range_map(u, lo, hi, curve, symmetric) -> float:
    return lib().oracle_range_map(float(u), float(lo), float(hi), float(curve), int(symmetric))


def adsr(t, attack, decay, sustain, release, alpha, d) -> float:
    return lib().oracle_adsr(float(t), float(attack), float(decay), float(sustain), float(release),
                             float(alpha), float(d))


def lfo_shape(shape: int, p: float) -> float:
    return lib().oracle_lfo_shape(int(shape), float(p))


def midi_to_hz(m: float) -> float:
    return lib().oracle_midi_to_hz(float(m))


def control(cfg: Config, u) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    P = num_control_points(cfg)
    u = np.ascontiguousarray(u, dtype=np.float64)
    env = np.zeros((6, P)); lfo = np.zeros((2, P)); dest = np.zeros((5, P))
    rc = lib().oracle_control(ctypes.byref(cfg), _p(u, ctypes.c_double), _p(env, ctypes.c_double),
                              _p(lfo, ctypes.c_double), _p(dest, ctypes.c_double))
    if rc != 0:
        raise ValueError("oracle_control: configuration not representable")
    return env, lfo, dest


def lfo_phase(cfg: Config, u) -> np.ndarray:
    """[2][K+1] LFO phases in cycles at the control points."""
    theta = np.zeros((2, num_control_points(cfg)))
    u = np.ascontiguousarray(u, dtype=np.float64)
    if lib().oracle_lfo_phase(ctypes.byref(cfg), _p(u, ctypes.c_double), _p(theta, ctypes.c_double)):
        raise ValueError("oracle_lfo_phase failed")
    return theta


def discontinuity_ties(cfg: Config, u, tol: float = 1e-9) -> np.ndarray:
    """Control points where an LFO phase sits within tol of a discontinuity of
    the square (0, 1/2) or saw shapes (0): there, two correct evaluations that
    round the running phase sum differently may take different sides."""
    th = lfo_phase(cfg, u)
    d0 = np.minimum(th, 1.0 - th)
    dh = np.abs(th - 0.5)
    near = (d0 < tol) | (dh < tol)
    # only a phase reached by adding nonzero increments can round either way
    moved = np.concatenate([np.zeros((2, 1), bool),
                            np.cumsum(np.diff(th, axis=1) != 0, axis=1) > 0], axis=1)
    return np.where((near & moved).any(axis=0))[0]


def render_voice(cfg: Config, u, seed: int, g: int, flags: int = 0) -> np.ndarray:
    out = np.zeros(num_samples(cfg))
    u = np.ascontiguousarray(u, dtype=np.float64)
    rc = lib().oracle_render_voice_ex(ctypes.byref(cfg), _p(u, ctypes.c_double), seed, g,
                                      _p(out, ctypes.c_double), flags)
    if rc != 0:
        raise ValueError("oracle_render_voice: configuration not representable")
    return out


FM_NUM_PARAMS = 30


def fm_draw_params(seed: int, g: int) -> np.ndarray:
    u = np.zeros(FM_NUM_PARAMS)
    lib().oracle_fm_draw_params(seed, g, _p(u, ctypes.c_double))
    return u


def fm_render_voice(cfg: Config, u) -> np.ndarray:
    """4-operator FM voice (the library's reading, see oracle.h), FP64."""
    out = np.zeros(num_samples(cfg))
    u = np.ascontiguousarray(u, dtype=np.float64)
    if lib().oracle_fm_render_voice(ctypes.byref(cfg), _p(u, ctypes.c_double),
                                    _p(out, ctypes.c_double)) != 0:
        raise ValueError("oracle_fm_render_voice: configuration not representable")
    return out


def fm_render_batch(cfg: Config, seed: int, batch_index: int, batch: int, u_in=None,
                    threads: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """FM audio [batch][N] float32 and normalized params [batch][30] float32."""
    N = num_samples(cfg)
    audio = np.zeros((batch, N), dtype=np.float32)
    params = np.zeros((batch, FM_NUM_PARAMS), dtype=np.float32)
    up = None
    if u_in is not None:
        u_in = np.ascontiguousarray(u_in, dtype=np.float64).reshape(batch, FM_NUM_PARAMS)
        up = _p(u_in, ctypes.c_double)
    if lib().oracle_fm_render_batch(ctypes.byref(cfg), seed, batch_index, batch, up,
                                    _p(audio, ctypes.c_float), _p(params, ctypes.c_float),
                                    threads) != 0:
        raise ValueError("oracle_fm_render_batch failed")
    return audio, params


def vco_phase(cfg: Config, u, vco: int) -> np.ndarray:
    out = np.zeros(num_samples(cfg))
    u = np.ascontiguousarray(u, dtype=np.float64)
    rc = lib().oracle_vco_phase(ctypes.byref(cfg), _p(u, ctypes.c_double), vco, _p(out, ctypes.c_double))
    if rc != 0:
        raise ValueError("oracle_vco_phase failed")
    return out


def render_batch(cfg: Config, seed: int, batch_index: int, batch: int, u_in=None,
                 threads: int = 0, voices=None) -> tuple[np.ndarray, np.ndarray]:
    """Audio [batch][N] float32 and normalized params [batch][78] float32.

    With ``voices`` only those voice slots are rendered (other rows stay 0)."""
    N = num_samples(cfg)
    audio = np.zeros((batch, N), dtype=np.float32)
    params = np.zeros((batch, NUM_PARAMS), dtype=np.float32)
    up = None
    if u_in is not None:
        u_in = np.ascontiguousarray(u_in, dtype=np.float64).reshape(batch, NUM_PARAMS)
        up = _p(u_in, ctypes.c_double)
    vp, nv = None, 0
    if voices is not None:
        va = np.ascontiguousarray(voices, dtype=np.int32)
        vp, nv = _p(va, ctypes.c_int32), len(va)
    rc = lib().oracle_render_batch(ctypes.byref(cfg), seed, batch_index, batch, up,
                                   _p(audio, ctypes.c_float), _p(params, ctypes.c_float), threads, vp, nv)
    if rc != 0:
        raise ValueError("oracle_render_batch failed")
    return audio, params


def render_vjp(cfg: Config, u, seed: int, g: int, w, threads: int = 0) -> np.ndarray:
    """sum_n w[n] d audio[n] / d u[p] for one voice (forward-mode dual numbers)."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    assert w.shape == (num_samples(cfg),)
    grad = np.zeros(NUM_PARAMS)
    rc = lib().oracle_render_vjp(ctypes.byref(cfg), _p(u, ctypes.c_double), seed, g,
                                 _p(w, ctypes.c_double), _p(grad, ctypes.c_double), threads)
    if rc != 0:
        raise ValueError("oracle_render_vjp failed")
    return grad


def peak_normalize(audio, threshold: float):
    """Per-voice peak normalisation with silence rejection, in FP64 -- the
    library's reading of a remedy for the nearly silent renders that Sec. 2
    expects from uniform parameter sampling: p = max_n |x[n]| per voice;
    a voice with p >= threshold (and p > 0) is divided by p, any other is
    left as it is and flagged silent. Returns (audio, peak, silent)."""
    a = np.array(audio, dtype=np.float64)
    peak = np.max(np.abs(a), axis=1) if a.shape[1] else np.zeros(a.shape[0])
    loud = (peak >= threshold) & (peak > 0.0)
    a[loud] = a[loud] / peak[loud, None]
    return a, peak, ~loud


def hardware_threads() -> int:
    return int(lib().oracle_hardware_threads())
