"""GB300 (sm_103a) batched Voice renderer -- Python binding of libsynth.so.

The binding only marshals arguments: every step of a render runs in the CUDA
kernels of ``libsynth.so`` (C ABI in ``include/synth.h``). PyTorch is used
for device memory and streams. There is no CPU fallback: if the library is not
built, importing the binding raises.

Paper: Turian et al., "One Billion Audio Sounds from GPU-enabled Modular
Synthesis" (DAFx 2021), Sec. 2-3.
"""
from __future__ import annotations

import ctypes
import os

NUM_PARAMS = 78
_HERE = os.path.dirname(os.path.abspath(__file__))
# SYNTH_CHECKED=1 in the environment selects, for the whole process, the
# bounds-checked build libsynth_checked.so (build.build(checks=True)).
LIB_PATH = os.path.join(_HERE, "libsynth_checked.so" if os.environ.get("SYNTH_CHECKED") == "1"
                        else "libsynth.so")

SYNTH_OK, SYNTH_ERR_ARG, SYNTH_ERR_CUDA, SYNTH_ERR_OOM = 0, 1, 2, 3
SYNTH_ERR_TIMEOUT, SYNTH_ERR_STATE, SYNTH_ERR_UNSUPPORTED, SYNTH_ERR_BOUNDS = 4, 5, 6, 7
SYNTH_CARRY_FIXED64, SYNTH_CARRY_FP32 = 0, 1
# Network input features = (log(mel + 1e-6) - FEATURE_SHIFT) / FEATURE_SCALE
# (the affine map synth_model_features applies; see include/synth.h).
FEATURE_SHIFT, FEATURE_SCALE = -2.5, 6.0


class SynthError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {synth_status_string(status)} (status {status})")
        self.status = status


class synth_nebula(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * NUM_PARAMS), ("hi", ctypes.c_double * NUM_PARAMS),
                ("curve", ctypes.c_double * NUM_PARAMS), ("symmetric", ctypes.c_int32 * NUM_PARAMS)]


class synth_config(ctypes.Structure):
    _fields_ = [("sample_rate", ctypes.c_double), ("control_rate", ctypes.c_double),
                ("seconds", ctypes.c_double), ("max_batch", ctypes.c_int32),
                ("carry", ctypes.c_int32), ("nebula", ctypes.POINTER(synth_nebula))]


_lib = None


def lib() -> ctypes.CDLL:
    """Loads libsynth.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                              "(the renderer has no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, u64, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64, ctypes.c_int64
        P = ctypes.POINTER
        L.synth_default_config.argtypes = [P(synth_config)]
        L.synth_default_config.restype = None
        L.synth_default_nebula.argtypes = [P(synth_nebula)]
        L.synth_default_nebula.restype = None
        L.synth_create.argtypes = [P(synth_config), P(vp)]
        L.synth_destroy.argtypes = [vp]
        L.synth_num_params.argtypes = [vp]
        L.synth_num_params.restype = i32
        L.synth_num_samples.argtypes = [vp]
        L.synth_num_samples.restype = i64
        L.synth_render.argtypes = [vp, u64, u64, i32, vp, vp, vp, vp]
        L.synth_render_normalized.argtypes = [vp, u64, u64, i32, vp, vp, vp, ctypes.c_float, vp,
                                              vp, vp]
        L.synth_render_plain_workspace_size.argtypes = [vp, i32, P(ctypes.c_size_t)]
        L.synth_render_plain.argtypes = [vp, u64, u64, i32, vp, vp, vp, vp, ctypes.c_size_t, vp]
        L.synth_render_backward_workspace_size.argtypes = [vp, i32, P(ctypes.c_size_t)]
        L.synth_render_backward.argtypes = [vp, u64, u64, i32, vp, vp, vp, vp, ctypes.c_size_t, vp]
        L.synth_gemm_bf16.argtypes = [vp, vp, i32, vp, i32, vp, i32, i32, i32, i32,
                                      ctypes.c_float, vp]
        L.synth_gemm_bf16.restype = ctypes.c_int
        L.synth_gemm_bf16_workspace_size.argtypes = [vp, i32, i32, P(ctypes.c_size_t)]
        L.synth_gemm_bf16_workspace_size.restype = ctypes.c_int
        L.synth_gemm_bf16_splitk.argtypes = [vp, vp, i32, vp, i32, vp, i32, i32, i32, i32,
                                             ctypes.c_float, vp, ctypes.c_size_t, vp]
        L.synth_gemm_bf16_splitk.restype = ctypes.c_int
        L.synth_mrstft_workspace_size.argtypes = [vp, i32, P(ctypes.c_size_t)]
        L.synth_mrstft.argtypes = [vp, vp, vp, i32, i32, vp, vp, vp, ctypes.c_size_t, vp]
        L.synth_param_adam.argtypes = [vp, vp, vp, vp, vp, i32, i32, ctypes.c_float, vp]
        L.synth_model_create.argtypes = [vp, i32, u64, P(vp)]
        L.synth_model_destroy.argtypes = [vp]
        L.synth_model_feature_dim.argtypes = [vp]
        L.synth_model_feature_dim.restype = i64
        L.synth_model_features.argtypes = [vp, vp, i32, vp, vp]
        L.synth_model_forward.argtypes = [vp, vp, i32, vp, vp]
        L.synth_model_train_features.argtypes = [vp, vp, vp, i32, ctypes.c_float, vp, vp]
        L.synth_model_train_step.argtypes = [vp, u64, u64, i32, ctypes.c_float, vp, vp]
        L.synth_propose.argtypes = [vp, vp, vp, i32, vp, vp]
        L.synth_model_get_tensor.argtypes = [vp, i32, i32, vp, ctypes.c_size_t, vp]
        L.synth_model_save.argtypes = [vp, ctypes.c_char_p]
        L.synth_model_load.argtypes = [vp, ctypes.c_char_p]
        for name in ("synth_mrstft_workspace_size", "synth_mrstft", "synth_param_adam",
                     "synth_model_create", "synth_model_destroy", "synth_model_features",
                     "synth_model_forward", "synth_model_train_features", "synth_model_train_step",
                     "synth_propose", "synth_model_get_tensor", "synth_model_save",
                     "synth_model_load", "synth_stream_features"):
            getattr(L, name).restype = ctypes.c_int
        L.synth_sync.argtypes = [vp, vp]
        L.synth_params_to_human.argtypes = [vp, vp, vp, i32]
        L.synth_is_test.argtypes = [u64]
        L.synth_is_test.restype = i32
        L.synth_render_batches.argtypes = [vp, u64, u64, u64, i32, i32, vp, vp, vp, vp]
        L.synth_render_batches.restype = ctypes.c_int
        L.synth_fm_render.argtypes = [vp, u64, u64, i32, vp, vp, vp, vp]
        L.synth_fm_render.restype = ctypes.c_int
        L.synth_split_voice.argtypes = [i32, u64]
        L.synth_split_voice.restype = u64
        L.synth_stream_features.argtypes = [vp, u64, i32, u64, ctypes.c_int64, i32, vp, vp, vp]
        L.synth_sfu_probe.argtypes = [i32, i32, i32, vp, P(i64), vp]
        L.synth_sfu_probe.restype = ctypes.c_int
        L.synth_l1_distances.argtypes = [vp, vp, i64, i32, i32, vp, vp]
        L.synth_l1_distances.restype = ctypes.c_int
        L.synth_mmd_trials.argtypes = [vp, vp, i32, vp, i32, vp, vp]
        L.synth_mmd_trials.restype = ctypes.c_int
        L.synth_selftest_wait_timeout.argtypes = [vp, vp]
        L.synth_selftest_wait_timeout.restype = ctypes.c_int
        L.synth_selftest_bounds.argtypes = [vp, vp]
        L.synth_selftest_bounds.restype = ctypes.c_int
        L.synth_checked_build.argtypes = []
        L.synth_checked_build.restype = i32
        L.synth_status_string.argtypes = [ctypes.c_int]
        L.synth_status_string.restype = ctypes.c_char_p
        for name in ("synth_create", "synth_destroy", "synth_render", "synth_render_normalized",
                     "synth_render_plain",
                     "synth_render_plain_workspace_size", "synth_sync", "synth_params_to_human",
                     "synth_render_backward", "synth_render_backward_workspace_size"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


# ---- thin wrappers with the C names -------------------------------------------
def synth_status_string(status: int) -> str:
    return lib().synth_status_string(int(status)).decode()


def _check(status: int, what: str) -> None:
    if status != SYNTH_OK:
        raise SynthError(status, what)


def synth_default_config() -> synth_config:
    cfg = synth_config()
    lib().synth_default_config(ctypes.byref(cfg))
    return cfg


def synth_default_nebula() -> synth_nebula:
    nb = synth_nebula()
    lib().synth_default_nebula(ctypes.byref(nb))
    return nb


def synth_create(cfg: synth_config) -> int:
    h = ctypes.c_void_p()
    _check(lib().synth_create(ctypes.byref(cfg), ctypes.byref(h)), "synth_create")
    return h.value


def synth_destroy(h: int) -> None:
    _check(lib().synth_destroy(h), "synth_destroy")


def synth_render(h, seed, batch_index, batch, params_in_ptr, audio_ptr, params_out_ptr, stream) -> int:
    return lib().synth_render(h, seed, batch_index, batch, params_in_ptr, audio_ptr, params_out_ptr,
                              stream)


def synth_render_plain(h, seed, batch_index, batch, params_in_ptr, audio_ptr, params_out_ptr,
                       workspace_ptr, workspace_bytes, stream) -> int:
    return lib().synth_render_plain(h, seed, batch_index, batch, params_in_ptr, audio_ptr,
                                    params_out_ptr, workspace_ptr, workspace_bytes, stream)


def synth_render_plain_workspace_size(h, batch) -> int:
    n = ctypes.c_size_t()
    _check(lib().synth_render_plain_workspace_size(h, batch, ctypes.byref(n)),
           "synth_render_plain_workspace_size")
    return n.value


def synth_render_backward_workspace_size(h, batch) -> int:
    n = ctypes.c_size_t()
    _check(lib().synth_render_backward_workspace_size(h, batch, ctypes.byref(n)),
           "synth_render_backward_workspace_size")
    return n.value


def synth_render_backward(h, seed, batch_index, batch, params_ptr, grad_audio_ptr, grad_params_ptr,
                          workspace_ptr, workspace_bytes, stream) -> int:
    return lib().synth_render_backward(h, seed, batch_index, batch, params_ptr, grad_audio_ptr,
                                       grad_params_ptr, workspace_ptr, workspace_bytes, stream)


def synth_sync(h, stream) -> int:
    return lib().synth_sync(h, stream)


def synth_is_test(g: int) -> bool:
    return bool(lib().synth_is_test(g))


SPLIT_ALL, SPLIT_TRAIN, SPLIT_TEST = 0, 1, 2
SFU_SIN, SFU_COS, SFU_EX2, SFU_RCP, SFU_LG2, SFU_TANH = 0, 1, 2, 3, 4, 5
FM_NUM_PARAMS = 30


def synth_split_voice(split: int, i: int) -> int:
    """Global voice index g of the i-th voice of a split (0 all, 1 train, 2 test)."""
    return int(lib().synth_split_voice(split, i))


def make_nebula(d: dict) -> synth_nebula:
    nb = synth_nebula()
    for p in range(NUM_PARAMS):
        nb.lo[p] = float(d["lo"][p])
        nb.hi[p] = float(d["hi"][p])
        nb.curve[p] = float(d["curve"][p])
        nb.symmetric[p] = int(d["symmetric"][p])
    return nb


def nebula_dict(nb: synth_nebula) -> dict:
    import numpy as np
    return {"lo": np.array(nb.lo[:]), "hi": np.array(nb.hi[:]), "curve": np.array(nb.curve[:]),
            "symmetric": np.array(nb.symmetric[:], dtype=np.int32)}


# ---- torch convenience layer ----------------------------------------------------
def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def _stream_ptr(stream) -> int | None:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Synth:
    """One renderer handle on the current CUDA device.

    ``render`` fills caller-visible torch tensors (float32, contiguous, on the
    handle's device) through the C ABI; nothing is computed in Python.
    """

    def __init__(self, seconds: float = 4.0, sample_rate: float = 44100.0,
                 control_rate: float = 441.0, max_batch: int = 128, carry: int = SYNTH_CARRY_FIXED64,
                 nebula: dict | None = None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Synth needs a CUDA device (there is no CPU fallback)")
        cfg = synth_default_config()
        cfg.sample_rate, cfg.control_rate, cfg.seconds = sample_rate, control_rate, seconds
        cfg.max_batch, cfg.carry = max_batch, carry
        self._nebula = make_nebula(nebula) if nebula is not None else None
        if self._nebula is not None:
            cfg.nebula = ctypes.pointer(self._nebula)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.handle = synth_create(cfg)
        self.max_batch = max_batch
        self.num_samples = int(lib().synth_num_samples(self.handle))
        self._workspace = None
        self._bwd_workspace = None

    def close(self) -> None:
        if getattr(self, "handle", None):
            synth_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check_tensor(self, t, shape, name):
        import torch
        if t is None:
            return
        if t.dtype != torch.float32 or not t.is_contiguous() or t.device != self.device:
            raise ValueError(f"{name} must be a contiguous float32 tensor on {self.device}")
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")

    def render(self, seed: int, batch_index: int, batch: int, params_in=None, out=None,
               params_out=None, stream=None, plain: bool = False):
        """Renders voices g = batch_index * batch + v; returns (audio, params)."""
        import torch
        if out is None:
            out = torch.empty((batch, self.num_samples), dtype=torch.float32, device=self.device)
        if params_out is None:
            params_out = torch.empty((batch, NUM_PARAMS), dtype=torch.float32, device=self.device)
        self._check_tensor(out, (batch, self.num_samples), "out")
        self._check_tensor(params_out, (batch, NUM_PARAMS), "params_out")
        self._check_tensor(params_in, (batch, NUM_PARAMS), "params_in")
        st = _stream_ptr(stream)
        if plain:
            need = synth_render_plain_workspace_size(self.handle, batch)
            if self._workspace is None or self._workspace.numel() < need:
                self._workspace = torch.empty(need, dtype=torch.uint8, device=self.device)
            status = synth_render_plain(self.handle, seed, batch_index, batch, _ptr(params_in),
                                        _ptr(out), _ptr(params_out), _ptr(self._workspace),
                                        self._workspace.numel(), st)
        else:
            status = synth_render(self.handle, seed, batch_index, batch, _ptr(params_in), _ptr(out),
                                  _ptr(params_out), st)
        _check(status, "synth_render_plain" if plain else "synth_render")
        return out, params_out

    def render_normalized(self, seed: int, batch_index: int, batch: int, threshold: float = 1e-3,
                          params_in=None, out=None, params_out=None, peak=None, silent=None,
                          stream=None):
        """Render with per-voice peak normalisation and silence rejection
        (synth_render_normalized); returns (audio, params, peak, silent)."""
        import torch
        if out is None:
            out = torch.empty((batch, self.num_samples), dtype=torch.float32, device=self.device)
        if params_out is None:
            params_out = torch.empty((batch, NUM_PARAMS), dtype=torch.float32, device=self.device)
        self._check_tensor(out, (batch, self.num_samples), "out")
        self._check_tensor(params_out, (batch, NUM_PARAMS), "params_out")
        self._check_tensor(params_in, (batch, NUM_PARAMS), "params_in")
        if peak is None:
            peak = torch.empty(batch, dtype=torch.float32, device=self.device)
        if silent is None:
            silent = torch.empty(batch, dtype=torch.int32, device=self.device)
        self._check_tensor(peak, (batch,), "peak")
        if silent.dtype != torch.int32 or not silent.is_contiguous() or tuple(silent.shape) != (batch,):
            raise ValueError(f"silent must be a contiguous int32 tensor of shape ({batch},)")
        status = lib().synth_render_normalized(self.handle, seed, batch_index, batch,
                                               _ptr(params_in), _ptr(out), _ptr(params_out),
                                               float(threshold), _ptr(peak), _ptr(silent),
                                               _stream_ptr(stream))
        _check(status, "synth_render_normalized")
        return out, params_out, peak, silent

    def render_batches(self, seed: int, seed_step: int, batch_index: int, batch: int, count: int,
                       params_in=None, out=None, params_out=None, stream=None):
        """`count` consecutive batches in one launch (synth_render_batches):
        batch k = render(seed + k seed_step, batch_index + k, batch); returns
        (audio [count * batch][N], params [count * batch][78])."""
        import torch
        total = batch * count
        if out is None:
            out = torch.empty((total, self.num_samples), dtype=torch.float32, device=self.device)
        if params_out is None:
            params_out = torch.empty((total, NUM_PARAMS), dtype=torch.float32, device=self.device)
        self._check_tensor(out, (total, self.num_samples), "out")
        self._check_tensor(params_out, (total, NUM_PARAMS), "params_out")
        self._check_tensor(params_in, (total, NUM_PARAMS), "params_in")
        _check(lib().synth_render_batches(self.handle, seed, seed_step, batch_index, batch, count,
                                          _ptr(params_in), _ptr(out), _ptr(params_out),
                                          _stream_ptr(stream)), "synth_render_batches")
        return out, params_out

    def fm_render(self, seed: int, batch_index: int, batch: int, params_in=None, out=None,
                  params_out=None, stream=None):
        """4-operator FM voices g = batch_index * batch + v (synth_fm_render);
        returns (audio, params [batch][30])."""
        import torch
        if out is None:
            out = torch.empty((batch, self.num_samples), dtype=torch.float32, device=self.device)
        if params_out is None:
            params_out = torch.empty((batch, FM_NUM_PARAMS), dtype=torch.float32, device=self.device)
        self._check_tensor(out, (batch, self.num_samples), "out")
        self._check_tensor(params_out, (batch, FM_NUM_PARAMS), "params_out")
        self._check_tensor(params_in, (batch, FM_NUM_PARAMS), "params_in")
        _check(lib().synth_fm_render(self.handle, seed, batch_index, batch, _ptr(params_in),
                                     _ptr(out), _ptr(params_out), _stream_ptr(stream)),
               "synth_fm_render")
        return out, params_out

    def sync(self, stream=None) -> None:
        _check(synth_sync(self.handle, _stream_ptr(stream)), "synth_sync")

    def backward(self, seed: int, batch_index: int, params, grad_audio, grad_params=None,
                 stream=None):
        """grad_params = (d audio / d u)^T grad_audio through the C-ABI adjoint."""
        import torch
        batch = params.shape[0]
        self._check_tensor(params, (batch, NUM_PARAMS), "params")
        self._check_tensor(grad_audio, (batch, self.num_samples), "grad_audio")
        if grad_params is None:
            grad_params = torch.empty((batch, NUM_PARAMS), dtype=torch.float32, device=self.device)
        self._check_tensor(grad_params, (batch, NUM_PARAMS), "grad_params")
        need = synth_render_backward_workspace_size(self.handle, batch)
        if self._bwd_workspace is None or self._bwd_workspace.numel() < need:
            self._bwd_workspace = torch.empty(need, dtype=torch.uint8, device=self.device)
        _check(synth_render_backward(self.handle, seed, batch_index, batch, _ptr(params),
                                     _ptr(grad_audio), _ptr(grad_params),
                                     _ptr(self._bwd_workspace), self._bwd_workspace.numel(),
                                     _stream_ptr(stream)), "synth_render_backward")
        return grad_params


def render_autograd(synth: "Synth", seed: int, batch_index: int, params):
    """Differentiable render: audio = Voice(params), with the hand-written
    adjoint as the backward (a torch.autograd.Function)."""
    import torch

    class _Render(torch.autograd.Function):
        @staticmethod
        def forward(ctx, u):
            u = u.detach().contiguous()
            audio, _ = synth.render(seed, batch_index, u.shape[0], params_in=u)
            ctx.save_for_backward(u)
            return audio

        @staticmethod
        def backward(ctx, grad_audio):
            (u,) = ctx.saved_tensors
            return synth.backward(seed, batch_index, u, grad_audio.contiguous())

    return _Render.apply(params)


# ---- spectral distance, refinement and the learned proposal -------------------
class MRSTFT:
    """Multi-resolution log-magnitude STFT distance on the tensor cores
    (synth_mrstft): per-voice loss and gradient w.r.t. x."""

    def __init__(self, synth: Synth, batch: int):
        import torch
        n = ctypes.c_size_t()
        _check(lib().synth_mrstft_workspace_size(synth.handle, batch, ctypes.byref(n)),
               "synth_mrstft_workspace_size")
        self.synth, self.batch = synth, batch
        self.ws = torch.empty(n.value, dtype=torch.uint8, device=synth.device)
        self.loss = torch.empty(batch, dtype=torch.float64, device=synth.device)

    def __call__(self, x, y, grad=True, target_ready=False, stream=None):
        import torch
        gx = torch.empty_like(x) if grad else None
        _check(lib().synth_mrstft(self.synth.handle, _ptr(x), _ptr(y), self.batch,
                                  1 if target_ready else 0, _ptr(self.loss), _ptr(gx),
                                  _ptr(self.ws), self.ws.numel(), _stream_ptr(stream)),
               "synth_mrstft")
        return self.loss, gx


def l1_distances(synth: Synth, emb, out=None, stream=None):
    """Pooled pairwise l1 distances [m][m] (FP32) of bf16 embeddings [m][dim]
    (synth_l1_distances)."""
    import torch
    m, dim = emb.shape
    if emb.dtype != torch.bfloat16 or emb.stride(1) != 1:
        raise ValueError("emb must be a bf16 tensor with contiguous rows")
    if out is None:
        out = torch.empty((m, m), dtype=torch.float32, device=emb.device)
    _check(lib().synth_l1_distances(synth.handle, _ptr(emb), emb.stride(0), m, dim, _ptr(out),
                                    _stream_ptr(stream)), "synth_l1_distances")
    return out


def mmd_trials(synth: Synth, dist, labels, out=None, stream=None):
    """One MMD per row of labels [trials][m] (int8: 0 in X, 1 in Y, else out)
    over the pooled distance matrix (synth_mmd_trials); FP64 [trials]."""
    import torch
    trials, m = labels.shape
    if labels.dtype != torch.int8 or not labels.is_contiguous():
        raise ValueError("labels must be a contiguous int8 tensor")
    if out is None:
        out = torch.empty(trials, dtype=torch.float64, device=dist.device)
    _check(lib().synth_mmd_trials(synth.handle, _ptr(dist), m, _ptr(labels), trials, _ptr(out),
                                  _stream_ptr(stream)), "synth_mmd_trials")
    return out


def param_adam(synth: Synth, u, grad, m, v, step: int, lr: float, stream=None) -> None:
    _check(lib().synth_param_adam(synth.handle, _ptr(u), _ptr(grad), _ptr(m), _ptr(v), u.numel(),
                                  step, lr, _stream_ptr(stream)), "synth_param_adam")


class ProposalModel:
    """Log-mel -> MLP -> sigmoid Voice parameters (synth_model_* calls)."""

    def __init__(self, synth: Synth, max_batch: int = 128, seed: int = 0):
        h = ctypes.c_void_p()
        _check(lib().synth_model_create(synth.handle, max_batch, seed, ctypes.byref(h)),
               "synth_model_create")
        self.synth, self.handle, self.max_batch = synth, h.value, max_batch
        self.feature_dim = int(lib().synth_model_feature_dim(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            lib().synth_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def features(self, audio, stream=None, out=None):
        import torch
        f = out if out is not None else torch.empty((audio.shape[0], self.feature_dim),
                                                    dtype=torch.bfloat16, device=audio.device)
        if f.dtype != torch.bfloat16 or not f.is_contiguous() or \
                tuple(f.shape) != (audio.shape[0], self.feature_dim):
            raise ValueError(f"out must be a contiguous bf16 tensor of shape "
                             f"({audio.shape[0]}, {self.feature_dim})")
        _check(lib().synth_model_features(self.handle, _ptr(audio), audio.shape[0], _ptr(f),
                                          _stream_ptr(stream)), "synth_model_features")
        return f

    def stream_features(self, seed: int, split: int, first: int, count: int, chunk: int = 0,
                        features=None, params=None, stream=None):
        """Features and parameters of voices g = synth_split_voice(split, first + i),
        i < count, rendered and transformed chunk by chunk
        (synth_stream_features); returns (features, params)."""
        import torch
        dev = self.synth.device
        if features is None:
            features = torch.empty((count, self.feature_dim), dtype=torch.bfloat16, device=dev)
        if params is None:
            params = torch.empty((count, NUM_PARAMS), dtype=torch.float32, device=dev)
        if features.dtype != torch.bfloat16 or not features.is_contiguous() or \
                tuple(features.shape) != (count, self.feature_dim):
            raise ValueError(f"features must be a contiguous bf16 tensor of shape "
                             f"({count}, {self.feature_dim})")
        self.synth._check_tensor(params, (count, NUM_PARAMS), "params")
        _check(lib().synth_stream_features(self.handle, seed, split, first, count, chunk,
                                           _ptr(features), _ptr(params), _stream_ptr(stream)),
               "synth_stream_features")
        return features, params

    def forward(self, feats, stream=None):
        import torch
        out = torch.empty((feats.shape[0], NUM_PARAMS), dtype=torch.float32, device=feats.device)
        _check(lib().synth_model_forward(self.handle, _ptr(feats), feats.shape[0], _ptr(out),
                                         _stream_ptr(stream)), "synth_model_forward")
        return out

    def train_features(self, feats, target, lr, loss=None, stream=None):
        _check(lib().synth_model_train_features(self.handle, _ptr(feats), _ptr(target),
                                                feats.shape[0], lr, _ptr(loss), _stream_ptr(stream)),
               "synth_model_train_features")

    def train_step(self, seed, batch_index, batch, lr, loss=None, stream=None):
        _check(lib().synth_model_train_step(self.handle, seed, batch_index, batch, lr, _ptr(loss),
                                            _stream_ptr(stream)), "synth_model_train_step")

    def propose(self, audio, stream=None):
        import torch
        out = torch.empty((audio.shape[0], NUM_PARAMS), dtype=torch.float32, device=audio.device)
        _check(lib().synth_propose(self.synth.handle, self.handle, _ptr(audio), audio.shape[0],
                                   _ptr(out), _stream_ptr(stream)), "synth_propose")
        return out

    def tensor(self, which: int, layer: int, batch: int | None = None):
        """which 0..3: weights, biases, weight / bias gradients of a layer;
        4: hidden activations H_layer [batch][1024] of the last call."""
        import torch
        dims = [self.feature_dim, 1024, 1024, 1024, NUM_PARAMS]
        if which == 4:
            shape = (batch, 1024)
        else:
            shape = (dims[layer + 1], dims[layer]) if which in (0, 2) else (dims[layer + 1],)
        t = torch.empty(shape, dtype=torch.float32, device=self.synth.device)
        _check(lib().synth_model_get_tensor(self.handle, which, layer, _ptr(t), t.numel(),
                                            _stream_ptr(None)), "synth_model_get_tensor")
        return t

    def save(self, path: str):
        _check(lib().synth_model_save(self.handle, path.encode()), "synth_model_save")

    def load(self, path: str):
        _check(lib().synth_model_load(self.handle, path.encode()), "synth_model_load")
