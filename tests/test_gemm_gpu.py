"""tcgen05 BF16 GEMM (the STFT/MLP contraction) against a plain PyTorch FP32
product of the same bf16 inputs, element by element, over tile-aligned,
ragged and STFT-sized shapes. The last four have more output tiles than the
persistent grid has CTAs (160, 320, 144 ragged, 1,384 for the MLP's first
weight gradient 1024 x 44160 x 128): each CTA then walks several tiles and
alternates its two TMEM accumulators, the epilogue of one tile running while
the next accumulates."""
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
    syn = pkg.Synth(seconds=0.01, max_batch=1)
    yield torch, pkg, syn
    syn.close()


@pytest.mark.parametrize("m,n,k", [(128, 128, 64), (256, 512, 1024), (100, 200, 72),
                                   (130, 300, 2056), (345, 2050, 2048), (128, 78, 1024),
                                   (1, 16, 8), (640, 8192, 256), (1280, 8192, 64),
                                   (1100, 4000, 136), (1024, 44160, 128)])
def test_gemm_matches_torch(env, m, n, k):
    torch, pkg, syn = env
    g = torch.Generator(device="cuda").manual_seed(m * 7 + n * 3 + k)
    a = torch.randn(m, k, device="cuda", generator=g).to(torch.bfloat16)
    b = torch.randn(n, k, device="cuda", generator=g).to(torch.bfloat16)
    c = torch.full((m, n), float("nan"), device="cuda")
    st = pkg.lib().synth_gemm_bf16(syn.handle, a.data_ptr(), k, b.data_ptr(), k, c.data_ptr(), n,
                                   m, n, k, 1.0, torch.cuda.current_stream().cuda_stream)
    assert st == 0
    syn.sync()
    ref = a.float() @ b.float().T
    # bf16 x bf16 products are exact in FP32; each side adds k of them with
    # at most k roundings of 2^-23 (truncating or not) relative to the sum
    # of |terms|, so the two results differ by at most k 2^-22 sum |a b|
    bar = (a.float().abs() @ b.float().abs().T) * (k * 2.0 ** -22) + 1e-6
    assert not torch.isnan(c).any()
    over = ((c - ref).abs() > bar).sum().item()
    assert over == 0, (over, (c - ref).abs().max().item())


def test_gemm_argument_errors(env):
    torch, pkg, syn = env
    L = pkg.lib()
    a = torch.zeros(16, 16, device="cuda", dtype=torch.bfloat16)
    c = torch.zeros(16, 16, device="cuda")
    assert L.synth_gemm_bf16(syn.handle, a.data_ptr(), 16, a.data_ptr(), 16, c.data_ptr(), 16,
                             16, 16, 12, 1.0, None) == pkg.SYNTH_ERR_ARG
    assert L.synth_gemm_bf16(syn.handle, None, 16, a.data_ptr(), 16, c.data_ptr(), 16,
                             16, 16, 16, 1.0, None) == pkg.SYNTH_ERR_ARG


@pytest.mark.parametrize("m,n,k", [(128, 1024, 44160), (128, 1024, 1024), (128, 78, 1024),
                                   (16, 1024, 2816), (200, 300, 4104)])
def test_gemm_splitk_matches_torch(env, m, n, k):
    """Split-K: fewer output tiles than SMs, K cut into slices (37 slices of
    19 k-blocks for the proposal network's first layer, 128 x 1024 x 44160),
    partial products added in slice order by the reduction kernel. Element by
    element within the FP32 accumulation bound, and bit-identical on a
    second call (fixed summation order)."""
    torch, pkg, syn = env
    L = pkg.lib()
    g = torch.Generator(device="cuda").manual_seed(m + 5 * n + k)
    a = torch.randn(m, k, device="cuda", generator=g).to(torch.bfloat16)
    b = torch.randn(n, k, device="cuda", generator=g).to(torch.bfloat16)
    import ctypes
    nb = ctypes.c_size_t()
    assert L.synth_gemm_bf16_workspace_size(syn.handle, m, n, ctypes.byref(nb)) == 0
    ws = torch.empty(nb.value // 4 + 1, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    outs = []
    for _ in range(2):
        c = torch.full((m, n), float("nan"), device="cuda")
        assert L.synth_gemm_bf16_splitk(syn.handle, a.data_ptr(), k, b.data_ptr(), k, c.data_ptr(),
                                        n, m, n, k, 1.0, ws.data_ptr(), nb.value, st) == 0
        outs.append(c)
    syn.sync()
    ref = a.float() @ b.float().T
    bar = (a.float().abs() @ b.float().abs().T) * (k * 2.0 ** -22) + 1e-6
    assert not torch.isnan(outs[0]).any()
    over = ((outs[0] - ref).abs() > bar).sum().item()
    assert over == 0, (over, (outs[0] - ref).abs().max().item())
    assert torch.equal(outs[0], outs[1])
