"""tcgen05 BF16 GEMM (the STFT/MLP contraction) against a plain PyTorch FP32
product of the same bf16 inputs, over tile-aligned, ragged and STFT-sized
shapes."""
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
                                   (1, 16, 8)])
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
    err = (c - ref).abs().max().item()
    assert err <= 1e-3 * (k ** 0.5) + 1e-4, err


def test_gemm_argument_errors(env):
    torch, pkg, syn = env
    L = pkg.lib()
    a = torch.zeros(16, 16, device="cuda", dtype=torch.bfloat16)
    c = torch.zeros(16, 16, device="cuda")
    assert L.synth_gemm_bf16(syn.handle, a.data_ptr(), 16, a.data_ptr(), 16, c.data_ptr(), 16,
                             16, 16, 12, 1.0, None) == pkg.SYNTH_ERR_ARG
    assert L.synth_gemm_bf16(syn.handle, None, 16, a.data_ptr(), 16, c.data_ptr(), 16,
                             16, 16, 16, 1.0, None) == pkg.SYNTH_ERR_ARG
