"""First launches from several host threads at once.

The persistent kernels' launch set-up (resident grid size, shared-memory
attribute) is kept per device and set up on first use under a lock. Four
threads of a fresh process, each with its own handle and stream, start the
MR-STFT distance, the log-mel features and the tensor-core GEMM at the same
moment; their results must equal the same calls made one at a time
afterwards, bit for bit (every kernel here sums in a fixed order).
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys, threading
sys.path.insert(0, sys.argv[1])
import torch
import paper_2104_12922_gb300 as pkg
B = 8
base = pkg.Synth(seconds=1.0, max_batch=B)
x, _ = base.render(1, 0, B)
y, _ = base.render(2, 1, B)
base.sync()
g = torch.Generator().manual_seed(5)
a = torch.randn(256, 512, generator=g).to(torch.bfloat16).cuda()
b = torch.randn(384, 512, generator=g).to(torch.bfloat16).cuda()
torch.cuda.synchronize()

def run(s, mr, pm, st):
    with torch.cuda.stream(st):
        loss, gx = mr(x, y, stream=st)
        f = pm.features(x, stream=st)
        c = torch.empty((256, 384), device="cuda")
        assert pkg.lib().synth_gemm_bf16(s.handle, a.data_ptr(), 512, b.data_ptr(), 512,
                                         c.data_ptr(), 384, 256, 384, 512, 1.0,
                                         st.cuda_stream) == 0
    st.synchronize()
    s.sync(st)
    return loss.clone(), gx.clone(), f.clone(), c.clone()

def setup():
    s = pkg.Synth(seconds=1.0, max_batch=B)
    return s, pkg.MRSTFT(s, B), pkg.ProposalModel(s, max_batch=B, seed=0), torch.cuda.Stream()

results = {}
errors = []
start = threading.Barrier(4)
def work(i):
    try:
        parts = setup()
        start.wait()
        results[i] = run(*parts)
    except Exception as e:
        errors.append(repr(e))
threads = [threading.Thread(target=work, args=(i,)) for i in range(4)]
for t in threads:
    t.start()
for t in threads:
    t.join()
assert not errors, errors
ref = run(*setup())
for i in range(4):
    for k, (got, want) in enumerate(zip(results[i], ref)):
        assert torch.equal(got, want), (i, k)
print("CONCURRENT-OK")
"""


def test_first_launches_from_several_threads():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_12922_gb300 import build as b
    b.build()
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "CONCURRENT-OK" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
