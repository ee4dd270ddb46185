"""Philox4x32-10 blocks from Triton's library implementation, run by Triton's
CPU interpreter in a child process (TRITON_INTERPRET must be set before Triton
is imported). Used only to pin the oracle's generator to an independent
implementation of the published algorithm."""
import json
import os
import subprocess
import sys

_CHILD = r'''
import json, os, sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def _blocks(c_ptr, out_ptr, seed, n: tl.constexpr):
    i = tl.arange(0, n)
    c0 = tl.load(c_ptr + 4 * i + 0)
    c1 = tl.load(c_ptr + 4 * i + 1)
    c2 = tl.load(c_ptr + 4 * i + 2)
    c3 = tl.load(c_ptr + 4 * i + 3)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + 4 * i + 0, a)
    tl.store(out_ptr + 4 * i + 1, b)
    tl.store(out_ptr + 4 * i + 2, c)
    tl.store(out_ptr + 4 * i + 3, d)

req = json.loads(sys.stdin.read())
res = []
for item in req:
    seed = int(item["seed"])
    ctrs = np.array(item["ctrs"], dtype=np.uint32).reshape(-1, 4)
    n = 1
    while n < len(ctrs):
        n *= 2
    buf = np.zeros((n, 4), dtype=np.uint32)
    buf[: len(ctrs)] = ctrs
    c = torch.from_numpy(buf.reshape(-1).view(np.int32).copy()).view(torch.uint32)
    o = torch.zeros(4 * n, dtype=torch.uint32)
    _blocks[(1,)](c, o, seed, n)
    res.append(o.view(torch.int32).numpy().view(np.uint32).reshape(n, 4)[: len(ctrs)].tolist())
print(json.dumps(res))
'''


def triton_philox(requests):
    """requests: list of {"seed": int64, "ctrs": [[c0,c1,c2,c3], ...]} ->
    list of [[w0,w1,w2,w3], ...]."""
    env = dict(os.environ)
    env["TRITON_INTERPRET"] = "1"
    out = subprocess.run([sys.executable, "-c", _CHILD], input=json.dumps(requests),
                         capture_output=True, text=True, env=env, timeout=600)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])
