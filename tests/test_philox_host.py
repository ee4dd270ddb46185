"""The render's noise generator in its split form (csrc/philox_noise.cuh),
built for the host with g++, against the oracle's plain Philox4x32-10
(Salmon et al., SC'11; the oracle's rounds are pinned to Triton's library
generator). The split form precomputes the key schedule and the two
products that the fixed counter words determine (Sec. 2.1 noise: counter
(g lo, g hi, block, stream)); every block must equal the plain rounds
bit for bit, including counters and keys at 0 and 2^32 - 1."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2104_12922_gb300", "csrc")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("phx") / "libphx.so")
    subprocess.run(["g++", "-O2", "-shared", "-fPIC", "-I", CSRC,
                    os.path.join(HERE, "philox_host_harness.cpp"), "-o", out], check=True)
    L = ctypes.CDLL(out)
    u32, pu = ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)
    L.h_philox_noise.argtypes = [u32, u32, u32, u32, u32, pu, ctypes.c_int, pu]
    return L


def split_blocks(lib, c0, c1, c3, k0, k1, qs):
    q = np.ascontiguousarray(qs, dtype=np.uint32)
    out = np.zeros((len(q), 4), dtype=np.uint32)
    lib.h_philox_noise(c0, c1, c3, k0, k1, q.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                       len(q), out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return out


def test_split_noise_philox_equals_plain_rounds(lib, oracle_mod):
    rng = np.random.default_rng(7)
    edge = [0, 1, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFF]
    cases = [(0, 0, 1, 0, 0), (0xFFFFFFFF, 0xFFFFFFFF, 1, 0xFFFFFFFF, 0xFFFFFFFF)]
    cases += [tuple(int(x) for x in rng.integers(0, 2**32, size=5, dtype=np.uint64))
              for _ in range(12)]
    for c0, c1, c3, k0, k1 in cases:
        qs = edge + [int(x) for x in rng.integers(0, 2**32, size=27, dtype=np.uint64)]
        got = split_blocks(lib, c0, c1, c3, k0, k1, qs)
        for q, row in zip(qs, got):
            ref = oracle_mod.philox4x32_10([c0, c1, q, c3], [k0, k1])
            assert np.array_equal(row, ref), (c0, c1, c3, k0, k1, q)


def test_split_noise_philox_voice_stream(lib, oracle_mod):
    """The render's own use: voice g = 0x1_0000_0005 of seed 2^40 + 3, stream 1,
    consecutive blocks from 0 (a tile's quads)."""
    g, seed = (1 << 32) + 5, (1 << 40) + 3
    c0, c1, k0, k1 = g & 0xFFFFFFFF, g >> 32, seed & 0xFFFFFFFF, seed >> 32
    qs = list(range(0, 64)) + [44099, 44100, 2**31]
    got = split_blocks(lib, c0, c1, 1, k0, k1, qs)
    for q, row in zip(qs, got):
        assert np.array_equal(row, oracle_mod.philox4x32_10([c0, c1, q, 1], [k0, k1]))
