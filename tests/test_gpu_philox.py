"""The oracle's Philox4x32-10 against curand's device generator (an
independent implementation, called): after curand_init(seed, subsequence,
offset = 4 b) the first curand4() is Philox4x32-10 with key (seed_lo,
seed_hi) and counter (b_lo, b_hi, subsequence_lo, subsequence_hi).  This pins
counter words 2 and 3 (the draw domain and the rejection attempt), which the
host generator of the CPU test leaves at small values / zero."""
import ctypes as C
import os
import subprocess
import tempfile

import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def probe():
    out = os.path.join(tempfile.mkdtemp(), "philox_probe.so")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                           "-Xcompiler", "-fPIC", "-o", out, os.path.join(HERE, "curand_philox_probe.cu")])
    L = C.CDLL(out)
    L.philox_probe.argtypes = [C.c_ulonglong, C.c_ulonglong, C.c_ulonglong, C.POINTER(C.c_uint)]
    return L


def test_philox_matches_curand_device(probe):
    checked = 0
    for seed in (0, 7, 0x123456789ABCDEF0, 0xFFFFFFFFFFFFFFFF):
        for b in (0, 1, (1 << 33) + 9):
            for sub in (0, 1, 5, (3 << 32) + 2, 0xFFFFFFFFFFFFFFFF):
                out = (C.c_uint * 4)()
                assert probe.philox_probe(seed, sub, 4 * b, out) == 0
                ctr = [b & 0xFFFFFFFF, b >> 32, sub & 0xFFFFFFFF, sub >> 32]
                assert O.philox(ctr, [seed & 0xFFFFFFFF, seed >> 32]) == list(out), (seed, b, sub)
                checked += 1
    assert checked == 60
