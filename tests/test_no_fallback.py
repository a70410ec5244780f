"""The product path has no CPU fallback: without a CUDA tensor, or without the
built library, every compute call raises instead of computing elsewhere.
(CPU only; the GPU tests exercise the same calls on a device.)"""
import os
import subprocess
import sys

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bm():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2609_00205_gb300 as m

    return m


def test_compute_calls_reject_host_tensors(bm):
    u = torch.zeros(9, 9, 9)
    buf = torch.zeros(1024, dtype=torch.uint8)
    calls = [
        lambda: bm.compress(u, 1e-2),
        lambda: bm.decompress(buf),
        lambda: bm.decompose(u),
        lambda: bm.recompose(torch.zeros(bm.coeff_count(u.shape)), u.shape),
        lambda: bm.stream_codes(buf),
        lambda: bm.huffman_encode(torch.zeros(64, dtype=torch.int16), 16),
        lambda: bm.compress_batch([u], [1e-2]),
    ]
    for f in calls:
        with pytest.raises(ValueError, match="CUDA device"):
            f()


def test_missing_library_raises():
    code = ("import torch, paper_2609_00205_gb300 as bm\n"
            "try:\n"
            "    bm.compress_bound((9, 9, 9))\n"
            "except RuntimeError as e:\n"
            "    print('raised', 'not built' in str(e))\n")
    env = dict(os.environ, BM_LIBRARY=os.path.join(ROOT, "_no_such_dir", "libbm.so"))
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-1000:]
    assert r.stdout.strip() == "raised True", r.stdout
