"""Block staging at every row alignment.

The forward block kernel stages a block that lies inside the field with one
bulk copy per row, rounded out to 16-byte boundaries, and drops the leading
elements of each slot; blocks on the far faces take the element-wise copy.
Rows start at every element offset modulo 16 bytes when the innermost extent
is not a multiple of the elements in 16 bytes, and when the field's first
element is not 16-byte aligned.  These cases place the same field at every
element offset of an aligned allocation, with innermost extents of every
residue, and require streams and coefficients identical to the aligned copy's
and (for one offset per case) the oracle's parity.
"""
import numpy as np
import pytest
import torch

import fields

from _util import check_stream_parity

pytestmark = pytest.mark.gpu

DEV = "cuda:0"

# (shape, dtype, B, K, M): innermost extents 68 (= 4 blocks of 17), 69, 70, 71
# and 37, 38 (B = 9); several interior blocks each, ragged far faces
CASES = [
    ((40, 36, 68), np.float32, 17, 2, 1),
    ((40, 35, 69), np.float32, 17, 2, 2),
    ((37, 34, 70), np.float32, 17, 1, 1),
    ((35, 40, 71), np.float32, 17, 2, 1),
    ((30, 28, 37), np.float32, 9, 2, 2),
    ((28, 30, 38), np.float64, 9, 2, 1),
    ((27, 27, 37), np.float64, 9, 1, 2),
]


@pytest.fixture(scope="module")
def bm():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2609_00205_gb300 as m

    return m


def _at_offset(u, off):
    """u copied into a fresh allocation starting `off` elements past its
    (256-byte aligned) start."""
    n = u.numel()
    buf = torch.empty(n + 8, dtype=u.dtype, device=DEV)
    v = buf[off:off + n].view(u.shape)
    v.copy_(u)
    assert v.is_contiguous() and v.data_ptr() % 16 == (off * u.element_size()) % 16
    return v


@pytest.mark.parametrize("case", CASES, ids=["x".join(map(str, c[0])) + f"_{np.dtype(c[1]).name}_b{c[2]}k{c[3]}m{c[4]}"
                                              for c in CASES])
def test_streams_identical_at_every_offset(bm, case):
    shape, dt, B, K, M = case
    u_np = fields.power_law_grf(shape, exponent=-3.0, seed=11, dtype=torch.float64).numpy().astype(dt)
    u = torch.from_numpy(u_np).to(DEV)
    esz = np.dtype(dt).itemsize
    kw = dict(block=B, levels=K, global_levels=M)
    ref = bm.compress(u, 1e-3, **kw).cpu().numpy()
    cref = bm.decompose(u, **kw).cpu().numpy()
    check_stream_parity(bm, u_np, ref, 1e-3, "rel", B, K, M, label=f"staging_{shape}_{np.dtype(dt).name}")
    for off in range(1, 16 // esz):
        v = _at_offset(u, off)
        s = bm.compress(v, 1e-3, **kw).cpu().numpy()
        np.testing.assert_array_equal(s, ref)
        np.testing.assert_array_equal(bm.decompose(v, **kw).cpu().numpy(), cref)


_VARIANT_SCRIPT = r"""
import sys
import numpy as np
import torch
import fields
import paper_2609_00205_gb300 as bm
from test_gpu_staging import CASES, _at_offset
out = {}
for ci, (shape, dt, B, K, M) in enumerate(CASES):
    u = torch.from_numpy(fields.power_law_grf(shape, exponent=-3.0, seed=11, dtype=torch.float64).numpy().astype(dt)).to("cuda:0")
    kw = dict(block=B, levels=K, global_levels=M)
    for off in range(16 // np.dtype(dt).itemsize):
        v = _at_offset(u, off) if off else u
        out[f"s{ci}_{off}"] = bm.compress(v, 1e-3, **kw).cpu().numpy()
        out[f"c{ci}_{off}"] = bm.decompose(v, **kw).cpu().numpy()
np.savez(sys.argv[1], **out)
"""


def test_bulk_staging_build_option(bm, tmp_path):
    """The build with bulk-copy staging (one cp.async.bulk per row of an
    interior block, BM_FWD_BULK=1) gives the default build's streams and
    coefficients at every row alignment."""
    import os
    import subprocess
    import sys

    from paper_2609_00205_gb300 import _build

    lib = _build.build(out=str(tmp_path / "libbm_bulk.so"), defines=("BM_FWD_BULK=1",))
    here = os.path.dirname(os.path.abspath(__file__))
    env = dict(os.environ, BM_LIBRARY=lib,
               PYTHONPATH=os.pathsep.join([here, os.path.dirname(here), os.environ.get("PYTHONPATH", "")]))
    res = tmp_path / "bulk.npz"
    subprocess.run([sys.executable, "-c", _VARIANT_SCRIPT, str(res)], env=env, check=True, timeout=600)
    got = np.load(res)
    for ci, (shape, dt, B, K, M) in enumerate(CASES):
        u = torch.from_numpy(fields.power_law_grf(shape, exponent=-3.0, seed=11,
                                                  dtype=torch.float64).numpy().astype(dt)).to(DEV)
        kw = dict(block=B, levels=K, global_levels=M)
        ref = bm.compress(u, 1e-3, **kw).cpu().numpy()
        cref = bm.decompose(u, **kw).cpu().numpy()
        for off in range(16 // np.dtype(dt).itemsize):
            np.testing.assert_array_equal(got[f"s{ci}_{off}"], ref)
            np.testing.assert_array_equal(got[f"c{ci}_{off}"], cref)
