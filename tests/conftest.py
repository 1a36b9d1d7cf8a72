import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: full-size workload")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle


def vb_from_dense_blocks(a: np.ndarray, sizes, drop_zero_blocks=True):
    """VBMat of a dense array under a square block partition (test helper)."""
    import oracle
    sizes = np.asarray(sizes, np.int32)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    bptr, bcol, voff, val = [0], [], [0], []
    for I in range(len(sizes)):
        for J in range(len(sizes)):
            blk = a[off[I]:off[I + 1], off[J]:off[J + 1]]
            if drop_zero_blocks and not blk.any():
                continue
            bcol.append(J)
            val.append(blk.ravel())
            voff.append(voff[-1] + blk.size)
        bptr.append(len(bcol))
    return oracle.VBMat(sizes.copy(), sizes.copy(), np.array(bptr, np.int64), np.array(bcol, np.int32),
                        np.array(voff, np.int64),
                        np.concatenate(val) if val else np.zeros(0))
