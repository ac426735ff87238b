"""The multi-block exclusive scan (Sec. IV-A) of the library, on the GPU:
the paper's worked example with four-element blocks, and random arrays
against numpy."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2004_13653_gb300 as kde  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "scan_example.txt")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    kde.load(build_if_stale=True)


def _golden():
    rows = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            k, *v = line.split()
            rows[k] = [int(x) for x in v]
    return rows


def test_paper_worked_example_two_blocks_of_four():
    g = _golden()
    x = torch.tensor(g["input"], dtype=torch.int32, device="cuda")
    got = kde.exclusive_scan(x, per_block=4).cpu().tolist()
    assert got == g["correct"]
    assert got[4:] != g["wrong1"]  # the propagation keeps block 0's last element


@pytest.mark.parametrize("n,per_block", [(1, 2048), (2047, 2048), (2048, 2048), (2049, 2048),
                                         (1000, 7), (5_000_001, 2048), (70_000, 4)])
def test_random_against_numpy(n, per_block):
    rng = np.random.default_rng(n)
    v = rng.integers(0, 50, n).astype(np.int32)
    got = kde.exclusive_scan(torch.as_tensor(v, device="cuda"), per_block=per_block).cpu().numpy()
    ref = np.concatenate([[0], np.cumsum(v, dtype=np.int64)[:-1]]).astype(np.int64)
    np.testing.assert_array_equal(got.astype(np.int64), ref)
