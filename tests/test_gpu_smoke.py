"""The entry point's smoke run (one staggered step of a 27 x 27 carpet in
FP64 and mixed precision against the oracle) passes on the GPU."""

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_smoke_runs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.smoke()
