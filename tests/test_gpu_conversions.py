"""The float64 <-> float32 conversions of the mixed-precision kernels (integer-pipe bit manipulation)
agree bit for bit with the hardware conversions: random patterns, ties, range edges, specials."""
import pytest

pytestmark = pytest.mark.gpu


def test_conversions_match_hardware():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_00706_gb300 import _lib, api
    _lib.build()
    for seed in (1, 2, 3):
        assert api.selftest_conversions(1 << 24, seed) == 0
