"""Host-side layout of the one-launch network (no GPU): the packed image's
size and the sizes the kernel refuses."""
import pytest

from paper_2207_06908_gb300 import _lib, mlp


def expected_bytes(sizes):
    """per layer, four cluster ranks each holding ceil(n / 4) output rows
    rounded up to 16, by the layer's inputs rounded up to 16, in BF16"""
    total = 0
    for k, n in zip(sizes[:-1], sizes[1:]):
        ns = ((n + 3) // 4 + 15) // 16 * 16
        total += 4 * ns * ((k + 15) // 16 * 16) * 2
    return total


@pytest.mark.parametrize("sizes", [[6, 256, 256, 256, 512], [6, 64, 64, 1], [13, 100, 37, 5], [256, 256],
                                   [24, 48, 200, 96, 64, 32, 16]])
def test_pack_bytes(sizes):
    assert mlp.net_pack_bytes(sizes) == expected_bytes(sizes)


@pytest.mark.parametrize("sizes", [[6, 512, 8],                  # a layer input above 256
                                   [6] * 8,                      # seven layers
                                   [6, 0, 4],                    # an empty layer
                                   [6, 1040],                    # a rank's output slice above one MMA's N
                                   [256, 256, 256, 256, 1024]])  # weight slices beyond shared memory
def test_pack_bytes_rejects(sizes):
    with pytest.raises(_lib.FdtdError):
        mlp.net_pack_bytes(sizes)
