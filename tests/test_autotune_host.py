"""The tile autotuner's search space (gp_tile_candidates), host logic only: no GPU."""
import pytest


@pytest.fixture(scope="module")
def abi():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2407_03608_gb300 import abi
    return abi


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("precision,rs", [(1, 4), (0, 8)])
@pytest.mark.parametrize("width", [4, 7, 9, 11])
def test_candidates_are_tiles_the_kernels_accept(abi, d, precision, rs, width):
    C = 9
    c = abi.gp_tile_candidates(d, C, precision, width)
    assert c, (d, precision, width)
    assert c == sorted(c, reverse=True) and len(set(c)) == len(c)
    for t in c:
        assert t >= width - 1                      # a tile holds a point's support
        if d >= 2:
            assert (t * rs) % 16 == 0              # TMA boxes start on 16 bytes along x


def test_wider_kernels_leave_fewer_tiles(abi):
    prev = None
    for width in range(4, 17):
        c = abi.gp_tile_candidates(3, 10, 1, width)
        if prev is not None:
            assert set(c) <= set(prev)
        prev = c
    # width 16 in 3-D FP64: the staged interp block (31^3 doubles) never fits
    assert abi.gp_tile_candidates(3, 25, 0, 16) == []


def test_invalid_arguments_are_rejected(abi):
    for args in [(0, 9, 1, 9), (4, 9, 1, 9), (2, 0, 1, 9), (2, 33, 1, 9), (2, 9, 3, 9), (2, 9, 1, 1), (2, 9, 1, 17)]:
        with pytest.raises(abi.GPError) as e:
            abi.gp_tile_candidates(*args)
        assert e.value.status == abi.GP_EINVAL
    abi.gp_tile_candidates(2, 9, 1, 9)             # a valid call clears the thread's error message
    assert abi.LIB.gp_last_error() == b""
