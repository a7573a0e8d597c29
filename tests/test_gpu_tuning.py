"""GPU: the micro-update tile chosen by the autotuner changes how work is split over CTAs, not the arithmetic of
any update, so every tile must give bitwise the same iterate; pinning a tile must round-trip."""
import numpy as np
import pytest

from paper_2605_03479_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SHAPES = [(4, 4), (4, 2), (2, 2), (8, 4)]


@pytest.fixture(scope="module")
def hb():
    from paper_2605_03479_gb300 import build, hbugks
    build.build()
    return hbugks


@pytest.mark.parametrize("precision", [0, 1])
def test_every_tile_gives_the_same_iterate(hb, precision):
    # 9 x 7 cells: ragged tiles for every shape, both walls of each axis inside partial tiles
    c = I.make_case("tile", 9, 10, kn=0.2, st=2.0, nh=2, pr=2 / 3, drive="thermal", amp=0.3, ncell_y=7,
                    precision=precision)
    state = I.initial_state(c, seed=7)
    s = hb.Solver(c)
    assert s.tile_shape(0) in SHAPES
    results = []
    for tx, ty in SHAPES:
        try:
            s.set_tile_shape(0, tx, ty)
        except hb.HbugksError:
            continue                     # the tile needs more shared memory than a CTA may have
        assert s.tile_shape(0) == (tx, ty)
        s.set_state(0, *state)
        s.iterate(6)
        results.append(s.get_state(0))
    assert len(results) >= 3
    for other in results[1:]:
        for a, b in zip(results[0], other):
            assert np.array_equal(a, b)


def test_unknown_tile_is_rejected(hb):
    c = I.make_case("bad", 6, 8, kn=0.1, st=1.0, nh=1, drive="shear")
    s = hb.Solver(c)
    before = s.tile_shape(0)
    with pytest.raises(hb.HbugksError):
        s.set_tile_shape(0, 3, 3)
    assert s.tile_shape(0) == before


def test_tuned_tile_is_reused_for_the_same_case(hb):
    c = I.make_case("same", 12, 12, kn=0.1, st=1.0, nh=3, pr=2 / 3, drive="thermal", precision=1)
    a = hb.Solver(c)
    b = hb.Solver(c)
    assert a.tile_shape(0) == b.tile_shape(0)
