"""GPU: the micro-update variant chosen by the autotuner (tile, velocity blocks per CTA) changes how work is
split over CTAs and lanes, not the arithmetic of any update, so every variant must give bitwise the same
iterate; pinning one must round-trip, and a variant a case cannot run must be refused."""
import numpy as np
import pytest

from paper_2605_03479_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SHAPES = [(4, 4), (4, 2), (2, 2), (8, 4)]
VARIANTS = [(4, 4, 1), (4, 2, 1), (2, 2, 1), (8, 4, 1), (4, 2, 2)]


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


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("implicit", [0, 1])
def test_every_variant_gives_the_same_iterate(hb, precision, implicit):
    # 9 x 7 cells, 16 x 16 velocities (two blocks per sign class, so the two-block variant can run in single
    # precision), N_H = 3: ragged tiles, walls inside partial tiles, both forms of the spectral source
    c = I.make_case("variant", 9, 16, kn=0.2, st=2.0, nh=3, pr=2 / 3, drive="thermal", amp=0.3, ncell_y=7,
                    precision=precision)
    c.spectral_implicit = implicit
    state = I.initial_state(c, seed=5)
    s = hb.Solver(c)
    assert s.micro_variant(0) in VARIANTS
    results = []
    for v in VARIANTS:
        try:
            s.set_micro_variant(0, *v)
        except hb.HbugksError:
            # FP64: two blocks per CTA is single precision only, and the 8 x 4 tile needs more shared memory
            # than a CTA may have at N_T = 7
            assert precision == 0 and v in ((4, 2, 2), (8, 4, 1))
            continue
        assert s.micro_variant(0) == v
        assert s.tile_shape(0) == v[:2]
        s.set_state(0, *state)
        s.iterate(5)
        results.append(s.get_state(0))
    assert len(results) == (5 if precision == 1 else 3)
    for other in results[1:]:
        for a, b in zip(results[0], other):
            assert np.array_equal(a, b)


def test_two_blocks_need_an_even_block_count_per_class(hb):
    # 10 x 10 velocities: 25 per sign class, one block each, so no CTA can take two blocks of one class
    c = I.make_case("odd", 6, 10, kn=0.1, st=1.0, nh=1, drive="shear", precision=1)
    s = hb.Solver(c)
    before = s.micro_variant(0)
    with pytest.raises(hb.HbugksError):
        s.set_micro_variant(0, 4, 2, 2)
    assert s.micro_variant(0) == before
    with pytest.raises(hb.HbugksError):
        s.set_micro_variant(0, 4, 4, 2)                 # not a variant at all


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
