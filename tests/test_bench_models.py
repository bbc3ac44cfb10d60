"""Host-side models of bench.py that feed the reported rooflines: the
algorithmic bytes of one gs_bin_sort and the pass counts of the two radix
sorts, checked on small hand-worked cases (no GPU)."""
import bench


def test_bin_sort_bytes_hand_worked_tight_plain():
    # 10 item slots, 6 visible items, 20 pairs, 4 tiles, 2 pair passes, tight
    # support (row tables: 16 B each), 3 depth passes
    #   pair count  10*4 + 6*(8 + 24 + 4 + 16 + 16 + 4)   = 472
    #   depth sort  10*8 + 6*8 + 2*6*20                   = 368
    #   offsets     6*(4 + 4 + 4 + 4 + 4)                 = 120
    #   emit        6*(4 + 4 + 4 + 16 + 16) + 8*20        = 424
    #   pair sort   2*20*20                               = 800
    #   ranges      4*20 + 16*4                           = 144
    assert bench.bin_sort_bytes(10, 6, 20, 4, 2, tight=True, fov=False, depth_passes=3) == 2328


def test_bin_sort_bytes_without_filters_has_no_row_tables():
    # no tight support, no foveation: no support reads, no row tables
    #   pair count  10*4 + 6*(8 + 4 + 16 + 4) = 232; depth 10*8 + 6*8 + 6*20 = 248
    #   offsets 120; emit 6*28 + 160 = 328; pair sort 800; ranges 144
    assert bench.bin_sort_bytes(10, 6, 20, 4, 2, tight=False, fov=False, depth_passes=2) == 1872
    # the foveation filter alone adds the row tables (16 B written, 16 B read)
    assert (bench.bin_sort_bytes(10, 6, 20, 4, 2, tight=False, fov=True, depth_passes=2)
            - bench.bin_sort_bytes(10, 6, 20, 4, 2, tight=False, fov=False, depth_passes=2)
            == 6 * 16 * 2)


def test_pair_passes_follow_the_tile_id_bits():
    # 1920x1080 with 16x16 tiles: 120 x 68 = 8160 tiles, ids below 2^13
    assert bench.pair_passes(8160) == 2            # balanced digits of at most 8 bits
    assert bench.pair_passes(8160, 7) == 2
    assert bench.pair_passes(8160, 5) == 3
    # a 64-view batch of ~350k tiles: 19 bits
    assert bench.pair_passes(350_000) == 3
    assert bench.pair_passes(350_000, 10) == 2
    # one tile: one pass; the histogram storage caps the count at four
    assert bench.pair_passes(1) == 1
    assert bench.pair_passes(1 << 20, 4) == 4
