"""The bench's roofline model (host logic, no GPU): pass-model bytes and pruned flops per stage.

The HBM roofline divides what each stage must move through HBM (read its input, write its output,
and for the middle stage read the symbol once) by its measured duration.  These checks fix the counts
of small cases by hand.
"""
import bench


def test_stage_bytes_2d_by_hand():
    # n = (3, 5), P = (8, 16): H1 = 5 row-spectrum bins, S1 holds 5 x 5 complex values
    eb = 8
    sb = bench.stage_bytes(2, (3, 5), (8, 16), eb)
    s1 = 5 * 5 * 2 * eb
    assert sb[0] == 15 * eb + s1                       # read u, write S1
    assert sb[1] == 2 * s1 + 5 * 9 * eb                # read + write S1, read the 5 x 9 symbol octant
    assert sb[2] == s1 + 15 * eb                       # read S1, write y
    # per unknown at 2047^2 in FP64: the 88 B/unknown pass model
    sb = bench.stage_bytes(2, (2047, 2047), (4096, 4096), 8)
    assert abs(sum(sb) / 2047 ** 2 - 88) < 0.2


def test_stage_bytes_3d_by_hand():
    eb = 4
    sb = bench.stage_bytes(3, (3, 5, 7), (8, 16, 16), eb)
    s1 = 5 * 5 * 7 * 2 * eb
    s2 = 5 * 16 * 7 * 2 * eb
    lam = 5 * 9 * 9 * eb
    assert sb == [105 * eb + s1, s1 + s2, 2 * s2 + lam, s2 + s1, s1 + 105 * eb]
    sb = bench.stage_bytes(3, (255, 255, 255), (512, 512, 512), 8)
    assert abs(sum(sb) / 255 ** 3 - 217) < 2.0


def test_pruned_flops_by_hand():
    # a transform of 16 points with half its input zero: 4 radix-2 stages, one trivial
    assert bench.pruned_fft_flops(16) == 5 * 16 * 3
    # a row of P_x = 32 real points: a half-length (16-point) pruned transform and 17 split bins
    assert bench.row_flops(32) == 5 * 16 * 3 + 6 * 17
    # a middle-stage line of 16 points: two pruned transforms and the symbol product
    assert bench.colmul_flops(16) == 2 * 240 + 32
    f = bench.stage_flops(2, (15, 15), (32, 16))
    assert f == [15 * bench.row_flops(32), 17 * bench.colmul_flops(16), 15 * bench.row_flops(32)]
