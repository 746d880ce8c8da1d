"""The bench's double-float roofline model (host logic, no GPU).

The peak of a double-float kernel is the FP32 issue rate over the FP32 instructions its butterflies
take per FP64-equivalent flop.  These checks fix the counts of the smallest transforms by hand, from the
operation costs (add 11, add without renormalisation 8, multiply 7, lazy complex product 32).
"""
import math

import bench


def test_dft_building_blocks():
    assert bench.DF_DFT4 == 4 * 2 * 8 + 4 * 2 * 11 == 152
    assert bench.DF_DFT16 == 8 * 152 + 8 * 32 == 1472
    assert bench.DF_DFT16_ZIN == 4 * 88 + 4 * 152 + 8 * 32 == 1216
    assert bench.DF_DFT8 == 2 * 152 + 72 + 176 == 552
    assert bench.DF_DFT8_ZIN == 176 + 72 + 176 == 424


def test_transform_counts_by_hand():
    # L = 16: one radix-16 butterfly, no stage twiddles
    assert bench.df_fft_instr(16, False) == 1472
    assert bench.df_fft_instr(16, True) == 1216
    # L = 32: two radix-16 butterflies, then 16 radix-2 butterflies with one twiddle product each
    assert bench.df_fft_instr(32, False) == 2 * 1472 + 16 * (32 + 44)
    # L = 64: radix-16 then radix-4 (3 twiddle products and one length-4 DFT per butterfly)
    assert bench.df_fft_instr(64, False) == 4 * 1472 + 16 * (96 + 152)
    # L = 128: radix-8 first, then one radix-16 stage with 15 stage twiddles per butterfly
    assert bench.df_fft_instr(128, True) == 16 * 424 + 8 * (1472 + 480)
    # L = 256: two radix-16 stages
    assert bench.df_fft_instr(256, False) == 16 * 1472 + 16 * (1472 + 480)


def test_instructions_per_flop_in_range():
    # a radix-16 butterfly with stage twiddles: 1952 instructions for 5 * 16 * 4 = 320 flops
    for P in [(4096, 4096), (512, 512, 512), (1024, 2048)]:
        r = bench.df64_instr_per_flop("colmul", P)
        assert 5.0 < r < 1952 / 320 + 0.5, (P, r)
    assert bench.df64_instr_per_flop("colmul", (4096, 4096)) == (
        bench.df_fft_instr(4096, True) + bench.df_fft_instr(4096, False) + 14 * 4096) / (10 * 4096 * 12 + 2 * 4096)
    peak = bench.FP32_ISSUE / bench.df64_instr_per_flop("colmul", (4096, 4096)) / 1e12
    assert 7.0 < peak < 7.6
    assert math.isclose(bench.FP32_ISSUE, 152 * 128 * 2.07e9)
