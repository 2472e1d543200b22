"""The algorithmic byte and instruction counts behind bench.py's roofline object,
checked against the counts written out by hand from the kernels' data flow (no
GPU): the fraction the bench reports is these numbers divided by measured time,
so a wrong count would misstate it."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_single_order_bytes():
    # T_{m-1}, T_{m-2}, T_m and l (16 B each, FP64), K = 3 slots of index (4 B) and
    # real hopping (8 B), the diagonal (8 B): 64 + 36 + 8
    assert bench.bytes_per_orbital_cheb(3, True, True, 1) == 108
    # l = r rows drop the l stream
    assert bench.bytes_per_orbital_cheb(3, True, True, 1) - 16 == 92
    # two recurrences: A and B of three orders (6 x 16) + the same H~ bytes
    assert bench.bytes_per_orbital_pair(3, True, 1) == 140
    # FP32 storage, R = 32, cubic K = 6: 4 x 8 x 32 + 6 x (4 + 4) + 4 per site
    assert bench.bytes_per_orbital_cheb(6, False, True, 32) == 4 * 8 * 32 + 6 * 8 + 4


def test_blocked_bytes():
    # per chain T_m, T_{m-1} read and T_{m+1}, T_{m+2} written (4 x 16 B), H~ as
    # FP32 pairs without the index array: 3 real hoppings (8 B each) + diagonal (8 B)
    assert bench.bytes_per_orbital_tiled(3, True, True) == 2 * 64 + 24 + 8 == 160
    assert bench.bytes_per_orbital_tiled(3, True, False) == 64 + 24 + 8 == 96
    # one common hopping: no hop array at all
    assert bench.bytes_per_orbital_tiled(3, True, True, uniform=True) == 136
    assert bench.bytes_per_orbital_tiled(3, True, False, uniform=True) == 72
    # complex hoppings: 16 B per slot
    assert bench.bytes_per_orbital_tiled(3, False, True) == 128 + 48 + 8


def test_paired_fp32_instruction_counts():
    # one pair multiply-accumulate = 12 FP32-pipe instructions; a real-hop recurrence
    # is (1 diagonal + K neighbours) x (Re, Im) of them plus two 6-instruction
    # renormalisations; a Re dot is two of them
    rec = 12 * (2 * (1 + 3)) + 12
    assert bench.df_fp32_ops_per_orbital(3, True, "dbl") == rec + 48 == 156
    assert bench.df_fp32_ops_per_orbital(3, True, "pair") == 2 * rec + 48 == 264
    # one common hopping: K - 1 pair additions (8) and two multiply-accumulates per part
    rec_u = 2 * (8 * 2 + 2 * 12) + 12
    assert bench.df_fp32_ops_per_orbital(3, True, "pair", uniform=True) == 2 * rec_u + 48 == 232
    assert bench.df_fp32_ops_per_orbital(3, True, "dbl", uniform=True) == rec_u + 48 == 140


def test_fp64_fma_counts():
    # diagonal 2 + 3 neighbours x 2 real FMAs per recurrence; Re dot 2, l = r dots 4
    assert bench.fp64_fma_per_orbital(3, True, "re") == 10
    assert bench.fp64_fma_per_orbital(3, True, "dbl") == 12
    assert bench.fp64_fma_per_orbital(3, True, "pair") == 20


def test_measured_traffic_records():
    """A committed ncu record is used only while its kernel sources are unchanged,
    and then lies near the algorithmic bytes (gathers re-read from L2, not DRAM)."""
    n = 1 << 24
    for fam, alg in (("k_cheb2_honey_df_pair_uh", 136), ("k_cheb2_honey_df_dbl_uh", 72),
                     ("k_cheb2_honey_df_pair", 160), ("k_cheb_pair_df", 140)):
        t = bench.measured_traffic(fam, n)
        if t is not None:
            assert 0.85 * alg < t / n < 1.25 * alg, (fam, t / n)
    assert bench.measured_traffic("no_such_family", n) is None
