"""The division-free integer arithmetic of the kernels' work layout, checked exhaustively on the CPU.

The Householder passes deal columns to warps and split them into row segments.  Their index arithmetic
avoids hardware integer division (about 80 cycles of dependent latency on this GPU) with two tricks,
restated here from csrc/la.cuh and compared with exact integer division over every input the kernels
can produce:
- floor(32 / cw) for cw in [3, 16] from a packed table of nibbles;
- lane / S as floor((lane + 1/2) * rcp(S)) in single precision, where rcp is the approximate
  reciprocal of PTX rcp.approx.f32.  (lane + 1/2) / S lies at least 1/(2S) from an integer, and the
  approximation's relative error is far smaller, so any reciprocal within a few ulp gives the same
  floor.  The test perturbs the reciprocal by up to 4 ulp either way.
"""
import numpy as np

NIBBLES = 0x2222223344568A  # floor(32 / cw) for cw = 3 .. 16, cw = 3 in the lowest nibble


def floor32_over(cw):
    """la.cuh hh_layout: floor(32 / cw) for cw >= 1 (cw > 16 gives 1)."""
    if cw <= 2:
        return 32 >> min(max(cw - 1, 0), 1)
    if cw > 16:
        return 1
    return (NIBBLES >> (4 * min(max(cw - 3, 0), 13))) & 0xF


def test_nibble_table_is_floor_32_over_cw():
    for cw in range(1, 200):
        assert floor32_over(cw) == max(1, 32 // cw), cw


def _perturbed_reciprocals(d):
    r = np.float32(1.0) / np.float32(d)
    out = [r]
    up, dn = r, r
    for _ in range(4):
        up = np.nextafter(up, np.float32(np.inf))
        dn = np.nextafter(dn, np.float32(0.0))
        out += [up, dn]
    return out


def test_half_offset_reciprocal_floor_is_exact_for_lane_over_segments():
    # lc = lane / S for lane in [0, 32), S in [1, 32] (hh_layout, the look-up of a lane's column)
    for S in range(1, 33):
        for r in _perturbed_reciprocals(S):
            for lane in range(32):
                lc = int(np.float32(np.float32(lane) + np.float32(0.5)) * r)
                assert lc == lane // S, (lane, S, r)


def test_shift_form_of_columns_per_warp_for_power_of_two_teams():
    # hh_layout: cw = (cnt + nw - 1) >> log2(nw) for the 1, 2, 4 or 8 warps a team may have
    for nw in (1, 2, 4, 8):
        sh = nw.bit_length() - 1
        for cnt in range(0, 400):
            assert (cnt + nw - 1) >> sh == -(-cnt // nw)


def layout(cnt, nr, nw):
    """la.cuh hh_layout for every lane of a team: (cw, S, lc[lane], sg[lane])."""
    cw = (cnt + nw - 1) >> (nw.bit_length() - 1)
    S = min(floor32_over(cw), nr)
    lanes = np.arange(32)
    return cw, S, lanes // S, lanes - (lanes // S) * S


def test_balanced_layout_visits_every_column_row_pair_once():
    # the segmented form (S > 1): warp w owns columns [w cw, w cw + cw), lane (lc, sg) takes column
    # w cw + lc and rows sg, sg + S, ...; the per-lane form (S == 1): lane takes columns w cw + lane + 32 j
    for nw in (1, 2, 4, 8):
        for cnt in range(0, 170):
            for nr in (1, 2, 3, 4, 5, 7, 8, 12, 16, 17, 24, 31, 32, 33, 48):
                cw, S, lc, sg = layout(cnt, nr, nw)
                seen = np.zeros((cnt, nr), dtype=np.int64)
                for w in range(nw):
                    pw0, pw1 = w * cw, min(w * cw + cw, cnt)
                    if S > 1:
                        for lane in range(32):
                            p = pw0 + lc[lane]
                            if lc[lane] < cw and p < pw1:
                                seen[p, sg[lane]::S] += 1
                    else:
                        for lane in range(32):
                            for p in range(pw0 + lane, pw1, 32):
                                seen[p, :] += 1
                assert (seen == 1).all(), (nw, cnt, nr)


def seg_sum(acc, sg, S):
    """la.cuh seg_sum over a warp: shuffle-down tree, the segment's first lane receives the total."""
    acc = list(acc)
    o = 1
    while 2 * o < S:
        o *= 2
    while o > 0:
        t = [acc[l + o] if l + o < 32 else acc[l] for l in range(32)]  # __shfl_down_sync
        acc = [acc[l] + t[l] if sg[l] + o < S else acc[l] for l in range(32)]
        o >>= 1
    return acc


def test_segment_sums_reach_each_segment_first_lane():
    rng = np.random.default_rng(0)
    for S in range(2, 33):
        lanes = np.arange(32)
        sg = lanes % S
        vals = [int(v) for v in rng.integers(-1000, 1000, 32)]
        out = seg_sum(vals, sg, S)
        for g in range(32 // S):
            assert out[g * S] == sum(vals[g * S:(g + 1) * S]), (S, g)
