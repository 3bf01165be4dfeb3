"""The chunk-level scan schedules of the CUDA path, restated and checked on the CPU for every chunk count.

csrc/api.cu launches the relation and cost-relation scans (k_rel_level, k_lqr_level) as radix-2
Kogge-Stone levels d = 1, 2, 4, ... while d < maxnch + 1, and the affine chains (k_aff_level) as radix-4
levels d = 1, 4, 16, ...; the level count is set by the longest problem of a group.  Each problem has
slots 0..nch: its chunks and one boundary element.  Elements here are exact (index tuples under
concatenation, integer affine maps), so every check is exact.
"""
import math

import pytest


def suffix_scan(nchs):
    """k_rel_level / k_lqr_level: slot t <- slot t o slot t + d when chunk c + d <= nch, else copied."""
    maxnch = max(nchs)
    levels = math.ceil(math.log2(maxnch + 1)) if maxnch > 0 else 0
    out = []
    for nch in nchs:
        cur = [(c,) for c in range(nch + 1)]  # slot nch: the terminal element
        for k in range(levels):
            d = 1 << k
            cur = [cur[c] + cur[c + d] if c + d <= nch else cur[c] for c in range(nch + 1)]
        out.append(cur)
    return out


@pytest.mark.parametrize("nchs", [[n] for n in range(1, 130)] + [[1, 7, 64], [3, 1, 1, 200], [147], [1024]])
def test_radix2_suffix_levels_leave_every_slot_its_suffix(nchs):
    for nch, slots in zip(nchs, suffix_scan(nchs)):
        for c in range(nch + 1):
            assert slots[c] == tuple(range(c, nch + 1)), (nch, c)


def compose(f, g):
    """f after g for affine maps y -> a y + b."""
    return (f[0] * g[0], f[0] * g[1] + f[1])


def affine_scan(maps, v, fwd):
    """k_aff_level over one problem's slots: values are ('v', y), maps ('m', (a, b)).
    Forward: slot 0 holds y_0, slot j the map of chunk j - 1.  Backward: slot nch holds y_N, slot j the
    map of chunk j.  Radix-4 levels d = 1, 4, 16, ... while d < nch + 1."""
    nch = len(maps)
    cur = ([("v", v)] + [("m", m) for m in maps]) if fwd else ([("m", m) for m in maps] + [("v", v)])
    d = 1
    while d < nch + 1:
        nxt = []
        for j in range(nch + 1):
            acc = cur[j]
            for q in (1, 2, 3):
                if acc[0] == "v":
                    break
                j2 = j - q * d if fwd else j + q * d
                if j2 < 0 or j2 > nch:
                    break
                oth = cur[j2]
                if oth[0] == "v":
                    acc = ("v", acc[1][0] * oth[1] + acc[1][1])
                else:
                    acc = ("m", compose(acc[1], oth[1]))
            nxt.append(acc)
        cur = nxt
        d *= 4
    return cur


@pytest.mark.parametrize("nch", list(range(1, 90)) + [147, 255, 256, 257, 1024])
@pytest.mark.parametrize("fwd", [True, False])
def test_radix4_affine_levels_give_every_slot_its_boundary_value(nch, fwd):
    maps = [(2 + (j % 3), (-1) ** j * (j + 1)) for j in range(nch)]
    v = 5
    cur = affine_scan(maps, v, fwd)
    # sequential chain: forward y_{j+1} = map_j(y_j) from y_0; backward y_j = map_j(y_{j+1}) from y_nch
    y = [None] * (nch + 1)
    if fwd:
        y[0] = v
        for j in range(nch):
            y[j + 1] = maps[j][0] * y[j] + maps[j][1]
    else:
        y[nch] = v
        for j in range(nch - 1, -1, -1):
            y[j] = maps[j][0] * y[j + 1] + maps[j][1]
    for j in range(nch + 1):
        assert cur[j] == ("v", y[j]), (nch, fwd, j)


@pytest.mark.parametrize("fwd", [True, False])
def test_single_chunk_keeps_its_boundary_value(fwd):
    """A problem that fits one chunk: k_aff_up leaves its chunk slot an empty map, and the level keeps the
    boundary slot that k_aff_down reads (forward slot 0, backward slot 1) unchanged."""
    cur = affine_scan([(0, 0)], 7, fwd)
    assert cur[0 if fwd else 1] == ("v", 7)
