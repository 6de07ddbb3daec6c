"""Host-side checks (no GPU) of the exact update's plan, read through the C ABI
(hk_update_plan): the Karatsuba expansion and its (offset, sign) terms
reproduce the product exactly at every depth; the unit table covers every limb
product of every sub-contraction exactly once; and every shared-memory read of
every unit lands in its piece, the zero gaps around it, or the zero pads of the
stage -- never in a neighbouring piece -- and inside its block's operand
window.  These are the properties the update kernel's exactness rests on."""
import random

import numpy as np
import pytest

UNT = 256  # compute threads (units) per block of the update kernel


@pytest.fixture(scope="module")
def hk():
    from paper_0902_0852_gb300 import build, hk as mod
    build.build()
    return mod


def expand(a, W, plan):
    """Pieces of a (W limbs) in slot order: each level splits every piece of
    width w at the plan's split point into lo, hi and lo + hi."""
    cur = [(a, W)]
    splits = [[plan["m1"]], plan["m2"], plan["m3"], plan["m4"]]
    for lv in range(plan["levels"]):
        nxt = []
        for u, (x, w) in enumerate(cur):
            m = splits[lv][u]
            assert m == (w + 1) // 2
            lo, hi = x & ((1 << (32 * m)) - 1), x >> (32 * m)
            nxt += [(lo, m), (hi, w - m), (lo + hi, max(m, w - m) + 1)]
        cur = nxt
    return cur


@pytest.mark.parametrize("W", [5, 13, 41, 64, 176, 400, 804])
@pytest.mark.parametrize("levels", [0, 1, 2, 3, 4])
def test_karatsuba_terms_reproduce_the_product(hk, W, levels):
    plan = hk.hk_update_plan(W, levels, with_units=False)
    if W < 64:
        levels = min(levels, 3)  # four levels need a window of at least 64 limbs
    assert plan["levels"] == levels and plan["npieces"] == 3 ** levels
    rng = random.Random(W * 10 + levels)
    for trial in range(6):
        a, b = rng.getrandbits(32 * W), rng.getrandbits(32 * W)
        if trial == 0:
            a = b = (1 << (32 * W)) - 1  # longest carries in the lo + hi sums
        pa, pb = expand(a, W, plan), expand(b, W, plan)
        total = 0
        for k, ((x, wx), (y, _), (off, w), terms) in enumerate(zip(pa, pb, plan["pieces"], plan["terms"])):
            assert wx == w and x < 1 << (32 * w) and y < 1 << (32 * w)
            # two terms (lo.lo: 0 and -m; hi.hi: 2m and -m) per lo or hi digit of
            # the piece's base-3 path, one (+m) per lo+hi digit
            digits = [(k // 3 ** (levels - 1 - i)) % 3 for i in range(levels)]
            assert len(terms) == 2 ** sum(dg != 2 for dg in digits)
            for toff, sign in terms:
                total += sign * (x * y << (32 * toff))
        assert total == a * b


@pytest.mark.parametrize("W", [13, 176, 804])
@pytest.mark.parametrize("levels", [1, 2, 3, 4])
def test_piece_slots_are_separated_by_zero_gaps(hk, W, levels):
    plan = hk.hk_update_plan(W, levels, with_units=False)
    G = plan["gap"]
    end = 0
    for off, w in plan["pieces"]:
        assert off >= end + G and off % 4 == 0  # 16-byte aligned slots for the bulk copies
        end = off + (w + 3) // 4 * 4
    assert plan["stride"] >= end + G and plan["stride"] % 4 == 0


def _plans():
    return [(176, -1), (400, -1), (804, -1), (804, 2), (300, 0), (804, 4), (300, 4)]


@pytest.mark.parametrize("W,levels", _plans())
def test_units_cover_every_product_once(hk, W, levels):
    plan = hk.hk_update_plan(W, levels)
    uc, upc = plan["uc"], plan["upc"]
    assert upc % uc == 0
    widths = [w for _, w in plan["pieces"]] if plan["levels"] > 0 else [W]
    counts = [np.zeros((w + upc, 2 * w + uc), dtype=np.int32) for w in widths]
    for q, d0, p0, ln in plan["units"]:
        assert ln % uc == 0 and 0 < ln <= upc
        counts[q][p0:p0 + ln, d0:d0 + uc] += 1
    for w, c in zip(widths, counts):
        p = np.arange(w + upc)[:, None]
        d = np.arange(2 * w + uc)[None, :]
        valid = (p < w) & (d - p >= 0) & (d - p < w)
        assert (c[valid] == 1).all()


@pytest.mark.parametrize("W,levels", _plans())
def test_unit_reads_stay_in_gaps_and_windows(hk, W, levels):
    plan = hk.hk_update_plan(W, levels)
    uc, upc, G = plan["uc"], plan["upc"], plan["gap"]
    pieces = plan["pieces"] if plan["levels"] > 0 else [(0, W)]
    for u, (q, d0, p0, ln) in enumerate(plan["units"]):
        off, w = pieces[q]
        # X limbs p0 .. p0 + ln - 1, Y limbs d - p over the stripe and chunk
        xlo, xhi = p0, p0 + ln - 1
        ylo, yhi = d0 - (p0 + ln - 1), d0 + uc - 1 - p0
        assert 0 <= xlo < w
        if uc == 8:
            assert p0 % 4 == 0 and off % 4 == 0  # X read as aligned quads
        if plan["levels"] > 0:
            # past the piece only into its own zero gaps
            assert xhi < w + G and ylo >= -G and yhi < w + G
            if plan["nxb"]:
                wlo, wlen = plan["windows"][u // UNT]
                assert wlo <= off + xlo and off + xhi < wlo + wlen
                assert wlo <= off + ylo and off + yhi < wlo + wlen
        else:
            # whole entries staged: past the entry only into the stage's zero pads
            assert xhi < W + (upc + 3) // 4 * 4
            assert ylo >= -((uc + upc + 3) // 4 * 4) and yhi < W + (uc + 6) // 4 * 4


def test_automatic_depth_follows_the_cost_model(hk):
    # three levels once the pieces stay wide enough to fill the unit grid;
    # four only where three update blocks still fit an SM with the staged
    # windows of 81 pieces (the plan assumes a factorisation of at least 768
    # rows; smaller ones stop at three)
    assert hk.hk_update_plan(400, -1, with_units=False)["levels"] == 3
    assert hk.hk_update_plan(560, -1, with_units=False)["levels"] == 3
    assert hk.hk_update_plan(804, -1, with_units=False)["levels"] == 4
    # deeper levels only as the window widens
    depths = [hk.hk_update_plan(W, -1, with_units=False)["levels"] for W in (8, 40, 100, 176, 300, 400, 804, 1100)]
    assert depths == sorted(depths) and depths[0] == 0
    for W in (8, 64, 176, 804, 1200):
        plan = hk.hk_update_plan(W, -1, with_units=False)
        assert 0 <= plan["levels"] <= 4 and plan["C"] >= 2 * W


def test_plan_argument_checks(hk):
    from paper_0902_0852_gb300.hk import HKError
    for W, lv in [(0, -1), (100, 5), (100, -2)]:
        with pytest.raises(HKError):
            hk.hk_update_plan(W, lv, with_units=False)
