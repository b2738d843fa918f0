"""Pins for the oracle's order / pack / select steps (Sec. 4.1-4.3)."""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2502_17712_gb300 import scenes as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_golden_worked_packings():
    g = json.load(open(os.path.join(GOLD, "pack_worked.json")))
    for case in g["cases"]:
        wh = np.array(case["boxes_wh"], np.uint32)
        fa, fb = wh[:, 0] * 256, wh[:, 1] * 256
        order = O.order(fb)
        assert (order == np.arange(len(wh))).all()  # listed tallest first
        r = O.pack_candidate(fa, fb, order, case["atlas_log2"], 1, n_scales=1,
                             min_box=case["min_box"])
        e = case["expected"]
        assert r["accepted"] == e["accepted"], case["name"]
        assert r["omega"] == e["omega"] and r["height"] == e["height"], case["name"]
        assert r["x"].tolist() == e["x"] and r["y"].tolist() == e["y"], case["name"]
        pk = O.pack(fa, fb, case["atlas_log2"], n_scales=1, min_box=case["min_box"])
        assert pk.status == (0 if e["accepted"] else 4)


def test_order_is_lexicographic_height_desc_index_asc():
    rng = np.random.default_rng(0)
    fb = rng.integers(1, 256 * 40, size=500).astype(np.uint32)
    fb[::7] = 0  # h0 clamps up to 1
    fb[::11] = 256 * 9000  # clamps down to 8192
    want = sorted(range(500), key=lambda c: (-min(max(math.ceil(int(fb[c]) / 256), 1), 8192), c))
    assert O.order(fb).tolist() == want


# ---------------------------------------------------------------- independent restatement


def restated_candidate(fa, fb, atlas_log2, k, n, min_box=2, gutter=0):
    """Fold with a running cursor and push by pairwise overlap (no frontline array):
    a box rests on the highest top among boxes of earlier rows that share an x."""
    om = 1 << atlas_log2
    order = sorted(range(len(fa)), key=lambda c: (-min(max(-(-int(fb[c]) // 256), 1), 8192), c))
    D = 256 * n
    boxes = []
    cursor = 0
    for c in order:
        w = max(-(-k * int(fa[c]) // D), min_box) + 2 * gutter
        h = max(-(-k * int(fb[c]) // D), min_box) + 2 * gutter
        boxes.append(dict(c=c, w=w, h=h, row=cursor // om, off=cursor % om))
        cursor += w
    m = max([0] + [b["off"] + b["w"] - om for b in boxes])
    Om = om + m
    for b in boxes:
        b["x"] = b["off"] if b["row"] % 3 == 0 else Om - b["off"] - b["w"]
    for b in boxes:
        below = [a["y"] + a["h"] for a in boxes if a["row"] < b["row"] and "y" in a
                 and a["x"] < b["x"] + b["w"] and b["x"] < a["x"] + a["w"]]
        b["y"] = max(below, default=0)
    H = max([0] + [b["y"] + b["h"] for b in boxes])
    return dict(boxes=boxes, omega=Om, height=H, accepted=H <= Om)


@pytest.mark.parametrize("seed", range(6))
def test_candidates_match_restatement(seed):
    fa, fb = S.lognormal_boxes(seed, 60, mean_texels=6, sigma=0.8, max_texels=60)
    order = O.order(fb)
    for atlas_log2 in (5, 6, 7):
        for k in (1, 7, 32, 50, 64):
            r = O.pack_candidate(fa, fb, order, atlas_log2, k)
            q = restated_candidate(fa, fb, atlas_log2, k, 64)
            assert r["omega"] == q["omega"] and r["height"] == q["height"]
            assert r["accepted"] == q["accepted"]
            assert r["x"].tolist() == [b["x"] for b in q["boxes"]]
            assert r["y"].tolist() == [b["y"] for b in q["boxes"]]
            assert r["w"].tolist() == [b["w"] for b in q["boxes"]]


def owners(place, om, Om):
    """Exact texel ownership after the uniform scale alpha = om / Om: texel t (centre
    t + 1/2) belongs to [x, x + w) iff 2 x om <= (2 t + 1) Om < 2 (x + w) om."""
    grid = np.zeros((om, om), np.int32)
    t2 = (2 * np.arange(om) + 1) * Om
    for x, y, w, h in place:
        cx = (t2 >= 2 * x * om) & (t2 < 2 * (x + w) * om)
        cy = (t2 >= 2 * y * om) & (t2 < 2 * (y + h) * om)
        grid[np.ix_(cy, cx)] += 1
    return grid


@pytest.mark.parametrize("seed", range(5))
def test_packing_is_disjoint_and_inside_atlas(seed):
    fa, fb = S.lognormal_boxes(10 + seed, 200, mean_texels=5, sigma=0.9, max_texels=80)
    for atlas_log2 in (6, 7, 8):
        pk = O.pack(fa, fb, atlas_log2)
        assert pk.status == 0
        om = 1 << atlas_log2
        P = pk.place.astype(np.int64)
        assert (P[:, 0] >= 0).all() and (P[:, 1] >= 0).all()
        assert (P[:, 0] + P[:, 2] <= pk.omega).all() and (P[:, 1] + P[:, 3] <= pk.omega).all()
        assert pk.height <= pk.omega
        # pairwise disjoint in the integer virtual grid
        x0, y0, x1, y1 = P[:, 0], P[:, 1], P[:, 0] + P[:, 2], P[:, 1] + P[:, 3]
        ov = (x0[:, None] < x1[None]) & (x0[None] < x1[:, None]) & (y0[:, None] < y1[None]) & (y0[None] < y1[:, None])
        np.fill_diagonal(ov, False)
        assert not ov.any()
        # every texel of the real om x om atlas has at most one owner
        assert owners(P, om, pk.omega).max() <= 1
        # area bound
        assert (P[:, 2] * P[:, 3]).sum() <= pk.omega * pk.omega


def sigma(k, n, om, Om):
    return Fraction(k, n) * Fraction(om, Om)


@pytest.mark.parametrize("nbox", [3, 4, 5])
def test_exhaustive_candidates_and_selection(nbox):
    rng = np.random.default_rng(nbox)
    for trial in range(8):
        wh = rng.integers(2, 40, size=(nbox, 2))
        fa = (np.minimum(wh[:, 0], wh[:, 1]) * 256 - rng.integers(0, 255, nbox)).astype(np.uint32)
        fb = (np.maximum(wh[:, 0], wh[:, 1]) * 256).astype(np.uint32)
        atlas_log2 = 5
        om = 32
        pk = O.pack(fa, fb, atlas_log2)
        acc = {}
        for k in range(1, 65):
            q = restated_candidate(fa, fb, atlas_log2, k, 64)
            assert bool(pk.cand_ok[k - 1]) == q["accepted"]
            assert int(pk.cand_omega[k - 1]) == q["omega"]
            if q["accepted"]:
                acc[k] = q["omega"]
        if not acc:
            assert pk.status == 4
            continue
        best = max(acc, key=lambda k: (sigma(k, 64, om, acc[k]), k))
        assert pk.k == best and pk.omega == acc[best]
        pk1 = O.pack(fa, fb, atlas_log2, select_mode=1)
        assert pk1.k == max(acc)
        # informational: the same fold/push over every order and orientation can only
        # do as well or better than the pinned (height desc) order
        if nbox == 5 or trial >= 4:
            continue
        best_enum = Fraction(0)
        for perm in itertools.permutations(range(nbox)):
            for rot in itertools.product((0, 1), repeat=nbox):
                a = np.array([fb[i] if r else fa[i] for i, r in zip(perm, rot)], np.uint32)
                b = np.array([fa[i] if r else fb[i] for i, r in zip(perm, rot)], np.uint32)
                od = np.arange(nbox, dtype=np.uint32)
                for k in range(64, 0, -1):
                    r = O.pack_candidate(a, b, od, atlas_log2, k)
                    if r["accepted"]:
                        best_enum = max(best_enum, sigma(k, 64, om, r["omega"]))
        assert sigma(pk.k, 64, om, pk.omega) <= best_enum


def test_degenerate_inputs():
    e = np.zeros(0, np.uint32)
    pk = O.pack(e, e, 11)
    assert pk.status == 0 and pk.k == 64 and pk.omega == 2048 and pk.height == 0
    # a box twice the atlas height can never fit (H >= h > Omega whenever w <= h)
    big_a = np.array([256 * 100], np.uint32)
    big_b = np.array([256 * 100000], np.uint32)
    pk = O.pack(big_a, big_b, 6)
    assert pk.status == 4
    # zero-size footprints still occupy min_box x min_box texels
    z = np.zeros(5, np.uint32)
    pk = O.pack(z, z, 4)
    assert pk.status == 0 and (pk.place[:, 2:] == 2).all()


def test_scale_64_when_everything_fits_without_overflow():
    # four 8x8 boxes in a 16x16 atlas: exact fit at scale 1 with Omega = omega
    fa = fb = np.full(4, 8 * 256, np.uint32)
    pk = O.pack(fa, fb, 4)
    assert pk.k == 64 and pk.omega == 16 and pk.height == 16
    assert sorted(map(tuple, pk.place[:, :2].tolist())) == [(0, 0), (0, 8), (8, 0), (8, 8)]


def test_gutter_and_min_box():
    fa, fb = S.lognormal_boxes(3, 40, mean_texels=4, sigma=0.5)
    pk = O.pack(fa, fb, 8, gutter=2, min_box=3)
    assert pk.status == 0
    assert (pk.place[:, 2] >= 3 + 4).all() and (pk.place[:, 3] >= 3 + 4).all()


def test_determinism():
    fa, fb = S.lognormal_boxes(9, 3000)
    a = O.pack(fa, fb, 11)
    b = O.pack(fa.copy(), fb.copy(), 11)
    assert (a.place == b.place).all() and a.k == b.k and a.omega == b.omega


# ---------------------------------------------------------------- one packing, two atlases

def _lowres_texels(pk, omega, gutter, d, fa, fb, n_scales):
    """Low-resolution texel ranges [x0, x1) x [y0, y1) of each chart's content: the
    content of box (x, y, w, h) spans [x + g, x + w - g) virtual texels, alpha = omega /
    Omega maps them to the atlas and 2^-d to the low-resolution atlas (exact
    rationals); the texels touched are floor(start) .. ceil(end) - 1."""
    from fractions import Fraction
    a = Fraction(omega, pk.omega) / (1 << d)
    out = []
    for x, y, w, h in pk.place:
        x0, x1 = a * (int(x) + gutter), a * (int(x) + int(w) - gutter)
        y0, y1 = a * (int(y) + gutter), a * (int(y) + int(h) - gutter)
        out.append((x0.__floor__(), -((-x1).__floor__()), y0.__floor__(), -((-y1).__floor__())))
    return out


@pytest.mark.parametrize("d,gutter,seed", [(2, 2, 0), (3, 4, 1), (3, 8, 2), (2, 3, 3)])
def test_lowres_packing_keeps_charts_apart(d, gutter, seed):
    fa, fb = S.lognormal_boxes(seed, 300, mean_texels=40.0)
    L = 12
    pk = O.pack(fa, fb, L, 64, 2, gutter, 0, d)
    assert pk.status == 0
    assert (pk.omega << d) <= 2 * gutter * (1 << L)
    r = _lowres_texels(pk, 1 << L, gutter, d, fa, fb, 64)
    for i in range(len(r)):
        for j in range(i + 1, len(r)):
            a, b = r[i], r[j]
            overlap = a[0] < b[1] and b[0] < a[1] and a[2] < b[3] and b[2] < a[3]
            assert not overlap, (i, j, a, b)
    # every candidate the constraint rejected broke it; the unconstrained choice is
    # at least as large a scale
    free = O.pack(fa, fb, L, 64, 2, gutter, 0, 0)
    assert free.status == 0 and free.k * pk.omega >= pk.k * free.omega
    for k in range(64):
        if free.cand_ok[k] and not pk.cand_ok[k]:
            assert (int(pk.cand_omega[k]) << d) > 2 * gutter * (1 << L)


def test_lowres_without_gutter_fails():
    fa, fb = S.lognormal_boxes(5, 50)
    assert O.pack(fa, fb, 11, 64, 2, 0, 0, 3).status == 4
