"""Host-side checks of the fixed geometry the n = 8 lane-tiled kernel
(paper_1004_3114_gb300/csrc/wl_tiled_tma8.cu) is compiled for: 315 lanes,
8 lane times per tile, at most 300 spans, slots of 8 alpha + 8 words.

The kernel takes these as constants for N coprime to 105 (and N % 4 == 0).
They follow from the stride candidates of that N (Section 3's strides, with
the candidate reading of this implementation: the odd divisors above one of
p^2 q r, p < q < r the smallest odd primes not dividing N) and from the lane
geometry of Eq. 1 (lane l from J_l = ceil(l N / L); span p of sub-vector i
starts at ceil(p N / m_i), m_i = L / alpha_i).  The constants are read from
the kernel source, the candidates from the oracle."""
import itertools
import math
import os
import random
import re

import pytest

from oracle import py_oracle as orc

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_1004_3114_gb300", "csrc", "wl_tiled_tma8.cu")


def _consts():
    text = open(SRC).read()
    vals = {}
    for name in ("T8_L", "T8_T", "T8_MAXSPANS", "T8_SPAN_PAD"):
        m = re.search(r"#define %s (\d+)" % name, text)
        assert m, name
        vals[name] = int(m.group(1))
    return vals


def _lcm(values):
    out = 1
    for v in values:
        out = out * v // math.gcd(out, v)
    return out


def test_candidates_for_n_coprime_to_105_are_the_divisors_of_315():
    for N in (1 << 14, 1 << 20, (1 << 21) + 32, 1 << 23, 100004):
        assert N % 3 and N % 5 and N % 7
        assert orc.stride_candidates(8, N) == [d for d in range(3, 316, 2) if 315 % d == 0]


def test_every_stride_set_has_315_lanes_and_fits_the_stage():
    c = _consts()
    L, T, maxsp, pad = c["T8_L"], c["T8_T"], c["T8_MAXSPANS"], c["T8_SPAN_PAD"]
    cand = orc.stride_candidates(8, 1 << 23)
    sdw = 8 * L * T + pad * maxsp   # the stage's data words the kernel reserves
    worst = 0
    for sub in itertools.combinations(cand, 8):
        assert _lcm(sub) == L
        nspans = sum(L // a for a in sub)
        assert nspans <= maxsp
        worst = max(worst, nspans)
        # slots of alpha T values plus the alignment lead and a wrap's rounding
        assert sum((L // a) * (T * a + pad) for a in sub) <= sdw
        # 16-byte aligned slots for the bulk copies
        assert all((T * a + pad) % 4 == 0 for a in sub)
    assert worst == maxsp   # the eight smallest candidates reach the bound


def _tile_reads(N, alpha, gamma, L, T, pad):
    """Every (sub-vector, lane, lane time) read of every tile through the span
    slots, as positions of the pool row; checks the bounds on the way."""
    J = [-((-l * N) // L) for l in range(L + 1)]
    maxlen = -(-N // L)
    assert max(J[l + 1] - J[l] for l in range(L)) <= maxlen
    seen = [[0] * N for _ in range(8)]
    for tile in range(-(-maxlen // T)):
        t0 = tile * T
        Tt = min(T, maxlen - t0)
        for i in range(8):
            a, m = alpha[i], L // alpha[i]
            for l in range(L):
                w, p = divmod(l, m)
                C = -((-p * N) // m)
                r = a * J[l] - w * N - C
                assert 0 <= r < a
                start = (C + a * t0 + gamma[i]) % N      # span p of this tile
                lead = start % 4
                # T % 4 == 0 and N % 4 == 0: the lead is the same in every tile
                assert lead == (C + gamma[i]) % 4
                words = 4 * ((lead + a * Tt + 3) // 4)
                assert words <= T * a + pad
                for t in range(min(Tt, J[l + 1] - J[l] - t0)):
                    off = lead + r + a * t
                    assert off < words
                    pos = (start - lead + off) % N
                    assert pos == (a * (J[l] + t0 + t) + gamma[i]) % N   # Eq. 1
                    seen[i][J[l] + t0 + t] += 1
    return seen


@pytest.mark.parametrize("N", [16384, 16388, 20012])
def test_lane_geometry_reads_eq1_positions_once(N):
    c = _consts()
    rng = random.Random(N)
    cand = orc.stride_candidates(8, N)
    for trial in range(2):
        alpha = list(cand[:8]) if trial == 0 else rng.sample(cand, 8)
        gamma = [rng.randrange(N) for _ in range(8)]
        seen = _tile_reads(N, alpha, gamma, c["T8_L"], c["T8_T"], c["T8_SPAN_PAD"])
        assert all(v == 1 for row in seen for v in row)


# ---- the two-CTA cluster form (paper_1004_3114_gb300/csrc/wl_tiled_tma8c.cu):
# each CTA stages four sub-vectors of a 315-lane x 16-lane-time tile

SRC_C = os.path.join(os.path.dirname(__file__), "..", "paper_1004_3114_gb300", "csrc", "wl_tiled_tma8c.cu")


def _consts_c():
    text = open(SRC_C).read()
    vals = {}
    for name in ("C8_L", "C8_T", "C8_STAGES", "C8_MAXSPANS", "C8_SPAN_PAD", "C8_CONS_WARPS", "C8_PROD_WARPS"):
        m = re.search(r"#define %s (\d+)" % name, text)
        assert m, name
        vals[name] = int(m.group(1))
    return vals


def test_cluster_halves_fit_the_stage_and_shared_memory():
    c = _consts_c()
    L, T, maxsp, pad = c["C8_L"], c["C8_T"], c["C8_MAXSPANS"], c["C8_SPAN_PAD"]
    cand = orc.stride_candidates(8, 1 << 23)
    sdw = 4 * L * T + pad * maxsp
    worst = 0
    # either CTA may hold any four of the drawn strides
    for half in itertools.combinations(cand, 4):
        nspans = sum(L // a for a in half)
        assert nspans <= maxsp
        worst = max(worst, nspans)
        assert sum((L // a) * (T * a + pad) for a in half) <= sdw
        assert all((T * a + pad) % 4 == 0 for a in half)
        # lane-table entries: slot word << 9 | span, in 31 bits
        assert sdw << 9 < 2 ** 31 and maxsp < 512
    assert worst == maxsp
    # the dynamic shared memory the kernel asks for, as its macros compute it
    items = (L + 3) // 4
    ipw = -(-items // c["C8_CONS_WARPS"])
    sw = (sdw + 31) & ~31
    xw = c["C8_CONS_WARPS"] * 2 * (2 * ipw) * 32
    cw = (L + 1) + 4 * L + 3 * maxsp
    assert 4 * (c["C8_STAGES"] * sw + xw + cw) <= 227 * 1024 - 2048
    # a thread reads lane times t and t + 8 of its lane: both inside the slot
    assert all(3 + (a - 1) + 15 * a < T * a + pad for a in cand)
    # every producer thread holds at most C8_KS spans
    ks = -(-maxsp // (32 * c["C8_PROD_WARPS"]))
    assert 32 * c["C8_PROD_WARPS"] * ks >= maxsp


def test_cluster_items_cover_each_tile_once_in_both_ctas():
    """Items of 4 lanes x 16 lane times (a thread: lane time t of lanes
    4 g + h and 4 g + 2 + h, a half-warp one lane's 16 lane times), dealt to
    consumer warp (tile items + g) mod W; warp w of both CTAs takes items
    g0 + u W, u < IPW, so the exchange slot (w, u, thread) names the same two
    tuples in both."""
    c = _consts_c()
    L, W_, T = c["C8_L"], c["C8_CONS_WARPS"], c["C8_T"]
    items = (L + 3) // 4
    ipw = -(-items // W_)
    for tile in range(0, 97):
        hits = [0] * items
        for w in range(W_):
            g0 = (w - (tile * items) % W_) % W_
            for u in range(ipw):
                g = g0 + u * W_
                if g < items:
                    hits[g] += 1
        assert hits == [1] * items
    # every (lane, lane time) of a tile is one thread's, once
    seen = sorted((4 * g + 2 * h + (th >> 4), th & 15)
                  for g in range(items) for th in range(32) for h in (0, 1) if 4 * g + 2 * h + (th >> 4) < L)
    assert seen == sorted((l, t) for l in range(L) for t in range(T))


@pytest.mark.parametrize("N", [16384, 16388, 20012])
def test_cluster_lane_geometry_reads_eq1_positions_once(N):
    c = _consts_c()
    rng = random.Random(N + 1)
    cand = orc.stride_candidates(8, N)
    for trial in range(2):
        alpha = list(cand[:8]) if trial == 0 else rng.sample(cand, 8)
        gamma = [rng.randrange(N) for _ in range(8)]
        seen = _tile_reads(N, alpha, gamma, c["C8_L"], c["C8_T"], c["C8_SPAN_PAD"])
        assert all(v == 1 for row in seen for v in row)
