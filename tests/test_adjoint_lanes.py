"""Row mapping of the one-angle-set reduction adjoint (``kAdjRedLow``), on the host.

The reduction step of a target t that lacks some of the bucket's variables
sums, for every target element, the products over its completions (the
values of the missing variables).  With one angle set the lanes of a warp
take the bucket's five lowest variables and the pass index the completion
bits above them, then the target bits (row q = (h << 5) | lane, h = k_h *
2^comp_bits + c_h, y = lane | pdep(c_h, C_H) | pdep(k_h, T_H)).  A warp tile
covers P passes; the lanes sum over the passes of one k_h, then over their
completion bits in a butterfly, and the lanes whose completion bits are 0 add
one term per target element.  This replays that mapping for random masks and
checks that every bucket row is visited once and that every target element
receives exactly its 2^|completions| rows, each with the right target index.
"""
import random

import pytest


def pdep(x, mask):
    r, j = 0, 0
    for b in range(32):
        if mask >> b & 1:
            if x >> j & 1:
                r |= 1 << b
            j += 1
    return r


def pext(y, mask):
    r, j = 0, 0
    for b in range(32):
        if mask >> b & 1:
            if y >> b & 1:
                r |= 1 << j
            j += 1
    return r


@pytest.mark.parametrize("seed", range(6))
def test_low_lane_reduction_covers_every_row_and_target(seed):
    rng = random.Random(seed)
    P = 32  # passes per warp tile (one angle set, the default tile)
    for _ in range(40):
        r = rng.randint(5, 12)  # bucket output rank (>= 5 completions make a reduction step)
        full = (1 << r) - 1
        while True:
            tmask = rng.getrandbits(r) & full
            if bin(full & ~tmask).count("1") >= 5:
                break
        comp = full & ~tmask
        CH, TH = comp & ~31, tmask & ~31
        cb = bin(CH).count("1")
        cl = ~tmask & 31  # completion bits among the lane bits
        seg = 1 << cb  # passes per target group
        n_pass = (1 << r) // 32
        seen, got = set(), {}
        for t0 in range(0, n_pass, P):
            group = []
            for q in range(min(P, n_pass - t0)):
                h = t0 + q
                yp = pdep(h & (seg - 1), CH) | pdep(h >> cb, TH)
                assert yp & 31 == 0
                group.append(yp)
                for lane in range(32):
                    assert (yp | lane) not in seen
                    seen.add(yp | lane)
                if (q + 1) % seg == 0 or q + 1 == P or h + 1 == n_pass:  # end of a target group
                    for lane in range(32):
                        if lane & cl:
                            continue
                        target = pext(yp, tmask) + pext(lane, tmask)  # table entry + lane part
                        rows = [g | l for g in group for l in range(32) if (l & ~cl & 31) == (lane & ~cl & 31)]
                        assert all(pext(y, tmask) == target for y in rows)
                        got[target] = got.get(target, 0) + len(rows)
                    group = []
        assert len(seen) == 1 << r
        assert len(got) == 1 << bin(tmask).count("1")
        assert set(got.values()) == {1 << bin(comp).count("1")}


@pytest.mark.parametrize("Bv", [1, 2, 3, 6, 8, 12, 16])
def test_multi_row_reduction_covers_every_completion(Bv):
    """The reduction adjoint on the multi-row layout (2 to 32 rows per warp
    pass, Bv vectors per row, lane l on row l // Bv and vector l % Bv): rows
    q = kt * 2^comp_bits + c with the lanes on the low completion bits, passes
    summed while the target row stays the same, then the RP lanes of each
    vector in a shuffle tree (lanes rip < off take rip + off, off = RP/2 .. 1).
    Every target element (and vector) gets each of its completions once, and
    the tree stays within the RP * Bv <= 32 busy lanes."""
    rng = random.Random(Bv)
    RP = 1
    while RP * 2 <= 32 // Bv:
        RP *= 2
    for P in (8, 32):
        for _ in range(12):
            r = rng.randint(5, 11)
            full = (1 << r) - 1
            while True:
                tmask = rng.getrandbits(r) & full
                if bin(full & ~tmask).count("1") >= 5:
                    break
            comp = full & ~tmask
            cb = bin(comp).count("1")
            seg = (1 << cb) // RP
            n_rows, R = 1 << r, P * RP
            got = {}
            for r0 in range(0, n_rows, R):
                r1 = min(r0 + R, n_rows)
                acc = {}
                for q in range(P):
                    if r0 + q * RP >= r1:
                        break
                    qq = r0 + q * RP
                    yp = pdep(qq >> cb, tmask) | pdep(qq & ((1 << cb) - 1), comp)
                    for lane in range(32):
                        rip, v0 = lane // Bv, lane % Bv
                        if rip < RP and qq + rip < r1:
                            acc.setdefault(v0, []).append(yp | pdep(rip, comp))
                    if (q + 1) % seg == 0 or q + 1 == P or r0 + (q + 1) * RP >= r1:
                        kt = (r0 + q * RP) >> cb
                        for v0, ys in acc.items():
                            assert all(pext(y, tmask) == kt for y in ys)
                            got[(kt, v0)] = got.get((kt, v0), 0) + len(ys)
                        acc = {}
            assert len(got) == (1 << bin(tmask).count("1")) * Bv
            assert set(got.values()) == {1 << cb}
    for lane in range(RP * Bv):
        off = RP // 2
        while off >= 1:
            if lane // Bv < off:
                assert lane + off * Bv < RP * Bv <= 32
            off //= 2
