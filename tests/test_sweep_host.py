"""Host emulation of the FP32 sweeps' reduction orders (no GPU needed).

The narrow-group kernel (k_tick_narrow in csrc/k_sweep.cu) claims bitwise the results of the ring
sweep's narrow tile for groups of four rows and at most 32 columns.  The per-(row, block) partial
sums are the same code; what could differ is the order in which the eight column blocks of a row
are added.  This test replays, in IEEE single precision, the ring's warp totals (group_totals in
csrc/qdse_internal.h: a transposed butterfly over 32 lanes, lane l holding row l / 8 and block
l % 8, zeros for the other rows) and the narrow kernel's butterfly over eight lanes (xor 4, 2, 1),
and checks that every total agrees bit for bit, over partials spread across many binades so that
any other order would round differently.
"""
import numpy as np

K_ROWS = 4
F = np.float32


def ring_totals(part):
    """part[r, cb]: the narrow tile's partial of row r, block cb (float32).  Returns the 8 totals
    (A of rows 0..3, then B of rows 0..3) as the ring's warp totals leave them: value qv on the
    lanes l with l // 4 == qv."""
    nv = 2 * K_ROWS
    lanes = []
    for lane in range(32):
        r, cb = lane // 8, lane % 8
        v = [F(0.0)] * nv
        v[r] = part[0][r, cb]              # sA[r] of this lane
        v[K_ROWS + r] = part[1][r, cb]     # sB[r]
        lanes.append(v)
    width = nv
    m = 16
    while m >= 1:
        new = [list(v) for v in lanes]
        if width > 1:
            half = width >> 1
            for lane in range(32):
                hi = (lane & m) != 0
                other = lanes[lane ^ m]
                for k in range(half):
                    keep = lanes[lane][k + half] if hi else lanes[lane][k]
                    send_other = other[k] if (lane ^ m) & m else other[k + half]
                    new[lane][k] = F(keep + send_other)
            width = half
        else:
            for lane in range(32):
                new[lane][0] = F(lanes[lane][0] + lanes[lane ^ m][0])
        lanes = new
        m >>= 1
    return [lanes[4 * qv][0] for qv in range(nv)]


def narrow_totals(part):
    """The narrow kernel: lane cb of the group's eight holds sA[r], sB[r] of block cb; butterfly
    xor 4, 2, 1; lane cb then stores value cb."""
    vals = [[part[c][r, cb] for cb in range(8)] for c in range(2) for r in range(K_ROWS)]
    out = []
    for row in vals:
        x = list(row)
        for m in (4, 2, 1):
            x = [F(x[cb] + x[cb ^ m]) for cb in range(8)]
        assert len({v.tobytes() for v in x}) == 1  # every lane holds the same total
        out.append(x[0])
    return out


def test_narrow_kernel_sums_in_the_ring_warp_totals_order():
    rng = np.random.default_rng(2012)
    for trial in range(300):
        part = []
        for c in range(2):
            mag = np.exp2(rng.integers(-30, 30, size=(K_ROWS, 8)))
            p = (rng.normal(size=(K_ROWS, 8)) * mag).astype(F)
            cut = rng.integers(0, 9)  # blocks beyond the band hold exact zeros
            p[:, cut:] = F(0.0)
            part.append(p)
        a = ring_totals(part)
        b = narrow_totals(part)
        for x, y in zip(a, b):
            assert x.tobytes() == y.tobytes(), (trial, x, y)


def test_another_order_would_round_differently():
    """The check has teeth: summing the eight blocks left to right instead differs in the last bit
    for some draws."""
    rng = np.random.default_rng(7)
    differs = 0
    for _ in range(200):
        x = (rng.normal(size=8) * np.exp2(rng.integers(-20, 20, size=8))).astype(F)
        tree = F(F(F(x[0] + x[4]) + F(x[2] + x[6])) + F(F(x[1] + x[5]) + F(x[3] + x[7])))
        seq = F(0.0)
        for v in x:
            seq = F(seq + v)
        differs += tree.tobytes() != seq.tobytes()
    assert differs > 20
