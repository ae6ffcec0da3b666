"""The batch kernel's incremental descent, checked in exact integers on the CPU.

When a ray steps into a refined neighbour, the FP32 kernels with links do not
redo the descent by mid-planes and the 64-bit exit-order terms.  They derive
the child cell and its terms from the parent's terms:

  e_xy = n_x |D_y| - n_y |D_x| = E s + r,  F = 2E + [r > 0]   (pair x < y)

with n_a the distance from the origin to the cell's exit plane on axis a and
s the cell size.  In units of the child size s' = s / 2, e = H s' + r' with
H = 2E + (the top bit of r) and r' the low bits of r.  The ray entered through
the face on axis ea, so on ea the child is the half next to that face; on
another axis a the entry point lies in the half the ray reaches first exactly
when e_(ea,a) < (2|D_a| - |D_ea|) s'.  With u_a = 1 for those first-reached
halves, the child's terms are E' = H - (u_x |D_y| - u_y |D_x|) and r = r'.

This test restates both sides in plain Python integers (the definitions:
exit-plane distances, pair terms, floor division, the side of each mid-plane
just after the entry event; and the incremental update) and requires them to
agree on random cells, directions and entry points, mid-plane ties included.
It exercises no GPU code; the GPU tests compare the kernel with the oracle.
"""
import random

import pytest

FIX = 36          # the origin's lattice: 2^-36 of the box
PAIRS = ((0, 1), (0, 2), (1, 2))


def exit_terms(X, D, k, lvl):
    """F and r of cell k at level lvl, from their definitions."""
    sh = FIX - lvl
    aD = [abs(d) for d in D]
    n = [((k[a] + 1) << sh) - X[a] if D[a] > 0 else X[a] - (k[a] << sh) for a in range(3)]
    F, r = [], []
    for x, y in PAIRS:
        e = n[x] * aD[y] - n[y] * aD[x]
        E = e >> sh                     # floor division by s
        r.append(e - (E << sh))
        F.append(2 * E + (r[-1] != 0))
    return F, r


def child_by_midplanes(X, D, k, lvl, ea):
    """The child holding the ray just after it enters cell k through its
    face on axis ea: the side of each mid-plane at the entry event."""
    sh = FIX - lvl
    aD = [abs(d) for d in D]
    m = (k[ea] << sh) - X[ea] if D[ea] > 0 else X[ea] - ((k[ea] + 1) << sh)
    kc = []
    for a in range(3):
        g = (X[a] - ((2 * k[a] + 1) << (sh - 1))) * aD[ea] + m * D[a]
        kc.append(2 * k[a] + (1 if g > 0 or (g == 0 and D[a] >= 0) else 0))
    return kc


def incremental_child(F, r, D, lvl, ea):
    """The kernel's update: child index bits and the child's F, r."""
    shc = FIX - lvl - 1
    low = (1 << shc) - 1
    aD = [abs(d) for d in D]
    H = [(F[p] & ~1) | ((r[p] >> shc) & 1) for p in range(3)]
    rl = [r[p] & low for p in range(3)]
    u = [0, 0, 0]
    u[ea] = 1
    for p, (x, y) in enumerate(PAIRS):
        if ea == x:                       # e_(ea,y) = e
            u[y] = int(H[p] < 2 * aD[y] - aD[ea])
        elif ea == y:                     # e_(ea,x) = -e
            u[x] = int(2 * (H[p] + 2 * aD[x] - aD[ea]) + (rl[p] != 0) > 0)
    dirbits = [1 if d < 0 else 0 for d in D]
    bits = [dirbits[a] if u[a] else dirbits[a] ^ 1 for a in range(3)]
    Fn = [2 * (H[p] - (u[x] * aD[y] - u[y] * aD[x])) + (rl[p] != 0) for p, (x, y) in enumerate(PAIRS)]
    return bits, Fn, rl


def random_case(rng):
    """A cell at level >= 4 and a ray entering it through its face on ea."""
    lvl = rng.randint(4, 21)
    D = [rng.choice((-1, 1)) * rng.randint(1, 1 << 23) for _ in range(3)]
    big = rng.randrange(3)
    D[big] = (1 << 23) if D[big] > 0 else -(1 << 23)
    ea = rng.randrange(3)
    sh = FIX - lvl
    k = [rng.randrange(1 << lvl) for _ in range(3)]
    P = []
    for a in range(3):
        if a == ea:
            P.append(k[a] << sh if D[a] > 0 else (k[a] + 1) << sh)
        else:
            P.append((k[a] << sh) + rng.randrange(1 << sh))
    if rng.random() < 0.25:               # on a mid-plane: the tie rule decides
        b = rng.choice([a for a in range(3) if a != ea])
        P[b] = (2 * k[b] + 1) << (sh - 1)
    t = rng.randint(0, 5)
    X = [P[a] - t * D[a] for a in range(3)]
    # ea must be the entry axis: its entry time is the latest
    entry = [(k[a] << sh) - X[a] if D[a] > 0 else X[a] - ((k[a] + 1) << sh) for a in range(3)]
    if any(entry[a] * abs(D[ea]) > entry[ea] * abs(D[a]) for a in range(3)):
        return None
    return X, D, k, lvl, ea


@pytest.mark.parametrize("seed", range(4))
def test_incremental_descent_matches_the_definitions(seed):
    rng = random.Random(seed)
    checked = 0
    while checked < 4000:
        case = random_case(rng)
        if case is None:
            continue
        X, D, k, lvl, ea = case
        F, r = exit_terms(X, D, k, lvl)
        kc = child_by_midplanes(X, D, k, lvl, ea)
        bits, Fn, rn = incremental_child(F, r, D, lvl, ea)
        assert bits == [kc[a] - 2 * k[a] for a in range(3)], case
        F_ref, r_ref = exit_terms(X, D, kc, lvl + 1)
        assert Fn == F_ref and rn == r_ref, case
        # a second level from the child, entered through the same face
        if lvl + 1 <= 21:
            kc2 = child_by_midplanes(X, D, kc, lvl + 1, ea)
            bits2, Fn2, rn2 = incremental_child(Fn, rn, D, lvl + 1, ea)
            assert bits2 == [kc2[a] - 2 * kc[a] for a in range(3)], case
            assert (Fn2, rn2) == exit_terms(X, D, kc2, lvl + 2), case
        checked += 1


def test_a_planted_mistake_fails():
    """Swapping the strict and non-strict near test (the mid-plane tie) must
    be caught by the cases above."""
    rng = random.Random(7)
    caught = False
    for _ in range(20000):
        case = random_case(rng)
        if case is None:
            continue
        X, D, k, lvl, ea = case
        F, r = exit_terms(X, D, k, lvl)
        shc = FIX - lvl - 1
        aD = [abs(d) for d in D]
        for p, (x, y) in enumerate(PAIRS):
            if ea == x:
                H = (F[p] & ~1) | ((r[p] >> shc) & 1)
                wrong = int(H <= 2 * aD[y] - aD[ea])
                right = int(H < 2 * aD[y] - aD[ea])
                if wrong != right:
                    kc = child_by_midplanes(X, D, k, lvl, ea)
                    near_bit = (1 if D[y] < 0 else 0)
                    assert (kc[y] - 2 * k[y] == near_bit) == bool(right)
                    caught = True
        if caught:
            break
    assert caught
