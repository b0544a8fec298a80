"""Index arithmetic of the candidate-list balancing (list32_balance in
csrc/select32.cuh, compiled into the 80-register launch shape), replayed on
the host: lane l's j-th entry sits at slot j*32 + l; with C entries in the
warp and T = ceil(C/32), lanes above T hand their last entries to lanes below
T through a 64-word table (excess entry e fills hole e, both numbered in lane
order from packed prefix sums).  Checked on random and extreme counts: every
table and slot index in range, no slot both read and written, every moved
entry lands in a hole, each lane's entries stay contiguous from slot 0, no
entry is lost or duplicated, and every lane holds at most T when at most 64
entries move."""
import numpy as np

XB32 = 64


def balance(cnt, qt):
    """One warp: returns (new counts, slot -> entry map) for entries (lane, j)."""
    slots = {j * 32 + l: (l, j) for l in range(32) for j in range(cnt[l])}
    C = int(cnt.sum())
    T = (C + 31) >> 5
    E = np.maximum(cnt - T, 0)
    D = np.maximum(T - cnt, 0)
    pk = (E.astype(np.int64) << 16) | D          # excess high, holes low
    inc = np.cumsum(pk)                          # the warp's inclusive scan
    M = min(int(inc[31] >> 16), XB32)            # entries that move
    if M == 0:
        return cnt.copy(), slots
    ex = inc - pk
    Epre, Dpre = ex >> 16, ex & 0xFFFF
    got = np.minimum(np.maximum(M - Dpre, 0), D)
    gave = np.minimum(np.maximum(M - Epre, 0), E)
    tab = [None] * XB32
    written = set()
    for l in range(32):                          # holes publish their slots
        for u in range(int(got[l])):
            h = int(Dpre[l]) + u
            assert 0 <= h < XB32 and tab[h] is None
            slot = (int(cnt[l]) + u) * 32 + l
            assert slot < qt * 32 and slot not in slots
            tab[h] = slot
    read = set()
    for l in range(32):                          # donors move their last entries
        for t in range(int(gave[l])):
            e = int(Epre[l]) + t
            assert 0 <= e < XB32 and tab[e] is not None
            src = (int(cnt[l]) - 1 - t) * 32 + l
            assert 0 <= src < qt * 32
            read.add(src)
            written.add(tab[e])
            slots[tab[e]] = slots.pop(src)
    assert not (read & written)
    return cnt + got - gave, slots


def test_balancing_moves_every_excess_entry_into_a_hole():
    rng = np.random.default_rng(11)
    for trial in range(3000):
        qt = int(rng.integers(1, 48))
        kind = trial % 5
        if kind == 0:
            cnt = np.minimum(rng.poisson(rng.uniform(0, qt), 32), qt)
        elif kind == 1:                          # one busy lane
            cnt = np.zeros(32, np.int64)
            cnt[rng.integers(0, 32)] = qt
        elif kind == 2:                          # all full
            cnt = np.full(32, qt)
        elif kind == 3:                          # many lanes over the mean
            cnt = np.where(rng.random(32) < 0.5, qt, 0)
        else:
            cnt = rng.integers(0, qt + 1, 32)
        cnt = np.asarray(cnt, np.int64)
        before = sorted((l, j) for l in range(32) for j in range(cnt[l]))
        new, slots = balance(cnt, qt)
        # each lane's entries are contiguous from slot 0, none lost or duplicated
        assert sorted(slots) == sorted(j * 32 + l for l in range(32) for j in range(new[l]))
        assert sorted(slots.values()) == before
        assert (new <= qt).all() and new.sum() == cnt.sum()
        T = (int(cnt.sum()) + 31) >> 5
        excess = int(np.maximum(cnt - T, 0).sum())
        if excess <= XB32:
            assert new.max() <= T
        else:                                    # only the first 64 move
            assert new.max() <= cnt.max()
