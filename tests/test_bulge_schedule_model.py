"""CPU models of the two schedules of the band -> tridiagonal stage (csrc/bulge.cu).  No GPU.

1. Bulge chasing.  Sweep s runs its tasks t = 0, 1, ... in order; task (s, t) starts once sweep
   s-1 has published progress >= t+3 (its tasks 0 .. t+2 done).  Chaining these waits, task (s2, t2)
   starts after every task (s1, u) with s1 < s2 and u <= t2 + 2 (s2 - s1).  The model lists the band
   cells each task reads and writes (the annihilated column or the stored L block, the diagonal block
   D, the block E below it, which the task keeps in shared memory and the sweep's next task stores)
   and checks that every pair of conflicting accesses from different sweeps is ordered by those
   waits, so the pipelined sweeps compute what the sweeps computed one after another do.  It also
   checks the compact-band offsets (0 <= i - j < 2b) and the reflector-store bound t < ntask.

2. Back-transform Y <- Q2 Y by levels.  Reflector H(s, t) acts on rows [p, p + len), p = s+1+tb.
   Group g holds the sweeps gb .. gb+b-1; its block for task t is applied at level
   L = t + (ngroups - 1 - g), its reflectors in decreasing s.  The model checks that the blocks of a
   level act on disjoint rows (they commute), that each block's rows fit its 2b-row staging buffer,
   and that for every two reflectors with overlapping rows, the one the reduction applied later is
   applied first in the back-transform; and which slots of the reflector store a level reads without
   the reduction having written them."""
import numpy as np
import pytest


def bulge_tasks(n, b):
    """(s, t, accesses) with accesses = [(kind, r0, r1, c0, c1)], rows [r0, r1) x cols [c0, c1)."""
    out = []
    for s in range(0, n - 2):
        pending = False
        t = 0
        while True:
            p = s + 1 + t * b
            ln = min(b, n - p) if p < n else 0
            if t > 0 and ln <= 1:
                acc = [("W", p, p + 1, p - b, p)] if (pending and ln == 1) else []
                out.append((s, t, acc))
                break
            p2 = p + ln
            ln2 = min(b, n - p2) if p2 < n else 0
            acc = []
            if t == 0:
                acc += [("R", s + 1, s + 1 + ln, s, s + 1), ("W", s + 1, s + 1 + ln, s, s + 1)]
            else:
                acc += [("W", p, p + ln, p - b, p)]  # the previous task's E, stored as this task's L
            acc += [("R", p, p + ln, p, p + ln), ("W", p, p + ln, p, p + ln)]
            if ln2 > 0:
                acc += [("R", p + ln, p + ln + ln2, p, p + ln)]
            pending = ln2 > 0
            out.append((s, t, acc))
            t += 1
    return out


def lower_overlap(a, b):
    """Rectangles a, b (r0, r1, c0, c1) share a cell (i, j) with i >= j (the stored triangle)."""
    r0, r1 = max(a[0], b[0]), min(a[1], b[1])
    c0, c1 = max(a[2], b[2]), min(a[3], b[3])
    return r0 < r1 and c0 < c1 and r1 - 1 >= c0


CASES = [(2, 16), (3, 16), (5, 16), (20, 16), (33, 16), (67, 16), (100, 16), (40, 32), (97, 32), (130, 32),
         (70, 64), (200, 64)]


@pytest.mark.parametrize("n,b", CASES)
def test_bulge_pipeline_orders_every_conflict(n, b):
    tasks = bulge_tasks(n, b)
    ntask = (n + b - 1) // b + 2
    rects = []
    for s, t, acc in tasks:
        assert t < ntask  # the reflector store holds ntask reflectors per sweep
        for kind, r0, r1, c0, c1 in acc:
            assert 0 <= c0 and r1 <= n
            # compact band: every stored cell (i >= j) of the block has i - j < 2b
            if r0 < r1 and c0 < c1:
                assert (r1 - 1) - c0 < 2 * b
            rects.append((s, t, kind == "W", r0, r1, c0, c1))
    if not rects:
        return
    R = np.array(rects, dtype=np.int64)
    s, t, w = R[:, 0], R[:, 1], R[:, 2].astype(bool)
    checked = 0
    for a in range(len(R)):
        later = s > s[a]
        ov = (later & (np.maximum(R[:, 3], R[a, 3]) < np.minimum(R[:, 4], R[a, 4]))
              & (np.maximum(R[:, 5], R[a, 5]) < np.minimum(R[:, 6], R[a, 6]))
              & (w | w[a]))
        for bidx in np.nonzero(ov)[0]:
            if not lower_overlap(R[a, 3:], R[bidx, 3:]):
                continue
            checked += 1
            # (s[bidx], t[bidx]) starts only after (s[a], u) for every u <= t[bidx] + 2 (s[bidx] - s[a])
            assert t[a] <= t[bidx] + 2 * (s[bidx] - s[a]), (tuple(R[a]), tuple(R[bidx]))
    if n >= 20:
        assert checked > 0  # the pipeline does overlap sweeps; the check is not vacuous


def test_a_looser_wait_is_caught():
    """Waiting for progress >= t+2 instead of t+3 lets a task run beside the previous sweep's next
    task, whose footprint it overlaps: the model must see a conflict that this wait leaves unordered."""
    n, b = 60, 16
    tasks = bulge_tasks(n, b)
    bad = 0
    for s1, t1, acc1 in tasks:
        for s2, t2, acc2 in tasks:
            if s2 != s1 + 1 or t1 <= t2 + 1:
                continue
            for k1, *r1 in acc1:
                for k2, *r2 in acc2:
                    if (k1 == "W" or k2 == "W") and lower_overlap(r1, r2) and t1 == t2 + 2:
                        bad += 1
    assert bad > 0


@pytest.mark.parametrize("n,b", CASES)
def test_back_transform_levels(n, b):
    last = n - 3
    if last < 0:
        return
    ntask = (n + b - 1) // b + 2
    ngroups = last // b + 1
    refl = {}  # (s, t) -> rows [p, p + len)
    for s, t, acc in bulge_tasks(n, b):
        p = s + 1 + t * b
        ln = min(b, n - p) if p < n else 0
        if ln >= 1 and any(k == "W" and r0 == p and c0 == p for k, r0, r1, c0, c1 in acc):
            refl[(s, t)] = (p, p + ln)
    applied = {}  # (s, t) -> (level, position inside its block)
    windows = {}
    unstored = set()
    for L in range(ngroups + ntask):
        for g in range(max(0, ngroups - 1 - L), ngroups):
            t = L - (ngroups - 1 - g)
            if t < 0 or t >= ntask:
                continue
            s0, s1 = g * b, min(g * b + b - 1, last)
            w0 = s0 + 1 + t * b
            if w0 >= n:
                continue
            w1 = min(n, s1 + 1 + t * b + b)
            assert w1 - w0 <= 2 * b  # staging buffer of 2b rows
            windows.setdefault(L, []).append((w0, w1))
            for pos, s in enumerate(range(s1, s0 - 1, -1)):
                if (s, t) in refl:
                    p0, p1 = refl[(s, t)]
                    assert w0 <= p0 and p1 <= w1
                    assert (s, t) not in applied
                    applied[(s, t)] = (L, pos)
                elif s + 1 + t * b < n:
                    unstored.add((s, t, s + 1 + t * b))
    assert set(applied) == set(refl)
    # slots inside the matrix that the reduction never stored: only a sweep's final single row.  The
    # FP32 level kernel reads their first entry with tau = 0 and no branch, which is why hb2st zeroes
    # the reflector store (not only tau) for FP32 data.
    assert all(p == n - 1 for _, _, p in unstored)
    for L, ws in windows.items():
        ws.sort()
        for (a0, a1), (b0, b1) in zip(ws, ws[1:]):
            assert a1 <= b0  # blocks of one level: disjoint rows
    keys = sorted(refl)  # the reduction's order: sweep by sweep, task by task
    for i, k1 in enumerate(keys):
        r1 = refl[k1]
        for k2 in keys[i + 1:]:
            r2 = refl[k2]
            if max(r1[0], r2[0]) < min(r1[1], r2[1]):
                assert applied[k2] < applied[k1], (k1, k2)  # the later reflector goes first
