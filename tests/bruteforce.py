"""Brute-force restatements used to pin the oracle on tiny inputs.

Everything here works on Python strings, sets and explicit loops over every
candidate (every window, every target start j), so that it shares no logic
with the oracle's event sweep, index or DP.
"""
from __future__ import annotations

import itertools
import math

_RC = str.maketrans("ACGTacgt", "TGCAtgca")
_CODE = str.maketrans("ACGT", "0123")


def kmer_codes(seq: bytes, st: int, en: int, k: int, min_unmasked: int = 1):
    """Per k-mer start p in [st, en-k]: (forward code, revcomp code, eligible)."""
    out = []
    s = seq.decode("latin1")
    for p in range(st, en - k + 1):
        km = s[p:p + k]
        up = km.upper()
        ok = all(c in "ACGT" for c in up)
        unmasked = sum(1 for c in km if not c.islower())
        if ok:
            f = int(up.translate(_CODE), 4)
            r = int(up.translate(_RC)[::-1].translate(_CODE), 4)
        else:
            f = r = -1
        out.append((f, r, ok and unmasked >= min_unmasked and f != r))
    return out


def sketch(seq: bytes, offsets, k: int, w: int, hash_fn, min_unmasked=1):
    """Winnowing by explicit window scan; set of (h, pos, strand)."""
    res = set()
    for s in range(len(offsets) - 1):
        st, en = int(offsets[s]), int(offsets[s + 1])
        codes = kmer_codes(seq, st, en, k, min_unmasked)
        hs = []
        for f, r, ok in codes:
            if ok:
                c = min(f, r)
                hs.append((hash_fn(c), 1 if r < f else 0))
            else:
                hs.append(None)
        for q in range(0, len(hs) - w + 1):
            win = [(hs[x][0], x) for x in range(q, q + w) if hs[x] is not None]
            if not win:
                continue
            mn = min(h for h, _ in win)
            x = max(x for h, x in win if h == mn)
            res.add((hs[x][0], st + x, hs[x][1]))
    return res


def windows(offsets, n, step):
    for s in range(len(offsets) - 1):
        i = int(offsets[s])
        while i + n <= int(offsets[s + 1]):
            yield s, i
            i += step


def m_of(tau, s):
    m = math.ceil(tau * s - 1e-9)
    return max(m, 0)


def filter_runs(qrecs, qoff, trecs, toff, p, tau):
    """Every query window x every valid target start j, by explicit sets."""
    k, n = p["k"], p["n"]
    span = n - k
    overlap = math.floor((p["delta_m"] + p["delta_g"]) * n)
    post = {}
    for h, t, sg in trecs:
        post.setdefault(h, []).append((t, sg))
    rows = []
    for qs_, i in windows(qoff, n, p["step"]):
        wq = {}
        for h, pos, sg in qrecs:
            if i <= pos <= i + span:
                wq.setdefault(h, set()).add(sg)
        if p["max_occ"] > 0:
            wq = {h: v for h, v in wq.items() if len(post.get(h, [])) <= p["max_occ"]}
        s = len(wq)
        if s == 0:
            continue
        m = m_of(tau, s)
        for o in (0, 1):
            def shared(j):
                hs = set()
                for h, t, sg in trecs:
                    if not (j <= t <= j + span):
                        continue
                    if p["self_mode"] and i <= t <= i + span:
                        continue
                    if h in wq and any((sq ^ sg) == o for sq in wq[h]):
                        hs.add(h)
                return len(hs)

            for u in range(len(toff) - 1):
                lo, hi = int(toff[u]), int(toff[u + 1]) - n
                if p["self_mode"]:
                    if u < qs_:
                        continue
                    if u == qs_:
                        lo = max(lo, i + n - overlap)
                    elif p["self_mode"] == 2:
                        continue
                run = None
                for j in range(lo, hi + 1):
                    c = shared(j)
                    if c >= m:
                        if run is None:
                            run = [j, j, c, j]
                        else:
                            run[1] = j
                            if c > run[2]:
                                run[2], run[3] = c, j
                    elif run is not None:
                        rows.append((i, o, *run, s, m))
                        run = None
                if run is not None:
                    rows.append((i, o, *run, s, m))
    return rows


def estimate(wq, trecs, i, j, p, o):
    """Winnowed MinHash estimate by explicit set construction."""
    span = p["n"] - p["k"]
    wt_all = set()
    wt_shared = set()
    for h, t, sg in trecs:
        if j <= t <= j + span:
            wt_all.add(h)
            if p["self_mode"] and i <= t <= i + span:
                continue
            if h in wq and any((sq ^ sg) == o for sq in wq[h]):
                wt_shared.add(h)
    s = len(wq)
    union = sorted(set(wq) | wt_all)
    U = union[:s]
    return sum(1 for h in U if h in wt_shared), len(U)


def best_chain_length(anchors, gap_max, diag_max):
    """Longest valid chain as the longest path of the 'may follow' relation,
    found by forward recursion over successors (tiny inputs only)."""
    A = sorted(set(anchors))
    nxt = {a: [] for a in range(len(A))}
    for a, b in itertools.permutations(range(len(A)), 2):
        dp = A[b][0] - A[a][0]
        dt = A[b][1] - A[a][1]
        if 0 < dp <= gap_max and 0 < dt <= gap_max and abs(dp - dt) <= diag_max:
            nxt[a].append(b)
    best = 0
    memo = {}

    def longest(a):
        if a in memo:
            return memo[a]
        r = 1 + max((longest(b) for b in nxt[a]), default=0)
        memo[a] = r
        return r

    for a in range(len(A)):
        best = max(best, longest(a))
    return best, A


def chain_is_valid(chain, gap_max, diag_max):
    for (p1, t1), (p2, t2) in zip(chain, chain[1:]):
        dp, dt = p2 - p1, t2 - t1
        if not (0 < dp <= gap_max and 0 < dt <= gap_max and abs(dp - dt) <= diag_max):
            return False
    return True


# ----------------------------------------------------------------- chains --
#
# Chaining restated from its definition (Section 3.3 on the seed's minimizer
# anchors), by exhaustive path enumeration instead of a DP.  `slip` names one
# plausible mistake to apply instead ("pred_tie", "end_tie", "span_short",
# "no_self", "no_flip", "keep_all"); the pin test uses it only to show that
# each mistake changes at least one row of its cases.

def _seq_index(offsets, pos):
    for s in range(len(offsets) - 1):
        if int(offsets[s]) <= pos < int(offsets[s + 1]):
            return s
    return -1


def seed_anchors(run, qrecs, trecs, p, slip=None):
    """Anchors of one kept run as (p, t', t): a query-window minimizer p in
    [i, i+n-k] and a target minimizer t in [j_a, j_b+n-k] with equal hash and
    strands differing by o; in self mode t outside [i, i+n-k]; t' = t, or
    j_b+n-k - t for o = 1.  Sorted by (p, t')."""
    i, o, ja, jb = (int(x) for x in run[:4])
    span = p["n"] - p["k"]
    t_hi = jb + span - (1 if slip == "span_short" else 0)
    occ = {}
    for h, _, _ in trecs:
        occ[h] = occ.get(h, 0) + 1
    out = []
    for hq, pq, sq in qrecs:
        if not (i <= pq <= i + span):
            continue
        if p["max_occ"] > 0 and occ.get(hq, 0) > p["max_occ"]:
            continue
        for ht, pt, st in trecs:
            if ht != hq or (sq ^ st) != o or not (ja <= pt <= t_hi):
                continue
            if p["self_mode"] and slip != "no_self" and i <= pt <= i + span:
                continue
            tp = t_hi - pt if (o == 1 and slip != "no_flip") else pt
            out.append((pq, tp, pt))
    return sorted(out)


def maximal_chains(anchors, gap_max, diag_max, cap=500_000):
    """Every source-to-sink path of the 'may follow' relation (index tuples).
    A longest chain can be extended at neither end, so it is one of them."""
    A = len(anchors)

    def follows(a, b):
        dp, dt = anchors[b][0] - anchors[a][0], anchors[b][1] - anchors[a][1]
        return 0 < dp <= gap_max and 0 < dt <= gap_max and abs(dp - dt) <= diag_max

    succ = [[b for b in range(A) if follows(a, b)] for a in range(A)]
    has_pred = [False] * A
    for a in range(A):
        for b in succ[a]:
            has_pred[b] = True
    paths = []
    stack = [(a,) for a in range(A) if not has_pred[a]]
    while stack:
        path = stack.pop()
        nxt = succ[path[-1]]
        if not nxt:
            paths.append(path)
            if len(paths) > cap:
                raise OverflowError("too many chains to enumerate")
        for b in nxt:
            stack.append(path + (b,))
    return paths


def chosen_chain(anchors, gap_max, diag_max, slip=None):
    """The chain the tie rule selects: among the longest chains, those ending
    at the earliest anchor; among these, walking back from the end, the later
    anchor at every step (lexicographically largest reversed index tuple)."""
    paths = maximal_chains(anchors, gap_max, diag_max)
    L = max(len(x) for x in paths)
    longest = [x for x in paths if len(x) == L]
    ends = {x[-1] for x in longest}
    end = max(ends) if slip == "end_tie" else min(ends)
    cands = [x for x in longest if x[-1] == end]
    key = lambda x: tuple(reversed(x))
    return min(cands, key=key) if slip == "pred_tie" else max(cands, key=key)


def chain_rows(runs, qrecs, qoff, trecs, toff, p, tau, slip=None):
    """Oracle chain rows (i, o, qseq, q0, q1, tseq, t0, t1, score, s) for
    every kept run, by explicit anchor sets and path enumeration."""
    span = p["n"] - p["k"]
    occ = {}
    for h, _, _ in trecs:
        occ[h] = occ.get(h, 0) + 1
    rows = []
    for run in runs:
        i, o, ja = int(run[0]), int(run[1]), int(run[2])
        if int(run[11]) != 1:
            continue
        wq = {h for h, pq, _ in qrecs if i <= pq <= i + span
              and not (p["max_occ"] > 0 and occ.get(h, 0) > p["max_occ"])}
        s = len(wq)
        anc = seed_anchors(run, qrecs, trecs, p, slip)
        if not anc:
            continue
        ch = chosen_chain([(a[0], a[1]) for a in anc], p["gap_max"], p["diag_max"], slip)
        score = len(ch)
        if score < m_of(tau, s) and slip != "keep_all":
            continue
        ps = [anc[x][0] for x in ch]
        ts = [anc[x][2] for x in ch]
        rows.append((i, o, _seq_index(qoff, i), min(ps), max(ps) + p["k"], _seq_index(toff, ja),
                     min(ts), max(ts) + p["k"], score, s))
    return rows


# -------------------------------------------------------------- extension --

def _region_estimate(qrecs, trecs, qa, qb, ta, tb, p, o):
    """Section 2.2 estimate of two regions from explicit sets: W_Q, W_T the
    minimizers whose k-mer lies in each region; s = |W_Q|; U = the s smallest
    of W_Q u W_T; est = hashes of U shared with relative strand o (in a self
    search a target minimizer inside the query's k-mer span is not shared)."""
    k = p["k"]
    Q = {}
    for h, pos, sg in qrecs:
        if qa <= pos <= qb - k:
            Q.setdefault(h, set()).add(sg)
    T_all, T_sh = set(), {}
    for h, pos, sg in trecs:
        if ta <= pos <= tb - k:
            T_all.add(h)
            if not (p["self_mode"] and qa <= pos <= qb - k):
                T_sh.setdefault(h, set()).add(sg)
    s = len(Q)
    U = sorted(set(Q) | T_all)[:s]
    est = sum(1 for h in U if h in Q and h in T_sh
              and any((a ^ b) == o for a in Q[h] for b in T_sh[h]))
    return est, len(U)


def extend_rows(runs, qrecs, qoff, trecs, toff, p, tau, max_len, slip=None):
    """Section 3.2 restated: every kept seed's regions grown one base per
    side per step, forward then backward, while the estimate of the grown
    regions (recomputed from scratch) stays >= m(s), inside the sequences,
    within max_len, and (self search, one sequence) without the regions
    overlapping more than before the step.  Rows (i, o, j*, qa, qb, ta, tb,
    est, den).  `slip` ("no_mirror": o = 1 targets grow like o = 0 ones) is
    used only to show that the pin sees such a mistake."""
    n = p["n"]
    rows = []
    for run in runs:
        if int(run[11]) != 1:
            continue
        i, o, js = int(run[0]), int(run[1]), int(run[9])
        qs, ts = _seq_index(qoff, i), _seq_index(toff, js)
        qlo, qhi = int(qoff[qs]), int(qoff[qs + 1])
        tlo, thi = int(toff[ts]), int(toff[ts + 1])
        same = p["self_mode"] and qs == ts
        qa, qb, ta, tb = i, i + n, js, js + n
        est, den = _region_estimate(qrecs, trecs, qa, qb, ta, tb, p, o)

        def ovl(a0, a1, b0, b1):
            return max(0, min(a1, b1) - max(a0, b0))

        if est >= m_of(tau, den):
            mirror = o == 1 and slip != "no_mirror"
            for direction in (0, 1):
                while True:
                    if direction == 0:
                        nqa, nqb = qa, qb + 1
                        nta, ntb = (ta - 1, tb) if mirror else (ta, tb + 1)
                    else:
                        nqa, nqb = qa - 1, qb
                        nta, ntb = (ta, tb + 1) if mirror else (ta - 1, tb)
                    if nqa < qlo or nqb > qhi or nta < tlo or ntb > thi:
                        break
                    if nqb - nqa > max_len:
                        break
                    if same and ovl(nqa, nqb, nta, ntb) > ovl(qa, qb, ta, tb):
                        break
                    e2, d2 = _region_estimate(qrecs, trecs, nqa, nqb, nta, ntb, p, o)
                    if e2 < m_of(tau, d2):
                        break
                    qa, qb, ta, tb, est, den = nqa, nqb, nta, ntb, e2, d2
        rows.append((i, o, js, qa, qb, ta, tb, est, den))
    return rows


# ------------------------------------------------------- two-tier chains --

_ACGT = set("ACGT")


def mems(X: str, Y: str, k2: int):
    """Maximal exact ACGT matches by scanning every diagonal."""
    out = []
    for d in range(-(len(X) - 1), len(Y)):
        x, y = (0, d) if d >= 0 else (-d, 0)
        run = 0
        while x < len(X) and y < len(Y):
            if X[x] == Y[y] and X[x] in _ACGT:
                run += 1
            else:
                if run >= k2:
                    out.append((x - run, y - run, run))
                run = 0
            x += 1
            y += 1
        if run >= k2:
            out.append((x - run, y - run, run))
    return sorted(out)


def _best_ending(items, link):
    """For every item b: the best score of a chain ending at b, by
    enumerating every chain (link(a, b) -> added score, or None)."""
    n = len(items)
    best = [None] * n

    def extend(path, score):
        b = path[-1]
        if best[b] is None or score > best[b]:
            best[b] = score
        for c in range(n):
            g = link(b, c)
            if g is not None:
                extend(path + [c], score + g)

    for a in range(n):
        extend([a], items[a][-1])
    return best


def _take_chains(items, best, link):
    """The greedy extraction: predecessors chosen from the enumerated best
    scores (the later item among those that reach the best), then chains
    taken by decreasing best score (earlier item on ties)."""
    n = len(items)
    pred = []
    for b in range(n):
        cand = [a for a in range(n) if link(a, b) is not None
                and best[a] + link(a, b) == best[b] and best[b] > items[b][-1]]
        pred.append(max(cand) if cand else -1)
    order = sorted(range(n), key=lambda b: (-best[b], b))
    used, chains = set(), []
    for b in order:
        if b in used:
            continue
        path = []
        c = b
        while c >= 0 and c not in used:
            used.add(c)
            path.append(c)
            c = pred[c]
        chains.append(path[::-1])
    return chains


def chain_tiers(seeds, g1, g2, gap_open, gap_div):
    """Both tiers of the Section 3.3 chaining on explicit seeds (x, y, L),
    with every best chain score found by enumerating chains; final chains
    (x0, x1, y0, y1, score, seeds, parts) in extraction order."""
    S = sorted(set(map(tuple, seeds)))

    def gain(a, b):
        P, Q = S[a], S[b]
        if P[0] >= Q[0] or P[1] >= Q[1]:
            return None
        if Q[0] - (P[0] + P[2]) > g1 or Q[1] - (P[1] + P[2]) > g1:
            return None
        g = min(Q[2], Q[0] + Q[2] - (P[0] + P[2]), Q[1] + Q[2] - (P[1] + P[2]))
        return g if g > 0 else None

    best = _best_ending(S, gain)
    init = []
    for ch in _take_chains(S, best, gain):
        score = S[ch[0]][2] + sum(gain(a, b) for a, b in zip(ch, ch[1:]))
        init.append((S[ch[0]][0], max(S[c][0] + S[c][2] for c in ch), S[ch[0]][1],
                     max(S[c][1] + S[c][2] for c in ch), len(ch), score))
    init.sort(key=lambda b: (b[0], b[2], b[1], b[3], b[5]))

    def pen(c, d):
        C, D = init[c], init[d]
        gq, gt = D[0] - C[1], D[2] - C[3]
        if gq < 0 or gt < 0 or gq > g2 or gt > g2:
            return None
        return gap_open + max(gq, gt) // gap_div

    def link2(c, d):
        p = pen(c, d)
        return None if p is None else init[d][5] - p

    # a link only counts when it raises the score (F = S + max(0, ...))
    best2 = _best_ending(init, lambda c, d: link2(c, d))
    best2 = [max(init[d][5], b) for d, b in enumerate(best2)]
    chains = _take_chains(init, best2, lambda c, d: (
        link2(c, d) if link2(c, d) is not None and best2[c] + link2(c, d) > init[d][5] else None))
    out = []
    for ch in chains:
        score = sum(init[c][5] for c in ch) - sum(pen(a, b) for a, b in zip(ch, ch[1:]))
        out.append((init[ch[0]][0], init[ch[-1]][1], init[ch[0]][2], init[ch[-1]][3], score,
                    sum(init[c][4] for c in ch), len(ch)))
    return out
