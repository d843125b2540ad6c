"""Brute-force checkers for tiny lattices -- TEST INFRASTRUCTURE.

Independent pure-Python restatements used to pin the C oracle against the
paper's definitions rather than against itself:

* :func:`wraps` -- a cluster wraps the torus (Sec. II.D) iff a breadth-first
  search that carries unwrapped ("lifted") coordinates reaches some occupied
  cell at two different lifts.  No union-find, no displacement bookkeeping.
* :func:`rsa_exact_distribution` -- the exact law of (n_j, n_c) for RSA
  (Sec. II.A, II.B) as a Markov chain over packings: each attempt picks one of
  the 2 L^2 (site, orientation) candidates uniformly, so the next accepted
  k-mer is uniform over the currently viable candidates.
* :func:`maximal_packings` -- every jammed configuration, for checking the
  Appendix A Proposition (every cluster of a jammed torus wraps).
"""
from __future__ import annotations

from collections import deque
from fractions import Fraction
from functools import lru_cache


def cells_of(L: int, k: int, idx: int):
    """Cells (y, x) of candidate idx = (o*L + y)*L + x."""
    o, r = divmod(idx, L * L)
    y, x = divmod(r, L)
    if o == 0:
        return [(y, (x + i) % L) for i in range(k)]
    return [((y + i) % L, x) for i in range(k)]


def wraps(L: int, occupied) -> bool:
    """True iff some 4-connected cluster of occupied cells on the L x L torus
    winds around it, in x or in y.  BFS assigns each reached cell an integer
    lift; an edge to an already-lifted cell at a different lift closes a cycle
    that goes round the torus."""
    occ = set(occupied)
    lift = {}
    for start in occ:
        if start in lift:
            continue
        lift[start] = start
        q = deque([start])
        while q:
            a = q.popleft()
            ly, lx = lift[a]
            for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)):
                b = ((a[0] + dy) % L, (a[1] + dx) % L)
                if b not in occ:
                    continue
                want = (ly + dy, lx + dx)
                if b in lift:
                    if lift[b] != want:
                        return True
                else:
                    lift[b] = want
                    q.append(b)
    return False


def wrap_dirs(L: int, occupied):
    """(winds along x, winds along y) for the occupied cells: the same lifted
    breadth-first search as :func:`wraps`, run to the end; every edge that
    reaches an already-lifted cell at another lift is a cycle whose winding is
    (lift difference) / L, and a direction counts if any such cycle moves
    along it."""
    occ = set(occupied)
    lift = {}
    wx = wy = False
    for start in occ:
        if start in lift:
            continue
        lift[start] = start
        q = deque([start])
        while q:
            a = q.popleft()
            ly, lx = lift[a]
            for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)):
                b = ((a[0] + dy) % L, (a[1] + dx) % L)
                if b not in occ:
                    continue
                want = (ly + dy, lx + dx)
                if b in lift:
                    wy |= lift[b][0] != want[0]
                    wx |= lift[b][1] != want[1]
                else:
                    lift[b] = want
                    q.append(b)
    return wx, wy


def clusters(L: int, occupied):
    """List of clusters (sets of cells), 4-neighbour connectivity on the torus."""
    occ = set(occupied)
    seen, out = set(), []
    for s in occ:
        if s in seen:
            continue
        comp, q = {s}, deque([s])
        seen.add(s)
        while q:
            a = q.popleft()
            for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)):
                b = ((a[0] + dy) % L, (a[1] + dx) % L)
                if b in occ and b not in seen:
                    seen.add(b)
                    comp.add(b)
                    q.append(b)
        out.append(comp)
    return out


def nc_bruteforce(L: int, k: int, accepted) -> int:
    """First m such that the first m accepted k-mers contain a wrapping
    cluster (0 if none)."""
    occ = []
    for m, idx in enumerate(accepted, start=1):
        occ.extend(cells_of(L, k, int(idx)))
        if wraps(L, occ):
            return m
    return 0


def greedy(L: int, k: int, order):
    """Accept candidates in the given order iff all cells are free."""
    occ, acc = set(), []
    for idx in order:
        c = cells_of(L, k, idx)
        if not any(p in occ for p in c):
            occ.update(c)
            acc.append(idx)
    return acc


def viable(L: int, k: int, occ):
    return [i for i in range(2 * L * L) if not any(p in occ for p in cells_of(L, k, i))]


def rsa_exact_distribution(L: int, k: int):
    """Exact law of (n_j, n_c) under RSA, as {(n_j, n_c): Fraction}."""
    n = 2 * L * L
    cell_sets = [frozenset(cells_of(L, k, i)) for i in range(n)]

    @lru_cache(maxsize=None)
    def go(occ: frozenset, m: int, nc: int):
        via = [i for i in range(n) if not (cell_sets[i] & occ)]
        if not via:
            return ((m, nc, Fraction(1)),)
        out = {}
        p = Fraction(1, len(via))
        for i in via:
            nocc = occ | cell_sets[i]
            nnc = nc if nc else (m + 1 if wraps(L, nocc) else 0)
            for (mj, mc, q) in go(nocc, m + 1, nnc):
                out[(mj, mc)] = out.get((mj, mc), Fraction(0)) + p * q
        return tuple((a, b, v) for (a, b), v in sorted(out.items()))

    return {(a, b): v for (a, b, v) in go(frozenset(), 0, 0)}


def maximal_packings(L: int, k: int):
    """All jammed packings (maximal sets of non-overlapping k-mers), as
    frozensets of occupied cells (orientation-free, so duplicates merge)."""
    n = 2 * L * L
    cell_sets = [frozenset(cells_of(L, k, i)) for i in range(n)]
    # a k-mer with k = L wraps onto itself; it is still a single candidate
    found = set()

    def rec(start: int, occ: frozenset):
        extended = False
        for i in range(start, n):
            if not (cell_sets[i] & occ):
                extended = True
                rec(i + 1, occ | cell_sets[i])
        if not extended:
            # maximal only if no candidate at all (even before start) fits
            if all(cell_sets[i] & occ for i in range(n)):
                found.add(occ)

    rec(0, frozenset())
    return found


def contacts(L: int, k: int, accepted):
    """Interspecific contacts by brute force: every unordered pair of
    4-adjacent occupied cells of different k-mers, once per lattice edge
    (so L = 2 counts both edges of a pair), classified by orientations."""
    owner = {}
    for m, idx in enumerate(accepted):
        for c in cells_of(L, k, int(idx)):
            owner[c] = (m, int(idx) >= L * L)
    nx = ny = nxy = 0
    for (y, x), (m, vert) in owner.items():
        for b in (((y + 1) % L, x), (y, (x + 1) % L)):
            if b in owner and owner[b][0] != m:
                ob = owner[b][1]
                if ob != vert:
                    nxy += 1
                elif vert:
                    ny += 1
                else:
                    nx += 1
    return nx, ny, nxy
