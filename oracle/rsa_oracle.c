/*
 * rsa_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, sequential CPU restatement of what the GPU path computes:
 * random sequential adsorption (RSA) of linear k-mers on an L x L torus run
 * to jamming, plus the k-mer count at which a wrapping cluster first appears.
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * leg may load this file's library.  It shares no code, header or table with
 * the CUDA library, and it never calls it.
 *
 * Paper: Slutskii, Barash, Tarasevich, "Percolation and jamming of random
 * sequential adsorption samples of large linear k-mers on a square lattice"
 * (arXiv:1810.06800).
 *
 *   Model (Sec. I, Sec. II.A): L x L lattice with periodic boundaries (a
 *   torus); a k-mer occupies k consecutive cells, horizontal or vertical;
 *   deposition is RSA until jamming (no further k-mer fits).
 *   Deposition (Sec. II.B): the viable-list form tries every (site,
 *   orientation) candidate exactly once, in uniformly random order, and
 *   accepts it iff all of its cells are free.  Here that random order is the
 *   ascending order of 64-bit priorities key(idx) (see oracle_key below);
 *   candidate idx = (o*L + y)*L + x, o = 0 horizontal, o = 1 vertical.
 *   Cluster labelling (Sec. II.C): union-find over k-mers, the smaller
 *   cluster is attached under the larger one (sizes are stored).
 *   Percolation (Sec. II.D): a cluster wraps the torus in one or both
 *   directions; found with per-node x/y displacements from the root
 *   (Machta / Newman-Ziff).  This file uses the exact rule "an edge inside
 *   one cluster whose lifted displacements disagree" and also evaluates the
 *   paper's |x1-x2|+|y1-y2| > 2k test so the two can be compared.
 *
 * Everything is integer arithmetic; there is no floating point here.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- splitmix64 (Steele, Lea, Flood, OOPSLA 2014; Vigna's public-domain
 * reference): state advances by the golden gamma 0x9E3779B97F4A7C15 and each
 * output is the "Mix13" finaliser of the new state. ------------------------ */
#define ORC_GAMMA 0x9E3779B97F4A7C15ULL

uint64_t oracle_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Per-sample stream base: the first splitmix64 output for state `seed`. */
uint64_t oracle_base(uint64_t seed) { return oracle_mix64(seed + ORC_GAMMA); }

/* Priority of candidate idx: output number idx+1 of splitmix64 started at the
 * sample base.  Smaller key = tried earlier. */
uint64_t oracle_key(uint64_t base, uint64_t idx)
{
    return oracle_mix64(base + ORC_GAMMA * (idx + 1));
}

void oracle_keys(uint32_t L, uint64_t seed, uint64_t *keys)
{
    uint64_t n = 2ULL * L * L, b = oracle_base(seed);
    for (uint64_t i = 0; i < n; ++i) keys[i] = oracle_key(b, i);
}

/* ---- sequential greedy scan (Sec. II.B) -------------------------------- */
typedef struct { uint64_t key; uint32_t idx; } orc_pair;

static int orc_cmp(const void *a, const void *b)
{
    const orc_pair *p = (const orc_pair *)a, *q = (const orc_pair *)b;
    if (p->key < q->key) return -1;
    if (p->key > q->key) return 1;
    return (p->idx < q->idx) ? -1 : (p->idx > q->idx);
}

/* cell (row y, column x) of cell number i of candidate idx */
static void orc_cell(uint32_t L, uint32_t idx, uint32_t i, uint32_t *y, uint32_t *x)
{
    uint32_t o = idx / (L * L), r = idx % (L * L);
    uint32_t y0 = r / L, x0 = r % L;
    if (o == 0) { *y = y0; *x = (x0 + i) % L; }
    else        { *y = (y0 + i) % L; *x = x0; }
}

/* Continue the scan over n (key, idx) pairs already sorted by key: accept a
 * candidate iff its k cells are free in occ, appending accepted idx to
 * accepted[*nj ..].  Returns 0, or -1 if two keys are equal (the order would
 * be undefined). */
static int orc_scan_more(uint32_t L, uint32_t k, const orc_pair *p, uint64_t n,
                         uint32_t *accepted, int64_t *nj, uint8_t *occ)
{
    for (uint64_t i = 1; i < n; ++i)
        if (p[i].key == p[i - 1].key) return -1;
    for (uint64_t s = 0; s < n; ++s) {
        uint32_t idx = p[s].idx, y, x, i, ok = 1;
        for (i = 0; i < k && ok; ++i) {
            orc_cell(L, idx, i, &y, &x);
            if (occ[(size_t)y * L + x]) ok = 0;
        }
        if (!ok) continue;
        for (i = 0; i < k; ++i) {
            orc_cell(L, idx, i, &y, &x);
            occ[(size_t)y * L + x] = 1;
        }
        accepted[(*nj)++] = idx;
    }
    return 0;
}

/* Scan n = 2L^2 (key, idx) pairs already sorted by key from an empty
 * lattice.  accepted[] receives the accepted idx in scan order.  Returns
 * n_j, or -1 if two keys are equal. */
static int64_t orc_scan_sorted(uint32_t L, uint32_t k, const orc_pair *p, uint64_t n,
                               uint32_t *accepted, uint8_t *occ)
{
    int64_t nj = 0;
    memset(occ, 0, (size_t)L * L);
    if (orc_scan_more(L, k, p, n, accepted, &nj, occ)) return -1;
    return nj;
}

/* Scan the 2L^2 candidates of caller-given keys in ascending key order
 * (Sec. II.B). */
int64_t oracle_scan(uint32_t L, uint32_t k, const uint64_t *keys,
                    uint32_t *accepted, uint8_t *occ)
{
    uint64_t n = 2ULL * L * L;
    orc_pair *p = (orc_pair *)malloc(n * sizeof(orc_pair));
    if (!p) return -2;
    for (uint64_t i = 0; i < n; ++i) { p[i].key = keys[i]; p[i].idx = (uint32_t)i; }
    qsort(p, n, sizeof(orc_pair), orc_cmp);
    int64_t nj = orc_scan_sorted(L, k, p, n, accepted, occ);
    free(p);
    return nj;
}

/* The same scan for the seeded priorities of oracle_keys, for the largest
 * lattices (L = 32768: 2^31 candidates): no key array is kept.  The top 16
 * bits of a key name its bucket (65536 buckets, in key order); a counting
 * pass gives each bucket's size.  The buckets are then taken in `parts`
 * consecutive runs, lowest keys first: for each run every key is generated
 * again and those of the run's buckets are written straight into their
 * bucket, each bucket is sorted by itself, and the run is scanned, the
 * lattice carrying over from the run before.  Only one run's pairs are held
 * (16 bytes x about 2L^2 / parts). */
int64_t oracle_scan_seed(uint32_t L, uint32_t k, uint64_t seed, uint32_t parts,
                         uint32_t *accepted, uint8_t *occ)
{
    const uint64_t n = 2ULL * L * L, b = oracle_base(seed), NB = 65536;
    if (parts < 1) parts = 1;
    if (parts > NB) parts = (uint32_t)NB;
    uint64_t *start = (uint64_t *)calloc(NB + 1, sizeof(uint64_t));
    uint64_t *at = (uint64_t *)malloc(NB * sizeof(uint64_t));
    if (!start || !at) { free(start); free(at); return -2; }
    for (uint64_t i = 0; i < n; ++i) start[(oracle_key(b, i) >> 48) + 1] += 1;
    for (uint64_t j = 0; j < NB; ++j) start[j + 1] += start[j];  /* bucket starts */
    uint64_t most = 0;                                          /* largest run */
    for (uint64_t q = 0; q < parts; ++q) {
        uint64_t lo = q * NB / parts, hi = (q + 1) * NB / parts;
        if (start[hi] - start[lo] > most) most = start[hi] - start[lo];
    }
    orc_pair *p = (orc_pair *)malloc((most ? most : 1) * sizeof(orc_pair));
    if (!p) { free(start); free(at); return -2; }
    memset(occ, 0, (size_t)L * L);
    int64_t nj = 0;
    for (uint64_t q = 0; q < parts; ++q) {
        const uint64_t lo = q * NB / parts, hi = (q + 1) * NB / parts, off = start[lo];
        for (uint64_t j = lo; j < hi; ++j) at[j] = start[j] - off;  /* write cursors */
        for (uint64_t i = 0; i < n; ++i) {
            uint64_t key = oracle_key(b, i), j = key >> 48;
            if (j < lo || j >= hi) continue;
            orc_pair *r = &p[at[j]++];
            r->key = key;
            r->idx = (uint32_t)i;
        }
        for (uint64_t j = lo; j < hi; ++j)
            if (start[j + 1] - start[j] > 1)
                qsort(p + (start[j] - off), start[j + 1] - start[j], sizeof(orc_pair), orc_cmp);
        if (orc_scan_more(L, k, p, start[hi] - off, accepted, &nj, occ)) { nj = -1; break; }
    }
    free(p);
    free(at);
    free(start);
    return nj;
}

/* ---- union-find with displacement vectors (Sec. II.C, II.D) ------------ */
typedef struct {
    int32_t *parent;   /* parent k-mer (scan order), self for a root   */
    int64_t *dx, *dy;  /* anchor of node minus anchor of parent (lift) */
    int64_t *size;     /* cells in the cluster (valid at roots)         */
} orc_uf;

/* Root of m, and the lifted displacement of m's anchor from that root.
 * Path compression keeps every stored displacement relative to the new
 * parent. */
static int32_t orc_find(orc_uf *u, int32_t m, int64_t *ox, int64_t *oy)
{
    int64_t sx = 0, sy = 0;
    int32_t r = m;
    while (u->parent[r] != r) { sx += u->dx[r]; sy += u->dy[r]; r = u->parent[r]; }
    /* compress: walk again, re-pointing each node straight at r */
    int64_t cx = sx, cy = sy;
    int32_t v = m;
    while (u->parent[v] != r && v != r) {
        int32_t nxt = u->parent[v];
        int64_t nx = cx - u->dx[v], ny = cy - u->dy[v];
        u->parent[v] = r; u->dx[v] = cx; u->dy[v] = cy;
        cx = nx; cy = ny; v = nxt;
    }
    *ox = sx; *oy = sy;
    return r;
}

static int64_t orc_iabs(int64_t a) { return a < 0 ? -a : a; }

/* Add accepted k-mers in scan order and return n_c: the number of k-mers
 * on the lattice when a wrapping cluster first exists (0 if none does after
 * all n_j).  *nc_paper receives the step at which the paper's test
 * |x1-x2|+|y1-y2| > 2k (comparing the root displacements of two contact
 * sites of one old cluster touched by the new k-mer) first fires.
 *
 * Exact rule: every lattice edge (a, a+d) between occupied cells is a
 * constraint lift(a) + d = lift(a+d).  An edge whose two ends already share
 * a root and whose displacements disagree closes a cycle of non-zero
 * winding, i.e. the cluster wraps. */
int64_t oracle_percolation(uint32_t L, uint32_t k, const uint32_t *accepted,
                           int64_t nj, int64_t *nc_paper)
{
    size_t LL = (size_t)L * L;
    int32_t *map = (int32_t *)malloc(LL * sizeof(int32_t));
    orc_uf u;
    u.parent = (int32_t *)malloc((size_t)(nj + 1) * sizeof(int32_t));
    u.dx = (int64_t *)malloc((size_t)(nj + 1) * sizeof(int64_t));
    u.dy = (int64_t *)malloc((size_t)(nj + 1) * sizeof(int64_t));
    u.size = (int64_t *)malloc((size_t)(nj + 1) * sizeof(int64_t));
    /* per new k-mer: the first contact site seen for each old root */
    int32_t *c_root = (int32_t *)malloc((size_t)(4 * k + 4) * sizeof(int32_t));
    int64_t *c_x = (int64_t *)malloc((size_t)(4 * k + 4) * sizeof(int64_t));
    int64_t *c_y = (int64_t *)malloc((size_t)(4 * k + 4) * sizeof(int64_t));
    if (!map || !u.parent || !u.dx || !u.dy || !u.size || !c_root || !c_x || !c_y) {
        free(map); free(u.parent); free(u.dx); free(u.dy); free(u.size);
        free(c_root); free(c_x); free(c_y);
        if (nc_paper) *nc_paper = -2;
        return -2;
    }
    for (size_t i = 0; i < LL; ++i) map[i] = -1;
    int64_t nc = 0, ncp = 0;
    static const int dirx[4] = {1, -1, 0, 0}, diry[4] = {0, 0, 1, -1};

    for (int64_t m = 0; m < nj; ++m) {
        uint32_t idx = accepted[m], o = idx / (uint32_t)LL;
        uint32_t y0 = (idx % (uint32_t)LL) / L, x0 = idx % L;
        int64_t ex = (o == 0), ey = (o == 1);   /* unit step along the k-mer */
        u.parent[m] = (int32_t)m; u.dx[m] = 0; u.dy[m] = 0; u.size[m] = k;

        /* (1) the paper's test, evaluated on the forest before m is merged */
        int nroots = 0, paper_hit = 0;
        for (uint32_t i = 0; i < k; ++i) {
            uint32_t ay, ax; orc_cell(L, idx, i, &ay, &ax);
            for (int d = 0; d < 4; ++d) {
                uint32_t by = (uint32_t)(((int64_t)ay + diry[d] + L) % L);
                uint32_t bx = (uint32_t)(((int64_t)ax + dirx[d] + L) % L);
                int32_t mp = map[(size_t)by * L + bx];
                if (mp < 0) continue;
                uint32_t idp = accepted[mp], op = idp / (uint32_t)LL;
                uint32_t yp = (idp % (uint32_t)LL) / L, xp = idp % L;
                int64_t j = (op == 0) ? (int64_t)((bx + L - xp) % L)
                                      : (int64_t)((by + L - yp) % L);
                int64_t rx, ry;
                int32_t r = orc_find(&u, mp, &rx, &ry);
                int64_t sx = rx + j * (op == 0), sy = ry + j * (op == 1);
                int c;
                for (c = 0; c < nroots; ++c) if (c_root[c] == r) break;
                if (c == nroots) { c_root[c] = r; c_x[c] = sx; c_y[c] = sy; ++nroots; }
                else if (orc_iabs(sx - c_x[c]) + orc_iabs(sy - c_y[c]) > 2 * (int64_t)k)
                    paper_hit = 1;
            }
        }

        /* (2) place m, then process every lattice edge at each of its cells */
        for (uint32_t i = 0; i < k; ++i) {
            uint32_t ay, ax; orc_cell(L, idx, i, &ay, &ax);
            map[(size_t)ay * L + ax] = (int32_t)m;
        }
        int wrap = 0;
        for (uint32_t i = 0; i < k; ++i) {
            uint32_t ay, ax; orc_cell(L, idx, i, &ay, &ax);
            for (int d = 0; d < 4; ++d) {
                uint32_t by = (uint32_t)(((int64_t)ay + diry[d] + L) % L);
                uint32_t bx = (uint32_t)(((int64_t)ax + dirx[d] + L) % L);
                int32_t mp = map[(size_t)by * L + bx];
                if (mp < 0) continue;
                uint32_t idp = accepted[mp], op = idp / (uint32_t)LL;
                uint32_t yp = (idp % (uint32_t)LL) / L, xp = idp % L;
                int64_t j = (op == 0) ? (int64_t)((bx + L - xp) % L)
                                      : (int64_t)((by + L - yp) % L);
                /* lift: anchor(mp) + j*e(mp) = anchor(m) + i*e(m) + d */
                int64_t r1x, r1y, r2x, r2y;
                int32_t r1 = orc_find(&u, (int32_t)m, &r1x, &r1y);
                int32_t r2 = orc_find(&u, mp, &r2x, &r2y);
                int64_t ax1 = r1x + (int64_t)i * ex + dirx[d];
                int64_t ay1 = r1y + (int64_t)i * ey + diry[d];
                int64_t bx2 = r2x + j * (op == 0), by2 = r2y + j * (op == 1);
                if (r1 == r2) {
                    if (ax1 != bx2 || ay1 != by2) wrap = 1;
                } else {
                    /* position of r2 relative to r1 */
                    int64_t Dx = ax1 - bx2, Dy = ay1 - by2;
                    if (u.size[r1] >= u.size[r2]) {
                        u.parent[r2] = r1; u.dx[r2] = Dx; u.dy[r2] = Dy;
                        u.size[r1] += u.size[r2];
                    } else {
                        u.parent[r1] = r2; u.dx[r1] = -Dx; u.dy[r1] = -Dy;
                        u.size[r2] += u.size[r1];
                    }
                }
            }
        }
        if (wrap && nc == 0) nc = m + 1;
        if (paper_hit && ncp == 0) ncp = m + 1;
        if (nc && ncp) break;
    }
    free(map); free(u.parent); free(u.dx); free(u.dy); free(u.size);
    free(c_root); free(c_x); free(c_y);
    if (nc_paper) *nc_paper = ncp;
    return nc;
}

/* One sample from its seed: n_j and n_c.  Returns 0, or a negative code. */
int oracle_sample(uint32_t L, uint32_t k, uint64_t seed, int64_t *nj, int64_t *nc,
                  int64_t *nc_paper)
{
    size_t n = 2ULL * L * L;
    uint64_t *keys = (uint64_t *)malloc(n * sizeof(uint64_t));
    uint32_t *acc = (uint32_t *)malloc(((size_t)L * L / k + 1) * sizeof(uint32_t));
    uint8_t *occ = (uint8_t *)malloc((size_t)L * L);
    if (!keys || !acc || !occ) { free(keys); free(acc); free(occ); return -2; }
    oracle_keys(L, seed, keys);
    int64_t j = oracle_scan(L, k, keys, acc, occ);
    int rc = 0;
    if (j < 0) rc = (int)j;
    else {
        *nj = j;
        *nc = oracle_percolation(L, k, acc, j, nc_paper);
        if (*nc < 0) rc = (int)*nc;
    }
    free(keys); free(acc); free(occ);
    return rc;
}

/* Same with caller-supplied keys (2L^2 distinct values). */
int oracle_sample_keys(uint32_t L, uint32_t k, const uint64_t *keys, int64_t *nj,
                       int64_t *nc, int64_t *nc_paper, uint32_t *accepted)
{
    uint8_t *occ = (uint8_t *)malloc((size_t)L * L);
    if (!occ) return -2;
    int64_t j = oracle_scan(L, k, keys, accepted, occ);
    free(occ);
    if (j < 0) return (int)j;
    *nj = j;
    *nc = oracle_percolation(L, k, accepted, j, nc_paper);
    return *nc < 0 ? (int)*nc : 0;
}

/* Jamming check: 1 iff no candidate has all of its k cells free. */
int oracle_is_jammed(uint32_t L, uint32_t k, const uint8_t *occ)
{
    for (uint32_t idx = 0; idx < 2u * L * L; ++idx) {
        uint32_t i, y, x, free_all = 1;
        for (i = 0; i < k && free_all; ++i) {
            orc_cell(L, idx, i, &y, &x);
            if (occ[(size_t)y * L + x]) free_all = 0;
        }
        if (free_all) return 0;
    }
    return 1;
}

/* Longest circular run of free cells along any row (horizontal) or column
 * (vertical) of an L x L occupancy map.  The lattice is jammed for k-mers iff
 * both are < k (a free run of k cells is exactly a placeable k-mer). */
void oracle_max_free_runs(uint32_t L, const uint8_t *occ, uint32_t *hrun, uint32_t *vrun)
{
    uint32_t hmax = 0, vmax = 0;
    for (int dir = 0; dir < 2; ++dir) {
        uint32_t best = 0;
        for (uint32_t line = 0; line < L; ++line) {
            /* walk the line twice to see runs that wrap round it */
            uint32_t run = 0, all_free = 1;
            for (uint32_t t = 0; t < 2 * L; ++t) {
                uint32_t i = t % L;
                uint8_t o = dir == 0 ? occ[(size_t)line * L + i] : occ[(size_t)i * L + line];
                if (o) { run = 0; all_free = 0; }
                else if (++run > best) best = run;
            }
            if (all_free) best = L;  /* an empty line holds any k <= L */
        }
        if (best > L) best = L;
        if (dir == 0) hmax = best; else vmax = best;
    }
    *hrun = hmax;
    *vrun = vmax;
}

/* Interspecific contacts (Sec. II.A, Eq. nxy): over every lattice edge
 * (cell, cell + x) and (cell, cell + y) of the torus whose two cells are
 * occupied by different k-mers, count the pairs of two horizontal k-mers
 * (nx), two vertical ones (ny) and perpendicular ones (nxy). */
int oracle_contacts(uint32_t L, uint32_t k, const uint32_t *accepted, int64_t nj,
                    int64_t *nx, int64_t *ny, int64_t *nxy)
{
    size_t LL = (size_t)L * L;
    int64_t *who = (int64_t *)malloc(LL * sizeof(int64_t));
    if (!who) return -2;
    for (size_t i = 0; i < LL; ++i) who[i] = -1;
    for (int64_t m = 0; m < nj; ++m)
        for (uint32_t i = 0; i < k; ++i) {
            uint32_t y, x;
            orc_cell(L, accepted[m], i, &y, &x);
            who[(size_t)y * L + x] = m;
        }
    int64_t cx = 0, cy = 0, cxy = 0;
    for (uint32_t y = 0; y < L; ++y)
        for (uint32_t x = 0; x < L; ++x) {
            int64_t a = who[(size_t)y * L + x];
            if (a < 0) continue;
            int64_t nb[2] = {who[(size_t)y * L + (x + 1) % L], who[(size_t)((y + 1) % L) * L + x]};
            for (int d = 0; d < 2; ++d) {
                int64_t b = nb[d];
                if (b < 0 || b == a) continue;
                int oa = accepted[a] >= LL, ob = accepted[b] >= LL;   /* 1 = vertical */
                if (oa != ob) ++cxy;
                else if (oa) ++cy;
                else ++cx;
            }
        }
    free(who);
    *nx = cx; *ny = cy; *nxy = cxy;
    return 0;
}

/* ---- the configuration of the first m accepted k-mers (Sec. II.C, II.D,
 * Sec. III "Structure of the percolating and jamming states") -------------
 *
 * Clusters are the connected components of occupied cells, 4-neighbours on
 * the torus.  Every lattice edge (a, a + e), e = +x or +y, whose two cells
 * are occupied is a constraint lift(a) + e = lift(a + e) on the lifted
 * (unwrapped) positions, lift(cell) = lift(anchor) + j e(k-mer) for the
 * cell's position j inside its k-mer.  Union-find over k-mers keeps the
 * exact int64 displacement of every k-mer's anchor from its root; an edge
 * inside one cluster whose two lifts disagree closes a cycle that winds
 * round the torus, by (mismatch_x / L, mismatch_y / L) turns.
 *
 *   counts[s] (s = 0 .. cap-1) = number of clusters made of exactly s
 *       k-mers (s k sites); needs cap >= m + 1, else -1.  May be NULL.
 *   *wrap (may be NULL) = bit 0: some cluster winds round the torus along
 *       x, bit 1: along y (any cycle with a non-zero x / y winding).
 * Returns 0, -1 on a short counts array, -2 on allocation failure. */
int oracle_configuration(uint32_t L, uint32_t k, const uint32_t *accepted, int64_t m,
                         int64_t *counts, int64_t cap, int32_t *wrap)
{
    size_t LL = (size_t)L * L;
    if (counts && cap < m + 1) return -1;
    int64_t *who = (int64_t *)malloc(LL * sizeof(int64_t));
    int64_t *jpos = (int64_t *)malloc(LL * sizeof(int64_t));
    orc_uf u;
    u.parent = (int32_t *)malloc((size_t)(m + 1) * sizeof(int32_t));
    u.dx = (int64_t *)malloc((size_t)(m + 1) * sizeof(int64_t));
    u.dy = (int64_t *)malloc((size_t)(m + 1) * sizeof(int64_t));
    u.size = (int64_t *)malloc((size_t)(m + 1) * sizeof(int64_t));
    if (!who || !jpos || !u.parent || !u.dx || !u.dy || !u.size) {
        free(who); free(jpos); free(u.parent); free(u.dx); free(u.dy); free(u.size);
        return -2;
    }
    for (size_t i = 0; i < LL; ++i) who[i] = -1;
    for (int64_t a = 0; a < m; ++a) {
        u.parent[a] = (int32_t)a; u.dx[a] = 0; u.dy[a] = 0; u.size[a] = 1;
        for (uint32_t i = 0; i < k; ++i) {
            uint32_t y, x;
            orc_cell(L, accepted[a], i, &y, &x);
            who[(size_t)y * L + x] = a;
            jpos[(size_t)y * L + x] = i;
        }
    }
    int32_t w = 0;
    for (uint32_t y = 0; y < L; ++y)
        for (uint32_t x = 0; x < L; ++x) {
            int64_t a = who[(size_t)y * L + x];
            if (a < 0) continue;
            for (int d = 0; d < 2; ++d) {             /* e = +x, then +y */
                uint32_t by = d ? (y + 1) % L : y, bx = d ? x : (x + 1) % L;
                int64_t b = who[(size_t)by * L + bx];
                if (b < 0) continue;
                int va = accepted[a] >= LL, vb = accepted[b] >= LL;   /* 1 = vertical */
                int64_t ja = jpos[(size_t)y * L + x], jb = jpos[(size_t)by * L + bx];
                int64_t oax, oay, obx, oby;
                int32_t ra = orc_find(&u, (int32_t)a, &oax, &oay);
                int32_t rb = orc_find(&u, (int32_t)b, &obx, &oby);
                /* lift(a) + e and lift(b), each relative to its own root */
                int64_t px = oax + (va ? 0 : ja) + (d == 0), py = oay + (va ? ja : 0) + (d == 1);
                int64_t qx = obx + (vb ? 0 : jb), qy = oby + (vb ? jb : 0);
                if (ra == rb) {
                    if (px != qx) w |= 1;
                    if (py != qy) w |= 2;
                } else if (u.size[ra] >= u.size[rb]) {   /* rb sits at p - q from ra */
                    u.parent[rb] = ra; u.dx[rb] = px - qx; u.dy[rb] = py - qy;
                    u.size[ra] += u.size[rb];
                } else {
                    u.parent[ra] = rb; u.dx[ra] = qx - px; u.dy[ra] = qy - py;
                    u.size[rb] += u.size[ra];
                }
            }
        }
    if (counts) {
        for (int64_t s = 0; s < cap; ++s) counts[s] = 0;
        for (int64_t a = 0; a < m; ++a)
            if (u.parent[a] == (int32_t)a) counts[u.size[a]] += 1;
    }
    if (wrap) *wrap = w;
    free(who); free(jpos); free(u.parent); free(u.dx); free(u.dy); free(u.size);
    return 0;
}
