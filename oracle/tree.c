/*
 * Oracle: the fully threaded octree (TEST INFRASTRUCTURE ONLY).
 *
 * Sec. 1 of the paper: RAMSES' mesh is an octree whose cubic cells split recursively
 * into eight octants (Khokhlov 1998), and space is ordered along the Peano-Hilbert
 * curve.  Conventions here: level l has 2^l cells per dimension; an oct at level l is
 * 2^3 level-l cells, has oct coordinates (ix,iy,iz) in [0, 2^(l-1)) and a father cell
 * at level l-1 with cell coordinates (ix,iy,iz).  Cell c = cx + 2 cy + 4 cz inside the
 * oct, cell id = oct*8 + c.  Octs are numbered by (level, Hilbert key).
 *
 * Tables are found by plain geometric search in an ordered map keyed by
 * (level, ix, iy, iz) -- independent of the Hilbert keys used for the numbering.
 */
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

/* Skilling 2004, "Programming the Hilbert curve": the coordinates are turned in place
   into the transposed Hilbert index (inverse undo, then Gray encoding), whose bits are
   interleaved most significant first with x as the high bit of each triple. */
uint64_t or_hilbert_key(int bits, uint32_t x, uint32_t y, uint32_t z)
{
    if (bits <= 0) return 0;
    uint32_t X[3] = { x, y, z };
    uint32_t M = 1u << (bits - 1);
    for (uint32_t Q = M; Q > 1; Q >>= 1) {
        uint32_t P = Q - 1;
        for (int i = 0; i < 3; i++) {
            if (X[i] & Q) {
                X[0] ^= P;
            } else {
                uint32_t t = (X[0] ^ X[i]) & P;
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    X[1] ^= X[0];
    X[2] ^= X[1];
    uint32_t t = 0;
    for (uint32_t Q = M; Q > 1; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1;
    for (int i = 0; i < 3; i++) X[i] ^= t;
    uint64_t key = 0;
    for (int b = bits - 1; b >= 0; b--)
        for (int i = 0; i < 3; i++) key = (key << 1) | ((X[i] >> b) & 1u);
    return key;
}

/* ---- ordered map (level, ix, iy, iz) -> oct ---------------------------------- */
static const or_tree *g_sort_tree;   /* qsort has no context argument */

static int cmp_lex(const void *a, const void *b)
{
    const or_tree *t = g_sort_tree;
    int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
    if (t->lvl[i] != t->lvl[j]) return t->lvl[i] < t->lvl[j] ? -1 : 1;
    if (t->ix[i] != t->ix[j]) return t->ix[i] < t->ix[j] ? -1 : 1;
    if (t->iy[i] != t->iy[j]) return t->iy[i] < t->iy[j] ? -1 : 1;
    if (t->iz[i] != t->iz[j]) return t->iz[i] < t->iz[j] ? -1 : 1;
    return 0;
}

int64_t or_lookup(const or_tree *t, int l, int64_t x, int64_t y, int64_t z)
{
    int64_t lo = 0, hi = t->noct - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2, o = t->lex[mid];
        int c;
        if (t->lvl[o] != l) c = t->lvl[o] < l ? -1 : 1;
        else if (t->ix[o] != x) c = t->ix[o] < x ? -1 : 1;
        else if (t->iy[o] != y) c = t->iy[o] < y ? -1 : 1;
        else if (t->iz[o] != z) c = t->iz[o] < z ? -1 : 1;
        else return o;
        if (c < 0) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

typedef struct { int32_t l, x, y, z; uint64_t key; } rec;
static int cmp_rec(const void *a, const void *b)
{
    const rec *p = a, *q = b;
    if (p->l != q->l) return p->l < q->l ? -1 : 1;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    return 0;
}

/* Apply the box boundary at level l (2^l cells per dimension) to one cell coordinate.
   Returns 0 and the wrapped coordinate, or 1 if it lies beyond an outflow boundary. */
static int bc_coord(const or_tree *t, int axis, int l, int64_t *c)
{
    int64_t n = (int64_t)1 << l;
    if (*c >= 0 && *c < n) return 0;
    int face = 2 * axis + (*c >= n ? 1 : 0);
    if (t->bc[face] == OR_BC_PERIODIC) {
        *c = ((*c % n) + n) % n;
        return 0;
    }
    return 1;
}

/* id of the cell at level l with cell coordinates (X,Y,Z) (already inside the box), or -1 */
static int64_t cell_at(const or_tree *t, int l, int64_t X, int64_t Y, int64_t Z)
{
    if (l < 1) return -1;
    int64_t o = or_lookup(t, l, X >> 1, Y >> 1, Z >> 1);
    if (o < 0) return -1;
    return o * 8 + (X & 1) + 2 * (Y & 1) + 4 * (Z & 1);
}

int or_tree_build(int32_t levelmin, const int32_t *bc, const int32_t *lxyz, int64_t n, or_tree **out)
{
    *out = NULL;
    if (n <= 0 || levelmin < 1 || levelmin > OR_MAXLEV) return OR_EINVAL;
    for (int f = 0; f < 6; f++) if (bc[f] != OR_BC_PERIODIC && bc[f] != OR_BC_OUTFLOW) return OR_EINVAL;
    for (int a = 0; a < 3; a++)
        if ((bc[2 * a] == OR_BC_PERIODIC) != (bc[2 * a + 1] == OR_BC_PERIODIC)) return OR_EINVAL;
    rec *r = malloc(sizeof(rec) * n);
    int lmax = 0;
    for (int64_t i = 0; i < n; i++) {
        int l = lxyz[4 * i];
        if (l < 1 || l > OR_MAXLEV) { free(r); return OR_EINVAL; }
        int64_t lim = (int64_t)1 << (l - 1);
        for (int a = 1; a < 4; a++)
            if (lxyz[4 * i + a] < 0 || lxyz[4 * i + a] >= lim) { free(r); return OR_EINVAL; }
        r[i].l = l; r[i].x = lxyz[4 * i + 1]; r[i].y = lxyz[4 * i + 2]; r[i].z = lxyz[4 * i + 3];
        r[i].key = or_hilbert_key(l - 1, r[i].x, r[i].y, r[i].z);
        if (l > lmax) lmax = l;
    }
    qsort(r, n, sizeof(rec), cmp_rec);
    for (int64_t i = 1; i < n; i++)
        if (r[i].l == r[i - 1].l && r[i].key == r[i - 1].key) { free(r); return OR_EINVAL; }

    or_tree *t = calloc(1, sizeof(or_tree));
    t->levelmin = levelmin; t->levelmax = lmax; t->noct = n;
    memcpy(t->bc, bc, sizeof(t->bc));
    t->lvl = malloc(4 * n); t->ix = malloc(4 * n); t->iy = malloc(4 * n); t->iz = malloc(4 * n);
    t->key = malloc(8 * n); t->son = malloc(4 * 8 * n); t->father = malloc(4 * n);
    t->nbor = malloc(4 * 6 * n); t->nb27 = malloc(4 * 27 * n); t->lex = malloc(8 * n);
    for (int64_t i = 0; i < n; i++) {
        t->lvl[i] = r[i].l; t->ix[i] = r[i].x; t->iy[i] = r[i].y; t->iz[i] = r[i].z; t->key[i] = r[i].key;
        t->lex[i] = i;
    }
    free(r);
    for (int l = 0; l <= OR_MAXLEV + 1; l++) {
        int64_t k = 0;
        while (k < n && t->lvl[k] < l) k++;
        t->lvl_off[l] = k;
    }
    g_sort_tree = t;
    qsort(t->lex, n, sizeof(int64_t), cmp_lex);

    int st = OR_OK;
    /* levels 1..levelmin are complete */
    for (int l = 1; l <= levelmin; l++) {
        int64_t want = (int64_t)1 << (3 * (l - 1));
        if (t->lvl_off[l + 1] - t->lvl_off[l] != want) st = OR_EINVAL;
    }
    for (int64_t o = 0; o < n && st == OR_OK; o++) {
        int l = t->lvl[o];
        for (int c = 0; c < 8; c++) {
            int64_t s = or_lookup(t, l + 1, 2 * (int64_t)t->ix[o] + (c & 1), 2 * (int64_t)t->iy[o] + ((c >> 1) & 1),
                                  2 * (int64_t)t->iz[o] + ((c >> 2) & 1));
            t->son[8 * o + c] = (int32_t)s;
        }
        if (l == 1) {
            t->father[o] = -1;
            for (int k = 0; k < 6; k++) t->nbor[6 * o + k] = -1;
            for (int k = 0; k < 27; k++) t->nb27[27 * o + k] = (k == 13) ? (int32_t)o : OR_OUTSIDE;
            continue;
        }
        int64_t f = cell_at(t, l - 1, t->ix[o], t->iy[o], t->iz[o]);
        if (f < 0) { st = OR_EINVAL; break; }   /* an oct without its father cell */
        t->father[o] = (int32_t)f;
        for (int k = 0; k < 6; k++) {
            int64_t P[3] = { t->ix[o], t->iy[o], t->iz[o] };
            P[k / 2] += (k & 1) ? 1 : -1;
            int out = 0;
            for (int a = 0; a < 3; a++) out |= bc_coord(t, a, l - 1, &P[a]);
            if (out) { t->nbor[6 * o + k] = -1; continue; }
            int64_t cid = cell_at(t, l - 1, P[0], P[1], P[2]);
            if (cid < 0) { st = OR_EUNBALANCED; break; }
            t->nbor[6 * o + k] = (int32_t)cid;
        }
        for (int dz = -1; dz <= 1 && st == OR_OK; dz++)
            for (int dy = -1; dy <= 1 && st == OR_OK; dy++)
                for (int dx = -1; dx <= 1 && st == OR_OK; dx++) {
                    int k = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
                    int64_t P[3] = { t->ix[o] + dx, t->iy[o] + dy, t->iz[o] + dz };
                    int out = 0;
                    for (int a = 0; a < 3; a++) out |= bc_coord(t, a, l - 1, &P[a]);
                    if (out) { t->nb27[27 * o + k] = OR_OUTSIDE; continue; }
                    /* 2:1 balance: every father-level neighbour of an oct's father exists */
                    int64_t cid = cell_at(t, l - 1, P[0], P[1], P[2]);
                    if (cid < 0) { st = OR_EUNBALANCED; break; }
                    int64_t s = or_lookup(t, l, P[0], P[1], P[2]);
                    t->nb27[27 * o + k] = s >= 0 ? (int32_t)s : (int32_t)(-1 - cid);
                }
    }
    if (st == OR_OK) {
        /* levels below levelmin carry no leaves */
        for (int64_t o = 0; o < t->lvl_off[levelmin]; o++)
            for (int c = 0; c < 8; c++) if (t->son[8 * o + c] < 0) st = OR_EINVAL;
    }
    if (st != OR_OK) { or_tree_free(t); return st; }
    *out = t;
    return OR_OK;
}

void or_tree_free(or_tree *t)
{
    if (!t) return;
    free(t->lvl); free(t->ix); free(t->iy); free(t->iz); free(t->key); free(t->son);
    free(t->father); free(t->nbor); free(t->nb27); free(t->lex); free(t);
}

int64_t or_tree_noct(const or_tree *t) { return t->noct; }

void or_tree_export(const or_tree *t, int32_t *lvl, int32_t *ix, int32_t *iy, int32_t *iz, uint64_t *key,
                    int32_t *son, int32_t *father, int32_t *nbor, int32_t *nb27, int64_t *lvl_off)
{
    int64_t n = t->noct;
    if (lvl) memcpy(lvl, t->lvl, 4 * n);
    if (ix) memcpy(ix, t->ix, 4 * n);
    if (iy) memcpy(iy, t->iy, 4 * n);
    if (iz) memcpy(iz, t->iz, 4 * n);
    if (key) memcpy(key, t->key, 8 * n);
    if (son) memcpy(son, t->son, 4 * 8 * n);
    if (father) memcpy(father, t->father, 4 * n);
    if (nbor) memcpy(nbor, t->nbor, 4 * 6 * n);
    if (nb27) memcpy(nb27, t->nb27, 4 * 27 * n);
    if (lvl_off) memcpy(lvl_off, t->lvl_off, 8 * (OR_MAXLEV + 2));
}
