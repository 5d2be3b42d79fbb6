/*
 * svt_oracle.c -- plain serial CPU oracle for the SVT track-fitting chain.
 *
 * TEST INFRASTRUCTURE ONLY (see svt_oracle.h): the definitions written out
 * one step at a time, with no blocking, fusion or reordering, so that each
 * function can be read against the paper's Sec. II / II-A and the readings
 * listed in svt_oracle.h.  Slow on purpose.
 */
#include "svt_oracle.h"

#include <stdlib.h>
#include <string.h>

#define N_LAYERS 5
#define MAX_HITS 8
#define MAX_ROADS_PER_EVENT 256

/* ------------------------------------------------------------------------ */
/* unpack (Sec. II-A: "unpacking of input data and filling of all the        */
/* necessary data structures")                                               */
/* ------------------------------------------------------------------------ */

static int word_fields_ok(uint32_t w)
{
    uint32_t ee = (w >> 31) & 1u, ep = (w >> 30) & 1u;
    uint32_t type = (w >> 27) & 7u, payload = w & 0x07FFFFFFu;
    (void)ee;
    (void)ep;
    if (type <= 4)
        return (payload >> 12) == 0;
    if (type == 5 || type == 6)
        return (payload >> 16) == 0;
    /* header */
    if ((payload >> 10) != 0)
        return 0;
    if ((payload & 15u) >= 12)
        return 0;
    if (((payload >> 4) & 7u) >= 6)
        return 0;
    if (((payload >> 7) & 7u) >= 5)
        return 0;
    return 1;
}

static int32_t sign_extend16(uint32_t v)
{
    v &= 0xFFFFu;
    return v >= 0x8000u ? (int32_t)v - 65536 : (int32_t)v;
}

/* Walk the words once.  Stores at most cap roads (roads may be NULL). */
int orc_unpack(const uint32_t *words, size_t n_words, orc_road *roads,
               size_t cap, size_t *n_roads, size_t *n_events, size_t *err_pos)
{
    size_t nr = 0, ne = 0;
    size_t pos_in_road = 0;          /* words seen so far in the open road */
    uint32_t road_in_event = 0;      /* roads closed so far in the open event */
    orc_road cur;
    memset(&cur, 0, sizeof cur);
    *n_roads = 0;
    *n_events = 0;
    *err_pos = 0;

    for (size_t i = 0; i < n_words; ++i) {
        uint32_t w = words[i];
        uint32_t ee = (w >> 31) & 1u, ep = (w >> 30) & 1u;
        uint32_t type = (w >> 27) & 7u, payload = w & 0x07FFFFFFu;

        /* 1. field checks */
        if (!word_fields_ok(w)) {
            *err_pos = i;
            return ORC_E_BADWORD;
        }
        /* 2. EE only together with EP */
        if (ee && !ep) {
            *err_pos = i;
            return ORC_E_BADWORD;
        }
        /* 3. type expected at this position of the road */
        if (pos_in_road == 0 && type != 7) { *err_pos = i; return ORC_E_BADWORD; }
        if (pos_in_road == 1 && type != 5) { *err_pos = i; return ORC_E_BADWORD; }
        if (pos_in_road == 2 && type != 6) { *err_pos = i; return ORC_E_BADWORD; }
        if (pos_in_road >= 3 && type > 4) { *err_pos = i; return ORC_E_BADWORD; }
        /* 4. a road has at least header, curvature and phi */
        if (ep && pos_in_road < 2) {
            *err_pos = i;
            return ORC_E_BADWORD;
        }
        /* 5. limits */
        if (pos_in_road == 0 && road_in_event >= MAX_ROADS_PER_EVENT) {
            *err_pos = i;
            return ORC_E_LIMIT;
        }
        if (pos_in_road >= 3 && cur.n[type] >= MAX_HITS) {
            *err_pos = i;
            return ORC_E_LIMIT;
        }

        /* the word is good: record it */
        if (pos_in_road == 0) {
            memset(&cur, 0, sizeof cur);
            cur.event = (uint32_t)ne;
            cur.road = road_in_event;
            cur.wedge = (int32_t)(payload & 15u);
            cur.barrel = (int32_t)((payload >> 4) & 7u);
            cur.excl = (int32_t)((payload >> 7) & 7u);
        } else if (pos_in_road == 1) {
            cur.curv = sign_extend16(payload);
        } else if (pos_in_road == 2) {
            cur.phi = sign_extend16(payload);
        } else {
            cur.coord[type][cur.n[type]] = (uint16_t)(payload & 0xFFFu);
            cur.n[type] += 1;
        }
        pos_in_road += 1;

        if (ep) {                       /* road closed */
            if (roads && nr < cap)
                roads[nr] = cur;
            nr += 1;
            road_in_event += 1;
            pos_in_road = 0;
        }
        if (ee) {                       /* event closed */
            ne += 1;
            road_in_event = 0;
        }
    }
    *n_roads = nr;
    *n_events = ne;
    if (pos_in_road != 0 || road_in_event != 0) {
        *err_pos = n_words;
        return ORC_E_TRUNCATED;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* fit (Sec. II: p_i = f_i . x_i + q_i with integer multiply and add)        */
/* ------------------------------------------------------------------------ */

/* floor(a / 4096): C division truncates toward zero, so a negative value
 * that is not a multiple of 4096 is one below the truncated quotient. */
static int64_t floor_div_4096(int64_t a)
{
    int64_t q = a / 4096;
    if (a < 0 && a % 4096 != 0)
        q -= 1;
    return q;
}

/* Fit one combination.  d[l] = hit index used on layer l. */
static void fit_one(const orc_road *r, const orc_consts *c, const int d[N_LAYERS],
                    int32_t p[3], int64_t *chi2)
{
    int32_t x[6];
    int j = 0;
    for (int l = 0; l < N_LAYERS; ++l) {
        if (l == r->excl)
            continue;
        x[j++] = (int32_t)r->coord[l][d[l]];
    }
    x[4] = r->curv;
    x[5] = r->phi;

    int s = (r->wedge * 6 + r->barrel) * 5 + r->excl;
    const int16_t *F = c->F + (size_t)s * 18;
    const int16_t *C = c->C + (size_t)s * 18;
    const int32_t *q = c->q + (size_t)s * 3;
    const int32_t *k = c->k + (size_t)s * 3;

    for (int i = 0; i < 3; ++i) {
        int64_t acc = 0;
        for (int jj = 0; jj < 6; ++jj) {
            int32_t prod = (int32_t)F[i * 6 + jj] * x[jj];   /* int32 product */
            acc += (int64_t)prod;                            /* int64 sum */
        }
        p[i] = (int32_t)(floor_div_4096(acc) + q[i]);
    }
    int64_t sum = 0;
    for (int kk = 0; kk < 3; ++kk) {
        int64_t acc = 0;
        for (int jj = 0; jj < 6; ++jj) {
            int32_t prod = (int32_t)C[kk * 6 + jj] * x[jj];
            acc += (int64_t)prod;
        }
        int64_t a = floor_div_4096(acc) + k[kk];
        sum += a * a;
    }
    *chi2 = sum;
}

/* ------------------------------------------------------------------------ */
/* growable arrays                                                           */
/* ------------------------------------------------------------------------ */

typedef struct {
    orc_fit *v;
    size_t n, cap;
} fit_vec;

static int fv_push(fit_vec *a, const orc_fit *f)
{
    if (a->n == a->cap) {
        size_t nc = a->cap ? a->cap * 2 : 1024;
        orc_fit *nv = (orc_fit *)realloc(a->v, nc * sizeof *nv);
        if (!nv)
            return ORC_E_NOMEM;
        a->v = nv;
        a->cap = nc;
    }
    a->v[a->n++] = *f;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* combine (Sec. II: "all possible combinations of hits inside a road")      */
/* ------------------------------------------------------------------------ */

/* Append every combination of road r (canonical comb order). */
static int combine_and_fit(const orc_road *r, const orc_consts *c, int64_t cut,
                           fit_vec *out)
{
    int S[N_LAYERS];
    S[0] = 1;
    for (int l = 1; l < N_LAYERS; ++l)
        S[l] = S[l - 1] * r->n[l - 1];

    int d[N_LAYERS];
    for (d[4] = 0; d[4] < r->n[4]; ++d[4])
        for (d[3] = 0; d[3] < r->n[3]; ++d[3])
            for (d[2] = 0; d[2] < r->n[2]; ++d[2])
                for (d[1] = 0; d[1] < r->n[1]; ++d[1])
                    for (d[0] = 0; d[0] < r->n[0]; ++d[0]) {
                        orc_fit f;
                        memset(&f, 0, sizeof f);
                        f.event = r->event;
                        f.road = r->road;
                        f.comb = 0;
                        for (int l = 0; l < N_LAYERS; ++l) {
                            f.comb += (uint32_t)(d[l] * S[l]);
                            f.coord[l] = r->coord[l][d[l]];
                        }
                        fit_one(r, c, d, f.p, &f.chi2);
                        f.pass = f.chi2 <= cut;
                        int rc = fv_push(out, &f);
                        if (rc)
                            return rc;
                    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* hit-warrior                                                               */
/* ------------------------------------------------------------------------ */

/* key(a) < key(b), key = (chi2, road, comb) */
static int key_less(const orc_fit *a, const orc_fit *b)
{
    if (a->chi2 != b->chi2)
        return a->chi2 < b->chi2;
    if (a->road != b->road)
        return a->road < b->road;
    return a->comb < b->comb;
}

static int shared_hits(const orc_fit *a, const orc_fit *b)
{
    int s = 0;
    for (int l = 0; l < N_LAYERS; ++l)
        s += a->coord[l] == b->coord[l];
    return s;
}

/* The rule as stated: t dropped iff a passing u with a lower key shares >= 3
 * hits with it.  O(n^2) per event. */
static void warrior_pairwise(const orc_fit *t, size_t n, char *dropped)
{
    for (size_t i = 0; i < n; ++i) {
        dropped[i] = 0;
        for (size_t j = 0; j < n; ++j) {
            if (j == i)
                continue;
            if (key_less(&t[j], &t[i]) && shared_hits(&t[j], &t[i]) >= 3) {
                dropped[i] = 1;
                break;
            }
        }
    }
}

/* The same rule through layer triples: sharing >= 3 hits means agreeing on
 * all three layers of at least one of the ten triples, so t is dropped iff,
 * in some triple's group of tracks with t's three coordinates, t is not the
 * lowest key.  One sort per triple. */
typedef struct {
    uint64_t group;          /* the three coordinates on the triple */
    const orc_fit *f;
    size_t idx;
} proj_rec;

static int proj_cmp(const void *pa, const void *pb)
{
    const proj_rec *a = (const proj_rec *)pa, *b = (const proj_rec *)pb;
    if (a->group != b->group)
        return a->group < b->group ? -1 : 1;
    if (key_less(a->f, b->f))
        return -1;
    if (key_less(b->f, a->f))
        return 1;
    return 0;
}

static int warrior_projection(const orc_fit *t, size_t n, char *dropped)
{
    static const int triples[10][3] = {
        {0, 1, 2}, {0, 1, 3}, {0, 1, 4}, {0, 2, 3}, {0, 2, 4},
        {0, 3, 4}, {1, 2, 3}, {1, 2, 4}, {1, 3, 4}, {2, 3, 4}};
    proj_rec *rec = (proj_rec *)malloc((n ? n : 1) * sizeof *rec);
    if (!rec)
        return ORC_E_NOMEM;
    for (size_t i = 0; i < n; ++i)
        dropped[i] = 0;
    for (int T = 0; T < 10; ++T) {
        for (size_t i = 0; i < n; ++i) {
            rec[i].group = ((uint64_t)t[i].coord[triples[T][0]] << 24) |
                           ((uint64_t)t[i].coord[triples[T][1]] << 12) |
                           (uint64_t)t[i].coord[triples[T][2]];
            rec[i].f = &t[i];
            rec[i].idx = i;
        }
        qsort(rec, n, sizeof *rec, proj_cmp);
        for (size_t i = 1; i < n; ++i)
            if (rec[i].group == rec[i - 1].group)   /* not first of its group */
                dropped[rec[i].idx] = 1;
    }
    free(rec);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* drivers                                                                   */
/* ------------------------------------------------------------------------ */

static int unpack_all(const uint32_t *words, size_t n_words, orc_road **roads,
                      size_t *n_roads, size_t *n_events)
{
    size_t err_pos, nr, ne;
    int rc = orc_unpack(words, n_words, NULL, 0, &nr, &ne, &err_pos);
    *roads = NULL;
    *n_roads = 0;
    *n_events = 0;
    if (rc)
        return rc;
    *roads = (orc_road *)malloc((nr ? nr : 1) * sizeof **roads);
    if (!*roads)
        return ORC_E_NOMEM;
    rc = orc_unpack(words, n_words, *roads, nr, &nr, &ne, &err_pos);
    *n_roads = nr;
    *n_events = ne;
    return rc;
}

int orc_fit_all(const uint32_t *words, size_t n_words, const orc_consts *c,
                int64_t cut, orc_fit **out, size_t *n_out)
{
    orc_road *roads;
    size_t nr, ne;
    fit_vec all = {0, 0, 0};
    *out = NULL;
    *n_out = 0;
    int rc = unpack_all(words, n_words, &roads, &nr, &ne);
    for (size_t r = 0; rc == ORC_OK && r < nr; ++r)
        rc = combine_and_fit(&roads[r], c, cut, &all);
    free(roads);
    if (rc) {
        free(all.v);
        return rc;
    }
    *out = all.v;
    *n_out = all.n;
    return ORC_OK;
}

int orc_chi2_all(const uint32_t *words, size_t n_words, const orc_consts *c,
                 int64_t **out, size_t *n_out)
{
    orc_road *roads;
    size_t nr, ne;
    *out = NULL;
    *n_out = 0;
    int rc = unpack_all(words, n_words, &roads, &nr, &ne);
    if (rc) {
        free(roads);
        return rc;
    }
    size_t total = 0;
    for (size_t r = 0; r < nr; ++r) {
        size_t m = 1;
        for (int l = 0; l < N_LAYERS; ++l)
            m *= (size_t)roads[r].n[l];
        total += m;
    }
    int64_t *chi = (int64_t *)malloc((total ? total : 1) * sizeof *chi);
    fit_vec tmp = {0, 0, 0};
    size_t k = 0;
    if (!chi)
        rc = ORC_E_NOMEM;
    for (size_t r = 0; rc == ORC_OK && r < nr; ++r) {
        tmp.n = 0;
        rc = combine_and_fit(&roads[r], c, 0, &tmp);
        for (size_t i = 0; rc == ORC_OK && i < tmp.n; ++i)
            chi[k++] = tmp.v[i].chi2;
    }
    free(tmp.v);
    free(roads);
    if (rc) {
        free(chi);
        return rc;
    }
    *out = chi;
    *n_out = k;
    return ORC_OK;
}

int orc_run(const uint32_t *words, size_t n_words, const orc_consts *c,
            int64_t cut, int warrior, orc_fit **out, size_t *n_out)
{
    orc_road *roads;
    size_t nr, ne;
    fit_vec ev_fits = {0, 0, 0}, passing = {0, 0, 0}, result = {0, 0, 0};
    char *dropped = NULL;
    size_t dropped_cap = 0;
    *out = NULL;
    *n_out = 0;
    int rc = unpack_all(words, n_words, &roads, &nr, &ne);

    size_t r = 0;
    while (rc == ORC_OK && r < nr) {
        /* one event at a time: combine + fit + cut over all its roads */
        uint32_t ev = roads[r].event;
        ev_fits.n = 0;
        passing.n = 0;
        for (; r < nr && roads[r].event == ev && rc == ORC_OK; ++r)
            rc = combine_and_fit(&roads[r], c, cut, &ev_fits);
        for (size_t i = 0; rc == ORC_OK && i < ev_fits.n; ++i)
            if (ev_fits.v[i].pass)
                rc = fv_push(&passing, &ev_fits.v[i]);
        if (rc)
            break;
        /* hit-warrior over the event's passing combinations */
        if (passing.n > dropped_cap) {
            free(dropped);
            dropped_cap = passing.n;
            dropped = (char *)malloc(dropped_cap);
            if (!dropped) {
                rc = ORC_E_NOMEM;
                break;
            }
        }
        if (warrior == 0)
            warrior_pairwise(passing.v, passing.n, dropped);
        else if (warrior == 1)
            rc = warrior_projection(passing.v, passing.n, dropped);
        else
            for (size_t i = 0; i < passing.n; ++i)
                dropped[i] = 0;
        for (size_t i = 0; rc == ORC_OK && i < passing.n; ++i)
            if (!dropped[i])
                rc = fv_push(&result, &passing.v[i]);
    }
    free(roads);
    free(ev_fits.v);
    free(passing.v);
    free(dropped);
    if (rc) {
        free(result.v);
        return rc;
    }
    *out = result.v;
    *n_out = result.n;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* one event at a time (the event-parallel driver, svt_oracle_mt.c, calls     */
/* these; they take the same steps as orc_run's loop over one event)          */
/* ------------------------------------------------------------------------ */

int orc_event_fits(const orc_road *roads, size_t n_roads, const orc_consts *c, int64_t cut,
                   orc_fit **passing, size_t *n_passing)
{
    fit_vec all = {0, 0, 0}, pass = {0, 0, 0};
    int rc = ORC_OK;
    *passing = NULL;
    *n_passing = 0;
    for (size_t r = 0; rc == ORC_OK && r < n_roads; ++r)
        rc = combine_and_fit(&roads[r], c, cut, &all);
    for (size_t i = 0; rc == ORC_OK && i < all.n; ++i)
        if (all.v[i].pass)
            rc = fv_push(&pass, &all.v[i]);
    free(all.v);
    if (rc) {
        free(pass.v);
        return rc;
    }
    *passing = pass.v;
    *n_passing = pass.n;
    return ORC_OK;
}

int orc_event_warrior(const orc_fit *passing, size_t n, int warrior, orc_fit **out, size_t *n_out)
{
    fit_vec result = {0, 0, 0};
    char *dropped = (char *)malloc(n ? n : 1);
    int rc = ORC_OK;
    *out = NULL;
    *n_out = 0;
    if (!dropped)
        return ORC_E_NOMEM;
    if (warrior == 0)
        warrior_pairwise(passing, n, dropped);
    else if (warrior == 1)
        rc = warrior_projection(passing, n, dropped);
    else
        for (size_t i = 0; i < n; ++i)
            dropped[i] = 0;
    for (size_t i = 0; rc == ORC_OK && i < n; ++i)
        if (!dropped[i])
            rc = fv_push(&result, &passing[i]);
    free(dropped);
    if (rc) {
        free(result.v);
        return rc;
    }
    *out = result.v;
    *n_out = result.n;
    return ORC_OK;
}

void orc_free(void *p)
{
    free(p);
}
