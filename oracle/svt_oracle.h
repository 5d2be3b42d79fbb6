/*
 * svt_oracle.h -- CPU oracle for the SVT track-fitting chain.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  The product (the CUDA
 * library and its Python binding) never includes, links, loads or calls it,
 * and it includes nothing of the product.
 *
 * What it computes (the paper, arXiv:1312.0917, Sec. II and Sec. II-A; where
 * the paper is silent the reading below is the library's and is marked R):
 *
 *  unpack   Sec. II-A, first function: walk the packed words, fill roads.
 *           Word: bit31 EE (end of event), bit30 EP (end of road),
 *           bits29..27 type, bits26..0 payload (R).
 *           type 0..4 hit on that layer, coordinate = bits 11..0, bits 26..12 zero;
 *           type 5 curvature, type 6 phi: int16 in bits 15..0, bits 26..16 zero;
 *           type 7 header: wedge bits 3..0 (<12), barrel bits 6..4 (<6),
 *           excluded layer bits 9..7 (<5), bits 26..10 zero.
 *           A road is header, curvature, phi, hits (R).  EP marks a road's
 *           last word, EE (always with EP) an event's last word.
 *           Limits (R): <= 8 hits per layer per road, <= 256 roads per event.
 *           The words are read in order; the first word that breaks a rule
 *           sets the batch status: a field or grammar fault -> ORC_E_BADWORD,
 *           else a limit -> ORC_E_LIMIT.  Faults are checked per word in the
 *           order: fields, EE without EP, type expected at this road position,
 *           EP before the road's third word, then the limits.  A stream whose
 *           last word is not an EE -> ORC_E_TRUNCATED (position = n_words).
 *
 *  combine  Sec. II, second function: every combination of one hit per layer;
 *           comb = sum_l d_l * S_l, S_0 = 1, S_l = S_{l-1} * n_{l-1}
 *           (layer 0 varies fastest) (R).  A layer with no hits -> no
 *           combinations.
 *
 *  fit      Sec. II, p_i = f_i . x_i + q_i.  x = (hits of the four layers
 *           other than the road's excluded layer, in ascending layer order,
 *           then curvature, then phi) (R).  Constant set index
 *           s = (wedge * 6 + barrel) * 5 + excluded layer (R).
 *           acc_i = sum_j F[s][i][j] * x_j  (int32 products, int64 sum)
 *           p_i   = floor(acc_i / 4096) + q[s][i]                     (R)
 *  chi2     Sec. II ("the chi^2 of the fitted track"); form (R):
 *           a_k = floor((sum_j C[s][k][j] * x_j) / 4096) + k[s][k],
 *           chi2 = a_0^2 + a_1^2 + a_2^2   (int64)
 *  cut      (R) a combination passes iff chi2 <= cut.
 *  warrior  (R) among the passing combinations of one event, t is dropped
 *           iff some passing u has key(u) < key(t) and shares >= 3 hits with
 *           t, where key = (chi2, road, comb) compared lexicographically and
 *           "shares a hit on layer l" means equal coordinate on layer l
 *           (all five layers count).  u need not survive itself.
 *
 * Output: the surviving combinations in (event, road, comb) order.
 */
#ifndef SVT_ORACLE_H
#define SVT_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    ORC_OK = 0,
    ORC_E_BADWORD = -2,
    ORC_E_TRUNCATED = -3,
    ORC_E_LIMIT = -4,
    ORC_E_NOMEM = -8
};

typedef struct {
    uint32_t event;          /* event index in the batch */
    uint32_t road;           /* road index within its event */
    int32_t wedge, barrel, excl, curv, phi;
    int32_t n[5];            /* hits per layer */
    uint16_t coord[5][8];    /* coordinate of hit d on layer l (0 beyond n) */
} orc_road;                  /* 128 bytes */

typedef struct {
    uint32_t event, road, comb;
    int32_t p[3];            /* d0, phi, pT-curvature (fixed point) */
    int64_t chi2;
    uint16_t coord[5];       /* coordinate used on each layer */
    uint16_t pad;
    int32_t pass;            /* chi2 <= cut */
} orc_fit;                   /* 48 bytes */

typedef struct {
    const int16_t *F;        /* [n_sets][3][6] */
    const int32_t *q;        /* [n_sets][3]    */
    const int16_t *C;        /* [n_sets][3][6] */
    const int32_t *k;        /* [n_sets][3]    */
    uint32_t n_sets;         /* 360 */
} orc_consts;

/* Unpack only.  roads may be NULL (count only); at most cap are stored.
 * Returns the status; *err_pos = offending word (n_words for TRUNCATED). */
int orc_unpack(const uint32_t *words, size_t n_words, orc_road *roads,
               size_t cap, size_t *n_roads, size_t *n_events, size_t *err_pos);

/* Every combination of every road, before the cut, in canonical order.
 * *out is malloc'ed by the oracle; release it with orc_free. */
int orc_fit_all(const uint32_t *words, size_t n_words, const orc_consts *c,
                int64_t cut, orc_fit **out, size_t *n_out);

/* chi2 of every combination (canonical order); *out malloc'ed. */
int orc_chi2_all(const uint32_t *words, size_t n_words, const orc_consts *c,
                 int64_t **out, size_t *n_out);

/* The whole chain.  warrior: 0 = pairwise definition, 1 = the same rule via
 * the ten layer-triple projections, -1 = no hit-warrior (passing only).
 * *out malloc'ed (survivors, canonical order, pass = 1). */
int orc_run(const uint32_t *words, size_t n_words, const orc_consts *c,
            int64_t cut, int warrior, orc_fit **out, size_t *n_out);

void orc_free(void *p);

/* One event: every combination of its roads (roads[0..n_roads), all of one
 * event, as orc_unpack returns them), fitted; the passing ones in canonical
 * order -> *passing (malloc'ed). */
int orc_event_fits(const orc_road *roads, size_t n_roads, const orc_consts *c, int64_t cut,
                   orc_fit **passing, size_t *n_passing);

/* The hit-warrior over one event's passing combinations (warrior as in
 * orc_run); the survivors in order -> *out (malloc'ed). */
int orc_event_warrior(const orc_fit *passing, size_t n, int warrior, orc_fit **out, size_t *n_out);

/* Host time of each stage of orc_run_mt, in seconds.  fit and warrior are
 * summed over the threads (CPU time of the stage); wall is the whole call. */
typedef struct {
    double unpack, fit, warrior, wall;
    int32_t threads;          /* threads of the event loop */
    int32_t pad;
} orc_times;

/* The chain of orc_run with the events spread over host threads (OpenMP, one
 * event at a time per thread; svt_oracle_mt.c).  n_threads <= 0: every core
 * OpenMP offers.  Output identical to orc_run.  times may be NULL. */
int orc_run_mt(const uint32_t *words, size_t n_words, const orc_consts *c, int64_t cut,
               int warrior, int n_threads, orc_fit **out, size_t *n_out, orc_times *times);

#ifdef __cplusplus
}
#endif
#endif
