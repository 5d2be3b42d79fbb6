/*
 * svt_oracle_mt.c -- the oracle's chain with the events of a batch spread
 * over the host cores.
 *
 * TEST INFRASTRUCTURE ONLY (see svt_oracle.h): the product never includes,
 * links or loads it.
 *
 * Every step after the unpack is local to one event: combinations, fits and
 * the cut belong to one road, and the hit-warrior compares tracks of one
 * event only.  The paper's many-core port therefore processes one event per
 * core with an OpenMP loop over events (arXiv:1312.0917, Sec. II-A, the Xeon
 * Phi version).  This driver does the same with the serial oracle's own
 * per-event functions: the words are unpacked once (a serial walk: an event's
 * road index depends on the words before it), then an OpenMP loop takes one
 * event at a time per thread, and the survivors are concatenated in event
 * order, so the output is orc_run's.  Each stage's host time is recorded
 * (the paper's time breakdown, Sec. IV-A).
 */
#define _POSIX_C_SOURCE 199309L
#include "svt_oracle.h"

#include <omp.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

static double now_s(void)
{
    struct timespec t;
    clock_gettime(CLOCK_MONOTONIC, &t);
    return (double)t.tv_sec + 1e-9 * (double)t.tv_nsec;
}

int orc_run_mt(const uint32_t *words, size_t n_words, const orc_consts *c, int64_t cut,
               int warrior, int n_threads, orc_fit **out, size_t *n_out, orc_times *times)
{
    const double t0 = now_s();
    size_t nr, ne, err_pos;
    *out = NULL;
    *n_out = 0;
    int rc = orc_unpack(words, n_words, NULL, 0, &nr, &ne, &err_pos);
    if (rc)
        return rc;
    orc_road *roads = (orc_road *)malloc((nr ? nr : 1) * sizeof *roads);
    size_t *first = (size_t *)malloc((ne + 1) * sizeof *first);   /* first road of each event */
    orc_fit **res = (orc_fit **)calloc(ne ? ne : 1, sizeof *res);
    size_t *cnt = (size_t *)calloc(ne ? ne : 1, sizeof *cnt);
    if (!roads || !first || !res || !cnt) {
        free(roads);
        free(first);
        free(res);
        free(cnt);
        return ORC_E_NOMEM;
    }
    rc = orc_unpack(words, n_words, roads, nr, &nr, &ne, &err_pos);
    for (size_t e = 0, r = 0; e <= ne; ++e) {   /* roads come in event order */
        while (r < nr && roads[r].event < e)
            ++r;
        first[e] = r;
    }
    const double t1 = now_s();

    const int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
    double *fit_s = (double *)calloc((size_t)nt, sizeof *fit_s);
    double *war_s = (double *)calloc((size_t)nt, sizeof *war_s);
    int failed = fit_s && war_s ? rc : ORC_E_NOMEM;
    if (!failed) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
        for (long e = 0; e < (long)ne; ++e) {
            int erc;
#pragma omp atomic read
            erc = failed;
            if (erc)
                continue;
            const int tid = omp_get_thread_num();
            orc_fit *passing = NULL;
            size_t np = 0;
            const double ta = now_s();
            erc = orc_event_fits(roads + first[e], first[e + 1] - first[e], c, cut, &passing, &np);
            const double tb = now_s();
            if (!erc)
                erc = orc_event_warrior(passing, np, warrior, &res[e], &cnt[e]);
            free(passing);
            fit_s[tid] += tb - ta;
            war_s[tid] += now_s() - tb;
            if (erc) {
#pragma omp atomic write
                failed = erc;
            }
        }
    }
    size_t total = 0;
    for (size_t e = 0; e < ne; ++e)
        total += cnt[e];
    orc_fit *all = failed ? NULL : (orc_fit *)malloc((total ? total : 1) * sizeof *all);
    if (!failed && !all)
        failed = ORC_E_NOMEM;
    size_t k = 0;
    for (size_t e = 0; e < ne; ++e) {
        if (!failed && cnt[e])
            memcpy(all + k, res[e], cnt[e] * sizeof *all);
        k += cnt[e];
        free(res[e]);
    }
    if (times) {
        times->unpack = t1 - t0;
        times->fit = 0.0;
        times->warrior = 0.0;
        for (int i = 0; fit_s && war_s && i < nt; ++i) {
            times->fit += fit_s[i];
            times->warrior += war_s[i];
        }
        times->threads = nt;
        times->pad = 0;
        times->wall = now_s() - t0;
    }
    free(fit_s);
    free(war_s);
    free(roads);
    free(first);
    free(res);
    free(cnt);
    if (failed) {
        free(all);
        return failed;
    }
    *out = all;
    *n_out = total;
    return ORC_OK;
}
