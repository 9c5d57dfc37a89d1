/*
 * kmpar_oracle.c -- plain, slow, FP64 CPU oracle for k-means|| (Bahmani et al.,
 * "Scalable K-Means++", arXiv:1203.6402).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file; only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or constant generator with the
 * CUDA library.
 *
 * Every function follows one passage of the paper, written out as the plain
 * definition (no blocking, no fusion, no reordering):
 *   - squared distance d^2(x, Y) and the cost phi_Y(C)          Sec. 3.1
 *   - centroid(Y)                                               Sec. 3.1
 *   - Algorithm 2 (k-means||) steps 1-2 (init), 4-5 (rounds),
 *     7 (weights), 8 (recluster with k-means++, Sec. 4.2)       Sec. 3.3
 *   - Algorithm 1 (k-means++), in its weighted form, for step 8 Sec. 3.1
 *     (one draw at a time, or the same law drawn in batches by rejection
 *     from a stale D^2 snapshot)                                Sec. 3.1
 *   - the exactly-l-per-round variant of step 4                  Sec. 5.3
 *   - Lloyd's iteration                                         Sec. 1, Sec. 3.1
 *   - Lloyd's iteration on the weighted candidates (the alternative
 *     reading of step 8: weighted k-means++, then local search on the
 *     weighted set, as Sec. 3.3 leaves the reclustering open)   Sec. 3.3
 *
 * Arithmetic: coordinates are read as FP32 and widened to FP64; every distance,
 * probability, prefix sum and centroid is FP64.  The file must be compiled with
 * -ffp-contract=off so that "s = s + t*t" is a rounded multiply followed by a
 * rounded add, exactly as written.
 *
 * Readings where the paper is silent:
 *   - p_x is capped at 1 (p = min(1, l*D^2/phi)); p = 0 when phi = 0.
 *   - ties in an argmin go to the lowest center index; candidates are numbered in
 *     insertion order (initial center 0, then each round's sample in ascending
 *     point order), so w sums to n.
 *   - the first reclustering draw is proportional to w (weighted k-means++).
 *   - Lloyd stops when no label changes; an empty cluster keeps its center.
 *   - if the reclustering runs out of positive mass (total w*D^2 = 0), the
 *     remaining centers repeat the first chosen one and a warning flag is set.
 *   - "exactly l points per round" (Sec. 5.3) is floor(l) successive draws
 *     without replacement, each proportional to D^2 among the points not drawn
 *     yet, with D^2 held at its value at the start of the round.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random
 * Numbers: As Easy as 1, 2, 3", SC'11), implemented here from its published
 * definition, key = (seed_lo, seed_hi), counter = (i_lo, i_hi, round, tag).  A
 * uniform double in [0,1) is built from the first two output words with the
 * 27+26-bit construction u = (a*2^26 + b) / 2^53, a = w0 >> 5, b = w1 >> 6.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TAG_INIT 1u
#define ORC_TAG_SAMPLE 2u
#define ORC_TAG_RECLUSTER 3u
#define ORC_TAG_EXACT 4u
#define ORC_TAG_RECLUSTER_RS 5u

/* ---------------------------------------------------------------------------
 * Philox4x32-10 (SC'11).  Each of the ten rounds multiplies the even words by the
 * two round multipliers, swaps and xors the high halves with the odd words and
 * the key; the key is bumped by the two Weyl constants between rounds.
 * ------------------------------------------------------------------------- */
static void orc_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                       uint32_t k0, uint32_t k1, uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    for (int r = 0; r < 10; ++r) {
        uint64_t prod0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    orc_philox(ctr[0], ctr[1], ctr[2], ctr[3], key[0], key[1], out);
}

/* uniform double in [0,1) for counter (i, round, tag) under key = seed */
double orc_uniform(uint64_t i, uint32_t round, uint32_t tag, uint64_t seed) {
    uint32_t w[4];
    orc_philox((uint32_t)i, (uint32_t)(i >> 32), round, tag,
               (uint32_t)seed, (uint32_t)(seed >> 32), w);
    double a = (double)(w[0] >> 5), b = (double)(w[1] >> 6);
    return (a * 67108864.0 + b) * (1.0 / 9007199254740992.0);
}

/* ---------------------------------------------------------------------------
 * Sec. 3.1: ||x - c||^2, FP64, difference form, dimensions in ascending order.
 * ------------------------------------------------------------------------- */
static double orc_dist2(const float *x, const double *c, int d) {
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
        double t = (double)x[j] - c[j];
        s = s + t * t;
    }
    return s;
}

double orc_dist2_ff(const float *x, const float *y, int d) {
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
        double t = (double)x[j] - (double)y[j];
        s = s + t * t;
    }
    return s;
}

/* near tie: two distinct values whose gap is at most 1e-6 of the larger */
static int orc_near(double a, double b) {
    double hi = a > b ? a : b, gap = fabs(a - b);
    return gap > 0.0 && gap <= 1e-6 * hi;
}

/* ---------------------------------------------------------------------------
 * Sec. 3.1: nearest center and cost.  For each x: label = argmin_i ||x - c_i||^2
 * (lowest i on ties), d2 = that minimum; phi = sum of d2 in ascending x.
 * near[x] = 1 when the runner-up is within 1e-6 (relative) of the minimum.
 * Any output pointer may be NULL.
 * ------------------------------------------------------------------------- */
double orc_assign(const float *X, int64_t n, int d, const double *C, int64_t k,
                  int64_t *label, double *d2, int8_t *near) {
    double phi = 0.0;
    for (int64_t x = 0; x < n; ++x) {
        const float *xr = X + x * (int64_t)d;
        double best = INFINITY, second = INFINITY;
        int64_t arg = -1;
        for (int64_t i = 0; i < k; ++i) {
            double v = orc_dist2(xr, C + i * (int64_t)d, d);
            if (v < best) {
                second = best; best = v; arg = i;
            } else if (v < second) {
                second = v;
            }
        }
        if (label) label[x] = arg;
        if (d2) d2[x] = best;
        if (near) near[x] = (int8_t)(k > 1 && orc_near(best, second));
        phi = phi + best;
    }
    return phi;
}

double orc_cost(const float *X, int64_t n, int d, const double *C, int64_t k) {
    return orc_assign(X, n, d, C, k, NULL, NULL, NULL);
}

/* ---------------------------------------------------------------------------
 * Algorithm 2, step 1: the first center, uniform over X.
 * i0 = floor(u * n) with u from counter (0, round 0, INIT).
 * ------------------------------------------------------------------------- */
int64_t orc_init_index(int64_t n, uint64_t seed) {
    double u = orc_uniform(0, 0, ORC_TAG_INIT, seed);
    int64_t i0 = (int64_t)floor(u * (double)n);
    if (i0 >= n) i0 = n - 1;
    return i0;
}

/* Algorithm 2, step 2: D^2(x) = ||x - x_i0||^2, idx = 0, psi = sum D^2. */
double orc_init(const float *X, int64_t n, int d, int64_t i0, double *D2, int64_t *idx) {
    double psi = 0.0;
    const float *c = X + i0 * (int64_t)d;
    for (int64_t x = 0; x < n; ++x) {
        D2[x] = orc_dist2_ff(X + x * (int64_t)d, c, d);
        idx[x] = 0;
        psi = psi + D2[x];
    }
    return psi;
}

/* ---------------------------------------------------------------------------
 * Algorithm 2, step 4: each x is drawn independently with
 * p_x = min(1, l * D^2(x) / phi), p = 0 when phi = 0; x is drawn iff u < p with
 * u from counter (x, round, SAMPLE).  Drawn points are written in ascending x.
 * p_out (optional) receives p_x; near (optional) flags |u - p| <= 1e-6.
 * Returns the number drawn (at most cap are written; the count is exact).
 * ------------------------------------------------------------------------- */
int64_t orc_sample(const double *D2, int64_t n, double phi, double ell, uint32_t round,
                   uint64_t seed, int64_t *out, int64_t cap, double *p_out, int8_t *near) {
    int64_t cnt = 0;
    for (int64_t x = 0; x < n; ++x) {
        double p = 0.0;
        if (phi > 0.0) {
            p = (ell * D2[x]) / phi;
            if (p > 1.0) p = 1.0;
        }
        double u = orc_uniform((uint64_t)x, round, ORC_TAG_SAMPLE, seed);
        if (p_out) p_out[x] = p;
        if (near) near[x] = (int8_t)(fabs(u - p) <= 1e-6);
        if (u < p) {
            if (cnt < cap) out[cnt] = x;
            cnt++;
        }
    }
    return cnt;
}

/* ---------------------------------------------------------------------------
 * Sec. 5.3 variant of Algorithm 2 step 4 (the runs of Fig. 5.1): exactly
 * L = floor(l) points per round from the D^2 distribution, without replacement.
 * Written as exponential clocks: point x rings at kappa_x = -ln(u_x) / D^2(x),
 * u_x from counter (x, round, EXACT).  The order in which the clocks ring is the
 * order of successive draws, each proportional to D^2 among the points not drawn
 * yet (D^2 as at the start of the round), so the L earliest clocks are the
 * sample.  Equal times go to the lower x.  Points with D^2 = 0 never ring: when
 * fewer than L points have D^2 > 0, all of those are drawn.  Drawn points are
 * written in ascending x.  *near (optional) is set to 1 when another clock rings
 * within w * kappa of the L-th one (only when more than L points can ring).
 * Returns the number drawn.
 * ------------------------------------------------------------------------- */
typedef struct {
    double key;
    int64_t x;
} orc_clock;

static int orc_clock_cmp(const void *pa, const void *pb) {
    const orc_clock *a = (const orc_clock *)pa, *b = (const orc_clock *)pb;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->x > b->x) - (a->x < b->x);
}

static int orc_i64_cmp(const void *pa, const void *pb) {
    const int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    return (a > b) - (a < b);
}

int64_t orc_sample_exact(const double *D2, int64_t n, double ell, uint32_t round, uint64_t seed, double w,
                         int64_t *out, int8_t *near) {
    if (near) *near = 0;
    const int64_t L = (int64_t)floor(ell);
    if (L < 1 || n < 1) return 0;
    orc_clock *cl = (orc_clock *)malloc(sizeof(orc_clock) * (size_t)n);
    if (!cl) return -1;
    int64_t npos = 0;
    for (int64_t x = 0; x < n; ++x) {
        if (D2[x] > 0.0) {
            double u = orc_uniform((uint64_t)x, round, ORC_TAG_EXACT, seed);
            cl[npos].key = -log(u) / D2[x];
            cl[npos].x = x;
            npos++;
        }
    }
    qsort(cl, (size_t)npos, sizeof(orc_clock), orc_clock_cmp);
    const int64_t cnt = npos < L ? npos : L;
    if (near && npos > L) {
        const double t = cl[L - 1].key;
        for (int64_t j = 0; j < npos; ++j)
            if (j != L - 1 && fabs(cl[j].key - t) <= w * t) {
                *near = 1;
                break;
            }
    }
    for (int64_t j = 0; j < cnt; ++j) out[j] = cl[j].x;
    qsort(out, (size_t)cnt, sizeof(int64_t), orc_i64_cmp);
    free(cl);
    return cnt;
}

/* ---------------------------------------------------------------------------
 * Algorithm 2, step 5: C <- C u C'.  The new centers are rows sel[0..cnt) of X,
 * numbered first_id, first_id+1, ... .  For every x and every new center c, in
 * ascending center number: if ||x - c||^2 < D^2(x) (strict), D^2(x) and idx(x)
 * take the new value.  Returns phi = sum D^2.  near[x] flags a runner-up within
 * 1e-6 (relative) of the new minimum among {old nearest, new centers}.
 * ------------------------------------------------------------------------- */
double orc_update(const float *X, int64_t n, int d, const int64_t *sel, int64_t cnt,
                  int64_t first_id, double *D2, int64_t *idx, int8_t *near) {
    double phi = 0.0;
    for (int64_t x = 0; x < n; ++x) {
        const float *xr = X + x * (int64_t)d;
        double best = D2[x], second = INFINITY;
        int64_t arg = idx[x];
        for (int64_t j = 0; j < cnt; ++j) {
            double v = orc_dist2_ff(xr, X + sel[j] * (int64_t)d, d);
            if (v < best) {
                second = best; best = v; arg = first_id + j;
            } else if (v < second) {
                second = v;
            }
        }
        D2[x] = best;
        idx[x] = arg;
        if (near) near[x] = (int8_t)orc_near(best, second);
        phi = phi + best;
    }
    return phi;
}

/* ---------------------------------------------------------------------------
 * Algorithm 2, step 7: w_c = number of x whose nearest center is c.
 * ------------------------------------------------------------------------- */
void orc_weights(const int64_t *idx, int64_t n, int64_t m, int64_t *w) {
    for (int64_t c = 0; c < m; ++c) w[c] = 0;
    for (int64_t x = 0; x < n; ++x) w[idx[x]] += 1;
}

/* ---------------------------------------------------------------------------
 * Algorithm 2, step 8 with k-means++ (Sec. 4.2), in weighted form: Algorithm 1
 * where each candidate j counts w_j times.
 *   draw 0: j with probability w_j / sum w;
 *   draw t: j with probability w_j D^2(j) / sum_j w_j D^2(j), D^2 to the centers
 *           drawn so far.
 * A draw takes u from counter (t, 0, RECLUSTER), target = u * total, and picks the
 * smallest j whose running prefix sum (FP64, ascending j) exceeds the target; if
 * rounding leaves none, the last j with positive mass.  cand is m x d (FP64).
 * chosen[t] receives the candidate number of draw t.  near[t] flags a target
 * within 1e-6 * total of a prefix boundary.  Returns 1 if the positive mass ran
 * out before k draws (remaining draws repeat chosen[0]), else 0.
 * ------------------------------------------------------------------------- */
int orc_recluster(const double *cand, const int64_t *w, int64_t m, int d, int64_t k,
                  uint64_t seed, int64_t *chosen, int8_t *near) {
    double *D2 = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    int warn = 0;
    for (int64_t t = 0; t < k; ++t) {
        double total = 0.0;
        for (int64_t j = 0; j < m; ++j) {
            double e = (t == 0) ? (double)w[j] : (double)w[j] * D2[j];
            total = total + e;
        }
        if (!(total > 0.0)) {
            for (int64_t s = t; s < k; ++s) { chosen[s] = (t > 0) ? chosen[0] : 0; if (near) near[s] = 0; }
            warn = 1;
            break;
        }
        double u = orc_uniform((uint64_t)t, 0, ORC_TAG_RECLUSTER, seed);
        double target = u * total;
        double prefix = 0.0;
        int64_t pick = -1, last_pos = -1;
        int8_t nt = 0;
        for (int64_t j = 0; j < m; ++j) {
            double e = (t == 0) ? (double)w[j] : (double)w[j] * D2[j];
            double before = prefix;
            prefix = prefix + e;
            if (e > 0.0) last_pos = j;
            if (pick < 0 && prefix > target) {
                pick = j;
                if (fabs(target - before) <= 1e-6 * total || fabs(prefix - target) <= 1e-6 * total) nt = 1;
            }
        }
        if (pick < 0) { pick = last_pos; nt = 1; }
        chosen[t] = pick;
        if (near) near[t] = nt;
        const double *c = cand + pick * (int64_t)d;
        for (int64_t j = 0; j < m; ++j) {
            double s = 0.0;
            const double *y = cand + j * (int64_t)d;
            for (int q = 0; q < d; ++q) {
                double dd = y[q] - c[q];
                s = s + dd * dd;
            }
            if (t == 0 || s < D2[j]) D2[j] = s;
        }
    }
    free(D2);
    return warn;
}

/* squared distance between two FP64 candidate rows, in ascending coordinates */
static double orc_dist2_dd(const double *x, const double *y, int d) {
    double s = 0.0;
    for (int q = 0; q < d; ++q) {
        double t = x[q] - y[q];
        s = s + t * t;
    }
    return s;
}

/* ---------------------------------------------------------------------------
 * Algorithm 2, step 8 with k-means++ (Sec. 4.2), weighted (Alg. 1 with
 * multiplicities w), the draws after the first taken in batches by rejection from
 * a stale snapshot of D^2.  The law of the chosen sequence is the one of
 * orc_recluster: every draw t >= 1 picks j with probability
 * w_j D^2(j) / sum_j w_j D^2(j), D^2 to all centers drawn before it.
 *
 *   draw 0: as in orc_recluster (u from counter (0, 0, RECLUSTER), mass w_j).
 *   then, until k centers: a snapshot S = D^2 fixes the masses e_j = w_j S_j
 *   (prefix sums in ascending j, FP64) and 2B proposals i = 0..2B-1 are drawn from
 *   them, proposal i with u from counter (p + i, 0, RS) and the inverse-CDF rule of
 *   orc_recluster.  In proposal order, proposal j is accepted as the next center
 *   iff v S_j < D(j), v from counter (p + i, 1, RS) and D(j) = the smaller of S_j
 *   and the distances from j to the centers accepted since the snapshot: a
 *   proposal is made with probability w_j S_j / sum e and kept with probability
 *   D(j) / S_j, so the kept j has probability proportional to w_j D(j).  The
 *   snapshot ends after 2B proposals, B acceptances or at k; D^2 then takes the
 *   new centers and the next snapshot starts at counter p + 2B.
 *
 * near[t] flags draw t when a proposal examined for it (since the previous
 * acceptance) had its target within 1e-6 of the snapshot total of a prefix
 * boundary, or v S_j within 1e-4 S_j of D(j) (the FP32 distances of a GPU path
 * can differ from these by up to ~(d + 2) 2^-24 relative).  *snapshots receives
 * the number of snapshots.  Returns 1 if the positive mass ran out before k
 * draws (the remaining draws repeat chosen[0]), else 0.
 * ------------------------------------------------------------------------- */
int orc_recluster_rejection(const double *cand, const int64_t *w, int64_t m, int d, int64_t k, int64_t B,
                            uint64_t seed, int64_t *chosen, int8_t *near, int64_t *snapshots) {
    if (snapshots) *snapshots = 0;
    if (k <= 0) return 0;
    const int64_t P = 2 * B;
    double *D2 = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *S = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *prefix = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    int64_t *prop = (int64_t *)malloc(sizeof(int64_t) * (size_t)P);
    int8_t *pnear = (int8_t *)malloc((size_t)P);
    int warn = 0;

    /* draw 0, proportional to w */
    double wtot = 0.0;
    for (int64_t j = 0; j < m; ++j) wtot = wtot + (double)w[j];
    if (!(wtot > 0.0)) {
        for (int64_t s = 0; s < k; ++s) { chosen[s] = 0; if (near) near[s] = 0; }
        free(D2); free(S); free(prefix); free(prop); free(pnear);
        return 1;
    }
    {
        double u = orc_uniform(0, 0, ORC_TAG_RECLUSTER, seed);
        double target = u * wtot, pre = 0.0;
        int64_t pick = -1, last_pos = -1;
        int8_t nt = 0;
        for (int64_t j = 0; j < m; ++j) {
            double before = pre;
            pre = pre + (double)w[j];
            if (w[j] > 0) last_pos = j;
            if (pick < 0 && pre > target) {
                pick = j;
                if (fabs(target - before) <= 1e-6 * wtot || fabs(pre - target) <= 1e-6 * wtot) nt = 1;
            }
        }
        if (pick < 0) { pick = last_pos; nt = 1; }
        chosen[0] = pick;
        if (near) near[0] = nt;
        for (int64_t j = 0; j < m; ++j) D2[j] = orc_dist2_dd(cand + j * (int64_t)d, cand + pick * (int64_t)d, d);
    }

    int64_t t = 1;
    uint64_t p = 0;
    int8_t pending = 0;
    while (t < k) {
        double total = 0.0;
        for (int64_t j = 0; j < m; ++j) {
            S[j] = D2[j];
            total = total + (double)w[j] * S[j];
            prefix[j] = total;
        }
        if (!(total > 0.0)) {
            for (int64_t s = t; s < k; ++s) { chosen[s] = chosen[0]; if (near) near[s] = 0; }
            warn = 1;
            break;
        }
        if (snapshots) *snapshots += 1;
        for (int64_t i = 0; i < P; ++i) {
            double u = orc_uniform(p + (uint64_t)i, 0, ORC_TAG_RECLUSTER_RS, seed);
            double target = u * total;
            int64_t pick = -1, last_pos = -1;
            int8_t nt = 0;
            for (int64_t j = 0; j < m; ++j) {
                double e = (double)w[j] * S[j];
                double before = j > 0 ? prefix[j - 1] : 0.0;
                if (e > 0.0) last_pos = j;
                if (pick < 0 && prefix[j] > target) {
                    pick = j;
                    if (fabs(target - before) <= 1e-6 * total || fabs(prefix[j] - target) <= 1e-6 * total) nt = 1;
                }
            }
            if (pick < 0) { pick = last_pos; nt = 1; }
            prop[i] = pick;
            pnear[i] = nt;
        }
        const int64_t first_new = t;
        for (int64_t i = 0; i < P && t < k && t - first_new < B; ++i) {
            const int64_t j = prop[i];
            double dj = S[j];
            for (int64_t a = first_new; a < t; ++a) {
                double s = orc_dist2_dd(cand + j * (int64_t)d, cand + chosen[a] * (int64_t)d, d);
                if (s < dj) dj = s;
            }
            double v = orc_uniform(p + (uint64_t)i, 1, ORC_TAG_RECLUSTER_RS, seed);
            double lhs = v * S[j];
            pending |= pnear[i];
            if (fabs(lhs - dj) <= 1e-4 * S[j]) pending = 1;
            if (lhs < dj) {
                chosen[t] = j;
                if (near) near[t] = pending;
                pending = 0;
                ++t;
            }
        }
        p += (uint64_t)P;
        for (int64_t a = first_new; a < t; ++a)
            for (int64_t j = 0; j < m; ++j) {
                double s = orc_dist2_dd(cand + j * (int64_t)d, cand + chosen[a] * (int64_t)d, d);
                if (s < D2[j]) D2[j] = s;
            }
    }
    free(D2); free(S); free(prefix); free(prop); free(pnear);
    return warn;
}

/* ---------------------------------------------------------------------------
 * Lloyd's iteration (Sec. 1, Sec. 3.1): assign every x to its nearest center
 * (lowest index on ties); stop if no label changed since the previous
 * assignment; otherwise replace each center by the centroid (Sec. 3.1) of its
 * cluster, summed in FP64 in ascending x (an empty cluster keeps its center).
 * At most max_iter center updates are made; the last assignment is always to the
 * final centers.  cost_hist (optional, max_iter+1 entries) receives the cost of
 * each assignment.  Returns the number of center updates made; *final_cost is the
 * cost of the final centers; labels receives the final assignment.
 * ------------------------------------------------------------------------- */
int64_t orc_lloyd(const float *X, int64_t n, int d, double *C, int64_t k, int64_t max_iter,
                  int64_t *labels, double *final_cost, double *cost_hist, int8_t *near) {
    int64_t *prev = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    double *sum = (double *)malloc(sizeof(double) * (size_t)(k * d > 0 ? k * d : 1));
    int64_t *count = (int64_t *)malloc(sizeof(int64_t) * (size_t)(k > 0 ? k : 1));
    int64_t t = 0;
    double cost = 0.0;
    for (;;) {
        cost = orc_assign(X, n, d, C, k, labels, NULL, near);
        if (cost_hist) cost_hist[t] = cost;
        if (t > 0) {
            int64_t changed = 0;
            for (int64_t x = 0; x < n; ++x) changed += (labels[x] != prev[x]);
            if (changed == 0) break;
        }
        if (t == max_iter) break;
        for (int64_t q = 0; q < k * d; ++q) sum[q] = 0.0;
        for (int64_t j = 0; j < k; ++j) count[j] = 0;
        for (int64_t x = 0; x < n; ++x) {
            int64_t j = labels[x];
            count[j] += 1;
            for (int q = 0; q < d; ++q) sum[j * d + q] = sum[j * d + q] + (double)X[x * (int64_t)d + q];
        }
        for (int64_t j = 0; j < k; ++j) {
            if (count[j] == 0) continue;
            for (int q = 0; q < d; ++q) C[j * d + q] = sum[j * d + q] / (double)count[j];
        }
        memcpy(prev, labels, sizeof(int64_t) * (size_t)n);
        t++;
    }
    if (final_cost) *final_cost = cost;
    free(prev); free(sum); free(count);
    return t;
}

/* ---------------------------------------------------------------------------
 * Step 8 alternative: Lloyd's iteration on the weighted candidate set (Sec. 3.3
 * step 8 reclusters the weighted candidates; Lloyd's local search of Sec. 1 /
 * Sec. 3.1 with every candidate counted w times).  Each iteration assigns every
 * candidate to its nearest center (FP64 difference form, lowest index on ties)
 * and stops if no label changed or max_iter updates were made; otherwise center
 * j becomes sum_c w_c c / sum_c w_c over its candidates (ascending candidate
 * order, FP64; a center with no candidate keeps its place).  Returns the number
 * of updates; *wcost = sum_c w_c d^2(c, nearest center) of the final centers.
 * ------------------------------------------------------------------------- */
int64_t orc_weighted_lloyd(const float *Cand, const int64_t *w, int64_t m, int d, double *C, int64_t k,
                           int64_t max_iter, int64_t *labels, double *wcost) {
    int64_t *prev = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    double *d2 = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *sum = (double *)malloc(sizeof(double) * (size_t)(k * d > 0 ? k * d : 1));
    int64_t *wsum = (int64_t *)malloc(sizeof(int64_t) * (size_t)(k > 0 ? k : 1));
    int64_t t = 0;
    for (;;) {
        orc_assign(Cand, m, d, C, k, labels, d2, NULL);
        if (t > 0) {
            int64_t changed = 0;
            for (int64_t c = 0; c < m; ++c) changed += (labels[c] != prev[c]);
            if (changed == 0) break;
        }
        if (t == max_iter) break;
        for (int64_t q = 0; q < k * d; ++q) sum[q] = 0.0;
        for (int64_t j = 0; j < k; ++j) wsum[j] = 0;
        for (int64_t c = 0; c < m; ++c) {
            const int64_t j = labels[c];
            wsum[j] += w[c];
            for (int q = 0; q < d; ++q)
                sum[j * d + q] = sum[j * d + q] + (double)w[c] * (double)Cand[c * (int64_t)d + q];
        }
        for (int64_t j = 0; j < k; ++j) {
            if (wsum[j] == 0) continue;
            for (int q = 0; q < d; ++q) C[j * d + q] = sum[j * d + q] / (double)wsum[j];
        }
        memcpy(prev, labels, sizeof(int64_t) * (size_t)m);
        t++;
    }
    double cost = 0.0;
    for (int64_t c = 0; c < m; ++c) cost = cost + (double)w[c] * d2[c];
    if (wcost) *wcost = cost;
    free(prev); free(d2); free(sum); free(wsum);
    return t;
}
