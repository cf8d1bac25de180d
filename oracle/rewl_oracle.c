/*
 * Plain serial CPU oracle of two-dimensional replica-exchange Wang-Landau
 * (REWL) sampling of the joint density of states g(E,M) of the periodic 2D
 * Ising model (Valentim et al., "Exploring Replica-Exchange Wang-Landau
 * sampling in higher-dimensional parameter space", arXiv:1508.02748).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this code.  It is slow on purpose:
 * int8 spins, one table per walker, walkers processed one after another,
 * every step in the order the paper states it.  It shares no code with the
 * device path.
 *
 * What follows which passage of the paper:
 *   model, E = -J sum s_i s_j, M = sum s_i, J = 1, periodic L x L  ... Sec. 1-2
 *   acceptance min[1, g(E',M')/g(E'',M'')]                      ... Eq. 1
 *   accept: g(E'',M'') *= f, H(E'',M'') += 1; reject: same on
 *   the current (E',M')                                            ... Sec. 2
 *   flat histogram ends an iteration, H reset, f -> sqrt(f)        ... Sec. 2
 *   80% criterion: every entry >= 0.8 x mean                       ... Sec. 3
 *   overlapping windows, several walkers per window                 ... Sec. 2 (Fig. 1b)
 *   exchange between adjacent windows, random pairs, only inside
 *   the overlap, acceptance of Eq. 2, no g/H update                 ... Eq. 2
 *   all walkers advance together; stop at f_final                   ... Sec. 2
 *   g(E) = sum_M g(E,M)                                             ... Eq. 3
 *   beta(E) = d ln g/dE, E_mat = argmin |beta_i - beta_j|, rescale,
 *   piecewise join                                                  ... Eq. 4
 *   E and M both split: match one dimension at a time               ... Sec. 2
 *   relative difference of two g(E,M) tables                        ... Eq. 5
 *
 * Readings of points the paper leaves open (each one is listed in the design
 * notes of the repository):
 *   - ln f_k = ln f_0 * factor^k; the last iteration is the first one with
 *     ln f <= ln f_final.
 *   - one uniformly random site per trial: site = floor(x * N / 2^32).
 *   - a proposal leaving the walker's window is rejected (the current bin is
 *     updated).
 *   - flatness is tested over the bins the walker has ever visited.
 *   - ln f halves only when every walker is flat (global AND).
 *   - exchange phases cycle E-even, E-odd, M-even, M-odd; walker k of the
 *     lower window pairs with walker pi(k) of the upper one, pi a random
 *     permutation (Fisher-Yates).
 *   - acceptance in log form: accept iff ln u < ln g(cur) - ln g(new), with
 *     u = (x + 1/2) 2^-32; identical to Eq. 1 because ln u < 0.
 *   - walkers of one window are merged only at the end (aligned mean).
 *   - the joined table is normalised to sum g = 2^N.
 *
 * Random numbers: Philox4x32-10 (philox.c), key = seed, counters:
 *   INIT  (c, 0, walker, 1)        initial spins, 128 sites per call
 *   DRIVE (d_lo, d_hi, walker, 2)  drive step d into the window
 *   TRIAL (c_lo, c_hi, walker, 3)  trial t uses call c = t/2, words
 *                                  (2h, 2h+1), h = t mod 2: site word, u word
 *   PERM  (x, pair, i, 4)          Fisher-Yates draw i of exchange step x
 *   EXCH  (x, pair, k, 5)          acceptance u of the k-th pair
 * where pair = 2 * (index of the lower window) + axis (0 = E, 1 = M).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

enum { ORC_OK = 0, ORC_E_INVALID = -1, ORC_E_UNREACHABLE = -4, ORC_E_JOIN = -7 };

typedef struct {
    int L, N;
    int nE, nM, W;            /* window grid and walkers per window */
    int nwin, nwalk;
    double lnf, lnf_final, lnf_factor;
    double flatness;
    uint64_t exch_interval;   /* trials per walker per cycle */
    int check_every;          /* cycles between flatness checks */
    uint32_t key[2];
    int *e0, *e1, *m0, *m1, *active;
    int8_t *spin;             /* nwalk * N, +1 / -1 */
    int *e, *m;               /* bins of the current configuration */
    uint64_t *t;              /* trials done by each walker */
    double *lng;              /* per walker: window table [e][m], window-local */
    int32_t *H;               /* same layout; -1 = never visited */
    size_t *toff;             /* table offset of each walker */
    int *flat;                /* last flatness verdict of each walker */
    uint64_t cycle, xstep;
    int iter, done;
    uint64_t exch_attempt, exch_accept;
} orc_rewl;

/* ---------------------------------------------------------------- model --- */

static int site_spin(const orc_rewl *s, int w, int i, int j)
{
    int L = s->L;
    i = ((i % L) + L) % L;
    j = ((j % L) + L) % L;
    return s->spin[(size_t)w * s->N + (size_t)i * L + j];
}

/* E = -sum over the 2N nearest-neighbour bonds (right and down, periodic). */
static void energy_magnetisation(const orc_rewl *s, int w, int *E, int *M)
{
    int L = s->L, e = 0, m = 0;
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L; ++j) {
            int si = site_spin(s, w, i, j);
            e -= si * site_spin(s, w, i, j + 1);
            e -= si * site_spin(s, w, i + 1, j);
            m += si;
        }
    *E = e; *M = m;
}

/* ------------------------------------------------------------- geometry --- */

/* Equal-sized overlapping windows over B bins: width w = ceil(B / (1 +
 * (n-1)(1-o))), starts rounded evenly from 0 to B - w (Sec. 2, Fig. 1b; Sec. 3
 * "equal-sized windows"). */
static void split_axis(int B, int n, double o, int *lo, int *hi)
{
    if (n <= 1) { lo[0] = 0; hi[0] = B - 1; return; }
    double span = 1.0 + (double)(n - 1) * (1.0 - o);
    double q = (double)B / span;
    int w = (int)ceil(q);
    if (w > B) w = B;
    if (w < 1) w = 1;
    for (int k = 0; k < n; ++k) {
        int64_t num = 2 * (int64_t)k * (B - w) + (n - 1);
        int st = (int)(num / (2 * (int64_t)(n - 1)));
        lo[k] = st; hi[k] = st + w - 1;
    }
}

/* Necessary conditions for a bin (e, m) to hold a configuration: with k =
 * min(m, N-m) minority spins, the number of broken bonds b = 2e satisfies
 *   b <= 2N - 2|2m - N|           (every minority spin breaks at most 4 bonds)
 *   b >= bmin(k) = min(2 ceil(2 sqrt k), 2L + 2 [k mod L != 0]) for k > 0
 *                                   (compact droplet or wrapping stripe).
 * Used only to decide which windows hold no configuration at all (Sec. 1:
 * the phase space has cusps and empty regions). */
static int bin_possible(int L, int e, int m)
{
    int N = L * L;
    int k = m < N - m ? m : N - m;
    int b = 2 * e;
    int dm = 2 * m - N; if (dm < 0) dm = -dm;
    if (b > 2 * N - 2 * dm) return 0;
    if (k == 0) return b == 0;
    int r = 0;
    while ((r + 1) * (r + 1) <= 4 * k) ++r;           /* r = floor(2 sqrt k) */
    int c = (r * r == 4 * k) ? r : r + 1;             /* ceil(2 sqrt k) */
    int bdrop = 2 * c;
    int bstripe = 2 * L + ((k % L) ? 2 : 0);
    int bmin = bdrop < bstripe ? bdrop : bstripe;
    return b >= bmin;
}

static int window_possible(int L, int e0, int e1, int m0, int m1)
{
    for (int e = e0; e <= e1; ++e)
        for (int m = m0; m <= m1; ++m)
            if (bin_possible(L, e, m)) return 1;
    return 0;
}

/* ------------------------------------------------------------ utilities --- */

static void philox(const orc_rewl *s, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t out[4])
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    orc_philox4x32_10(ctr, s->key, out);
}

static uint32_t mulhi32(uint32_t a, uint32_t b) { return (uint32_t)(((uint64_t)a * b) >> 32); }

static double unit_open(uint32_t x) { return ((double)x + 0.5) * (1.0 / 4294967296.0); }

static int win_of(const orc_rewl *s, int w) { return w / s->W; }

static int in_rect(const orc_rewl *s, int win, int e, int m)
{
    return e >= s->e0[win] && e <= s->e1[win] && m >= s->m0[win] && m <= s->m1[win];
}

static size_t tidx(const orc_rewl *s, int win, int e, int m)
{
    int wM = s->m1[win] - s->m0[win] + 1;
    return (size_t)(e - s->e0[win]) * wM + (size_t)(m - s->m0[win]);
}

static size_t tsize(const orc_rewl *s, int win)
{
    return (size_t)(s->e1[win] - s->e0[win] + 1) * (size_t)(s->m1[win] - s->m0[win] + 1);
}

static int l1_dist(const orc_rewl *s, int win, int e, int m)
{
    int d = 0;
    if (e < s->e0[win]) d += s->e0[win] - e;
    if (e > s->e1[win]) d += e - s->e1[win];
    if (m < s->m0[win]) d += s->m0[win] - m;
    if (m > s->m1[win]) d += m - s->m1[win];
    return d;
}

/* Change of the bins (e, m) if the spin at `site` is flipped: with s the spin
 * and n_up the number of up neighbours, dE = 2 s sum_nb = 4 s (n_up - 2), so
 * de = s (n_up - 2); dM = -2 s, so dm = -s. */
static void flip_delta(const orc_rewl *s, int w, int site, int *de, int *dm)
{
    int L = s->L, i = site / L, j = site % L;
    int sp = site_spin(s, w, i, j);
    int sum = site_spin(s, w, i - 1, j) + site_spin(s, w, i + 1, j)
            + site_spin(s, w, i, j - 1) + site_spin(s, w, i, j + 1);
    int nup = (sum + 4) / 2;
    *de = sp * (nup - 2);
    *dm = -sp;
}

/* --------------------------------------------------------------- create --- */

void orc_destroy(orc_rewl *s)
{
    if (!s) return;
    free(s->e0); free(s->e1); free(s->m0); free(s->m1); free(s->active);
    free(s->spin); free(s->e); free(s->m); free(s->t);
    free(s->lng); free(s->H); free(s->toff); free(s->flat);
    free(s);
}

/* init_spins: NULL for Philox INIT spins, else nwalk*N bytes of 0/1 (1 = up).
 * Returns NULL on invalid input; *err gets the reason code. */
orc_rewl *orc_create(int L, int nE, int nM, double oE, double oM, int W,
                     double lnf_init, double lnf_final, double lnf_factor, double flatness,
                     uint64_t exch_interval, int check_every, uint64_t seed,
                     const uint8_t *init_spins, uint64_t drive_budget, int *err)
{
    *err = ORC_E_INVALID;
    if (L < 3 || L > 64 || nE < 1 || nM < 1 || W < 1 || check_every < 1) return NULL;
    if (!(oE >= 0.0 && oE < 1.0 && oM >= 0.0 && oM < 1.0)) return NULL;
    if (!(lnf_init > 0.0 && lnf_final > 0.0 && lnf_factor > 0.0 && lnf_factor < 1.0)) return NULL;
    if (!(flatness > 0.0 && flatness <= 1.0)) return NULL;
    int N = L * L;
    if (nE > N + 1 || nM > N + 1) return NULL;

    orc_rewl *s = (orc_rewl *)calloc(1, sizeof(orc_rewl));
    s->L = L; s->N = N; s->nE = nE; s->nM = nM; s->W = W;
    s->nwin = nE * nM; s->nwalk = s->nwin * W;
    s->lnf = lnf_init; s->lnf_final = lnf_final; s->lnf_factor = lnf_factor;
    s->flatness = flatness; s->exch_interval = exch_interval; s->check_every = check_every;
    s->key[0] = (uint32_t)seed; s->key[1] = (uint32_t)(seed >> 32);

    int *eloA = (int *)malloc(sizeof(int) * nE), *ehiA = (int *)malloc(sizeof(int) * nE);
    int *mloA = (int *)malloc(sizeof(int) * nM), *mhiA = (int *)malloc(sizeof(int) * nM);
    split_axis(N + 1, nE, oE, eloA, ehiA);
    split_axis(N + 1, nM, oM, mloA, mhiA);
    s->e0 = (int *)malloc(sizeof(int) * s->nwin); s->e1 = (int *)malloc(sizeof(int) * s->nwin);
    s->m0 = (int *)malloc(sizeof(int) * s->nwin); s->m1 = (int *)malloc(sizeof(int) * s->nwin);
    s->active = (int *)malloc(sizeof(int) * s->nwin);
    for (int b = 0; b < nM; ++b)
        for (int a = 0; a < nE; ++a) {
            int win = b * nE + a;
            s->e0[win] = eloA[a]; s->e1[win] = ehiA[a];
            s->m0[win] = mloA[b]; s->m1[win] = mhiA[b];
            s->active[win] = window_possible(L, eloA[a], ehiA[a], mloA[b], mhiA[b]);
        }
    free(eloA); free(ehiA); free(mloA); free(mhiA);

    s->spin = (int8_t *)malloc((size_t)s->nwalk * N);
    s->e = (int *)calloc(s->nwalk, sizeof(int));
    s->m = (int *)calloc(s->nwalk, sizeof(int));
    s->t = (uint64_t *)calloc(s->nwalk, sizeof(uint64_t));
    s->flat = (int *)calloc(s->nwalk, sizeof(int));
    s->toff = (size_t *)malloc(sizeof(size_t) * (s->nwalk + 1));
    size_t off = 0;
    for (int w = 0; w < s->nwalk; ++w) { s->toff[w] = off; off += tsize(s, win_of(s, w)); }
    s->toff[s->nwalk] = off;
    s->lng = (double *)calloc(off, sizeof(double));
    s->H = (int32_t *)malloc(off * sizeof(int32_t));
    for (size_t i = 0; i < off; ++i) s->H[i] = -1;

    /* Initial spins: i.i.d. +-1 from the INIT stream, or given. */
    for (int w = 0; w < s->nwalk; ++w) {
        for (int site = 0; site < N; ++site) {
            int up;
            if (init_spins) {
                up = init_spins[(size_t)w * N + site] != 0;
            } else {
                uint32_t x[4];
                philox(s, (uint32_t)(site / 128), 0u, (uint32_t)w, 1u, x);
                up = (x[(site / 32) % 4] >> (site % 32)) & 1u;
            }
            s->spin[(size_t)w * N + site] = up ? 1 : -1;
        }
        int E, M;
        energy_magnetisation(s, w, &E, &M);
        s->e[w] = (E + 2 * N) / 4;
        s->m[w] = (M + N) / 2;
    }

    /* Drive each walker of an active window into its window: a random site is
     * flipped iff the L1 distance of (e, m) to the window does not grow. */
    for (int w = 0; w < s->nwalk; ++w) {
        int win = win_of(s, w);
        if (!s->active[win]) continue;
        uint64_t d = 0;
        while (l1_dist(s, win, s->e[w], s->m[w]) > 0) {
            if (d >= drive_budget) { orc_destroy(s); *err = ORC_E_UNREACHABLE; return NULL; }
            uint32_t x[4];
            philox(s, (uint32_t)d, (uint32_t)(d >> 32), (uint32_t)w, 2u, x);
            int site = (int)mulhi32(x[0], (uint32_t)N);
            int de, dm;
            flip_delta(s, w, site, &de, &dm);
            if (l1_dist(s, win, s->e[w] + de, s->m[w] + dm) <= l1_dist(s, win, s->e[w], s->m[w])) {
                s->spin[(size_t)w * N + site] = (int8_t)-s->spin[(size_t)w * N + site];
                s->e[w] += de; s->m[w] += dm;
            }
            ++d;
        }
    }
    *err = ORC_OK;
    return s;
}

/* ---------------------------------------------------------- WL sampling --- */

/* n trials of one walker (Eq. 1 and the update rule of Sec. 2). */
static void walker_trials(orc_rewl *s, int w, uint64_t n)
{
    int win = win_of(s, w), N = s->N;
    double *lng = s->lng + s->toff[w];
    int32_t *H = s->H + s->toff[w];
    for (uint64_t q = 0; q < n; ++q) {
        uint64_t t = s->t[w];
        uint32_t x[4];
        uint64_t c = t >> 1;
        int h = (int)(t & 1u);
        philox(s, (uint32_t)c, (uint32_t)(c >> 32), (uint32_t)w, 3u, x);
        int site = (int)mulhi32(x[2 * h], (uint32_t)N);
        double u = unit_open(x[2 * h + 1]);
        int de, dm;
        flip_delta(s, w, site, &de, &dm);
        int en = s->e[w] + de, mn = s->m[w] + dm;
        int accept = 0;
        if (in_rect(s, win, en, mn)) {
            /* Eq. 1: P = min[1, g(E',M')/g(E'',M'')], in logarithms. */
            double delta = lng[tidx(s, win, s->e[w], s->m[w])] - lng[tidx(s, win, en, mn)];
            accept = (delta >= 0.0) || (log(u) < delta);
        }
        if (accept) {
            s->spin[(size_t)w * N + site] = (int8_t)-s->spin[(size_t)w * N + site];
            s->e[w] = en; s->m[w] = mn;
        }
        /* g(cur) *= f, H(cur) += 1 for the state the walker is now in. */
        size_t ci = tidx(s, win, s->e[w], s->m[w]);
        lng[ci] += s->lnf;
        H[ci] = (H[ci] < 0 ? 0 : H[ci]) + 1;
        s->t[w] = t + 1;
    }
}

void orc_sweep(orc_rewl *s, uint64_t n)
{
    if (s->done) return;
    for (int w = 0; w < s->nwalk; ++w)
        if (s->active[win_of(s, w)]) walker_trials(s, w, n);
}

/* ----------------------------------------------------------- flatness --- */

/* 80% rule of Sec. 3 over visited bins: every visited H >= flatness x mean,
 * i.e. min H * n_seen >= flatness * sum H.  The flatness parameter is read as
 * a decimal with six digits, q = round(flatness * 10^6), so 0.8 is exactly
 * 4/5, and the test min H * n_seen * 10^6 >= q * sum H is done in exact
 * 64-bit integers (sum H < 2^42 keeps both sides below 2^63). */
static int walker_flat(const orc_rewl *s, int w)
{
    const int32_t *H = s->H + s->toff[w];
    size_t n = s->toff[w + 1] - s->toff[w];
    int64_t seen = 0, sum = 0;
    int32_t mn = INT32_MAX;
    for (size_t i = 0; i < n; ++i) {
        if (H[i] < 0) continue;
        ++seen; sum += H[i];
        if (H[i] < mn) mn = H[i];
    }
    if (seen == 0) return 0;
    int64_t q = (int64_t)llround(s->flatness * 1e6);
    return (int64_t)mn * seen * 1000000 >= q * sum;
}

/* Checks every walker; when all are flat, ends the iteration: H reset on the
 * visited bins, ln f -> ln f * factor (f -> sqrt f for factor 1/2), or stop
 * once the finished iteration had ln f <= ln f_final (Sec. 2). Returns 1 if
 * an iteration ended. */
int orc_check_advance(orc_rewl *s)
{
    if (s->done) return 0;
    int all = 1;
    for (int w = 0; w < s->nwalk; ++w) {
        if (!s->active[win_of(s, w)]) { s->flat[w] = 1; continue; }
        s->flat[w] = walker_flat(s, w);
        all &= s->flat[w];
    }
    if (!all) return 0;
    size_t tot = s->toff[s->nwalk];
    for (size_t i = 0; i < tot; ++i)
        if (s->H[i] > 0) s->H[i] = 0;
    if (s->lnf <= s->lnf_final) s->done = 1;
    else s->lnf *= s->lnf_factor;
    s->iter += 1;
    return 1;
}

/* ----------------------------------------------------------- exchange --- */

static void swap_configs(orc_rewl *s, int wi, int wj)
{
    int N = s->N;
    for (int k = 0; k < N; ++k) {
        int8_t tmp = s->spin[(size_t)wi * N + k];
        s->spin[(size_t)wi * N + k] = s->spin[(size_t)wj * N + k];
        s->spin[(size_t)wj * N + k] = tmp;
    }
    int te = s->e[wi], tm = s->m[wi];
    s->e[wi] = s->e[wj]; s->m[wi] = s->m[wj];
    s->e[wj] = te; s->m[wj] = tm;
}

/* One exchange sweep (Eq. 2) of the phase x mod 4. */
void orc_exchange(orc_rewl *s)
{
    if (s->done) { return; }
    uint64_t x = s->xstep;
    int phase = (int)(x % 4), axis = phase / 2, parity = phase % 2;
    int W = s->W;
    int *perm = (int *)malloc(sizeof(int) * W);
    for (int b = 0; b < s->nM; ++b)
        for (int a = 0; a < s->nE; ++a) {
            int lo_idx = axis == 0 ? a : b;
            int n_axis = axis == 0 ? s->nE : s->nM;
            if (lo_idx % 2 != parity || lo_idx + 1 >= n_axis) continue;
            int A = b * s->nE + a;
            int B = axis == 0 ? A + 1 : A + s->nE;
            if (!s->active[A] || !s->active[B]) continue;
            uint32_t pair = (uint32_t)(2 * A + axis);
            for (int k = 0; k < W; ++k) perm[k] = k;
            for (int i = W - 1; i >= 1; --i) {
                uint32_t r[4];
                philox(s, (uint32_t)x, pair, (uint32_t)i, 4u, r);
                int j = (int)mulhi32(r[0], (uint32_t)(i + 1));
                int tmp = perm[i]; perm[i] = perm[j]; perm[j] = tmp;
            }
            for (int k = 0; k < W; ++k) {
                int wi = A * W + k, wj = B * W + perm[k];
                int eX = s->e[wi], mX = s->m[wi], eY = s->e[wj], mY = s->m[wj];
                if (!in_rect(s, B, eX, mX) || !in_rect(s, A, eY, mY)) continue;
                const double *gi = s->lng + s->toff[wi], *gj = s->lng + s->toff[wj];
                double lnP = (gi[tidx(s, A, eX, mX)] - gi[tidx(s, A, eY, mY)])
                           + (gj[tidx(s, B, eY, mY)] - gj[tidx(s, B, eX, mX)]);
                uint32_t r[4];
                philox(s, (uint32_t)x, pair, (uint32_t)k, 5u, r);
                double u = unit_open(r[0]);
                s->exch_attempt += 1;
                if (lnP >= 0.0 || log(u) < lnP) {
                    swap_configs(s, wi, wj);
                    s->exch_accept += 1;
                }
            }
        }
    free(perm);
    s->xstep = x + 1;
}

/* ------------------------------------------------------------- cycle --- */

/* One cycle: every walker does exch_interval trials; one exchange sweep; a
 * flatness check (and iteration advance) every check_every cycles. */
void orc_run_cycles(orc_rewl *s, uint64_t ncyc)
{
    for (uint64_t c = 0; c < ncyc && !s->done; ++c) {
        orc_sweep(s, s->exch_interval);
        orc_exchange(s);
        s->cycle += 1;
        if (s->cycle % (uint64_t)s->check_every == 0) orc_check_advance(s);
    }
}

/* ------------------------------------------------------------ accessors --- */

void orc_info(const orc_rewl *s, int64_t *out)
{
    out[0] = s->L; out[1] = s->N; out[2] = s->nwin; out[3] = s->nwalk;
    out[4] = (int64_t)s->cycle; out[5] = (int64_t)s->xstep; out[6] = s->iter; out[7] = s->done;
    out[8] = (int64_t)s->toff[s->nwalk];
    out[9] = (int64_t)s->exch_attempt; out[10] = (int64_t)s->exch_accept;
}

double orc_lnf(const orc_rewl *s) { return s->lnf; }

void orc_windows(const orc_rewl *s, int32_t *out /* nwin x 5 */)
{
    for (int w = 0; w < s->nwin; ++w) {
        out[5 * w + 0] = s->e0[w]; out[5 * w + 1] = s->e1[w];
        out[5 * w + 2] = s->m0[w]; out[5 * w + 3] = s->m1[w];
        out[5 * w + 4] = s->active[w];
    }
}

/* Walker state: e, m, t, flat (nwalk x 4 int64) and spins (nwalk x N, 0/1). */
void orc_walkers(const orc_rewl *s, int64_t *st, uint8_t *spins)
{
    for (int w = 0; w < s->nwalk; ++w) {
        st[4 * w + 0] = s->e[w]; st[4 * w + 1] = s->m[w];
        st[4 * w + 2] = (int64_t)s->t[w]; st[4 * w + 3] = s->flat[w];
        if (spins)
            for (int k = 0; k < s->N; ++k) spins[(size_t)w * s->N + k] = s->spin[(size_t)w * s->N + k] > 0;
    }
}

/* All walker tables concatenated (walker w at toff[w]); toff has nwalk+1. */
void orc_tables(const orc_rewl *s, double *lng, int32_t *H, int64_t *toff)
{
    size_t tot = s->toff[s->nwalk];
    if (lng) memcpy(lng, s->lng, tot * sizeof(double));
    if (H) memcpy(H, s->H, tot * sizeof(int32_t));
    if (toff) for (int w = 0; w <= s->nwalk; ++w) toff[w] = (int64_t)s->toff[w];
}

/* Overwrite the tables (tests use this to set up join cases). */
void orc_set_tables(orc_rewl *s, const double *lng, const int32_t *H)
{
    size_t tot = s->toff[s->nwalk];
    if (lng) memcpy(s->lng, lng, tot * sizeof(double));
    if (H) memcpy(s->H, H, tot * sizeof(int32_t));
}

int orc_bin_possible(int L, int e, int m) { return bin_possible(L, e, m); }

/* ------------------------------------------------------ merge and join --- */

static double logsumexp(const double *v, size_t n, size_t stride)
{
    double mx = -INFINITY;
    for (size_t i = 0; i < n; ++i) if (v[i * stride] > mx) mx = v[i * stride];
    if (mx == -INFINITY) return -INFINITY;
    double acc = 0.0;
    for (size_t i = 0; i < n; ++i)
        if (v[i * stride] != -INFINITY) acc += exp(v[i * stride] - mx);
    return mx + log(acc);
}

/* Walkers of one window merged into one table: each walker is shifted by the
 * mean, over the bins every walker visited, of its difference to the first
 * walker; each bin is the mean over the walkers that visited it; -inf if none
 * did.  Walker `excl` of the window (-1: none) is left out entirely (the
 * jackknife replicates of Sec. 2). */
static int merge_window(const orc_rewl *s, int win, double *out, int excl)
{
    int W = s->W;
    int ref = excl == 0 ? 1 : 0;
    size_t n = tsize(s, win);
    double *off = (double *)calloc(W, sizeof(double));
    size_t common = 0;
    for (size_t i = 0; i < n; ++i) {
        int all = 1;
        for (int k = 0; k < W; ++k) if (k != excl && s->H[s->toff[win * W + k] + i] < 0) { all = 0; break; }
        common += all;
    }
    if (W - (excl >= 0) > 1 && common == 0) { free(off); return ORC_E_JOIN; }
    for (int k = 0; k < W; ++k) {
        if (k == ref || k == excl) continue;
        double acc = 0.0;
        const double *g0 = s->lng + s->toff[win * W + ref], *gk = s->lng + s->toff[win * W + k];
        for (size_t i = 0; i < n; ++i) {
            int all = 1;
            for (int q = 0; q < W; ++q) if (q != excl && s->H[s->toff[win * W + q] + i] < 0) { all = 0; break; }
            if (all) acc += gk[i] - g0[i];
        }
        off[k] = acc / (double)common;
    }
    for (size_t i = 0; i < n; ++i) {
        double acc = 0.0;
        int cnt = 0;
        for (int k = 0; k < W; ++k) {
            if (k == excl) continue;
            size_t j = s->toff[win * W + k] + i;
            if (s->H[j] < 0) continue;
            acc += s->lng[j] - off[k];
            ++cnt;
        }
        out[i] = cnt ? acc / (double)cnt : -INFINITY;
    }
    free(off);
    return ORC_OK;
}

/* Matching point between two pieces on one axis (Eq. 4): over positions p of
 * the overlap [lo, hi] with p >= floor_p, where both pieces have finite
 * marginals at p and p+1, beta = (G(p+1) - G(p)) / step; the point minimising
 * |beta_a - beta_b| (lowest on ties).  Without such a p: the lowest p >=
 * floor_p where both are finite.  Returns -1 if there is none. */
static int match_point(const double *Ga, const double *Gb, int lo, int hi, int floor_p,
                       double step)
{
    int best = -1;
    double bestd = INFINITY;
    int start = lo > floor_p ? lo : floor_p;
    for (int p = start; p + 1 <= hi; ++p) {
        if (Ga[p] == -INFINITY || Ga[p + 1] == -INFINITY) continue;
        if (Gb[p] == -INFINITY || Gb[p + 1] == -INFINITY) continue;
        double ba = (Ga[p + 1] - Ga[p]) / step;
        double bb = (Gb[p + 1] - Gb[p]) / step;
        double d = fabs(ba - bb);
        if (d < bestd) { bestd = d; best = p; }
    }
    if (best >= 0) return best;
    for (int p = start; p <= hi; ++p)
        if (Ga[p] != -INFINITY && Gb[p] != -INFINITY) return p;
    return -1;
}

/* Final merge, join and normalisation.  out: (N+1) x (N+1) ln g in [e][m]
 * order, -inf where no walker visited, normalised so sum g = 2^N.
 * ematch: nM x (nE-1) E matching points (-1 where unused);
 * mmatch: (nM-1) M matching points. */
int orc_join_rule(const orc_rewl *s, int excl, int rule, double *out, int32_t *ematch, int32_t *mmatch);

int orc_join(const orc_rewl *s, double *out, int32_t *ematch, int32_t *mmatch)
{
    return orc_join_rule(s, -1, 0, out, ematch, mmatch);
}

/* The join with walker `excl` of every window left out of the merge (-1:
 * none); excl >= 0 needs at least two walkers per window. */
int orc_join_excl(const orc_rewl *s, int excl, double *out, int32_t *ematch, int32_t *mmatch)
{
    return orc_join_rule(s, excl, 0, out, ematch, mmatch);
}

/* Rescaling rule of a join step (Eq. 4 and the sentence before it: the
 * surface is rescaled at g(E_mat, M), read in two ways).
 *   rule 0: one constant per piece, the difference of the two pieces'
 *           marginals (Eq. 3) at the matching point;
 *   rule 1: one constant per slice: for every M of the piece, the
 *           difference ln g_i(E_mat, M) - ln g_j(E_mat, M) where both pieces
 *           have that bin, else the marginal difference of rule 0; joining
 *           rows along M, the same per E at M_mat. */
int orc_join_rule(const orc_rewl *s, int excl, int rule, double *out, int32_t *ematch, int32_t *mmatch)
{
    if (excl >= s->W || (excl >= 0 && s->W < 2) || rule < 0 || rule > 1) return ORC_E_INVALID;
    int N = s->N, B = N + 1, nE = s->nE, nM = s->nM;
    for (size_t i = 0; i < (size_t)B * B; ++i) out[i] = -INFINITY;
    double **piece = (double **)calloc(s->nwin, sizeof(double *));
    int rc = ORC_OK;
    for (int w = 0; w < s->nwin; ++w) {
        if (!s->active[w]) continue;
        piece[w] = (double *)malloc(sizeof(double) * tsize(s, w));
        if (merge_window(s, w, piece[w], excl) != ORC_OK) rc = ORC_E_JOIN;
    }
    for (int i = 0; i < nM * (nE > 1 ? nE - 1 : 1); ++i) ematch[i] = -1;
    for (int i = 0; i < (nM > 1 ? nM - 1 : 1); ++i) mmatch[i] = -1;
    /* rows[b]: full-width table B x B for row b (-inf outside). */
    double **rows = (double **)calloc(nM, sizeof(double *));
    double *Ga = (double *)malloc(sizeof(double) * B), *Gb = (double *)malloc(sizeof(double) * B);
    double *sl = (double *)malloc(sizeof(double) * B), *sl_next = (double *)malloc(sizeof(double) * B);
    int *row_ok = (int *)calloc(nM, sizeof(int));
    for (int b = 0; b < nM && rc == ORC_OK; ++b) {
        int first = -1, last = -1;
        for (int a = 0; a < nE; ++a)
            if (s->active[b * nE + a]) { if (first < 0) first = a; last = a; }
        if (first < 0) continue;
        for (int a = first; a <= last; ++a)
            if (!s->active[b * nE + a]) { rc = ORC_E_JOIN; break; }
        if (rc != ORC_OK) break;
        rows[b] = (double *)malloc(sizeof(double) * B * B);
        for (size_t i = 0; i < (size_t)B * B; ++i) rows[b][i] = -INFINITY;
        row_ok[b] = 1;
        double shift = 0.0;      /* shift of the current piece */
        for (int m = 0; m < B; ++m) sl[m] = 0.0;   /* rule 1: shift of each M slice */
        int from = s->e0[b * nE + first];
        for (int a = first; a <= last; ++a) {
            int A = b * nE + a;
            int wM = s->m1[A] - s->m0[A] + 1;
            int to;              /* piece a covers [from, to) */
            double next_shift = 0.0;
            if (a < last) {
                int Bw = A + 1;
                /* Eq. 3: E marginals of both pieces over the row's M range. */
                for (int e = 0; e < B; ++e) { Ga[e] = -INFINITY; Gb[e] = -INFINITY; }
                for (int e = s->e0[A]; e <= s->e1[A]; ++e)
                    Ga[e] = logsumexp(piece[A] + (size_t)(e - s->e0[A]) * wM, (size_t)wM, 1);
                for (int e = s->e0[Bw]; e <= s->e1[Bw]; ++e)
                    Gb[e] = logsumexp(piece[Bw] + (size_t)(e - s->e0[Bw]) * wM, (size_t)wM, 1);
                int p = match_point(Ga, Gb, s->e0[Bw], s->e1[A], from, 4.0);
                if (p < 0) { rc = ORC_E_JOIN; break; }
                ematch[b * (nE - 1) + a] = p;
                next_shift = shift + (Ga[p] - Gb[p]);
                for (int m = 0; m < B; ++m) sl_next[m] = sl[m] + (Ga[p] - Gb[p]);
                if (rule == 1)
                    for (int m = s->m0[A]; m <= s->m1[A]; ++m) {
                        double va = piece[A][(size_t)(p - s->e0[A]) * wM + (m - s->m0[A])];
                        double vb = piece[Bw][(size_t)(p - s->e0[Bw]) * wM + (m - s->m0[Bw])];
                        if (va != -INFINITY && vb != -INFINITY) sl_next[m] = sl[m] + (va - vb);
                    }
                to = p;
            } else {
                to = s->e1[A] + 1;
            }
            for (int e = from; e < to; ++e)
                for (int m = s->m0[A]; m <= s->m1[A]; ++m) {
                    double v = piece[A][(size_t)(e - s->e0[A]) * wM + (m - s->m0[A])];
                    double c = rule == 1 ? sl[m] : shift;
                    rows[b][(size_t)e * B + m] = v == -INFINITY ? v : v + c;
                }
            shift = next_shift;
            for (int m = 0; m < B; ++m) sl[m] = sl_next[m];
            from = to;
        }
    }
    /* Join the rows along M with the same rule on g(M) = sum_E g(E,M). */
    if (rc == ORC_OK) {
        int first = -1, last = -1;
        for (int b = 0; b < nM; ++b) if (row_ok[b]) { if (first < 0) first = b; last = b; }
        for (int b = first; b >= 0 && b <= last; ++b) if (!row_ok[b]) { rc = ORC_E_JOIN; break; }
        if (first < 0) rc = ORC_E_JOIN;
        double shift = 0.0;
        for (int e = 0; e < B; ++e) sl[e] = 0.0;   /* rule 1: shift of each E slice */
        int from = rc == ORC_OK ? s->m0[first * nE] : 0;
        for (int b = first; rc == ORC_OK && b <= last; ++b) {
            int to;
            double next_shift = 0.0;
            if (b < last) {
                for (int m = 0; m < B; ++m) {
                    Ga[m] = logsumexp(rows[b] + m, (size_t)B, (size_t)B);
                    Gb[m] = logsumexp(rows[b + 1] + m, (size_t)B, (size_t)B);
                }
                int lo = s->m0[(b + 1) * nE], hi = s->m1[b * nE];
                int p = match_point(Ga, Gb, lo, hi, from, 2.0);
                if (p < 0) { rc = ORC_E_JOIN; break; }
                mmatch[b] = p;
                next_shift = shift + (Ga[p] - Gb[p]);
                for (int e = 0; e < B; ++e) {
                    double va = rows[b][(size_t)e * B + p], vb = rows[b + 1][(size_t)e * B + p];
                    double d = (rule == 1 && va != -INFINITY && vb != -INFINITY) ? va - vb : Ga[p] - Gb[p];
                    sl_next[e] = sl[e] + d;
                }
                to = p;
            } else {
                to = s->m1[b * nE] + 1;
            }
            for (int e = 0; e < B; ++e)
                for (int m = from; m < to; ++m) {
                    double v = rows[b][(size_t)e * B + m];
                    double c = rule == 1 ? sl[e] : shift;
                    out[(size_t)e * B + m] = v == -INFINITY ? v : v + c;
                }
            shift = next_shift;
            for (int e = 0; e < B; ++e) sl[e] = sl_next[e];
            from = to;
        }
    }
    /* Normalise: sum g = 2^N. */
    if (rc == ORC_OK) {
        double lz = logsumexp(out, (size_t)B * B, 1);
        double c = (double)N * log(2.0) - lz;
        for (size_t i = 0; i < (size_t)B * B; ++i)
            if (out[i] != -INFINITY) out[i] += c;
    }
    for (int w = 0; w < s->nwin; ++w) free(piece[w]);
    for (int b = 0; b < nM; ++b) free(rows[b]);
    free(piece); free(rows); free(Ga); free(Gb); free(sl); free(sl_next); free(row_ok);
    return rc;
}

/* E marginal of a joined table (Eq. 3): out[e] = ln sum_m g(e, m). */
void orc_marginal_e(int N, const double *joined, double *out)
{
    int B = N + 1;
    for (int e = 0; e < B; ++e) out[e] = logsumexp(joined + (size_t)e * B, (size_t)B, 1);
}

/* Relative difference of two density-of-states tables, Eq. 5:
 * |g_a - g_b| / gbar with gbar = (g_a + g_b) / 2, per bin, from ln g_a and
 * ln g_b.  Numerator and denominator are both scaled by exp(-max(ln g_a,
 * ln g_b)) so that the exponentials stay finite at any size; a bin empty in
 * one table only gives 2, a bin empty in both NaN (no value). */
void orc_rel_diff(size_t n, const double *lga, const double *lgb, double *out)
{
    for (size_t i = 0; i < n; ++i) {
        const double a = lga[i], b = lgb[i];
        if (a == -INFINITY && b == -INFINITY) { out[i] = NAN; continue; }
        const double s = a > b ? a : b;
        const double ga = exp(a - s), gb = exp(b - s);
        const double gbar = (ga + gb) / 2.0;
        out[i] = fabs(ga - gb) / gbar;
    }
}
