/*
 * Exact joint density of states g(E,M) of the periodic L x L Ising model
 * (J = 1, E = -sum over the 2N bonds, M = sum of spins; Sec. 1-2 of the
 * paper).  TEST INFRASTRUCTURE ONLY: these pin the oracle, nothing else.
 *
 * Bins: e = (E + 2N)/4 = (broken bonds)/2, m = (M + N)/2 = number of up
 * spins; out is (N+1) x (N+1) in [e][m] order.
 *
 * orc_enum_gEM: brute force over all 2^N configurations (L <= 5), visited in
 * Gray-code order so that each step flips one spin.
 * orc_tm_gEM:   site-by-site transfer matrix (L <= 8).  Row 0 is fixed; the
 * state is the profile of the last L placed spins together with the broken
 * bond count and up count so far; the periodic closures are the bond from
 * the last to the first site of each row and, at the end, the bonds from row
 * L-1 to row 0.  Row-0 configurations related by a cyclic shift give the
 * same counts, so each shift class is computed once and weighted by its
 * size.  Arithmetic is modulo 2^64: every final count is below 2^64 for
 * L <= 8 (the total is 2^N <= 2^64 and more than one bin is occupied), so
 * the residues are the counts.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int spin_at(uint64_t cfg, int L, int i, int j)
{
    i = ((i % L) + L) % L;
    j = ((j % L) + L) % L;
    return (int)((cfg >> (i * L + j)) & 1u);
}

int orc_enum_gEM(int L, uint64_t *out)
{
    if (L < 3 || L > 5) return -1;
    int N = L * L, B = N + 1;
    memset(out, 0, sizeof(uint64_t) * (size_t)B * B);
    uint64_t cfg = 0;                  /* all down: m = 0, no broken bond */
    int broken = 0, up = 0;
    uint64_t total = (uint64_t)1 << N;
    for (uint64_t g = 0; g < total; ++g) {
        out[(size_t)(broken / 2) * B + up] += 1;
        if (g + 1 == total) break;
        /* Gray code: the bit to flip is the lowest set bit of g + 1. */
        uint64_t nx = g + 1;
        int site = 0;
        while (!((nx >> site) & 1u)) ++site;
        int i = site / L, j = site % L;
        int s = spin_at(cfg, L, i, j);
        int nb[4] = {spin_at(cfg, L, i - 1, j), spin_at(cfg, L, i + 1, j),
                     spin_at(cfg, L, i, j - 1), spin_at(cfg, L, i, j + 1)};
        for (int k = 0; k < 4; ++k) broken += (nb[k] == s) ? 1 : -1;
        up += s ? -1 : 1;
        cfg ^= (uint64_t)1 << site;
    }
    return 0;
}

static uint32_t rot_row(uint32_t r, int L, int k)
{
    uint32_t mask = (L == 32) ? 0xFFFFFFFFu : ((1u << L) - 1u);
    k %= L;
    if (k == 0) return r;
    return ((r << k) | (r >> (L - k))) & mask;
}

static int popc(uint32_t x) { int c = 0; while (x) { c += x & 1u; x >>= 1; } return c; }

int orc_tm_gEM(int L, uint64_t *out)
{
    if (L < 3 || L > 8) return -1;
    int N = L * L, B = N + 1;
    int NB = 2 * N + 1;                 /* broken bonds 0..2N */
    uint32_t P = 1u << L;
    size_t per = (size_t)NB * B;
    uint64_t *cur = (uint64_t *)malloc(sizeof(uint64_t) * P * per);
    uint64_t *nxt = (uint64_t *)malloc(sizeof(uint64_t) * P * per);
    if (!cur || !nxt) { free(cur); free(nxt); return -2; }
    memset(out, 0, sizeof(uint64_t) * (size_t)B * B);
    for (uint32_t r0 = 0; r0 < P; ++r0) {
        /* Only the smallest member of each cyclic-shift class is run. */
        int rep = 1, orbit = 0;
        for (int k = 0; k < L; ++k) {
            uint32_t rr = rot_row(r0, L, k);
            if (rr < r0) { rep = 0; break; }
        }
        if (!rep) continue;
        for (int k = 0; k < L; ++k) {
            uint32_t rr = rot_row(r0, L, k);
            int dup = 0;
            for (int q = 0; q < k; ++q) if (rot_row(r0, L, q) == rr) { dup = 1; break; }
            orbit += !dup;
        }
        memset(cur, 0, sizeof(uint64_t) * P * per);
        int b0 = popc(r0 ^ rot_row(r0, L, 1));          /* row 0's horizontal bonds */
        cur[(size_t)r0 * per + (size_t)b0 * B + popc(r0)] = 1;
        for (int i = 1; i < L; ++i)
            for (int j = 0; j < L; ++j) {
                memset(nxt, 0, sizeof(uint64_t) * P * per);
                for (uint32_t pr = 0; pr < P; ++pr) {
                    const uint64_t *src = cur + (size_t)pr * per;
                    for (int x = 0; x <= 1; ++x) {
                        int db = (((pr >> j) & 1u) != (uint32_t)x);            /* up bond */
                        if (j >= 1) db += (((pr >> (j - 1)) & 1u) != (uint32_t)x); /* left */
                        if (j == L - 1) db += ((pr & 1u) != (uint32_t)x);          /* wrap */
                        uint32_t np = (pr & ~(1u << j)) | ((uint32_t)x << j);
                        uint64_t *dst = nxt + (size_t)np * per;
                        for (int b = 0; b + db < NB; ++b)
                            for (int k = 0; k + x < B; ++k) {
                                uint64_t v = src[(size_t)b * B + k];
                                if (v) dst[(size_t)(b + db) * B + k + x] += v;
                            }
                    }
                }
                uint64_t *t = cur; cur = nxt; nxt = t;
            }
        /* Close the torus vertically: row L-1 (the profile) against row 0. */
        for (uint32_t pr = 0; pr < P; ++pr) {
            int db = popc(pr ^ r0);
            const uint64_t *src = cur + (size_t)pr * per;
            for (int b = 0; b + db < NB; ++b)
                for (int k = 0; k < B; ++k) {
                    uint64_t v = src[(size_t)b * B + k];
                    if (!v) continue;
                    int bb = b + db;
                    if (bb & 1) { free(cur); free(nxt); return -3; }   /* impossible */
                    out[(size_t)(bb / 2) * B + k] += v * (uint64_t)orbit;
                }
        }
    }
    free(cur); free(nxt);
    return 0;
}
