/*
 * Philox4x32-10 counter-based generator, oracle side (test infrastructure only).
 *
 * Written from the published definition (Salmon, Moraes, Dror, Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC'11, Sec. 4): a 4x32-bit counter and a
 * 2x32-bit key; each round multiplies counter words 0 and 2 by two fixed
 * constants (full 64-bit products), recombines the high halves with the other
 * counter words and the key by XOR, and swaps the low halves across; the key is
 * bumped by two Weyl constants between rounds; 10 rounds.
 *
 * The paper (Sec. 2) only requires uniform random trial moves and random
 * exchange pairing; this generator is how both the oracle and the device path
 * draw them, so that trajectories can be compared trial by trial.  The oracle
 * shares no code with the device path: the CUDA side has its own
 * implementation of the same published definition.
 *
 * Pinned in tests against an independent implementation (PyTorch's
 * header-only philox_engine, compiled and run, not read for values).
 */
#include <stdint.h>

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        philox_round(c, k);
        k[0] += PHILOX_W0;
        k[1] += PHILOX_W1;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Batch form for tests: n counters (4 words each) under one key. */
void orc_philox_batch(uint64_t n, const uint32_t *ctrs, const uint32_t key[2], uint32_t *outs)
{
    for (uint64_t i = 0; i < n; ++i)
        orc_philox4x32_10(ctrs + 4 * i, key, outs + 4 * i);
}
