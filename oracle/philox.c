/* Philox4x32-10 counter-based generator -- oracle (test infrastructure).
 *
 * Written from the definition in Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3" (SC'11): a 10-round Feistel-like network over
 * four 32-bit words.  Each round multiplies words 0 and 2 by the two round
 * multipliers, mixes the high halves with the other words and the key, and
 * the key is advanced by the two Weyl constants between rounds.
 */
#include "oracle.h"

static void mul_hi_lo(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t mult0 = 0xD2511F53u, mult1 = 0xCD9E8D57u;   /* round multipliers */
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;   /* key schedule */
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += weyl0;
            k1 += weyl1;
        }
        uint32_t hi_a, lo_a, hi_b, lo_b;
        mul_hi_lo(mult0, x0, &hi_a, &lo_a);
        mul_hi_lo(mult1, x2, &hi_b, &lo_b);
        uint32_t y0 = hi_b ^ x1 ^ k0;
        uint32_t y1 = lo_b;
        uint32_t y2 = hi_a ^ x3 ^ k1;
        uint32_t y3 = lo_a;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

double orc_u01(uint32_t u)
{
    return (double)(u >> 8) * (1.0 / 16777216.0);
}
