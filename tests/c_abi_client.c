/*
 * A plain C client of libqubo.so (no Python): solves two instances through qubo_solve and checks
 * them against closed forms.
 *
 * 1. A dense planted instance, n = 34.  With a planted state a (bits a_i), weights w_i > 0 and
 *    couplings c_ij >= 0, let s_i = x_i XOR a_i.  E(x) = sum_i w_i (1 - 2 a_i) x_i
 *    + sum_{i<j} c_ij (s_i s_j - a_i a_j) expands into an upper-triangular integer Q (below).
 *    The first sum is minimised exactly at x = a; the coupling sum is >= -sum c_ij a_i a_j with
 *    equality at x = a (s = 0 there).  So a is the unique minimiser and
 *    E_min = -sum_{a_i = 1} w_i - sum_{i<j} c_ij a_i a_j.
 * 2. Q = 0, n = 20: every state ties at 0; with room for 16 codes the call returns
 *    QUBO_TRUNCATED, the exact count 2^20 and the codes 0..15.
 *
 * Exit status 0 when every check holds.  Build: cc -I include tests/c_abi_client.c
 * -L paper_2607_04857_gb300 -lqubo -Wl,-rpath,<that directory>.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "qubo.h"

static uint64_t lcg_state = 0x2545F4914F6CDD1DULL;

static uint32_t next_u32(void)
{
    lcg_state = lcg_state * 6364136223846793005ULL + 1442695040888963407ULL;
    return (uint32_t)(lcg_state >> 33);
}

static int fail(const char *what)
{
    fprintf(stderr, "c_abi_client: %s\n", what);
    return 1;
}

int main(void)
{
    enum { N = 34 };
    static int32_t Q[N * N];
    int a[N];
    int64_t w[N];
    int64_t expect = 0;
    memset(Q, 0, sizeof(Q));
    uint64_t planted = 0;
    for (int i = 0; i < N; ++i) {
        a[i] = (int)(next_u32() & 1u);
        w[i] = 1 + (int64_t)(next_u32() % 100u);
        planted |= (uint64_t)a[i] << i;
        Q[i * N + i] += (int32_t)(w[i] * (1 - 2 * a[i]));
        if (a[i])
            expect -= w[i];
    }
    for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j) {
            const int64_t c = (int64_t)(next_u32() % 50u);
            /* c (s_i s_j - a_i a_j) with s = a + (1 - 2a) x */
            Q[i * N + j] += (int32_t)(c * (1 - 2 * a[i]) * (1 - 2 * a[j]));
            Q[i * N + i] += (int32_t)(c * a[j] * (1 - 2 * a[i]));
            Q[j * N + j] += (int32_t)(c * a[i] * (1 - 2 * a[j]));
            expect -= c * a[i] * a[j];
        }

    int64_t mn = 0;
    uint64_t ties[4], top[2];
    int64_t topE[2];
    qubo_result info;
    int st = qubo_solve(Q, N, QUBO_I32, 0, 2, &mn, ties, 4, top, topE, &info, NULL);
    if (st != QUBO_OK) {
        fprintf(stderr, "qubo_solve: %s\n", qubo_strerror(st));
        return 1;
    }
    if (mn != expect || info.min_i != expect)
        return fail("planted instance: wrong minimum");
    if (info.n_ties != 1 || info.n_written != 1 || ties[0] != planted)
        return fail("planted instance: wrong minimiser");
    if (info.states_scanned != (1ULL << N) || info.n_topk != 2 || top[0] != planted || topE[0] != expect ||
        topE[1] <= expect)
        return fail("planted instance: wrong scan count or K lowest");

    static int16_t Z[20 * 20];
    memset(Z, 0, sizeof(Z));
    uint64_t codes[16];
    st = qubo_solve(Z, 20, QUBO_I16, 0, 0, &mn, codes, 16, NULL, NULL, &info, NULL);
    if (st != QUBO_TRUNCATED || mn != 0 || info.n_ties != (1ULL << 20) || info.n_written != 16 || !info.truncated)
        return fail("zero instance: wrong status, minimum or count");
    for (int t = 0; t < 16; ++t)
        if (codes[t] != (uint64_t)t)
            return fail("zero instance: wrong tie codes");

    if (qubo_solve(Q, 0, QUBO_I32, 0, 0, &mn, NULL, 0, NULL, NULL, NULL, NULL) != QUBO_ERR_ARG)
        return fail("n = 0 not rejected");
    printf("c_abi_client ok: %s; planted min %lld at %llx\n", qubo_version(), (long long)expect,
           (unsigned long long)planted);
    return 0;
}
