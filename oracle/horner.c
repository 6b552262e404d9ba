/* Algorithm 2 (fast evaluation of a linear recurrence) for the oracle.
 *
 * TEST INFRASTRUCTURE ONLY: part of the CPU oracle.  Plain loops, exact
 * arithmetic with unsigned __int128 for a modulus q < 2^63; the same
 * computation as oracle.zeta.horner_python, tested against it.
 *
 * A chunk of k steps in direction v from the exponent x + k v (Sec. 3.2):
 *   M(y) = R_{x + y v, v} = y A + B,  A = sum_i v_i A_i,  B = sum_i x_i A_i + A_{n+1}
 *   W <- M(0) M(1) ... M(k-1) W   (mod q)
 * evaluated as in Algorithm 2: M <- (k-1) A + B; repeat k times
 * { W <- M W; M <- M - A }.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q) {
    return (uint64_t)(((u128)a * b) % q);
}

/* parts: (n1 + 1) matrices s x s row-major (A_0..A_{n1-1}, A_{n1}); x, v: n1 entries.
 * W: s x c row-major, overwritten.  Returns 0 on success. */
int oracle_horner_chunk(int n1, int s, int c, int k, const uint64_t *parts,
                        const int64_t *x, const int64_t *v, uint64_t *W, uint64_t q) {
    size_t ss = (size_t)s * s;
    uint64_t *A = malloc(ss * sizeof(uint64_t));
    uint64_t *M = malloc(ss * sizeof(uint64_t));
    uint64_t *T = malloc((size_t)s * c * sizeof(uint64_t));
    if (!A || !M || !T) { free(A); free(M); free(T); return 1; }
    const uint64_t *Alast = parts + (size_t)n1 * ss;
    for (size_t e = 0; e < ss; e++) {
        u128 a = 0, b = Alast[e];
        for (int i = 0; i < n1; i++) {
            a += (u128)((uint64_t)v[i] % q) * parts[(size_t)i * ss + e];
            b += (u128)((uint64_t)x[i] % q) * parts[(size_t)i * ss + e];
            a %= q;
            b %= q;
        }
        A[e] = (uint64_t)a;
        /* M = (k-1) A + B */
        M[e] = (uint64_t)(((u128)(k - 1) * A[e] + b) % q);
    }
    for (int step = 0; step < k; step++) {
        for (int r = 0; r < s; r++) {
            for (int col = 0; col < c; col++) {
                u128 acc = 0;
                for (int j = 0; j < s; j++) {
                    acc += (u128)M[(size_t)r * s + j] * W[(size_t)j * c + col];
                    if (acc >> 127) acc %= q;
                }
                T[(size_t)r * c + col] = (uint64_t)(acc % q);
            }
        }
        memcpy(W, T, (size_t)s * c * sizeof(uint64_t));
        for (size_t e = 0; e < ss; e++) M[e] = (M[e] >= A[e]) ? M[e] - A[e] : M[e] + q - A[e];
    }
    free(A); free(M); free(T);
    return 0;
}

/* Plain matrix product mod q (used by tests of the helper itself). */
void oracle_matmul_mod(int r, int s, int c, const uint64_t *M, const uint64_t *W,
                       uint64_t *out, uint64_t q) {
    for (int i = 0; i < r; i++)
        for (int col = 0; col < c; col++) {
            u128 acc = 0;
            for (int j = 0; j < s; j++) {
                acc += (u128)M[(size_t)i * s + j] * W[(size_t)j * c + col];
                if (acc >> 127) acc %= q;
            }
            out[(size_t)i * c + col] = (uint64_t)(acc % q);
        }
    (void)mulmod;
}
