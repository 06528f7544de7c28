/* Fast random walk over matmul schemes modulo 2 (the discrete half of the
 * offline search for base cases <M,K,N;R>, Section 2.3): the flip-graph
 * method of Kauers and Moosbauer ("Flip graphs for matrix multiplication",
 * 2022), with the plus transitions of their later work, written here from
 * the published description.
 *
 * A scheme is a list of rank-one terms u (x) v (x) w whose sum is the matmul
 * tensor of <M,K,N> over GF(2); each factor is a bitmask over the MK, KN or
 * MN block entries (row-order vec, Section 2.2.2).  Moves:
 *   flip       x(y1)(z1) + x(y2)(z2) = x(y1+y2)(z1) + x(y2)(z1+z2)   (mod 2)
 *   reduction  two terms sharing two factors merge; a zero factor drops a term.
 * The walk starts from the classical scheme (MKN terms) and restarts after a
 * plateau without reductions.  Once the rank is <= R it keeps flipping at that
 * rank and prints up to `emit` schemes, one per `gap` flips, as lines
 * "u v w;u v w;..." of hexadecimal masks.  The Python side lifts each scheme
 * to exact rationals (Hensel lifting) and checks Eq. (2) exactly.
 *
 * A scheme at rank R can be isolated (no two terms share a factor, so no flip
 * applies).  The walk then leaves it by a plus transition, which splits two
 * terms into three,
 *   a(b)(c) + a'(b')(c') = (a+a')(b)(c) + a'(b+b')(c') + a'(b)(c+c')   (mod 2),
 * and walks on until the rank is back at R; emitted schemes are the sparsest
 * (fewest nonzero factor entries, i.e. the shortest addition chains of
 * Section 3.2) seen in each window of `gap` schemes at rank R.
 *
 * usage: flipwalk M K N R seed max_steps plateau emit gap
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#define MAXT 512

static uint64_t rng_state;
static inline uint64_t rnd(void) {
    /* xorshift64* */
    rng_state ^= rng_state >> 12;
    rng_state ^= rng_state << 25;
    rng_state ^= rng_state >> 27;
    return rng_state * 2685821657736338717ULL;
}
static inline uint32_t rndu(uint32_t n) { return (uint32_t)((rnd() >> 32) % n); }

static uint32_t T[MAXT][3];
static int nt;

static void classical(int M, int K, int N) {
    nt = 0;
    for (int a = 0; a < M; a++)
        for (int b = 0; b < K; b++)
            for (int c = 0; c < N; c++) {
                T[nt][0] = 1u << (a * K + b);
                T[nt][1] = 1u << (b * N + c);
                T[nt][2] = 1u << (a * N + c);
                nt++;
            }
}

static void drop(int i) {
    nt--;
    T[i][0] = T[nt][0];
    T[i][1] = T[nt][1];
    T[i][2] = T[nt][2];
}

/* Remove zero terms and merge terms that share two factors; returns the
 * number of terms removed. */
static int reduce_all(void) {
    int removed = 0;
    int changed = 1;
    while (changed) {
        changed = 0;
        for (int i = 0; i < nt && !changed; i++) {
            if (!T[i][0] || !T[i][1] || !T[i][2]) {
                drop(i);
                removed++;
                changed = 1;
                break;
            }
            for (int j = i + 1; j < nt && !changed; j++) {
                for (int keep = 0; keep < 3; keep++) {
                    int o1 = (keep + 1) % 3, o2 = (keep + 2) % 3;
                    if (T[i][o1] == T[j][o1] && T[i][o2] == T[j][o2]) {
                        T[i][keep] ^= T[j][keep];
                        drop(j);
                        removed++;
                        changed = 1;
                        break;
                    }
                }
            }
        }
    }
    return removed;
}

/* One random flip; returns 1 if a flip was applied. */
static int flip(void) {
    int i = (int)rndu((uint32_t)nt);
    int mode = (int)rndu(3);
    int cand[MAXT], nc = 0;
    for (int j = 0; j < nt; j++)
        if (j != i && T[j][mode] == T[i][mode]) cand[nc++] = j;
    if (!nc) return 0;
    int j = cand[rndu((uint32_t)nc)];
    int p = (mode + 1) % 3, q = (mode + 2) % 3;
    if (rnd() & 1) { int t = p; p = q; q = t; }
    T[i][p] ^= T[j][p];
    T[j][q] ^= T[i][q];
    return 1;
}

static int weight(void) {
    int w = 0;
    for (int i = 0; i < nt; i++)
        w += __builtin_popcount(T[i][0]) + __builtin_popcount(T[i][1]) + __builtin_popcount(T[i][2]);
    return w;
}

static void emit_terms(uint32_t (*S)[3], int n) {
    for (int i = 0; i < n; i++)
        printf("%s%x %x %x", i ? ";" : "", S[i][0], S[i][1], S[i][2]);
    printf("\n");
    fflush(stdout);
}

/* Plus transition: two random terms become three (rank + 1). */
static void plus(void) {
    if (nt < 2 || nt + 1 > MAXT) return;
    int i = (int)rndu((uint32_t)nt), j = (int)rndu((uint32_t)(nt - 1));
    if (j >= i) j++;
    uint32_t a = T[i][0], b = T[i][1], c = T[i][2];
    uint32_t a2 = T[j][0], b2 = T[j][1], c2 = T[j][2];
    T[i][0] = a ^ a2;                                  /* (a+a') b c   */
    T[j][0] = a2; T[j][1] = b ^ b2; T[j][2] = c2;      /* a' (b+b') c' */
    T[nt][0] = a2; T[nt][1] = b; T[nt][2] = c ^ c2;    /* a' b (c+c')  */
    nt++;
    reduce_all();
}

int main(int argc, char **argv) {
    if (argc < 10) {
        fprintf(stderr, "usage: flipwalk M K N R seed max_steps plateau emit gap\n");
        return 2;
    }
    int M = atoi(argv[1]), K = atoi(argv[2]), N = atoi(argv[3]), R = atoi(argv[4]);
    rng_state = 0x9E3779B97F4A7C15ULL ^ (uint64_t)strtoull(argv[5], 0, 10) * 0xBF58476D1CE4E5B9ULL;
    if (!rng_state) rng_state = 1;
    long long max_steps = atoll(argv[6]), plateau = atoll(argv[7]);
    int emit = atoi(argv[8]);
    long long gap = atoll(argv[9]);
    static uint32_t base[MAXT][3], best[MAXT][3];
    int base_n = 0, best_n = 0, best_w = 1 << 30;
    if (M * K > 32 || K * N > 32 || M * N > 32 || M * K * N > MAXT) {
        fprintf(stderr, "sizes too large\n");
        return 2;
    }
    classical(M, K, N);
    long long since = 0;
    int emitted = 0, reached = 0;
    long long window = 0;
    for (long long step = 0; step < max_steps; step++) {
        if (nt <= R) {
            /* a scheme at rank R: score it, keep it as the restart point,
             * then leave it by a plus transition */
            reached = 1;
            int w = weight();
            if (w < best_w) {
                best_w = w;
                best_n = nt;
                for (int i = 0; i < nt; i++) { best[i][0] = T[i][0]; best[i][1] = T[i][1]; best[i][2] = T[i][2]; }
            }
            base_n = nt;
            for (int i = 0; i < nt; i++) { base[i][0] = T[i][0]; base[i][1] = T[i][1]; base[i][2] = T[i][2]; }
            if (++window == gap) {
                emit_terms(best, best_n);
                best_w = 1 << 30;
                window = 0;
                if (++emitted >= emit) return 0;
            }
            plus();
            since = 0;
            continue;
        }
        if (!flip()) continue;
        if (reduce_all()) since = 0; else since++;
        if (since > plateau) {
            if (reached) {
                nt = base_n;
                for (int i = 0; i < nt; i++) { T[i][0] = base[i][0]; T[i][1] = base[i][1]; T[i][2] = base[i][2]; }
                plus();
            } else {
                classical(M, K, N);
            }
            since = 0;
        }
    }
    return emitted ? 0 : 1;
}
