/*
 * pt_mt.c -- the paper's multi-threaded CPU Parallel Tempering (Sec. 4, Figs. 4-5): a
 * stronger CPU baseline than the plain oracle. See pt_mt.h for what it computes.
 *
 * Layout: each chain row i holds its P/2 even copies, then its P/2 odd copies, so that the
 * copies one parity group updates together are contiguous (Sec. 5's two groups of
 * independent regions: at one site the even copies depend only on the odd ones and on the
 * neighbours' same copies, and the other way round).
 */
#define _POSIX_C_SOURCE 200809L  /* pthread barriers */
#include "pt_mt.h"

#include <math.h>
#include <pthread.h>
#include <stdatomic.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- Philox4x32-10
 * Salmon, Moraes, Dror, Shaw (SC'11): ten rounds of
 *   (c0, c1, c2, c3) -> (hi(B c2) ^ c1 ^ k0, lo(B c2), hi(A c0) ^ c3 ^ k1, lo(A c0))
 * with A = 0xD2511F53, B = 0xCD9E8D57 and the key bumped by (0x9E3779B9, 0xBB67AE85)
 * after each round. */
static void philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1, uint32_t out[4]) {
    for (int round = 0; round < 10; ++round) {
        const uint64_t pa = (uint64_t)0xD2511F53u * c0;
        const uint64_t pb = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(pb >> 32) ^ c1 ^ k0;
        const uint32_t n2 = (uint32_t)(pa >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)pb;
        c3 = (uint32_t)pa;
        c0 = n0;
        c2 = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* exp(x) for x in (-23, 0] from IEEE basic operations: Cody-Waite reduction by a two-part
 * ln 2 (the high part with 28 fraction bits, so n * hi is exact), the degree-13 Taylor
 * polynomial by Horner's rule, and an exact scaling by 2^n. The three constants are the
 * ones the swap rule of this repository fixes as data. */
static double exp_swap(double x) {
    const double hi = 0x1.62e42ff000000p-1, lo = -0x1.718432a1b0e26p-35, inv_ln2 = 0x1.71547652b82fep+0;
    const double n = nearbyint(x * inv_ln2);
    const double r = (x - n * hi) - n * lo;
    double fact = 1.0, c[14];
    for (int k = 0; k < 14; ++k) {
        if (k > 1) fact *= (double)k;
        c[k] = 1.0 / fact;
    }
    double poly = c[13];
    for (int k = 12; k >= 0; --k) poly = poly * r + c[k];
    return ldexp(poly, (int)n);
}

struct cpt {
    int32_t N, P, R, Lmax, H, odd, row;   /* H copies per parity (1 for P = 1), row = bytes per site */
    int32_t *adj_off, *adj_j, *adj_J, *h;
    uint32_t* thr;
    double* coef;
    uint32_t k0, k1;
    int8_t* s;                            /* [R][N][row]: even copies, then odd copies */
    int64_t *E, *M;                       /* by chain */
    int32_t *rung_of, *replica_at;
    int64_t *n_meas, *sum_E, *sum_E2, *sum_M, *sum_M2, *flip_acc, *swap_att, *swap_acc;  /* by rung / pair */
    int64_t* hard;                        /* flips of each chain in the last interval */
    int32_t* order;                       /* work pool order, hardest first */
    int64_t t, q;
    int32_t threads;
};

static int8_t* copy_ptr(const cpt* c, int32_t rep, int32_t i, int32_t k) {
    /* copy k of site i: even k at k/2, odd k at H + k/2 */
    return c->s + ((size_t)rep * c->N + i) * c->row + (k & 1) * c->H + (k >> 1);
}

static void chain_sums(cpt* c, int32_t rep) {
    int64_t e = 0, m = 0;
    for (int32_t k = 0; k < c->P; ++k)
        for (int32_t i = 0; i < c->N; ++i) {
            const int32_t si = *copy_ptr(c, rep, i, k);
            int32_t f = c->h[i];
            for (int32_t a = c->adj_off[i]; a < c->adj_off[i + 1]; ++a)
                if (c->adj_j[a] > i) f += c->adj_J[a] * *copy_ptr(c, rep, c->adj_j[a], k);
            e += (int64_t)si * f;
            m += (int64_t)si * *copy_ptr(c, rep, i, (k + 1) % c->P);
        }
    c->E[rep] = e;
    c->M[rep] = m;
}

int32_t cpt_lmax(const cpt* c) { return c->Lmax; }

cpt* cpt_create(int32_t n, int32_t n_edges, const int32_t* ei, const int32_t* ej, const int32_t* J,
                const int32_t* h, int32_t P, int32_t R, const uint32_t* thr, const double* coef, uint64_t seed,
                int32_t threads) {
    if (n < 1 || n_edges < 0 || R < 1 || (P != 1 && (P < 2 || (P & 1))) || !thr || (R > 1 && !coef) || !h ||
        (n_edges > 0 && (!ei || !ej || !J)))
        return NULL;
    cpt* c = (cpt*)calloc(1, sizeof(cpt));
    c->N = n;
    c->P = P;
    c->R = R;
    c->H = P == 1 ? 1 : P / 2;
    c->odd = P == 1 ? 0 : 1;
    c->row = P == 1 ? 1 : P;
    c->threads = threads < 1 ? 1 : threads;
    c->adj_off = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
    c->adj_j = (int32_t*)malloc(sizeof(int32_t) * (2 * (size_t)n_edges + 1));
    c->adj_J = (int32_t*)malloc(sizeof(int32_t) * (2 * (size_t)n_edges + 1));
    c->h = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    memcpy(c->h, h, sizeof(int32_t) * (size_t)n);
    for (int32_t b = 0; b < n_edges; ++b) {
        if (ei[b] < 0 || ei[b] >= n || ej[b] < 0 || ej[b] >= n || ei[b] == ej[b]) {
            cpt_destroy(c);
            return NULL;
        }
        c->adj_off[ei[b] + 1]++;
        c->adj_off[ej[b] + 1]++;
    }
    for (int32_t i = 0; i < n; ++i) c->adj_off[i + 1] += c->adj_off[i];
    int32_t* pos = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    memcpy(pos, c->adj_off, sizeof(int32_t) * (size_t)n);
    for (int32_t b = 0; b < n_edges; ++b) {
        c->adj_j[pos[ei[b]]] = ej[b];
        c->adj_J[pos[ei[b]]++] = J[b];
        c->adj_j[pos[ej[b]]] = ei[b];
        c->adj_J[pos[ej[b]]++] = J[b];
    }
    free(pos);
    c->Lmax = 0;
    for (int32_t i = 0; i < n; ++i) {
        int32_t l = abs(h[i]);
        for (int32_t a = c->adj_off[i]; a < c->adj_off[i + 1]; ++a) l += abs(c->adj_J[a]);
        if (l > c->Lmax) c->Lmax = l;
    }
    const size_t nthr = (size_t)R * (2 * (size_t)c->Lmax + 1) * 3;
    c->thr = (uint32_t*)malloc(sizeof(uint32_t) * nthr);
    memcpy(c->thr, thr, sizeof(uint32_t) * nthr);
    c->coef = (double*)calloc(2 * (size_t)R, sizeof(double));
    if (R > 1) memcpy(c->coef, coef, sizeof(double) * 2 * (size_t)(R - 1));
    c->k0 = (uint32_t)(seed & 0xFFFFFFFFu);
    c->k1 = (uint32_t)(seed >> 32);
    c->s = (int8_t*)malloc((size_t)R * n * c->row);
    c->E = (int64_t*)calloc((size_t)R, sizeof(int64_t));
    c->M = (int64_t*)calloc((size_t)R, sizeof(int64_t));
    c->rung_of = (int32_t*)malloc(sizeof(int32_t) * (size_t)R);
    c->replica_at = (int32_t*)malloc(sizeof(int32_t) * (size_t)R);
    c->order = (int32_t*)malloc(sizeof(int32_t) * (size_t)R);
    c->hard = (int64_t*)calloc((size_t)R, sizeof(int64_t));
    int64_t** stats[] = {&c->n_meas, &c->sum_E, &c->sum_E2, &c->sum_M, &c->sum_M2, &c->flip_acc, &c->swap_att,
                         &c->swap_acc};
    for (size_t k = 0; k < sizeof(stats) / sizeof(stats[0]); ++k) *stats[k] = (int64_t*)calloc((size_t)R, sizeof(int64_t));
    /* initial spins: chain rho starts on rung rho; copy k of site i is -1 iff bit 31 of word
     * k % 4 of philox((0, i, rho, 2 << 28 | k / 4)) is set */
    for (int32_t rep = 0; rep < R; ++rep) {
        c->rung_of[rep] = rep;
        c->replica_at[rep] = rep;
        c->order[rep] = R - 1 - rep;
        for (int32_t i = 0; i < n; ++i)
            for (int32_t k = 0; k < P; k += 4) {
                uint32_t u[4];
                philox10(0u, (uint32_t)i, (uint32_t)rep, (2u << 28) | (uint32_t)(k >> 2), c->k0, c->k1, u);
                for (int32_t w = 0; w < 4 && k + w < P; ++w) *copy_ptr(c, rep, i, k + w) = (u[w] >> 31) ? -1 : 1;
            }
        chain_sums(c, rep);
    }
    return c;
}

void cpt_destroy(cpt* c) {
    if (!c) return;
    void* ptrs[] = {c->adj_off, c->adj_j, c->adj_J, c->h,      c->thr,    c->coef,    c->s,        c->E,
                    c->M,       c->rung_of, c->replica_at, c->order, c->hard, c->n_meas, c->sum_E, c->sum_E2,
                    c->sum_M,   c->sum_M2, c->flip_acc, c->swap_att, c->swap_acc};
    for (size_t k = 0; k < sizeof(ptrs) / sizeof(ptrs[0]); ++k) free(ptrs[k]);
    free(c);
}

/* ---------------------------------------------------------------- one chain, one interval
 * len sweeps of chain rep, starting at sweep t0, on the rung it holds for the interval.
 * Sweep t visits sites in index order; at each site the even copies, then the odd ones.
 * Copy k = p + 2x of site i draws word x % 4 of philox((t, i, rep, p << 24 | x / 4)). The
 * statistics of the rung are gathered after every sweep. */
static void sweep_interval(cpt* c, int32_t rep, int64_t t0, int32_t len) {
    const int32_t N = c->N, H = c->H, row = c->row, L0 = c->Lmax, r = c->rung_of[rep];
    const uint32_t* thr = c->thr + (size_t)r * (2 * (size_t)L0 + 1) * 3;
    int8_t* base = c->s + (size_t)rep * N * row;
    int32_t* field = (int32_t*)malloc(sizeof(int32_t) * (size_t)H);
    int64_t E = c->E[rep], M = c->M[rep], flips = 0;
    for (int32_t s = 0; s < len; ++s) {
        const uint32_t t = (uint32_t)(t0 + s);
        for (int32_t i = 0; i < N; ++i) {
            int8_t* site = base + (size_t)i * row;
            for (int32_t p = 0; p <= c->odd; ++p) {
                int8_t* own = site + p * H;
                const int8_t* opp = site + (1 - p) * H;
                for (int32_t x = 0; x < H; ++x) field[x] = c->h[i];
                for (int32_t a = c->adj_off[i]; a < c->adj_off[i + 1]; ++a) {
                    const int8_t* nb = base + (size_t)c->adj_j[a] * row + p * H;
                    const int32_t Jv = c->adj_J[a];
                    for (int32_t x = 0; x < H; ++x) field[x] += Jv * nb[x];
                }
                uint32_t u[4] = {0, 0, 0, 0};
                for (int32_t x = 0; x < H; ++x) {
                    if ((x & 3) == 0)
                        philox10(t, (uint32_t)i, (uint32_t)rep, ((uint32_t)p << 24) | (uint32_t)(x >> 2), c->k0, c->k1, u);
                    const int32_t si = own[x];
                    const int32_t L = si * field[x];
                    int32_t m = 0;
                    if (c->odd) {
                        /* Trotter neighbours k - 1 and k + 1 (periodic) are opposite-parity copies */
                        const int32_t left = p == 0 ? opp[x == 0 ? H - 1 : x - 1] : opp[x];
                        const int32_t right = p == 0 ? opp[x] : opp[x + 1 == H ? 0 : x + 1];
                        m = si * (left + right);
                    }
                    const uint32_t th = thr[(size_t)(L + L0) * 3 + (size_t)(m / 2 + 1)];
                    if (th == 0xFFFFFFFFu || u[x & 3] < th) {
                        own[x] = (int8_t)(-si);
                        E -= 2 * (int64_t)L;
                        M -= 2 * (int64_t)m;
                        ++flips;
                    }
                }
            }
        }
        /* measurements after every sweep (Fig. 4); this chain alone holds rung r */
        c->n_meas[r] += 1;
        c->sum_E[r] += E;
        c->sum_E2[r] += E * E;
        c->sum_M[r] += M;
        c->sum_M2[r] += M * M;
    }
    c->flip_acc[r] += flips;
    c->hard[rep] = flips;
    c->E[rep] = E;
    c->M[rep] = M;
    free(field);
}

/* Pair (r, r + 1) of swap pass q (Sec. 2): accept iff Delta >= 0, or Delta > -23 and
 * u < min(floor(2^32 exp(Delta)), 2^32 - 1) with u = word 0 of philox((q, r, 0, 1 << 28)),
 * Delta = a_r (E_X - E_Y) + c_r (M_X - M_Y) for X on rung r and Y on rung r + 1. */
static void swap_pair(cpt* c, int32_t r, int64_t q) {
    const int32_t X = c->replica_at[r], Y = c->replica_at[r + 1];
    const double dE = (double)(c->E[X] - c->E[Y]);
    const double dM = (double)(c->M[X] - c->M[Y]);
    const double delta = c->coef[r] * dE + c->coef[(c->R - 1) + r] * dM;
    int accept = 0;
    if (delta >= 0.0) {
        accept = 1;
    } else if (delta > -23.0) {
        uint32_t u[4];
        philox10((uint32_t)q, (uint32_t)r, 0u, 1u << 28, c->k0, c->k1, u);
        const double v = floor(exp_swap(delta) * 4294967296.0);
        const uint32_t ts = v >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)v;
        accept = u[0] < ts;
    }
    c->swap_att[r] += 1;
    if (accept) {
        c->swap_acc[r] += 1;
        c->replica_at[r] = Y;
        c->replica_at[r + 1] = X;
        c->rung_of[X] = r + 1;
        c->rung_of[Y] = r;
    }
}

/* ---------------------------------------------------------------- persistent threads
 * Fig. 5: the threads stay alive for the whole run. Per interval they take chains from a
 * shared pool (hardest first) until it is empty, meet at a barrier, decide the swap pass's
 * disjoint pairs in parallel, meet again, and one thread orders the next pool. */
typedef struct {
    cpt* c;
    int64_t n_sweeps;
    int32_t sps;
    atomic_int next;
    pthread_barrier_t bar;
} run_state;

typedef struct {
    run_state* rs;
    int32_t tid;
} worker_arg;


static const cpt* g_sort_ctx;  /* the pool order is set by one thread between barriers */
static int cmp_hard(const void* a, const void* b) {
    const int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    const int64_t hx = g_sort_ctx->hard[x], hy = g_sort_ctx->hard[y];
    if (hx != hy) return hx > hy ? -1 : 1;
    return x < y ? -1 : (x > y);
}

static void* worker(void* p) {
    worker_arg* wa = (worker_arg*)p;
    run_state* rs = wa->rs;
    cpt* c = rs->c;
    const int32_t T = c->threads;
    int64_t done = 0;
    while (done < rs->n_sweeps) {
        const int64_t left = rs->n_sweeps - done;
        const int swap = rs->sps > 0 && left >= rs->sps;
        const int32_t len = (int32_t)(rs->sps > 0 ? (swap ? rs->sps : left) : left);
        const int64_t t0 = c->t;
        for (int k; (k = atomic_fetch_add(&rs->next, 1)) < c->R;) sweep_interval(c, c->order[k], t0, len);
        pthread_barrier_wait(&rs->bar);
        if (swap)
            for (int32_t r = (int32_t)(c->q & 1) + 2 * wa->tid; r + 1 < c->R; r += 2 * T) swap_pair(c, r, c->q);
        pthread_barrier_wait(&rs->bar);
        if (wa->tid == 0) {
            c->t += len;
            if (swap) c->q += 1;
            g_sort_ctx = c;
            qsort(c->order, (size_t)c->R, sizeof(int32_t), cmp_hard);
            atomic_store(&rs->next, 0);
        }
        pthread_barrier_wait(&rs->bar);
        done += len;
    }
    return NULL;
}

void cpt_run(cpt* c, int64_t n_sweeps, int32_t sps) {
    if (!c || n_sweeps <= 0) return;
    if (sps > 0 && c->R == 1) {
        /* a one-rung ladder has no pairs; its passes only count */
        cpt_run(c, n_sweeps, 0);
        c->q += n_sweeps / sps;
        return;
    }
    run_state rs;
    rs.c = c;
    rs.n_sweeps = n_sweeps;
    rs.sps = sps;
    atomic_init(&rs.next, 0);
    const int32_t T = c->threads;
    pthread_barrier_init(&rs.bar, NULL, (unsigned)T);
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)T);
    worker_arg* args = (worker_arg*)malloc(sizeof(worker_arg) * (size_t)T);
    for (int32_t k = 0; k < T; ++k) {
        args[k].rs = &rs;
        args[k].tid = k;
        if (k > 0) pthread_create(&th[k], NULL, worker, &args[k]);
    }
    worker(&args[0]);
    for (int32_t k = 1; k < T; ++k) pthread_join(th[k], NULL);
    pthread_barrier_destroy(&rs.bar);
    free(th);
    free(args);
}

void cpt_read_state(const cpt* c, int8_t* out) {
    for (int32_t r = 0; r < c->R; ++r) {
        const int32_t rep = c->replica_at[r];
        for (int32_t i = 0; i < c->N; ++i)
            for (int32_t k = 0; k < c->P; ++k) out[((size_t)r * c->N + i) * c->P + k] = *copy_ptr(c, rep, i, k);
    }
}

void cpt_read_obs(const cpt* c, int64_t* tq, int64_t* E, int64_t* M, int64_t* n_meas, int64_t* sum_E,
                  int64_t* sum_E2, int64_t* sum_M, int64_t* sum_M2, int64_t* flip_acc, int64_t* swap_att,
                  int64_t* swap_acc, int32_t* replica_at) {
    tq[0] = c->t;
    tq[1] = c->q;
    for (int32_t r = 0; r < c->R; ++r) {
        const int32_t rep = c->replica_at[r];
        E[r] = c->E[rep];
        M[r] = c->M[rep];
        n_meas[r] = c->n_meas[r];
        sum_E[r] = c->sum_E[r];
        sum_E2[r] = c->sum_E2[r];
        sum_M[r] = c->sum_M[r];
        sum_M2[r] = c->sum_M2[r];
        flip_acc[r] = c->flip_acc[r];
        replica_at[r] = rep;
        if (r + 1 < c->R) {
            swap_att[r] = c->swap_att[r];
            swap_acc[r] = c->swap_acc[r];
        }
    }
}
