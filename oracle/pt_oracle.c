/*
 * pt_oracle.c -- plain, slow, obviously correct CPU oracle for the PT-QMC hot path.
 *
 * TEST INFRASTRUCTURE ONLY (see pt_oracle.h). Compiled with -ffp-contract=off so that
 * every floating-point operation below is one IEEE basic operation in the order written.
 *
 * Model (Sec. 2 parallel tempering; Sec. 6 "many copies (128) of the corresponding
 * classical system" = the Suzuki-Trotter mapping of the transverse-field Ising model):
 *   spins s in {-1,+1}; one copy's problem energy E(s) = sum_edges J_ij s_i s_j + sum_i h_i s_i
 *   chain state X = s[i][k], copy index k periodic mod P
 *   rung r: beta_r = 1/T_r, a_r = beta_r*Gamma_r/P, K_r = -1/2 ln tanh(a_r)
 *   action S_r(X) = (beta_r/P) * sum_k E(s^k) - K_r * M(X),  M(X) = sum_k sum_i s_i^k s_i^{k+1}
 *   each chain samples exp(-S_r) at the rung r it currently sits on.
 */
#include "pt_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
 * 1, 2, 3", SC'11). One round maps (c0,c1,c2,c3) with round key (k0,k1) to
 *   (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0));
 * the key is bumped by the Weyl constants (W0,W1) between rounds; 10 rounds.
 * ------------------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t prod0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(prod1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)prod1;
        uint32_t n2 = (uint32_t)(prod0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)prod0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* Stream tags in the top nibble of counter word 3 keep the three uses apart. */
#define TAG_FLIP 0u
#define TAG_SWAP 1u
#define TAG_INIT 2u

/* ------------------------------------------------------------------------------------
 * det_exp: exp(x) for x in (-23, 0] from IEEE basic operations only (Cody & Waite
 * argument reduction, "Software Manual for the Elementary Functions", 1980, followed
 * by the Taylor series of exp evaluated by Horner's rule).
 *   n = rint(x * (1/ln2));  r = (x - n*LN2_HI) - n*LN2_LO;  exp(r) ~ sum_{k<=13} r^k/k!
 *   result = p * 2^n.
 * LN2_HI is ln 2 rounded to 28 fraction bits, so n*LN2_HI is exact for |n| < 2^24;
 * LN2_LO = ln 2 - LN2_HI rounded to double; INV_LN2 = 1/ln 2 rounded to double.
 * ------------------------------------------------------------------------------------ */
static const double DE_LN2_HI = 0x1.62e42ff000000p-1;
static const double DE_LN2_LO = -0x1.718432a1b0e26p-35;
static const double DE_INV_LN2 = 0x1.71547652b82fep+0;

double orc_det_exp(double x) {
    double inv_fact[14];
    double fact = 1.0;
    for (int k = 0; k < 14; k++) {
        if (k > 0) fact = fact * (double)k; /* k! is exact in double for k <= 13 */
        inv_fact[k] = 1.0 / fact;
    }
    double nd = rint(x * DE_INV_LN2);
    double r = (x - nd * DE_LN2_HI) - nd * DE_LN2_LO;
    double p = inv_fact[13];
    for (int k = 12; k >= 0; k--) p = p * r + inv_fact[k];
    return ldexp(p, (int)nd);
}

void orc_det_exp_array(const double* x, double* y, int64_t n) {
    for (int64_t i = 0; i < n; i++) y[i] = orc_det_exp(x[i]);
}

/* ------------------------------------------------------------------------------------ */

struct orc {
    int32_t N, P, R, n_edges, Lmax;
    int32_t* ei;
    int32_t* ej;
    int32_t* Jv;
    int32_t* h;
    /* adjacency: neighbours of site i are adj_j[adj_off[i] .. adj_off[i+1]) with couplings adj_J */
    int32_t* adj_off;
    int32_t* adj_j;
    int32_t* adj_J;
    uint32_t* thr;  /* [R][2*Lmax+1][3] */
    double* coef;   /* a[0..R-2], c[0..R-2] */
    uint32_t key[2];
    int8_t* s;          /* [replica][i][k] */
    int32_t* rung_of;   /* [replica] */
    int32_t* replica_at; /* [rung] */
    int64_t* E;         /* [replica] sum_k E(s^k) */
    int64_t* M;         /* [replica] sum_k sum_i s_i^k s_i^{k+1} */
    int64_t t, q;
    int64_t *n_meas, *sum_E, *sum_E2, *sum_M, *sum_M2, *flip_acc; /* [rung] */
    int64_t *swap_att, *swap_acc;                                  /* [pair] */
    int32_t threads;
};

static char orc_errbuf[256];
const char* orc_error(void) { return orc_errbuf; }
static void set_err(const char* m) {
    strncpy(orc_errbuf, m, sizeof(orc_errbuf) - 1);
    orc_errbuf[sizeof(orc_errbuf) - 1] = 0;
}

static int8_t* spin_ptr(const orc* o, int32_t rep, int32_t i, int32_t k) {
    return o->s + ((size_t)rep * o->N + (size_t)i) * o->P + (size_t)k;
}

/* sum_k E(s^k) straight from the definition of E. */
static int64_t chain_energy(const orc* o, int32_t rep) {
    int64_t e = 0;
    for (int32_t k = 0; k < o->P; k++) {
        for (int32_t b = 0; b < o->n_edges; b++)
            e += (int64_t)o->Jv[b] * *spin_ptr(o, rep, o->ei[b], k) * *spin_ptr(o, rep, o->ej[b], k);
        for (int32_t i = 0; i < o->N; i++) e += (int64_t)o->h[i] * *spin_ptr(o, rep, i, k);
    }
    return e;
}

/* M(X) = sum_k sum_i s_i^k s_i^{(k+1) mod P} straight from its definition. */
static int64_t chain_trotter(const orc* o, int32_t rep) {
    int64_t m = 0;
    for (int32_t k = 0; k < o->P; k++)
        for (int32_t i = 0; i < o->N; i++)
            m += (int64_t)*spin_ptr(o, rep, i, k) * *spin_ptr(o, rep, i, (k + 1) % o->P);
    return m;
}

/* Metropolis acceptance table (Sec. 2: flips follow the Metropolis rule at the chain's
 * temperature; Sec. 5 keeps the real-valued part of a sweep in a table-driven form).
 * Flipping s_i^k changes the action by dS = -(2 beta/P) L + 2 K m with
 *   L = s_i^k (h_i + sum_j J_ij s_j^k),  m = s_i^k (s_i^{k-1} + s_i^{k+1}),
 * so the Metropolis probability is p = min(1, exp((2 beta/P) L - 2 K m)).
 * thr = 0xFFFFFFFF means "always accept"; otherwise accept iff u < thr = floor(p 2^32). */
static void build_tables(orc* o, const double* T, const double* gamma) {
    int32_t nL = 2 * o->Lmax + 1;
    double* K = (double*)malloc(sizeof(double) * o->R);
    double* b = (double*)malloc(sizeof(double) * o->R);
    for (int32_t r = 0; r < o->R; r++) {
        double beta = 1.0 / T[r];
        double a = beta * gamma[r] / (double)o->P;
        /* classical (P = 1): no Trotter coupling */
        K[r] = o->P == 1 ? 0.0 : -0.5 * log(tanh(a));
        b[r] = beta / (double)o->P;
        double c1 = 2.0 * beta / (double)o->P;
        double c2 = 2.0 * K[r];
        for (int32_t L = -o->Lmax; L <= o->Lmax; L++) {
            for (int32_t mi = 0; mi < 3; mi++) {
                int32_t m = 2 * mi - 2;
                double x = c1 * (double)L - c2 * (double)m;
                uint32_t thr;
                if (x >= 0.0) {
                    thr = 0xFFFFFFFFu;
                } else {
                    double v = floor(ldexp(exp(x), 32));
                    thr = (v >= 4294967295.0) ? 0xFFFFFFFFu : (uint32_t)v;
                }
                o->thr[((size_t)r * nL + (size_t)(L + o->Lmax)) * 3 + (size_t)mi] = thr;
            }
        }
    }
    /* swap coefficients (Sec. 2: probability of the two chains' states occurring at each
     * other's temperature): exchanging X at rung r with Y at rung r+1 has
     * log ratio = a_r (E_X - E_Y) + c_r (M_X - M_Y), a_r = beta_r/P - beta_{r+1}/P, c_r = K_{r+1} - K_r */
    for (int32_t r = 0; r + 1 < o->R; r++) {
        o->coef[r] = b[r] - b[r + 1];
        o->coef[(o->R - 1) + r] = K[r + 1] - K[r];
    }
    free(K);
    free(b);
}

orc* orc_create(int32_t n, int32_t n_edges, const int32_t* ei, const int32_t* ej,
                const int32_t* J, const int32_t* h, int32_t P, int32_t R,
                const double* T, const double* gamma, const uint32_t* flip_thr,
                const double* swap_coef, uint64_t seed) {
    if (n < 1 || n_edges < 0 || (P != 1 && (P < 2 || (P & 1))) || R < 1) {
        set_err("need n >= 1, n_edges >= 0, P = 1 or even P >= 2, R >= 1");
        return NULL;
    }
    for (int32_t b = 0; b < n_edges; b++) {
        if (ei[b] < 0 || ei[b] >= n || ej[b] < 0 || ej[b] >= n || ei[b] == ej[b] || J[b] == 0) {
            set_err("edge endpoints must be distinct sites in range and J must be non-zero");
            return NULL;
        }
        for (int32_t c = 0; c < b; c++)
            if ((ei[c] == ei[b] && ej[c] == ej[b]) || (ei[c] == ej[b] && ej[c] == ei[b])) {
                set_err("duplicate edge");
                return NULL;
            }
    }
    /* P >= 2: the Suzuki-Trotter chain of the transverse-field problem, Gamma > 0 (K finite).
     * P = 1: classical parallel tempering over T, Gamma = 0 (one copy, no Trotter coupling). */
    if (!flip_thr || !swap_coef)
        for (int32_t r = 0; r < R; r++)
            if (!(T[r] > 0.0) || (P == 1 ? !(gamma[r] == 0.0) : !(gamma[r] > 0.0))) {
                set_err("T must be positive; Gamma positive for P >= 2 and zero for P = 1");
                return NULL;
            }

    orc* o = (orc*)calloc(1, sizeof(orc));
    o->N = n;
    o->P = P;
    o->R = R;
    o->n_edges = n_edges;
    o->threads = 1;
    o->ei = (int32_t*)malloc(sizeof(int32_t) * (n_edges + 1));
    o->ej = (int32_t*)malloc(sizeof(int32_t) * (n_edges + 1));
    o->Jv = (int32_t*)malloc(sizeof(int32_t) * (n_edges + 1));
    o->h = (int32_t*)malloc(sizeof(int32_t) * n);
    memcpy(o->ei, ei, sizeof(int32_t) * n_edges);
    memcpy(o->ej, ej, sizeof(int32_t) * n_edges);
    memcpy(o->Jv, J, sizeof(int32_t) * n_edges);
    memcpy(o->h, h, sizeof(int32_t) * n);

    /* adjacency lists */
    o->adj_off = (int32_t*)calloc(n + 1, sizeof(int32_t));
    for (int32_t b = 0; b < n_edges; b++) {
        o->adj_off[ei[b] + 1]++;
        o->adj_off[ej[b] + 1]++;
    }
    for (int32_t i = 0; i < n; i++) o->adj_off[i + 1] += o->adj_off[i];
    o->adj_j = (int32_t*)malloc(sizeof(int32_t) * (2 * n_edges + 1));
    o->adj_J = (int32_t*)malloc(sizeof(int32_t) * (2 * n_edges + 1));
    int32_t* fill = (int32_t*)calloc(n, sizeof(int32_t));
    for (int32_t b = 0; b < n_edges; b++) {
        int32_t u = ei[b], v = ej[b];
        o->adj_j[o->adj_off[u] + fill[u]] = v;
        o->adj_J[o->adj_off[u] + fill[u]++] = J[b];
        o->adj_j[o->adj_off[v] + fill[v]] = u;
        o->adj_J[o->adj_off[v] + fill[v]++] = J[b];
    }
    free(fill);

    /* Lmax = max_i (|h_i| + sum_j |J_ij|) bounds |L| */
    o->Lmax = 0;
    for (int32_t i = 0; i < n; i++) {
        int32_t l = abs(h[i]);
        for (int32_t a = o->adj_off[i]; a < o->adj_off[i + 1]; a++) l += abs(o->adj_J[a]);
        if (l > o->Lmax) o->Lmax = l;
    }

    size_t nthr = (size_t)R * (2 * o->Lmax + 1) * 3;
    o->thr = (uint32_t*)malloc(sizeof(uint32_t) * nthr);
    o->coef = (double*)malloc(sizeof(double) * (2 * (size_t)R));
    if (!flip_thr || !swap_coef) build_tables(o, T, gamma);
    if (flip_thr) memcpy(o->thr, flip_thr, sizeof(uint32_t) * nthr);
    if (swap_coef) memcpy(o->coef, swap_coef, sizeof(double) * 2 * (size_t)(R - 1));

    o->key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
    o->key[1] = (uint32_t)(seed >> 32);

    o->s = (int8_t*)malloc((size_t)R * n * P);
    o->rung_of = (int32_t*)malloc(sizeof(int32_t) * R);
    o->replica_at = (int32_t*)malloc(sizeof(int32_t) * R);
    o->E = (int64_t*)calloc(R, sizeof(int64_t));
    o->M = (int64_t*)calloc(R, sizeof(int64_t));
    o->n_meas = (int64_t*)calloc(R, sizeof(int64_t));
    o->sum_E = (int64_t*)calloc(R, sizeof(int64_t));
    o->sum_E2 = (int64_t*)calloc(R, sizeof(int64_t));
    o->sum_M = (int64_t*)calloc(R, sizeof(int64_t));
    o->sum_M2 = (int64_t*)calloc(R, sizeof(int64_t));
    o->flip_acc = (int64_t*)calloc(R, sizeof(int64_t));
    o->swap_att = (int64_t*)calloc(R, sizeof(int64_t));
    o->swap_acc = (int64_t*)calloc(R, sizeof(int64_t));

    /* Initial state: chain rho starts on rung rho; each spin from the chain's own stream
     * (Sec. 3: every chain has its own random state) with counter (0, i, rho, INIT|k/4),
     * word k%4, spin = -1 if the top bit is set. */
    for (int32_t rep = 0; rep < R; rep++) {
        o->rung_of[rep] = rep;
        o->replica_at[rep] = rep;
        for (int32_t i = 0; i < n; i++)
            for (int32_t k = 0; k < P; k++) {
                uint32_t ctr[4] = {0u, (uint32_t)i, (uint32_t)rep, (TAG_INIT << 28) | (uint32_t)(k >> 2)};
                uint32_t u[4];
                orc_philox(ctr, o->key, u);
                *spin_ptr(o, rep, i, k) = (u[k & 3] >> 31) ? (int8_t)-1 : (int8_t)1;
            }
        o->E[rep] = chain_energy(o, rep);
        o->M[rep] = chain_trotter(o, rep);
    }
    return o;
}

void orc_destroy(orc* o) {
    if (!o) return;
    free(o->ei); free(o->ej); free(o->Jv); free(o->h);
    free(o->adj_off); free(o->adj_j); free(o->adj_J);
    free(o->thr); free(o->coef); free(o->s);
    free(o->rung_of); free(o->replica_at); free(o->E); free(o->M);
    free(o->n_meas); free(o->sum_E); free(o->sum_E2); free(o->sum_M); free(o->sum_M2);
    free(o->flip_acc); free(o->swap_att); free(o->swap_acc);
    free(o);
}

void orc_set_threads(orc* o, int32_t threads) { o->threads = threads < 1 ? 1 : threads; }
int32_t orc_lmax(const orc* o) { return o->Lmax; }
void orc_flip_table(const orc* o, uint32_t* out) {
    memcpy(out, o->thr, sizeof(uint32_t) * (size_t)o->R * (2 * o->Lmax + 1) * 3);
}
void orc_swap_coef(const orc* o, double* out) {
    memcpy(out, o->coef, sizeof(double) * 2 * (size_t)(o->R - 1));
}

/* One Metropolis sweep of chain rep at sweep index t (Sec. 2 "sweeps through all of the
 * chains, flipping bits with the Metropolis algorithm"; Sec. 5: the chain is split into
 * two groups of independent regions, swept one group after the other). Sites are visited
 * in index order; at each site all even copies k = 0, 2, ... are updated, then all odd
 * copies k = 1, 3, .... The uniform for copy k = p + 2*hh (p = k mod 2) comes from the
 * chain's stream with counter (t, i, rep, FLIP | p<<24 | hh/4), word hh mod 4. */
static void sweep_chain(orc* o, int32_t rep, int64_t t, int64_t* flips_out) {
    const int32_t P = o->P, nL = 2 * o->Lmax + 1;
    const uint32_t* thr = o->thr + (size_t)o->rung_of[rep] * nL * 3;
    int64_t dE = 0, dM = 0, flips = 0;
    for (int32_t i = 0; i < o->N; i++) {
        for (int32_t p = 0; p < 2; p++) {
            uint32_t u[4] = {0, 0, 0, 0};
            for (int32_t hh = 0; 2 * hh + p < P; hh++) {
                int32_t k = p + 2 * hh;
                if ((hh & 3) == 0) {
                    uint32_t ctr[4] = {(uint32_t)t, (uint32_t)i, (uint32_t)rep,
                                       (TAG_FLIP << 28) | ((uint32_t)p << 24) | (uint32_t)(hh >> 2)};
                    orc_philox(ctr, o->key, u);
                }
                int32_t si = *spin_ptr(o, rep, i, k);
                int32_t field = o->h[i];
                for (int32_t a = o->adj_off[i]; a < o->adj_off[i + 1]; a++)
                    field += o->adj_J[a] * *spin_ptr(o, rep, o->adj_j[a], k);
                int32_t L = si * field;
                /* the lone copy of a classical chain (P = 1) has no Trotter neighbours */
                int32_t m = P == 1 ? 0
                                   : si * (*spin_ptr(o, rep, i, (k + P - 1) % P) + *spin_ptr(o, rep, i, (k + 1) % P));
                uint32_t th = thr[(size_t)(L + o->Lmax) * 3 + (size_t)(m / 2 + 1)];
                if (th == 0xFFFFFFFFu || u[hh & 3] < th) {
                    *spin_ptr(o, rep, i, k) = (int8_t)(-si);
                    dE -= 2 * (int64_t)L;
                    dM -= 2 * (int64_t)m;
                    flips++;
                }
            }
        }
    }
    o->E[rep] += dE;
    o->M[rep] += dM;
    *flips_out = flips;
}

/* Measurements after every sweep (Fig. 4 "gather statistics"; Sec. 5 accumulates in high
 * precision): per rung, the count and the sums of E, E^2, M, M^2 of the chain on it. */
static void accumulate(orc* o) {
    for (int32_t r = 0; r < o->R; r++) {
        int32_t rep = o->replica_at[r];
        o->n_meas[r] += 1;
        o->sum_E[r] += o->E[rep];
        o->sum_E2[r] += o->E[rep] * o->E[rep];
        o->sum_M[r] += o->M[rep];
        o->sum_M2[r] += o->M[rep] * o->M[rep];
    }
}

void orc_sweep(orc* o, int64_t n) {
    int64_t* flips = (int64_t*)calloc(o->R, sizeof(int64_t));
    for (int64_t s = 0; s < n; s++) {
        /* chains are independent during a sweep (Sec. 4); the optional threads only split them */
#ifdef _OPENMP
#pragma omp parallel for num_threads(o->threads) schedule(dynamic, 1)
#endif
        for (int32_t rep = 0; rep < o->R; rep++) sweep_chain(o, rep, o->t, &flips[rep]);
        for (int32_t rep = 0; rep < o->R; rep++) o->flip_acc[o->rung_of[rep]] += flips[rep];
        o->t += 1;
        accumulate(o);
    }
    free(flips);
}

/* One swap pass q (Sec. 2: only neighbouring chains are swap candidates, taken two at a
 * time, so up to R/2 disjoint pairs): pairs (r, r+1) for r = q mod 2, q mod 2 + 2, ....
 * X on rung r and Y on rung r+1 exchange rungs with probability min(1, exp(Delta)),
 * Delta = a_r (E_X - E_Y) + c_r (M_X - M_Y). The uniform is word 0 of the counter
 * (q, r, 0, SWAP). Accept iff Delta >= 0, or Delta > -23 and u < min(floor(2^32 e^Delta), 2^32-1). */
void orc_swap(orc* o) {
    const double* a = o->coef;
    const double* c = o->coef + (o->R - 1);
    for (int32_t r = (int32_t)(o->q & 1); r + 1 < o->R; r += 2) {
        int32_t X = o->replica_at[r], Y = o->replica_at[r + 1];
        double dE = (double)(o->E[X] - o->E[Y]);
        double dM = (double)(o->M[X] - o->M[Y]);
        double delta = a[r] * dE + c[r] * dM;
        int accept;
        if (delta >= 0.0) {
            accept = 1;
        } else if (!(delta > -23.0)) {
            accept = 0;
        } else {
            uint32_t ctr[4] = {(uint32_t)o->q, (uint32_t)r, 0u, TAG_SWAP << 28};
            uint32_t u[4];
            orc_philox(ctr, o->key, u);
            double v = floor(ldexp(orc_det_exp(delta), 32));
            uint32_t ts = (v >= 4294967295.0) ? 0xFFFFFFFFu : (uint32_t)v;
            accept = u[0] < ts;
        }
        o->swap_att[r] += 1;
        if (accept) {
            o->swap_acc[r] += 1;
            o->replica_at[r] = Y;
            o->replica_at[r + 1] = X;
            o->rung_of[X] = r + 1;
            o->rung_of[Y] = r;
        }
    }
    o->q += 1;
}

/* The loop of Fig. 4: sweeps, with a swap pass after every sweeps_per_swap-th sweep. */
void orc_run(orc* o, int64_t n_sweeps, int32_t sweeps_per_swap) {
    for (int64_t s = 0; s < n_sweeps; s++) {
        orc_sweep(o, 1);
        if (sweeps_per_swap > 0 && (s + 1) % sweeps_per_swap == 0) orc_swap(o);
    }
}

void orc_read_state(const orc* o, int8_t* out) {
    size_t chain = (size_t)o->N * o->P;
    for (int32_t r = 0; r < o->R; r++)
        memcpy(out + (size_t)r * chain, o->s + (size_t)o->replica_at[r] * chain, chain);
}

void orc_read_replica_state(const orc* o, int8_t* out) {
    memcpy(out, o->s, (size_t)o->R * o->N * o->P);
}

int orc_write_state(orc* o, const int8_t* in) {
    size_t chain = (size_t)o->N * o->P;
    for (size_t x = 0; x < (size_t)o->R * chain; x++)
        if (in[x] != 1 && in[x] != -1) return -1;
    for (int32_t r = 0; r < o->R; r++) {
        int32_t rep = o->replica_at[r];
        memcpy(o->s + (size_t)rep * chain, in + (size_t)r * chain, chain);
        o->E[rep] = chain_energy(o, rep);
        o->M[rep] = chain_trotter(o, rep);
    }
    return 0;
}

void orc_read_obs(const orc* o, int64_t* tq, int64_t* E, int64_t* M, int64_t* n_meas,
                  int64_t* sum_E, int64_t* sum_E2, int64_t* sum_M, int64_t* sum_M2,
                  int64_t* flip_acc, int64_t* swap_att, int64_t* swap_acc,
                  int32_t* replica_at) {
    tq[0] = o->t;
    tq[1] = o->q;
    for (int32_t r = 0; r < o->R; r++) {
        E[r] = o->E[o->replica_at[r]];
        M[r] = o->M[o->replica_at[r]];
        n_meas[r] = o->n_meas[r];
        sum_E[r] = o->sum_E[r];
        sum_E2[r] = o->sum_E2[r];
        sum_M[r] = o->sum_M[r];
        sum_M2[r] = o->sum_M2[r];
        flip_acc[r] = o->flip_acc[r];
        replica_at[r] = o->replica_at[r];
    }
    for (int32_t r = 0; r + 1 < o->R; r++) {
        swap_att[r] = o->swap_att[r];
        swap_acc[r] = o->swap_acc[r];
    }
}
