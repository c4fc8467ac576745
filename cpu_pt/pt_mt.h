/*
 * pt_mt.h -- the paper's multi-threaded CPU Parallel Tempering (Sec. 4, Figs. 4-5) for the
 * PT-QMC problem of this repository, as a CPU comparison baseline.
 *
 * Persistent worker threads sweep the chains of one swap interval from a work pool ordered
 * hardest first (Sec. 4: chains with more flips take longer, so they are handed out first,
 * first come first served), meet at a barrier, then run the swap pass in parallel over the
 * disjoint pairs, and meet again. It computes the same Markov chain as the GPU library and
 * the CPU oracle: the same Philox4x32-10 counters, site and copy order, threshold tables
 * and swap rule, so its state and statistics are identical for any thread count.
 *
 * Not part of the GPU library (which never calls it) and not the oracle (which stays the
 * plain reference the tests trust); the benchmark times it beside the oracle.
 */
#ifndef PT_MT_H
#define PT_MT_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cpt cpt;

/* thr: R*(2*lmax+1)*3 Metropolis thresholds [r][L+lmax][m/2+1] with lmax = max_i(|h_i| +
 * sum_j |J_ij|); coef: 2*(R-1) swap coefficients (a_0.., c_0..). Both are copied. P = 1
 * (classical, no Trotter coupling) or even P >= 2. Returns NULL on invalid input. */
cpt* cpt_create(int32_t n, int32_t n_edges, const int32_t* ei, const int32_t* ej, const int32_t* J,
                const int32_t* h, int32_t P, int32_t R, const uint32_t* thr, const double* coef, uint64_t seed,
                int32_t threads);
/* n_sweeps sweeps with a swap pass after every sweeps_per_swap-th (0 = none). */
void cpt_run(cpt* c, int64_t n_sweeps, int32_t sweeps_per_swap);
/* state in rung order, copy index fastest: out[(r*n + i)*P + k] */
void cpt_read_state(const cpt* c, int8_t* out);
/* tq[0] = sweeps, tq[1] = swap passes; per rung: E, M, n_meas, sums of E, E^2, M, M^2, flips;
 * per pair: swap attempts and accepts; replica_at[r] = chain on rung r. */
void cpt_read_obs(const cpt* c, int64_t* tq, int64_t* E, int64_t* M, int64_t* n_meas, int64_t* sum_E,
                  int64_t* sum_E2, int64_t* sum_M, int64_t* sum_M2, int64_t* flip_acc, int64_t* swap_att,
                  int64_t* swap_acc, int32_t* replica_at);
void cpt_destroy(cpt* c);
int32_t cpt_lmax(const cpt* c);

#ifdef __cplusplus
}
#endif
#endif
