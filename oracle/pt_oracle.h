/*
 * pt_oracle.h -- plain CPU oracle for the parallel-tempering quantum Monte Carlo
 * (PT-QMC) hot path of Karimi, Dickson & Hamze, "High-Performance Physics
 * Simulations Using Multi-Core CPUs and GPGPUs in a Volunteer Computing Context".
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, loads or calls
 * this code. Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may use it. It shares no code with the CUDA path.
 *
 * What it computes (each function cites the passage it follows):
 *   - Parallel Tempering over R chains (replicas), each chain a Suzuki-Trotter
 *     stack of P coupled copies of an N-spin Ising problem (Sec. 2, Sec. 6 / Table 1).
 *   - Metropolis sweeps in a fixed site order, each site updating its even copies
 *     and then its odd copies (the "two groups of independent regions", Sec. 5).
 *   - Neighbouring-pair swaps with alternating pairing (Sec. 2).
 *   - Per-chain counter-based random numbers (Sec. 3 gives each chain its own
 *     stream; here Philox4x32-10 of Salmon et al., SC'11).
 *   - Integer energies and int64 statistics (Sec. 5 accumulates in high precision).
 *
 * Parity: every function is pinned by CPU tests (brute-force enumeration,
 * transfer matrix, exact diagonalisation, closed forms, curand's host Philox,
 * libm exp). None is "parity unpinned".
 */
#ifndef PT_ORACLE_H
#define PT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc orc;

/* Philox4x32-10 block: out = philox(ctr, key). */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* exp(x) for x in (-23, 0], Cody-Waite reduction + degree-13 Taylor/Horner. */
double orc_det_exp(double x);
void orc_det_exp_array(const double* x, double* y, int64_t n);

/* Returns NULL on invalid input (message in orc_error()). flip_thr / swap_coef may be
 * NULL (then built from the ladder in FP64). */
orc* orc_create(int32_t n, int32_t n_edges, const int32_t* ei, const int32_t* ej,
                const int32_t* J, const int32_t* h, int32_t P, int32_t R,
                const double* T, const double* gamma, const uint32_t* flip_thr,
                const double* swap_coef, uint64_t seed);
const char* orc_error(void);
void orc_destroy(orc* o);
void orc_set_threads(orc* o, int32_t threads);

int32_t orc_lmax(const orc* o);
void orc_flip_table(const orc* o, uint32_t* out);  /* R*(2*Lmax+1)*3 */
void orc_swap_coef(const orc* o, double* out);     /* 2*(R-1): a_0..a_{R-2}, c_0..c_{R-2} */

void orc_sweep(orc* o, int64_t n);
void orc_swap(orc* o);
void orc_run(orc* o, int64_t n_sweeps, int32_t sweeps_per_swap);

/* state in rung order: out[(r*N + i)*P + k] = spin of copy k of site i in the chain at rung r */
void orc_read_state(const orc* o, int8_t* out);
/* state in replica order (replica = chain identity, fixed at creation) */
void orc_read_replica_state(const orc* o, int8_t* out);
/* writes rung-ordered state; recomputes E and M of every chain from scratch */
int orc_write_state(orc* o, const int8_t* in);

/* observables; arrays sized R (per rung) or R-1 (per pair) */
void orc_read_obs(const orc* o, int64_t* tq, int64_t* E, int64_t* M, int64_t* n_meas,
                  int64_t* sum_E, int64_t* sum_E2, int64_t* sum_M, int64_t* sum_M2,
                  int64_t* flip_acc, int64_t* swap_att, int64_t* swap_acc,
                  int32_t* replica_at);

#ifdef __cplusplus
}
#endif
#endif
