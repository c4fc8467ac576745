/*
 * pt.h -- C ABI of the GB300 parallel-tempering quantum Monte Carlo (PT-QMC) library.
 *
 * The method is the data-parallel core of Karimi, Dickson & Hamze, "High-Performance
 * Physics Simulations Using Multi-Core CPUs and GPGPUs in a Volunteer Computing
 * Context": Parallel Tempering over R chains (Sec. 2), each chain a Suzuki-Trotter stack
 * of P coupled copies of an N-spin Ising problem (Sec. 6, Table 1), swept with the
 * Metropolis rule in two groups of independent regions (Sec. 5), and neighbouring
 * chains swapped in disjoint pairs (Sec. 2). Every step runs in sm_103a CUDA kernels.
 *
 * Conventions for every entry point:
 *   - Return 0 (PT_OK) or a negative PT_E* code. Errors are sticky per context: once a
 *     call on a context fails with PT_ECUDA or PT_ETIMEDOUT, later calls return the same
 *     code. pt_last_error() gives a one-line message.
 *   - Inputs are copied at create; the caller keeps ownership of every pointer passed.
 *   - Outputs go into caller-allocated HOST buffers; the calls that fill them synchronise
 *     the context's stream.
 *   - pt_sweep / pt_swap / pt_run only enqueue work on the context's stream (asynchronous).
 *   - Spin states cross the boundary as int8 +1/-1 in rung order:
 *       state[(r*N + i)*P + k] = copy k of site i of the chain currently on rung r.
 *   - The library needs a CUDA device (sm_103a). There is no CPU fallback: without one,
 *     pt_create fails with PT_ENODEV.
 *
 * The model (Sec. 6's coupled classical copies of a quantum Ising problem):
 *   E(s) = sum_edges J_ij s_i s_j + sum_i h_i s_i, integer;
 *   rung r: beta = 1/T_r, a = beta*Gamma_r/P, K_r = -1/2 ln tanh(a);
 *   a chain X = s[i][k] (k periodic mod P) on rung r samples exp(-S_r(X)) with
 *   S_r = (beta/P) sum_k E(s^k) - K_r M(X),  M(X) = sum_k sum_i s_i^k s_i^{k+1}.
 */
#ifndef PT_H
#define PT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PT_OK 0
#define PT_EINVAL -1     /* invalid argument (message in pt_last_error) */
#define PT_ENOMEM -2     /* device or host allocation failed */
#define PT_ECUDA -3      /* a CUDA call failed (sticky) */
#define PT_EOVERFLOW -4  /* a counter or int64 accumulator could overflow */
#define PT_ETIMEDOUT -5  /* a device-side wait gave up (sticky) */
#define PT_EBUSY -6      /* no free slot or device memory for a request */
#define PT_ENODEV -7     /* no usable CUDA device */

typedef struct pt_ctx pt_ctx;

/* One Ising instance. Edges (ei[b], ej[b]) are distinct unordered pairs of distinct
 * sites in [0, n) with J[b] != 0; |h_i| + sum_j |J_ij| <= 127 for every site; n <= 65535. */
typedef struct {
    int32_t n;
    int32_t n_edges;
    const int32_t* ei;
    const int32_t* ej;
    const int32_t* J;
    const int32_t* h;
} pt_instance;

/* One rung of the ladder: temperature T > 0 and transverse field gamma > 0 (gamma = 0 for
 * classical parallel tempering, P = 1). */
typedef struct {
    double T;
    double gamma;
} pt_rung;

/* Optional settings (zero-initialised = defaults). */
typedef struct {
    int32_t threads_per_block;  /* 0 = choose automatically; else a multiple of 32 <= 1024 */
    int32_t wait_timeout_ms;    /* limit of every device-side wait; 0 = 5000 ms */
    int32_t swap_mode;          /* 0 = auto, 1 = swaps inside one cooperative launch,
                                   2 = one launch per sweep interval + a swap launch */
    int32_t test_withhold_rung; /* test hook, 0 = off: if r+1, the chain on rung r never
                                   publishes its swap mailbox, so its partner's wait runs out
                                   and the call fails with PT_ETIMEDOUT (no fault, no hang) */
    int32_t kernel_path;        /* 0 = auto, 1 = byte-wise, 2 = packed with inline random
                                   words, 3 = packed with random words produced one sweep
                                   ahead by dedicated warps, 4 = packed with one bit per
                                   copy in shared memory (paths 2-6 need P % 8 == 0 and
                                   degree <= 7), 5 = path 3 with each chain split over a
                                   cluster of two CTAs, one half of the Trotter copies each
                                   (needs P % 16 == 0 and all R chains resident at once;
                                   for short ladders that leave SMs idle), 6 = path 5 with
                                   the random words computed inline (no producer warps),
                                   7 = every chain of the problem resident on the CTAs of one
                                   thread-block cluster (cluster_size CTAs, 0 = the fewest
                                   that hold them), each chain swept by a group of
                                   group_threads threads, swap passes decided in shared memory
                                   (needs what paths 2-6 need; for problems too small to fill
                                   the GPU, whose sweeps would otherwise wait on the swap
                                   mailboxes between SMs), 8 = path 3 with every thread
                                   sweeping and the random words made by a second CTA of a
                                   two-CTA cluster per chain, written into the first one's
                                   shared memory one sweep ahead (needs all R clusters
                                   resident at once; for ladders that leave SMs idle),
                                   9 = path 2 (or path 3 with producer_threads > 0) with the
                                   CTAs of all R chains in one thread-block cluster and the
                                   swap mailboxes in every CTA's shared memory, so that a
                                   chain waits for its partner on its own SM (needs what
                                   paths 2-6 need, R <= 16 and threads_per_block <= 384),
                                   10 = classical chains (P = 1) packed several to a CTA,
                                   chain fastest in shared memory, on one thread-block cluster
                                   of about cluster_size CTAs (0 = 16 chains a CTA; at most 16
                                   CTAs) with the swap mailboxes in every CTA's shared memory */
    int32_t producer_threads;   /* paths 3 and 5: threads producing random words (0 = auto);
                                   path 9: 0 = random words inline, else this many producer
                                   threads (a multiple of 32 below threads_per_block) */
    int32_t test_exact_swaps;   /* test hook: 1 = skip the FP32 pre-decision of swaps and always
                                   evaluate the FP64 rule (results are identical either way) */
    int32_t cluster_size;       /* path 10: CTAs of its cluster (see kernel_path);
                                   batched launches: CTAs per thread-block cluster (1..16), or
                                   0 = autotune (pt_batch_create times a short run of each
                                   layout and keeps the fastest, remembered per batch shape --
                                   every request's N, P, R, degree class, levels and sweeps --
                                   for the process; results never depend on it) */
    int32_t no_autotune;        /* 0: when kernel_path and threads_per_block are automatic and
                                   the chains are int8 in shared memory, pt_create times a
                                   short run of each candidate plan (paths 2, 3, 5, 6, 7, 8 and
                                   9, block sizes 128-512, clusters of 1-16 CTAs; for P = 1,
                                   paths 1 and 10), keeps the fastest
                                   and resets the context to its initial state; the choice is
                                   remembered per shape for the process. Results never depend
                                   on it. 1: off. */
    int32_t group_threads;      /* kernel_path 7: threads sweeping one chain (32, 64, ..., 512),
                                   0 = the narrowest that keeps every chain resident */
    int32_t reserved[2];
} pt_options;

/* Statistics (Fig. 4 "gather statistics"; Sec. 5 accumulates in high precision).
 * Per-rung arrays have R entries, per-pair arrays R-1. All caller-allocated. */
typedef struct {
    int64_t t;          /* sweeps done */
    int64_t q;          /* swap passes done */
    int64_t* E;         /* [R] sum_k E(s^k) of the chain on rung r */
    int64_t* M;         /* [R] M(X) of the chain on rung r */
    int64_t* n_meas;    /* [R] sweeps accumulated (one measurement after every sweep) */
    int64_t* sum_E;     /* [R] sum over measurements of E */
    int64_t* sum_E2;    /* [R] ... of E^2 */
    int64_t* sum_M;     /* [R] ... of M */
    int64_t* sum_M2;    /* [R] ... of M^2 */
    int64_t* flip_acc;  /* [R] accepted spin flips while on rung r */
    int64_t* swap_att;  /* [R-1] swap attempts of pair (r, r+1) */
    int64_t* swap_acc;  /* [R-1] accepted swaps of pair (r, r+1) */
    int32_t* replica_at;/* [R] chain (replica id, = its starting rung) now on rung r */
} pt_observables;

/* Layout and schedule facts of a context (for tests and the benchmark). */
typedef struct {
    int32_t n, P, R, lmax, max_degree;
    int32_t n_levels;          /* dependency levels of one sweep (see pt_create) */
    int32_t threads_per_block;
    int32_t cooperative;       /* 1 if swaps run inside one launch */
    int32_t kernel_path;       /* path chosen (see pt_options.kernel_path) */
    int32_t producer_threads;  /* random-word producer threads per CTA (path 3) */
    int64_t device_bytes;      /* device memory held by the context */
    int64_t kernel_launches;   /* kernels this context has launched so far */
    int64_t h2d_bytes;         /* bytes copied host -> device so far */
    int32_t tuned_plans;       /* candidate plans timed by pt_create (0: none, or cached) */
    int32_t reserved;
} pt_info;

/* Create a PT-QMC problem on the current CUDA device (Sec. 2: chains and temperatures
 * are fixed before the run, Sec. 5 / Fig. 6: data moved to the device once).
 *   inst        Ising instance (copied).
 *   P           Trotter copies, even, 2 <= P <= 4096; or P = 1 with gamma = 0 on every rung:
 *               classical parallel tempering over the temperatures (one copy per chain,
 *               no Trotter coupling: K = 0, m = 0, M = N). Classical chains run on the
 *               byte-wise kernel; batched launches and the server need P % 8 == 0.
 *   ladder, R   R >= 1 rungs (copied), 1 <= R <= 65535.
 *   flip_thr    NULL to build the Metropolis table in FP64 on the host, or R*(2*Lmax+1)*3
 *               uint32 thresholds [r][L+Lmax][m/2+1] (accept iff thr == 0xFFFFFFFF or
 *               u < thr) where Lmax = max_i(|h_i| + sum_j |J_ij|).
 *   swap_coef   NULL to build from the ladder, or 2*(R-1) doubles a_0..a_{R-2}, c_0..c_{R-2}
 *               (swap of X on r with Y on r+1 has log-ratio a_r (E_X-E_Y) + c_r (M_X-M_Y)).
 *   seed        64-bit Philox4x32-10 key; every random number is a function of
 *               (seed, counter), independent of the launch layout.
 *   opt         NULL for defaults.
 *   cuda_stream cudaStream_t to use, or NULL for a stream owned by the context.
 * Initial spins come from the key: copy k of site i of chain rho is -1 iff bit 31 of
 * word k%4 of philox((0, i, rho, 2<<28 | k/4), seed) is set.
 * With an automatic plan (see pt_options.no_autotune) pt_create first times a short run of
 * each candidate kernel plan, then returns the context to exactly that initial state.
 * Returns PT_EINVAL, PT_ENOMEM, PT_ECUDA or PT_ENODEV on failure (*out untouched). */
int pt_create(const pt_instance* inst, int32_t P, const pt_rung* ladder, int32_t R,
              const uint32_t* flip_thr, const double* swap_coef, uint64_t seed,
              const pt_options* opt, void* cuda_stream, pt_ctx** out);

/* n >= 0 Metropolis sweeps of every chain (Sec. 2, Sec. 5). Sweep t visits sites in
 * index order; at each site it updates the even copies, then the odd copies. Copy
 * k = p + 2h of site i of chain rho draws word h%4 of philox((t, i, rho, p<<24 | h/4)).
 * Statistics are accumulated after every sweep. Asynchronous. */
int pt_sweep(pt_ctx* ctx, int64_t n);

/* One swap pass q (Sec. 2: neighbouring chains, disjoint pairs): pairs (r, r+1) for
 * r = q%2, q%2+2, ...; accept iff Delta >= 0, or Delta > -23 and u < min(floor(2^32
 * exp(Delta)), 2^32-1) with u = word 0 of philox((q, r, 0, 1<<28)) and exp evaluated by
 * the Cody-Waite/Taylor sequence of IEEE operations. Asynchronous. */
int pt_swap(pt_ctx* ctx);

/* Fig. 4's loop: n_sweeps sweeps with a swap pass after every sweeps_per_swap-th sweep
 * (0 = no swaps, at most 2^30). Bit-identical to the equivalent sequence of pt_sweep /
 * pt_swap calls. */
int pt_run(pt_ctx* ctx, int64_t n_sweeps, int32_t sweeps_per_swap);

/* Copy the state, rung-ordered int8 (+1/-1), into out (bytes >= R*N*P). Synchronises.
 * (Fig. 6's copy of the chains back to the host, here only when the caller asks.) */
int pt_read_state(pt_ctx* ctx, int8_t* out, size_t bytes);

/* Overwrite the state (rung-ordered int8 +1/-1, bytes = R*N*P) and recompute E and M
 * of every chain on the device. Counters and statistics are kept. Synchronises. */
int pt_write_state(pt_ctx* ctx, const int8_t* in, size_t bytes);

/* Fill the caller's arrays with the current statistics. Synchronises. */
int pt_read_observables(pt_ctx* ctx, pt_observables* out);

/* Checkpoint restore: put a context back into the state that pt_read_state (into `in`) and
 * pt_read_observables (into `snap`) captured from a context of the same problem and seed.
 * The chains return to their rungs (snap->replica_at; the random streams belong to the
 * chains), the statistics and the sweep / pass counters (snap->t, snap->q) are restored,
 * and E and M are recomputed from the spins. The following sweeps and swaps are then
 * bit-identical to those of the context the snapshot came from. Every array of `snap`
 * except E and M is required. PT_EINVAL for a bad buffer or permutation, PT_EOVERFLOW
 * for counters out of range. Synchronises. */
int pt_restore(pt_ctx* ctx, const int8_t* in, size_t bytes, const pt_observables* snap);

/* Copy the tables the context uses: thr (R*(2*Lmax+1)*3) and coef (2*(R-1)); either
 * pointer may be NULL. Host data, no synchronisation. */
int pt_read_tables(const pt_ctx* ctx, uint32_t* thr, size_t thr_count, double* coef,
                   size_t coef_count);

int pt_get_info(const pt_ctx* ctx, pt_info* out);

/* Host-only helpers (no device needed): the exact setup data pt_create uses.
 * pt_make_tables fills thr[R*(2*lmax+1)*3] and coef[2*(R-1)] from the ladder in FP64
 * (either may be NULL). pt_make_schedule writes the sweep's level schedule: items[2n]
 * ((i<<1)|parity, grouped by level) and level_off[n_levels+1] (room for 2n+1 entries);
 * update (i,1) comes after (i,0), and (i,p) after (j,p) for every neighbour j < i. */
int pt_make_tables(int32_t P, const pt_rung* ladder, int32_t R, int32_t lmax, uint32_t* thr,
                   double* coef);
int pt_make_schedule(const pt_instance* inst, uint32_t* items, int32_t* level_off,
                     int32_t* n_levels);
/* The same dependencies and the same number of levels, with the updates spread over the
 * levels for a kernel that takes items_per_round items of a level at a time: each update
 * lies between the earliest level its predecessors allow and the latest its successors
 * allow, and levels are filled in whole rounds, most urgent updates first. Any such
 * assignment replays the sequential order exactly (Sec. 5's regions, swept in dependency
 * order), so results do not depend on it. items_per_round = 0 gives pt_make_schedule's
 * as-early-as-possible levels. pt_create uses this with its kernel's round size. */
int pt_make_schedule_balanced(const pt_instance* inst, int32_t items_per_round, uint32_t* items,
                              int32_t* level_off, int32_t* n_levels);

/* ---- Many independent problems in one launch ----------------------------------------
 * The paper solves many problem instances (Sec. 1) one application run at a time; here a
 * batch of independent requests shares one persistent launch. A thread-block cluster takes
 * one request at a time (largest first) and runs all of its sweeps and swap passes; each
 * request gets exactly the bits pt_create + pt_run would give it alone. Batched requests
 * need P % 8 == 0, degree <= 7, R <= 1024 and one chain's spins plus its instance data
 * within one CTA's shared memory. */
typedef struct {
    pt_instance inst;            /* copied at pt_batch_create */
    int32_t P;                   /* Trotter copies */
    const pt_rung* ladder;       /* R rungs (copied) */
    int32_t R;
    uint64_t seed;               /* Philox key of this request */
    int64_t n_sweeps;            /* sweeps per pt_batch_run (<= 2^30) */
    int32_t sweeps_per_swap;     /* a swap pass after every sweeps_per_swap-th sweep (0 = none) */
} pt_request;

typedef struct pt_batch pt_batch;

typedef struct {
    int32_t count;              /* requests */
    int32_t cluster;            /* CTAs per cluster */
    int32_t n_clusters;         /* clusters in the persistent grid */
    int32_t threads_per_block;
    int64_t smem_bytes;         /* dynamic shared memory per CTA */
    int64_t device_bytes;
    int64_t kernel_launches;
    int64_t h2d_bytes;
    int32_t tuned_layouts;      /* layouts the autotuner timed (0 = layout given, or reused:
                                   the choice is remembered per batch shape for the process) */
    int32_t group_widen;        /* threads per chain: doublings (> 0) or halvings (< 0) of the
                                   width that gives about one update unit per thread in an
                                   average level; fixed layouts use -4 (narrowest that fits) */
    int32_t graph;              /* 1 = runs replay a captured CUDA graph */
    int32_t reserved;
} pt_batch_info;

/* Copy and prepare every request (tables, schedules, initial spins as in pt_create). */
int pt_batch_create(const pt_request* reqs, int32_t count, const pt_options* opt, void* cuda_stream,
                    pt_batch** out);
/* One persistent launch running every request's n_sweeps (with its swap passes). Async.
 * The first call captures the launch into a CUDA graph and later calls replay it. On a
 * stream that is itself being captured the launch is recorded into the caller's graph;
 * every replay of that graph is one more run (the sweep and pass counters live on the
 * device and advance with it), but only runs made through pt_batch_run are checked
 * against the counter limits (PT_EOVERFLOW). */
int pt_batch_run(pt_batch* b);
int pt_batch_read_state(pt_batch* b, int32_t index, int8_t* out, size_t bytes);   /* syncs */
int pt_batch_read_observables(pt_batch* b, int32_t index, pt_observables* out);  /* syncs */
int pt_batch_get_info(const pt_batch* b, pt_batch_info* out);
int pt_batch_sync(pt_batch* b);
int pt_batch_destroy(pt_batch* b);
const char* pt_batch_last_error(const pt_batch* b);

/* ---- Serving: continuous batching ----------------------------------------------------
 * A request (pt_request) is copied and queued by pt_server_submit. pt_server_step never
 * blocks: it reports the requests that have finished, then admits queued requests in
 * arrival order while a slot (max_active) and room in the device arena are free, and while
 * the chains in flight (one CTA each, a batched launch's CTAs until it ends) plus the
 * request's own R stay within the device's SM count, so that every admitted request is
 * resident at once (a request larger than that is admitted when nothing else runs). An
 * admitted request's state and counters live in the arena; all of its sweeps are launched
 * at once on the least-loaded stream of a pool (one CTA per chain), so requests that arrive
 * while others run overlap with them on the device. When a backlog of 8 or more requests waits, they
 * start together in one persistent batched launch (as pt_batch_run) instead; each of them
 * is reported finished as soon as its own chains are written back, not when the whole
 * launch ends. In stepped
 * mode each step instead advances every admitted request by quantum_sweeps sweeps in one
 * launch and waits for it. Results are read with pt_server_read_result and the arena room
 * is returned by pt_server_release. Each result equals pt_create + pt_run of that request
 * alone. Same request limits as pt_batch. */
typedef struct pt_server pt_server;

typedef struct {
    int64_t arena_bytes;    /* device memory for admitted requests (0 = half of the free memory) */
    int32_t max_active;     /* requests on the device at once (0 = 512) */
    int32_t quantum_sweeps; /* sweeps per request per step (0 = 100) */
    int32_t cluster_size;   /* CTAs per cluster of batched launches (1..16), or 0: 2 in
                               stepped mode; a backlog launch in streamed mode takes the
                               largest of 8, 4 and 2 at which every request of the backlog
                               gets a cluster of its own at once (else 2) */
    int32_t reserved[3];    /* reserved[1] = 1: stepped mode (a quantum of sweeps per launch);
                               reserved[0] = 1: stepped mode with chains packed on clusters only */
} pt_server_options;

typedef struct {
    int32_t active;         /* requests on the device */
    int32_t queued;         /* requests waiting for a slot or arena room */
    int64_t arena_bytes;
    int64_t arena_used;
    int64_t steps;
    int64_t kernel_launches;
    int64_t wide_steps;     /* steps that ran one CTA per chain (the rest packed chains) */
    int64_t group_launches; /* streamed mode: backlogs started together in one batched launch */
} pt_server_info;

int pt_server_create(const pt_server_options* opt, void* cuda_stream, pt_server** out);
/* PT_EINVAL for an invalid request, PT_ENOMEM if it could never fit the arena. */
int pt_server_submit(pt_server* s, const pt_request* req, int64_t* id);
/* Admit, run one step, and write up to max_done finished ids (the rest come next call). */
int pt_server_step(pt_server* s, int64_t* done_ids, int32_t max_done, int32_t* n_done);
/* For a finished request: state (rung order, may be NULL) and statistics (may be NULL). */
int pt_server_read_result(pt_server* s, int64_t id, int8_t* state, size_t bytes, pt_observables* obs);
/* Forget a queued or finished request (PT_EBUSY while it runs). */
int pt_server_release(pt_server* s, int64_t id);
int pt_server_get_info(const pt_server* s, pt_server_info* out);
int pt_server_destroy(pt_server* s);
const char* pt_server_last_error(const pt_server* s);

/* ---- Running on caller-owned device memory, without allocating ----------------------
 * The paper has no counterpart to this entry point. It is for callers that cannot allocate
 * device memory, neither themselves nor through this library: latency-critical loops that
 * must not enter the allocator (cudaMalloc / cudaFree can synchronise the device and take
 * locks other threads hold), and embedding runtimes or frameworks that hand out device
 * memory only from their own accounted pool, or fix the process's device memory at start-up.
 * pt_create allocates; such a caller instead builds the problem with pt_make_tables and
 * pt_make_schedule, copies it into device memory it owns, and calls pt_run_noalloc, which
 * allocates nothing (no cudaMalloc, no cudaFree, no library routine that allocates).
 *
 * The only scratch memory the kernel needs, the swap mailboxes, is one fixed array of
 * PT_NOALLOC_MAILBOXES 16-byte entries (256 KiB) that every GPU loading this library holds
 * until the process exits. All calls share it and it keeps the last call's contents; each
 * launch clears the entries it uses. Calls that overlap on the GPU (other streams, other
 * threads) race on it: serialise them. The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress, with that device current) and caches it for the
 * process; make that first call before any stream capture. cuda_stream must belong to the
 * current device, and a device reset (cudaDeviceReset) makes the cached address stale: do
 * not call this on a device after its reset. */
#define PT_NOALLOC_MAILBOXES 16384  /* swap passes x rungs one launch can hold */

typedef struct {
    int32_t n, P, R;            /* sites, Trotter copies (even, or 1: classical), rungs (R <= PT_NOALLOC_MAILBOXES) */
    int32_t lmax;               /* max_i(|h_i| + sum_j |J_ij|) <= 127 */
    int32_t row_stride;         /* entries per row of nbr: 4, 8 or 32, >= the largest degree */
    int32_t n_levels;           /* level count returned by pt_make_schedule */
    const uint32_t* nbr;        /* [n][row_stride]: (j << 8) | (uint8_t)J_ij; unused entries (i << 8) */
    const int8_t* h;            /* [n] */
    const uint32_t* items;      /* [2n] from pt_make_schedule */
    const int32_t* level_off;   /* [n_levels + 1] from pt_make_schedule */
    const uint32_t* thr;        /* [R][(2*lmax+1)*3] from pt_make_tables */
    const double* coef;         /* [2(R-1)] from pt_make_tables (read only when R > 1) */
    int8_t* spins;              /* in/out [R][n*P rounded up to 16] by replica, copy index fastest;
                                   16-byte aligned */
    int64_t* E;                 /* in/out [R] by replica: sum_k E(s^k) of its spins */
    int64_t* M;                 /* in/out [R] by replica: M(X) of its spins */
    int32_t* rung_of_slot;      /* in/out [R] rung of each replica */
    int32_t* slot_of_rung;      /* in/out [R] replica on each rung (inverse permutation) */
    uint64_t* stats;            /* in/out [R][6] per rung: count, sum E, sum E^2, sum M, sum M^2,
                                   accepted flips (added to) */
    uint64_t* swap_stats;       /* in/out [R][2] per pair r: attempts, accepts (added to) */
    int32_t* status;            /* in/out: 0, or PT_ETIMEDOUT if a swap wait gave up */
    uint64_t seed;              /* Philox key */
    int64_t t0;                 /* sweeps done so far (the caller advances it by n_sweeps) */
    int64_t q0;                 /* swap passes done so far (advance by n_sweeps/sweeps_per_swap) */
} pt_device_problem;

/* Same arithmetic and bits as pt_run(n_sweeps, sweeps_per_swap) on a context in the same
 * state, launched on cuda_stream (asynchronous). All pointers are device pointers owned by
 * the caller. A call whose swap passes x R exceed PT_NOALLOC_MAILBOXES runs as several
 * launches of whole swap intervals, each clearing the mailboxes it uses first. Returns
 * PT_EINVAL (message in pt_noalloc_last_error) for R beyond the fixed mailbox array, a chain
 * beyond the shared memory of one CTA, or sweeps_per_swap > 2^30; PT_EOVERFLOW for counters
 * past 2^32 - 1; PT_ECUDA if a launch fails. */
int pt_run_noalloc(const pt_device_problem* prob, int64_t n_sweeps, int32_t sweeps_per_swap,
                   int32_t wait_timeout_ms, void* cuda_stream);
const char* pt_noalloc_last_error(void);

/* Wait for all queued work of the context. */
int pt_sync(pt_ctx* ctx);

/* Free the context (synchronises first). NULL is a no-op. (Fig. 6: the device's copy of
 * the problem is released once the run ends.) */
int pt_destroy(pt_ctx* ctx);

/* One-line message of the last error on ctx (or of the last failed create if ctx is NULL).
 * The paper's kernel launches can fail and are retried by the host (Fig. 7); here a failure
 * is reported once, with its reason, and stays (sticky) on the context. */
const char* pt_last_error(const pt_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
