// pt_internal.h -- structures shared by the host side (pt_host.cu) and the kernels
// (pt_kernels.cu) of the PT-QMC library. Not part of the public ABI (include/pt.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "pt.h"

namespace ptq {

// Stream tags in the top nibble of Philox counter word 3.
constexpr uint32_t kTagFlip = 0u;
constexpr uint32_t kTagSwap = 1u;
constexpr uint32_t kTagInit = 2u;

// One (pass, rung) mailbox of the in-kernel swap: two self-validating 64-bit words that the
// chain on rung r writes after the sweep preceding pass q,
//   a = E << 24 | tag,   b = (uint32)M << 32 | tag,   tag = q mod (2^24 - 1) + 1 (never 0),
// so a partner that sees the pass's tag in both words has a consistent (E, M) from one round
// trip of two relaxed loads. |E| < 2^39 and |M| < 2^31 are checked at create; the host
// clears the mailboxes before a tag value could repeat.
struct alignas(16) Mailbox {
    unsigned long long a;
    unsigned long long b;
};
constexpr long long kTagPeriod = 16777215ll;
constexpr int kClusterMailPasses = 4;  // path 9: swap passes whose mailboxes each CTA holds at once

// Per-rung statistics, in this order, as unsigned 64-bit two's-complement sums.
enum { kAccN = 0, kAccE, kAccE2, kAccM, kAccM2, kAccFlip, kAccCount };

// Device view of one PT problem. All pointers are device pointers.
struct DevProblem {
    // instance (read-only)
    const uint32_t* nbr;       // [N][dmax]: (j << 8) | (uint8_t)J; padding has J = 0, j = i
    const int8_t* h;           // [N]
    const uint32_t* items;     // [2N] (i << 1) | parity, grouped by dependency level
    const int32_t* level_off;  // [n_levels + 1]
    const uint32_t* desc;      // [N][8 or 12] packed-path site descriptors
    const uint32_t* thr;       // [R][nL*3] Metropolis thresholds
    const double* coef;        // [2(R-1)] a_r then c_r
    // state
    int8_t* spins;             // [R slots][slot_stride] int8, copy index fastest
    long long* E;              // [slot]
    long long* M;              // [slot]
    int32_t* rung_of_slot;     // [slot]
    int32_t* slot_of_rung;     // [rung]
    unsigned long long* acc;   // [rung][kAccCount]
    unsigned long long* swap_stats;  // [pair][2] attempts, accepts
    Mailbox* mbox;             // [max_passes][R]
    int* status;               // 0 or a PT_E* code set by a kernel
    int N, P, R, Lmax, nL3, n_levels;
    int dmax;                  // row stride of `nbr` (4, 8 or 32)
    int slot_stride;           // bytes between slots in `spins` (multiple of 16)
    int withhold_rung;         // test hook: rung whose chain never publishes (-1 = off)
    int acc_in_smem;           // 1: per-rung statistics gathered in shared memory per launch
    int tables_in_smem;        // 1: every rung's threshold row resident in shared memory
    int exact_swaps;           // test hook: 1 = always take the FP64 swap decision
    uint32_t key0, key1;
};

// Sweep kernel variants: byte-wise (any shape), packed with Philox inline, packed with the
// random words produced one sweep ahead by dedicated warps, bit-packed, and the produced-words
// kernel with each chain split over a cluster of two CTAs.
// Path 7 runs the batched kernel on the one problem: all chains packed on the CTAs of one
// cluster (thread groups per chain), resident in shared memory, swaps in shared memory.
enum {
    kPathGeneric = 1,
    kPathPackedInline = 2,
    kPathPacked = 3,
    kPathBits = 4,
    kPathSplit = 5,
    kPathSplitInline = 6,
    kPathPackedChains = 7,
    kPathPeer = 8,  // path 3's sweep on every thread of rank 0 of a two-CTA cluster; rank 1 makes its random words
    kPathCluster = 9,   // paths 2 / 3 with every chain's CTA in one cluster; swap mailboxes in shared memory
    kPathClassical = 10  // P = 1: chains packed several to a CTA, one cluster, swap mailboxes in shared memory
};

struct LaunchPlan {
    int path;            // kPath*
    int threads;         // threads per CTA
    int n_consumer;      // threads running the levels (the rest produce random words)
    int dclass;          // padded neighbour slots the kernel is built for
    size_t smem_bytes;   // dynamic shared memory per CTA
    int cluster = 1;     // path 7: CTAs in the one cluster
    int group_threads = 0;  // path 7: threads sweeping one chain
    int thr_resident = 0;   // path 7: every rung's threshold row in shared memory
    int chains_per_cta = 1; // path 10: chains packed on one CTA (cluster = ceil(R / chains_per_cta))
};

// Sizes of the dynamic shared-memory carve-up of the sweep kernel for a path.
// cluster_pre: path 9 with producer warps (its plan's n_consumer < threads)
size_t sweep_smem_bytes(const DevProblem& p, int path, int dclass, bool cluster_pre = false);
// path 10: the shared memory of a CTA holding `chains` classical chains
size_t classical_smem_bytes(const DevProblem& p, int chains);

// One request of a batched launch (device view). Every chain of the request is swept by
// one CTA of the thread-block cluster that takes the request; the cluster's CTAs split the
// chains and exchange (E, M) through distributed shared memory for the swap passes.
struct BatchInstance {
    const uint32_t* sdesc;     // [N][DW] packed-path site descriptors
    const uint32_t* items;     // [2N] schedule, grouped by level
    const int32_t* level_off;  // [n_levels + 1]
    const uint32_t* thr;       // [R][nL3]
    const double* coef;        // [2(R-1)] (at least 2 entries)
    int8_t* spins;             // [R][slot_stride]
    long long* E;              // [R] by replica
    long long* M;
    int32_t* rung_of_slot;     // [R]
    int32_t* slot_of_rung;     // [R]
    unsigned long long* acc;   // [R][kAccCount] by rung
    unsigned long long* swap_stats;  // [R][2] by pair
    int N, P, R, Lmax, nL3, n_levels, dc, slot_stride;
    int group_threads;         // threads sweeping one chain (a divisor of the CTA size)
    int resident;              // 1: a CTA keeps all its chains in shared memory for the run
    int thr_resident;          // 1: every rung's threshold row stays in shared memory for the run
    uint32_t key0, key1;
    long long t0, q0;          // counters before this run
    int n_sweeps, sweeps_per_swap;
};

struct BatchParams {
    BatchInstance* inst;        // [count]; t0 / q0 of a finished problem advance in place
    const int32_t* order;       // [count] request indices, most work first
    int count;
    int* next_job;              // work counter, zero at launch
    int* status;
    int* done = nullptr;        // [count] or null: done[k] = done_token once problem k is written back
    int done_token = 1;         // nonzero, different per launch, so stale flags never match
    int single = 0;             // 1: one cluster runs `one` (passed by value) once; inst, order,
                                // next_job and done are unused and the counters stay on the host
    BatchInstance one;
};

// Kernel launchers (pt_kernels.cu). Each returns a cudaError_t from the launch.
cudaError_t launch_init(const DevProblem& p, cudaStream_t s);
cudaError_t launch_energy(const DevProblem& p, cudaStream_t s);
cudaError_t launch_sweeps(const DevProblem& p, const LaunchPlan& plan, long long t0,
                          long long q0, int n_sweeps, int sweeps_per_swap, long long timeout_ns,
                          bool cooperative, cudaStream_t s);
cudaError_t launch_swap(const DevProblem& p, long long q, cudaStream_t s);
cudaError_t launch_gather_state(const DevProblem& p, int8_t* out, cudaStream_t s);
cudaError_t launch_scatter_state(const DevProblem& p, const int8_t* in, cudaStream_t s);
cudaError_t sweep_kernel_occupancy(const DevProblem& p, const LaunchPlan& plan, int* blocks_per_sm);
// Chains that can be resident at once for a plan (CTAs, or clusters of the split kernel).
cudaError_t sweep_resident_chains(const DevProblem& p, const LaunchPlan& plan, long long* chains);
cudaError_t prepare_sweep_kernel(const LaunchPlan& plan);

// One problem of a multi-problem cooperative launch (one CTA per chain of every problem).
struct MultiProblem {
    DevProblem p;
    int dc;                    // packed neighbour slots: 4 or 8
    int n_sweeps, sweeps_per_swap;
    long long t0, q0, timeout_ns;
};
size_t multi_smem_bytes(const DevProblem& p, int dc);
cudaError_t multi_prepare(int threads, size_t smem, int* blocks_per_sm);
cudaError_t launch_multi(const MultiProblem* probs, const int2* map, int n_blocks, int threads, size_t smem,
                         cudaStream_t s);

// Host-side preparation shared by single and batched problems (pt_host.cu).
void build_tables(int R, int P, int Lmax, const pt_rung* ladder, std::vector<uint32_t>& thr,
                  std::vector<double>& coef);
// per_round > 0: levels balanced for a kernel that takes per_round items of a level at a
// time (same level count, same dependencies); 0: every update as early as possible.
// row_words > 0: each level's items ordered for a packed kernel whose rows are row_words
// 4-byte words (see level_schedule); 0: in site order.
void level_schedule(int N, const std::vector<std::vector<int>>& adj, std::vector<uint32_t>& items,
                    std::vector<int32_t>& level_off, int per_round = 0, int row_words = 0);
void build_site_desc(int N, int row_bytes, int dclass, const std::vector<std::vector<int>>& adj,
                     const std::vector<std::vector<int>>& adjJ, const int32_t* h, std::vector<uint32_t>& desc);

// Host-side preparation of one batched request (pt_batch.cu).
struct Prepared {
    int N, P, R, Lmax, dc, n_levels, slot_stride;
    std::vector<uint32_t> sdesc, items, thr;
    std::vector<int32_t> level_off;
    std::vector<double> coef;
    size_t off_sdesc, off_items, off_loff, off_thr, off_coef, off_spins, off_E, off_M, off_rung, off_slot, off_acc,
        off_sw, off_mbox = 0, off_inst = 0, off_map = 0, off_status = 0;
    long long sweep_limit;
};
// per_round > 0: the level schedule is balanced for a kernel taking per_round items at a time.
int prepare_request(const pt_request& r, Prepared& pr, char* why, size_t why_len, int per_round = 0);
size_t request_block_layout(Prepared& p, size_t mailbox_entries = 0);
void fill_instance(BatchInstance& I, const Prepared& p, unsigned char* base, const pt_request& r);
// Group width of a fixed layout: narrowest that fits (one warp per chain where possible),
// which the autotuner picks on the batched size mix.
constexpr int kGroupWidenDefault = -4;
void choose_groups(BatchInstance& I, int cluster, int threads, size_t smem_cap, int widen = kGroupWidenDefault);

// Batched launchers (pt_batch.cu).
size_t batch_smem_bytes(const BatchInstance& I, int cluster, int threads);
cudaError_t launch_batch(const BatchParams& bp, int cluster, int n_clusters, int threads, size_t smem,
                         cudaStream_t s);
cudaError_t batch_max_clusters(int cluster, int threads, size_t smem, int* n_clusters);
cudaError_t launch_batch_init(const BatchInstance* inst, const int2* map, int n_chains, cudaStream_t s);
// One problem on one cluster of `cluster` CTAs (path 7); I carries t0, q0, n_sweeps, sweeps_per_swap.
cudaError_t launch_batch_single(const BatchInstance& I, int cluster, int threads, size_t smem, cudaStream_t s);
// The largest shared-memory need of the batched kernel: the device's opt-in maximum less
// the kernel's static shared memory.
size_t batch_smem_cap();

}  // namespace ptq
