// pt_kernels.cu -- sm_103a kernels of the PT-QMC hot path.
//
// Sweep (Sec. 2 Metropolis sweeps; Sec. 5 "two groups of independent regions", swept one
// after the other with a barrier between them): one CTA owns one chain (replica) for the
// whole launch, with its spins, the instance and the chain's current Metropolis table in
// shared memory. The sequential order (sites in index order, even copies then odd copies)
// is replayed exactly by a static level schedule computed on the host: update (i, p)
// (site i, copy parity p, all P/2 copies of that parity) must follow (i, 0) when p = 1
// and (j, p) for every neighbour j < i; updates in one level touch disjoint spins, so
// running a level in parallel and putting a CTA barrier between levels reproduces the
// sequential result bit for bit. Random numbers are a pure function of the counter
// (Philox4x32-10), so the thread layout does not change any result.
//
// Swap (Sec. 2: neighbouring chains, disjoint pairs): inside a cooperative launch each
// chain publishes (E, M) for pass q in a per-(pass, rung) mailbox and waits, with a time
// limit, only for its pair partner; both partners evaluate the same decision.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pt.h"
#include "pt_device.cuh"
#include "pt_internal.h"

namespace ptq {

namespace cg = cooperative_groups;

// ------------------------------------------------------------------------- smem layouts

// Threshold rows and per-rung statistics in shared memory (when they fit).
__host__ __device__ inline size_t thr_bytes(const DevProblem& p) {
    return up16((size_t)(p.tables_in_smem ? p.R : 1) * p.nL3 * 4);
}
__host__ __device__ inline size_t acc_bytes(const DevProblem& p) {
    return p.acc_in_smem ? (size_t)p.R * kAccCount * 8 : 0;
}

// Byte-wise path (any even P, any degree up to 32).
struct GenericLayout {
    size_t spins, nbr, h, items, loff, thr, acc, red, ctl, total;
    __host__ __device__ explicit GenericLayout(const DevProblem& p) {
        const int N = p.N, P = p.P;
        size_t o = 0;
        spins = o; o += up16((size_t)N * P);
        nbr = o;   o += up16((size_t)N * p.dmax * 4);
        h = o;     o += up16((size_t)N);
        items = o; o += up16((size_t)2 * N * 4);
        loff = o;  o += up16((size_t)(p.n_levels + 1) * 4);
        thr = o;   o += thr_bytes(p);
        acc = o;   o += acc_bytes(p);
        red = o;   o += 32 * 3 * 8;
        ctl = o;   o += 16;
        total = o;
    }
};

// Packed path (P % 8 == 0, degree + 1 <= 8): spins, one row of +1 copies (the field's h
// slot points at it), per-site descriptors, the schedule, level offsets, the threshold
// row(s), statistics, reduction scratch, control words and, when
// the random words are produced ahead, two buffers of one sweep's words each.
// With bits, the chain is P/8 bytes per site, the constant row holds +1 copies as zero bits,
// and two 256-entry tables spread parity bits into +1/-1 bytes.
// With cswap (path 9), each CTA also holds the swap mailboxes of the cluster's chains: four
// passes of R (E, M) words each (see eos_decide_cluster).
struct FastLayout {
    size_t spins, ones, lut, desc, items, loff, thr, acc, red, ctl, cmb, rbuf, total;
    __host__ __device__ FastLayout(const DevProblem& p, int dc, bool pre, bool bits = false, bool cswap = false) {
        const int N = p.N, P = p.P;
        const size_t row = bits ? (size_t)P / 8 : (size_t)P;
        size_t o = 0;
        spins = o; o += up16((size_t)N * row);
        ones = o;  o += up16(row);
        lut = o;   o += bits ? 2048 : 0;
        desc = o;  o += (size_t)N * (dc == 4 ? 32 : 48);
        items = o; o += up16((size_t)2 * N * 4);
        loff = o;  o += up16((size_t)(p.n_levels + 1) * 4);
        thr = o;   o += thr_bytes(p);
        acc = o;   o += acc_bytes(p);
        red = o;   o += 32 * 3 * 8;
        ctl = o;   o += 32;
        cmb = o;   o += cswap ? (size_t)kClusterMailPasses * p.R * 16 : 0;
        rbuf = o;
        if (pre) o += (size_t)2 * (2 * N) * (P / 8) * 16;
        total = o;
    }
};

size_t split_smem_bytes(const DevProblem& p, int dclass, bool pre);

size_t sweep_smem_bytes(const DevProblem& p, int path, int dclass, bool cluster_pre) {
    if (path == kPathGeneric) return GenericLayout(p).total;
    if (path == kPathCluster) return FastLayout(p, dclass, cluster_pre, false, true).total;
    if (path == kPathPeer) return FastLayout(p, dclass, true, false).total;
    if (path == kPathSplit || path == kPathSplitInline) return split_smem_bytes(p, dclass, path == kPathSplit);
    return FastLayout(p, dclass, path == kPathPacked, path == kPathBits).total;
}


// ------------------------------------------------------------------------- end of a sweep
// Tag of pass q0 + pass, from qmod0 = q0 mod kTagPeriod (taken once per launch): a 32-bit
// remainder by a constant instead of a 64-bit one on the path to the partner.
__device__ __forceinline__ unsigned long long mbox_tag(uint32_t qmod0, int pass) {
    return (unsigned long long)((qmod0 + (uint32_t)pass) % (uint32_t)kTagPeriod) + 1ull;
}

// A chain's side of the swap pass that follows a sweep: rl is the lower rung of its pair,
// partner the other rung; active = 0 when no pass follows or the chain has no partner.
struct SwapSide {
    int active, rl, partner, pass;
    long long q;
    unsigned long long tag;
};

// Thread 0 of a chain's CTA, after the sweep's changes are reduced: update E and M, add the
// statistics of the rung the chain sits on (to `acc`, shared or global) and, when a swap
// pass follows this sweep, publish (E, M) in the pass's mailbox. Does not wait.
// pass >= 0: a swap pass with this index (within the launch) follows the sweep.
// write = false: a CTA that shares the chain with the one that publishes (split kernel).
__device__ SwapSide eos_publish(const DevProblem& p, int rung, long long& E, long long& M, long long dE,
                                long long dM, int pass, long long q0, uint32_t qmod0, bool write = true) {
    E += dE;
    M += dM;
    SwapSide w;
    w.active = 0;
    if (pass >= 0) {
        const int R = p.R;
        w.pass = pass;
        w.q = q0 + w.pass;
        w.tag = mbox_tag(qmod0, w.pass);
        Mailbox* mb = p.mbox + (size_t)w.pass * R;
        if (write && rung != p.withhold_rung) {
            st_relaxed_u64(&mb[rung].a, ((unsigned long long)E << 24) | w.tag);
            st_relaxed_u64(&mb[rung].b, ((unsigned long long)(uint32_t)(int32_t)M << 32) | w.tag);
        }
        if ((rung & 1) == (int)(w.q & 1)) {
            w.rl = rung;
            w.partner = rung + 1;
        } else {
            w.rl = rung - 1;
            w.partner = rung - 1;
        }
        w.active = (w.rl >= 0 && w.rl + 1 < R) ? 1 : 0;
    }
    return w;
}

static_assert(kAccN == 0 && kAccE == 1 && kAccE2 == 2 && kAccM == 3 && kAccM2 == 4 && kAccFlip == 5 && kAccCount == 6,
              "eos_stats pairs the counters in this order");

// Thread 0: the statistics of the rung the chain sat on during the sweep (to `acc`, shared or
// global), from the updated E and M.
__device__ __forceinline__ void eos_stats(const DevProblem& p, unsigned long long* acc, int rung, long long E,
                                          long long M, long long nflip) {
    unsigned long long* a = acc + (size_t)rung * kAccCount;
    if (p.acc_in_smem) {
        // the rung's six counters (48 bytes, 16-byte aligned) in three paired loads and stores
        ulonglong2* a2 = reinterpret_cast<ulonglong2*>(a);
        ulonglong2 v0 = a2[0], v1 = a2[1], v2 = a2[2];
        v0.x += 1ull;                                // kAccN
        v0.y += (unsigned long long)E;               // kAccE
        v1.x += (unsigned long long)(E * E);         // kAccE2
        v1.y += (unsigned long long)M;               // kAccM
        v2.x += (unsigned long long)(M * M);         // kAccM2
        v2.y += (unsigned long long)nflip;           // kAccFlip
        a2[0] = v0;
        a2[1] = v1;
        a2[2] = v2;
    } else {
        atomicAdd(a + kAccN, 1ull);
        atomicAdd(a + kAccE, (unsigned long long)E);
        atomicAdd(a + kAccE2, (unsigned long long)(E * E));
        atomicAdd(a + kAccM, (unsigned long long)M);
        atomicAdd(a + kAccM2, (unsigned long long)(M * M));
        atomicAdd(a + kAccFlip, (unsigned long long)nflip);
    }
}

// Thread 0 again: wait for the partner's mailbox (bounded by timeout_ns) and take the
// decision both chains of the pair take. Returns the chain's rung for the next sweep; sets
// *abort when the partner's mailbox never arrived within the time limit. count = false: the
// pair's attempt and acceptance are counted by another CTA of the chain (split kernel).
__device__ int eos_decide(const DevProblem& p, const SwapSide& w, int rung, long long E, long long M,
                          long long timeout_ns, const PhiloxKey& key, int* abort, bool count = true) {
    *abort = 0;
    if (!w.active) return rung;
    const int R = p.R;
    const Mailbox* mb = p.mbox + (size_t)w.pass * R;
    long long pE, pM;
    const unsigned long long start = globaltimer_ns();
    // the first polls spin (the partner usually publishes within an L2 round trip); later
    // ones back off with __nanosleep, doubling up to 256 ns, so that a CTA waiting on a slow
    // partner leaves its issue slots and the L2 to the CTAs sharing its SM
    unsigned int nap = 0;
    for (int polls = 0;; ++polls) {
        const unsigned long long wa = ld_relaxed_u64(&mb[w.partner].a);
        const unsigned long long wb = ld_relaxed_u64(&mb[w.partner].b);
        if ((wa & 0xFFFFFFull) == w.tag && (wb & 0xFFFFFFull) == w.tag) {
            pE = (long long)wa >> 24;
            pM = (long long)(int32_t)(uint32_t)(wb >> 32);
            break;
        }
        if ((long long)(globaltimer_ns() - start) > timeout_ns) {
            atomicCAS(p.status, 0, PT_ETIMEDOUT);
            *abort = 1;
            return rung;
        }
        if (polls >= 32) {
            nap = nap ? min(2u * nap, 256u) : 16u;
            __nanosleep(nap);
        }
    }
    const int rl = w.rl;
    const bool lower = (rung == rl);
    const bool acc_swap = swap_accept_fast(lower ? E : pE, lower ? pE : E, lower ? M : pM, lower ? pM : M,
                                           p.coef[rl], p.coef[(R - 1) + rl], (uint32_t)w.q, (uint32_t)rl, key,
                                           p.exact_swaps != 0);
    if (lower && count) {
        atomicAdd(p.swap_stats + 2 * rl, 1ull);
        if (acc_swap) atomicAdd(p.swap_stats + 2 * rl + 1, 1ull);
    }
    return acc_swap ? w.partner : rung;
}

// Path 9 (one cluster holds every chain): the same decision with the partner's (E, M) read
// from this CTA's own copy of the cluster mailboxes. Every chain that publishes for a pass
// writes its two tagged words into every CTA of the cluster, at [pass mod 4][rung], so the
// wait polls local shared memory. Four slots suffice: the chain that would overwrite the
// slot a waiting chain reads (the holder of that rung three passes later) must first finish
// the pass two later, in which it waits for the reader's own publication again.
__device__ int eos_decide_cluster(const DevProblem& p, const unsigned long long* s_cmb, const SwapSide& w, int rung,
                                  long long E, long long M, long long timeout_ns, const PhiloxKey& key, int* abort) {
    *abort = 0;
    if (!w.active) return rung;
    const int R = p.R;
    const unsigned long long* mb = s_cmb + ((size_t)(w.pass & (kClusterMailPasses - 1)) * R + w.partner) * 2;
    long long pE, pM;
    const unsigned long long start = globaltimer_ns();
    unsigned int nap = 0;
    for (int polls = 0;; ++polls) {
        const unsigned long long wa = ld_cluster_local_u64(mb);
        const unsigned long long wb = ld_cluster_local_u64(mb + 1);
        if ((wa & 0xFFFFFFull) == w.tag && (wb & 0xFFFFFFull) == w.tag) {
            pE = (long long)wa >> 24;
            pM = (long long)(int32_t)(uint32_t)(wb >> 32);
            break;
        }
        if ((long long)(globaltimer_ns() - start) > timeout_ns) {
            atomicCAS(p.status, 0, PT_ETIMEDOUT);
            *abort = 1;
            return rung;
        }
        if (polls >= 32) {
            nap = nap ? min(2u * nap, 256u) : 16u;
            __nanosleep(nap);
        }
    }
    const int rl = w.rl;
    const bool lower = (rung == rl);
    const bool acc_swap = swap_accept_fast(lower ? E : pE, lower ? pE : E, lower ? M : pM, lower ? pM : M,
                                           p.coef[rl], p.coef[(R - 1) + rl], (uint32_t)w.q, (uint32_t)rl, key,
                                           p.exact_swaps != 0);
    if (lower) {
        atomicAdd(p.swap_stats + 2 * rl, 1ull);
        if (acc_swap) atomicAdd(p.swap_stats + 2 * rl + 1, 1ull);
    }
    return acc_swap ? w.partner : rung;
}

// Both steps at once (the byte-wise kernel).
__device__ int end_of_sweep(const DevProblem& p, unsigned long long* acc, int rung, long long& E, long long& M,
                            long long dE, long long dM, long long nflip, int s, long long q0, int sweeps_per_swap,
                            long long timeout_ns, const PhiloxKey& key, int* abort) {
    const int pass = (sweeps_per_swap > 0 && (s + 1) % sweeps_per_swap == 0) ? (s + 1) / sweeps_per_swap - 1 : -1;
    const SwapSide w = eos_publish(p, rung, E, M, dE, dM, pass, q0, (uint32_t)(q0 % kTagPeriod));
    eos_stats(p, acc, rung, E, M, nflip);
    return eos_decide(p, w, rung, E, M, timeout_ns, key, abort);
}

// Shared-memory threshold rows: every rung's row when they fit, else the current one.
__device__ __forceinline__ void load_thr(const DevProblem& p, uint32_t* s_thr, int rung, int tid, int nt) {
    if (p.tables_in_smem) {
        for (int x = tid; x < p.R * p.nL3; x += nt) s_thr[x] = p.thr[x];
    } else {
        for (int x = tid; x < p.nL3; x += nt) s_thr[x] = p.thr[(size_t)rung * p.nL3 + x];
    }
}
__device__ __forceinline__ const uint32_t* thr_row(const DevProblem& p, const uint32_t* s_thr, int rung) {
    return p.tables_in_smem ? s_thr + (size_t)rung * p.nL3 : s_thr;
}

// Per-launch statistics gathered in shared memory are added to the global rows once.
__device__ __forceinline__ void flush_acc(const DevProblem& p, const unsigned long long* s_acc, int tid, int nt) {
    if (!p.acc_in_smem) return;
    for (int x = tid; x < p.R * kAccCount; x += nt)
        if (s_acc[x]) atomicAdd(p.acc + x, s_acc[x]);
}

// ------------------------------------------------------------------------- generic sweep
// One CTA per chain (slot); byte-wise spins, Philox inline in each 4-copy unit. Used when
// P is not a multiple of 8 or a site has more than 7 neighbours.
template <int DCLASS>
__global__ void __launch_bounds__(512, 1)
sweep_kernel(DevProblem p, long long t0, long long q0, int n_sweeps, int sweeps_per_swap,
             long long timeout_ns, int n_consumer) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = p.N, P = p.P;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int slot = blockIdx.x;
    const GenericLayout L(p);
    int8_t* sp = reinterpret_cast<int8_t*>(smem + L.spins);
    uint32_t* s_nbr = reinterpret_cast<uint32_t*>(smem + L.nbr);
    int8_t* s_h = reinterpret_cast<int8_t*>(smem + L.h);
    uint32_t* s_items = reinterpret_cast<uint32_t*>(smem + L.items);
    int32_t* s_loff = reinterpret_cast<int32_t*>(smem + L.loff);
    uint32_t* s_thr = reinterpret_cast<uint32_t*>(smem + L.thr);
    long long* s_red = reinterpret_cast<long long*>(smem + L.red);
    int* s_ctl = reinterpret_cast<int*>(smem + L.ctl);
    unsigned long long* s_acc = reinterpret_cast<unsigned long long*>(smem + L.acc);
    (void)n_consumer;

    {
        const int4* src = reinterpret_cast<const int4*>(p.spins + (size_t)slot * p.slot_stride);
        int4* dst = reinterpret_cast<int4*>(sp);
        const int n16 = (int)(up16((size_t)N * P) / 16);
        for (int x = tid; x < n16; x += nt) dst[x] = src[x];
        for (int x = tid; x < N * DCLASS; x += nt) s_nbr[x] = p.nbr[x];
        for (int x = tid; x < N; x += nt) s_h[x] = p.h[x];
        for (int x = tid; x < 2 * N; x += nt) s_items[x] = p.items[x];
        for (int x = tid; x <= p.n_levels; x += nt) s_loff[x] = p.level_off[x];
    }
    int rung = p.rung_of_slot[slot];
    load_thr(p, s_thr, rung, tid, nt);
    if (p.acc_in_smem)
        for (int x = tid; x < p.R * kAccCount; x += nt) s_acc[x] = 0ull;
    long long E = p.E[slot], M = p.M[slot];  // meaningful in thread 0 only
    __syncthreads();
    const uint32_t* thr = thr_row(p, s_thr, rung);

    const PhiloxKey key = philox_schedule(p.key0, p.key1);
    const int G = (((P + 1) >> 1) + 3) >> 2;  // 4-copy groups per parity (P = 1: one even copy)
    int lg = 0;
    while ((1 << lg) < G) ++lg;
    const int gmask = (1 << lg) - 1;
    const int Lmax = p.Lmax;
    const int lane = tid & 31, warp = tid >> 5, nwarps = (nt + 31) >> 5;

    for (int s = 0; s < n_sweeps; ++s) {
        const uint32_t t = (uint32_t)(t0 + s);
        int dE = 0, dM = 0, nf = 0;
        for (int lev = 0; lev < p.n_levels; ++lev) {
            const int base = s_loff[lev];
            const int units = (s_loff[lev + 1] - base) << lg;
            for (int u = tid; u < units; u += nt) {
                const int g = u & gmask;
                if (g >= G) continue;
                const uint32_t it = s_items[base + (u >> lg)];
                const int i = (int)(it >> 1), par = (int)(it & 1u);
                const uint4 r4 = philox(make_uint4(t, (uint32_t)i, (uint32_t)slot,
                                                   ((uint32_t)par << 24) | (uint32_t)g), key);
                const uint32_t rw[4] = {r4.x, r4.y, r4.z, r4.w};
                uint32_t nb[DCLASS];
#pragma unroll
                for (int d = 0; d < DCLASS; ++d) nb[d] = s_nbr[i * DCLASS + d];
                const int hi = s_h[i];
                int8_t* row = sp + (size_t)i * P;
                const int n_par = (P + 1 - par) >> 1;  // copies of this parity
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    const int hh = 4 * g + w;
                    if (hh < n_par) {
                        const int k = par + 2 * hh;
                        const int sk = row[k];
                        int f = hi;
#pragma unroll
                        for (int d = 0; d < DCLASS; ++d) {
                            const int j = (int)(nb[d] >> 8);
                            const int J = (int)(int8_t)(nb[d] & 0xFFu);
                            f += J * (int)sp[(size_t)j * P + k];
                        }
                        const int Lf = sk * f;
                        const int km1 = (k == 0) ? P - 1 : k - 1;
                        const int kp1 = (k + 1 == P) ? 0 : k + 1;
                        // a classical chain's lone copy (P = 1) has no Trotter neighbours
                        const int m = P == 1 ? 0 : sk * ((int)row[km1] + (int)row[kp1]);
                        const uint32_t th = thr[(Lf + Lmax) * 3 + (m >> 1) + 1];
                        if (th == 0xFFFFFFFFu || rw[w] < th) {
                            row[k] = (int8_t)(-sk);
                            dE -= 2 * Lf;
                            dM -= 2 * m;
                            nf += 1;
                        }
                    }
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            dE += __shfl_xor_sync(0xFFFFFFFFu, dE, o);
            dM += __shfl_xor_sync(0xFFFFFFFFu, dM, o);
            nf += __shfl_xor_sync(0xFFFFFFFFu, nf, o);
        }
        if (lane == 0) {
            s_red[warp * 3 + 0] = dE;
            s_red[warp * 3 + 1] = dM;
            s_red[warp * 3 + 2] = nf;
        }
        __syncthreads();
        if (tid == 0) {
            long long sE = 0, sM = 0, sF = 0;
            for (int w = 0; w < nwarps; ++w) {
                sE += s_red[w * 3 + 0];
                sM += s_red[w * 3 + 1];
                sF += s_red[w * 3 + 2];
            }
            int abort_flag = 0;
            s_ctl[0] = end_of_sweep(p, p.acc_in_smem ? s_acc : p.acc, rung, E, M, sE, sM, sF, s, q0,
                                    sweeps_per_swap, timeout_ns, key, &abort_flag);
            s_ctl[1] = abort_flag;
        }
        __syncthreads();
        if (s_ctl[1]) return;  // a partner never arrived; status holds PT_ETIMEDOUT
        const int nr = s_ctl[0];
        if (nr != rung) {
            rung = nr;
            if (!p.tables_in_smem) load_thr(p, s_thr, rung, tid, nt);
            thr = thr_row(p, s_thr, rung);
        }
        __syncthreads();
    }
    flush_acc(p, s_acc, tid, nt);

    {
        int4* dst = reinterpret_cast<int4*>(p.spins + (size_t)slot * p.slot_stride);
        const int4* src = reinterpret_cast<const int4*>(sp);
        const int n16 = (int)(up16((size_t)N * P) / 16);
        for (int x = tid; x < n16; x += nt) dst[x] = src[x];
    }
    if (tid == 0) {
        p.E[slot] = E;
        p.M[slot] = M;
        p.rung_of_slot[slot] = rung;
        p.slot_of_rung[rung] = slot;
    }
}

// ------------------------------------------------------------------------- classical sweep
// Path 10 (P = 1, classical tempering): the R chains packed C to a CTA (C a power of two),
// chain fastest in shared memory (site i of chain c at byte i C + c), on one cluster of
// K = ceil(R / C) CTAs. A level's updates are (site, chain) pairs, chain fastest, and every
// thread keeps one chain (blockDim is a multiple of C), so a warp reads one site's neighbour
// list for up to 32 chains and their bytes side by side, and the thread's threshold row is
// its chain's. After a sweep thread c of the CTA ends chain c's sweep: statistics, then the
// swap publication into every CTA of the cluster and the partner's wait in its own shared
// memory, as path 9 does (eos_decide_cluster). The update, its counter and its table entry
// are the byte-wise kernel's for P = 1.
struct ClassicalLayout {
    size_t spins, nbr, h, items, loff, thr, acc, cmb, E, M, rung, sums, ctl, total;
    __host__ __device__ ClassicalLayout(const DevProblem& p, int C) {
        size_t o = 0;
        spins = o; o += up16((size_t)p.N * C);
        nbr = o;   o += up16((size_t)p.N * p.dmax * 4);
        h = o;     o += up16((size_t)p.N);
        items = o; o += up16((size_t)2 * p.N * 4);
        loff = o;  o += up16((size_t)(p.n_levels + 1) * 4);
        thr = o;   o += up16((size_t)p.R * p.nL3 * 4);  // every rung's row
        acc = o;   o += (size_t)p.R * kAccCount * 8;      // this launch's statistics, by rung
        cmb = o;   o += (size_t)kClusterMailPasses * p.R * 16;
        E = o;     o += up16((size_t)C * 8);
        M = o;     o += up16((size_t)C * 8);
        rung = o;  o += up16((size_t)C * 4);
        sums = o;  o += up16((size_t)C * 8);               // per chain: dE and flips of the sweep
        ctl = o;   o += 16;
        total = o;
    }
};

size_t classical_smem_bytes(const DevProblem& p, int chains) { return ClassicalLayout(p, chains).total; }

template <int DCLASS>
__global__ void __launch_bounds__(512, 1)
    sweep_classical_kernel(DevProblem p, long long t0, long long q0, int n_sweeps, int sweeps_per_swap,
                           long long timeout_ns, int C) {
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cluster = cg::this_cluster();
    const int K = (p.R + C - 1) / C;
    if (cluster.num_blocks() != (unsigned)K || gridDim.x != (unsigned)K || p.P != 1 || C < 1 || (C & (C - 1)) ||
        (blockDim.x % (unsigned)C) || (blockDim.x & 31u)) {
        if (threadIdx.x == 0) atomicCAS(p.status, 0, PT_ECUDA);
        return;  // every CTA returns here, before any cluster barrier
    }
    const int N = p.N, R = p.R;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    const int rank = (int)cluster.block_rank();
    const int c0 = rank * C, nc = min(C, R - c0);  // this CTA's chains: slots c0 .. c0 + nc - 1
    const ClassicalLayout L(p, C);
    int8_t* sp = reinterpret_cast<int8_t*>(smem + L.spins);
    uint32_t* s_nbr = reinterpret_cast<uint32_t*>(smem + L.nbr);
    int8_t* s_h = reinterpret_cast<int8_t*>(smem + L.h);
    uint32_t* s_items = reinterpret_cast<uint32_t*>(smem + L.items);
    int32_t* s_loff = reinterpret_cast<int32_t*>(smem + L.loff);
    uint32_t* s_thr = reinterpret_cast<uint32_t*>(smem + L.thr);
    unsigned long long* s_acc = reinterpret_cast<unsigned long long*>(smem + L.acc);
    unsigned long long* s_cmb = reinterpret_cast<unsigned long long*>(smem + L.cmb);
    long long* s_E = reinterpret_cast<long long*>(smem + L.E);
    long long* s_M = reinterpret_cast<long long*>(smem + L.M);
    int* s_rung = reinterpret_cast<int*>(smem + L.rung);
    int* s_sums = reinterpret_cast<int*>(smem + L.sums);  // [c][0] = dE, [c][1] = flips
    int* s_ctl = reinterpret_cast<int*>(smem + L.ctl);

    for (int x = tid; x < N * C; x += nt) {
        const int i = x / C, c = x - i * C;
        sp[x] = c < nc ? p.spins[(size_t)(c0 + c) * p.slot_stride + i] : (int8_t)1;
    }
    for (int x = tid; x < N * DCLASS; x += nt) s_nbr[x] = p.nbr[x];
    for (int x = tid; x < N; x += nt) s_h[x] = p.h[x];
    for (int x = tid; x < 2 * N; x += nt) s_items[x] = p.items[x];
    for (int x = tid; x <= p.n_levels; x += nt) s_loff[x] = p.level_off[x];
    for (int x = tid; x < R * p.nL3; x += nt) s_thr[x] = p.thr[x];
    for (int x = tid; x < R * kAccCount; x += nt) s_acc[x] = 0ull;
    for (int x = tid; x < kClusterMailPasses * R * 2; x += nt) s_cmb[x] = 0ull;
    for (int c = tid; c < C; c += nt) {
        s_E[c] = c < nc ? p.E[c0 + c] : 0;
        s_M[c] = c < nc ? p.M[c0 + c] : 0;
        s_rung[c] = c < nc ? p.rung_of_slot[c0 + c] : 0;
        s_sums[2 * c] = s_sums[2 * c + 1] = 0;
    }
    if (tid == 0) s_ctl[0] = 0;
    __syncthreads();
    cluster_barrier();  // every CTA's mailboxes are clear before anyone publishes

    const PhiloxKey key = philox_schedule(p.key0, p.key1);
    const int Lmax = p.Lmax;
    const int my_c = tid & (C - 1);  // this thread's chain, the same in every level
    int lgC = 0;
    while ((1 << lgC) < C) ++lgC;
    const bool live = my_c < nc;
    const uint32_t my_slot = (uint32_t)(c0 + my_c);
    const uint32_t* thr = s_thr + (size_t)s_rung[my_c] * p.nL3 + 1;  // m = 0 column
    const uint32_t qmod0 = (uint32_t)(q0 % kTagPeriod);
    int since_pass = 0, next_pass = 0;  // thread c < nc: chain c's swap schedule

    for (int s = 0; s < n_sweeps; ++s) {
        const uint32_t t = (uint32_t)(t0 + s);
        int dE = 0, nf = 0;
        for (int lev = 0; lev < p.n_levels; ++lev) {
            const int base = s_loff[lev];
            const int units = (s_loff[lev + 1] - base) << lgC;
            if (live)
                for (int u = tid; u < units; u += nt) {
                    const int i = (int)(s_items[base + (u >> lgC)] >> 1);
                    const uint32_t r = philox(make_uint4(t, (uint32_t)i, my_slot, 0u), key).x;
                    int f = s_h[i];
#pragma unroll
                    for (int d = 0; d < DCLASS; ++d) {
                        const uint32_t nb = s_nbr[i * DCLASS + d];
                        f += (int)(int8_t)(nb & 0xFFu) * (int)sp[(size_t)(nb >> 8) * C + my_c];
                    }
                    int8_t* own = sp + (size_t)i * C + my_c;
                    const int sk = *own;
                    const int Lf = sk * f;
                    const uint32_t th = thr[(Lf + Lmax) * 3];
                    if (th == 0xFFFFFFFFu || r < th) {
                        *own = (int8_t)(-sk);
                        dE -= 2 * Lf;
                        nf += 1;
                    }
                }
            __syncthreads();
        }
        // the sweep's changes of each chain: lanes of a warp that share a chain are C apart
        for (int o = 16; o >= C; o >>= 1) {
            dE += __shfl_xor_sync(0xFFFFFFFFu, dE, o);
            nf += __shfl_xor_sync(0xFFFFFFFFu, nf, o);
        }
        if (live && lane < C && (dE | nf)) {
            atomicAdd(s_sums + 2 * my_c, dE);
            atomicAdd(s_sums + 2 * my_c + 1, nf);
        }
        __syncthreads();
        // chain tid's end of sweep, in two phases: every chain of the CTA publishes before
        // any of them waits, so partners on one CTA never wait on a thread that has not
        // published yet (spreading the copies over the CTA's threads, behind one more
        // barrier, measured slower)
        SwapSide side;
        long long E = 0, M = 0;
        int rung = 0;
        if (tid < nc) {
            const int c = tid;
            E = s_E[c];
            M = s_M[c];
            rung = s_rung[c];
            const int sE = s_sums[2 * c], sF = s_sums[2 * c + 1];
            s_sums[2 * c] = s_sums[2 * c + 1] = 0;
            int pass = -1;
            if (sweeps_per_swap > 0 && ++since_pass == sweeps_per_swap) {
                since_pass = 0;
                pass = next_pass++;
            }
            side = eos_publish(p, rung, E, M, sE, 0, pass, q0, qmod0, false);
            eos_stats(p, s_acc, rung, E, M, sF);
            if (side.active && rung != p.withhold_rung) {
                const int idx = ((side.pass & (kClusterMailPasses - 1)) * R + rung) * 2;
                const unsigned long long wa = ((unsigned long long)E << 24) | side.tag;
                const unsigned long long wb = ((unsigned long long)(uint32_t)(int32_t)M << 32) | side.tag;
                for (int r = 0; r < K; ++r) st_cluster_u64x2(s_cmb + idx, (unsigned)r, wa, wb);
            }
        }
        __syncthreads();
        if (tid < nc) {
            const int c = tid;
            int abort_flag = 0;
            s_rung[c] = eos_decide_cluster(p, s_cmb, side, rung, E, M, timeout_ns, key, &abort_flag);
            s_E[c] = E;
            s_M[c] = M;
            if (abort_flag) s_ctl[0] = 1;  // a partner never arrived
        }
        __syncthreads();
        if (s_ctl[0]) break;  // to the cluster barrier that every CTA passes before leaving
        thr = s_thr + (size_t)s_rung[my_c] * p.nL3 + 1;
    }
    __syncthreads();
    // no CTA leaves while another may still write its mailboxes (every wait is bounded)
    cluster_barrier();
    if (s_ctl[0]) return;  // status holds PT_ETIMEDOUT
    for (int x = tid; x < R * kAccCount; x += nt)
        if (s_acc[x]) atomicAdd(p.acc + x, s_acc[x]);
    for (int x = tid; x < N * nc; x += nt) {
        const int c = x / N, i = x - c * N;
        p.spins[(size_t)(c0 + c) * p.slot_stride + i] = sp[(size_t)i * C + c];
    }
    for (int c = tid; c < nc; c += nt) {
        const int rung = s_rung[c];
        p.E[c0 + c] = s_E[c];
        p.M[c0 + c] = s_M[c];
        p.rung_of_slot[c0 + c] = rung;
        p.slot_of_rung[rung] = c0 + c;
    }
}

// ------------------------------------------------------------------------- packed sweep
// Random words of one sweep for the producer warps: word w of philox((t, i, slot,
// p<<24 | g)) goes with copy 8g + p + 2w of site i (the same counter the update would use).
__device__ __forceinline__ void produce_words(uint4* buf, uint32_t t, const uint32_t* s_items, int n_items, int G,
                                              int lg, int gmask, int ptid, int np, uint32_t slot,
                                              const PhiloxKey& key) {
    if (ptid < 0 || np <= 0) return;  // producer threads only
    const int total = n_items << lg;
    for (int x = ptid; x < total; x += np) {
        const int g = x & gmask;
        if (g >= G) continue;
        const int q = x >> lg;
        const uint32_t it = s_items[q];
        // stored as min(u, 2^32 - 2): then u < thr alone is the acceptance rule, the
        // "accept always" entry 0xFFFFFFFF included
        const uint4 r = philox(make_uint4(t, it >> 1, slot, ((it & 1u) << 24) | (uint32_t)g), key);
        buf[q * G + g] = make_uint4(min(r.x, 0xFFFFFFFEu), min(r.y, 0xFFFFFFFEu), min(r.z, 0xFFFFFFFEu),
                                    min(r.w, 0xFFFFFFFEu));
    }
}

// One CTA per chain with the chain, the unit descriptors and the threshold row in shared
// memory. PRE: the last (blockDim - n_consumer) threads are producer warps that write the
// random words of sweep s+1 into one shared buffer while the consumer warps run the levels
// of sweep s out of the other; consumers synchronise levels on named barrier 1 and both
// groups meet once per sweep.
// PEER (path 8): the CTA is rank 0 of a cluster of two, and rank 1 (peer_producer below)
// writes the random words into this CTA's buffers through distributed shared memory; every
// thread here sweeps, and the two CTAs meet at a cluster barrier once per sweep.
// CSWAP (path 9): the CTAs of all R chains form one cluster (slot = rank) and the swap
// mailboxes live in every CTA's shared memory (eos_decide_cluster); the CTAs meet at a
// cluster barrier only after the mailboxes are cleared and before they leave.
template <int DC, bool PRE, bool BITS = false, bool SPEC = true, bool PEER = false, bool CSWAP = false>
__device__ __forceinline__ void sweep_packed_body(const DevProblem& p, int slot, long long t0, long long q0,
                                                  int n_sweeps, int sweeps_per_swap, long long timeout_ns,
                                                  int n_consumer, unsigned char* smem) {
    const int N = p.N, P = p.P;
    const int tid = threadIdx.x, nt = blockDim.x;
    const FastLayout L(p, DC, PRE, BITS, CSWAP);
    int8_t* sp = reinterpret_cast<int8_t*>(smem + L.spins);
    uint8_t* bp = reinterpret_cast<uint8_t*>(smem + L.spins);
    uint32_t* s_lut = reinterpret_cast<uint32_t*>(smem + L.lut);
    uint32_t* s_desc = reinterpret_cast<uint32_t*>(smem + L.desc);
    uint32_t* s_items = reinterpret_cast<uint32_t*>(smem + L.items);
    int32_t* s_loff = reinterpret_cast<int32_t*>(smem + L.loff);
    uint32_t* s_thr = reinterpret_cast<uint32_t*>(smem + L.thr);
    long long* s_red = reinterpret_cast<long long*>(smem + L.red);
    int* s_ctl = reinterpret_cast<int*>(smem + L.ctl);
    uint4* rbuf = reinterpret_cast<uint4*>(smem + L.rbuf);
    unsigned long long* s_acc = reinterpret_cast<unsigned long long*>(smem + L.acc);
    unsigned long long* s_cmb = reinterpret_cast<unsigned long long*>(smem + L.cmb);
    const int NC = PRE ? n_consumer : nt;
    const bool consumer = tid < NC;
    const int DW = SiteDesc<DC>::DW;

    if (BITS) {
        // int8 chain in global memory -> one bit per copy in shared memory
        const uint2* src = reinterpret_cast<const uint2*>(p.spins + (size_t)slot * p.slot_stride);
        for (int x = tid; x < N * (P / 8); x += nt) {
            const uint2 v = src[x];
            uint32_t b = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                b |= ((v.x >> (8 * k + 7)) & 1u) << k;
                b |= ((v.y >> (8 * k + 7)) & 1u) << (k + 4);
            }
            bp[x] = (uint8_t)b;
        }
        uint8_t* zeros = reinterpret_cast<uint8_t*>(smem + L.ones);
        for (int x = tid; x < P / 8; x += nt) zeros[x] = 0;
        for (int x = tid; x < 512; x += nt) {
            const uint32_t par = (uint32_t)x >> 8, byte = (uint32_t)x & 0xFFu;
            uint32_t v = 0;
#pragma unroll
            for (int w = 0; w < 4; ++w) v |= (((byte >> (par + 2 * w)) & 1u) ? 0xFFu : 0x01u) << (8 * w);
            s_lut[x] = v;
        }
    } else {
        // interleaved int8 chain in global memory -> parity-split rows in shared memory
        load_split(sp, p.spins + (size_t)slot * p.slot_stride, N, P, P >> 3, chunk_ginv(P >> 3), tid, nt);
        int8_t* ones = reinterpret_cast<int8_t*>(smem + L.ones);
        for (int x = tid; x < P; x += nt) ones[x] = 1;
    }
    {
        const int4* dsrc = reinterpret_cast<const int4*>(p.desc);
        int4* ddst = reinterpret_cast<int4*>(s_desc);
        for (int x = tid; x < N * DW / 4; x += nt) ddst[x] = dsrc[x];
        for (int x = tid; x < 2 * N; x += nt) s_items[x] = p.items[x];
        for (int x = tid; x <= p.n_levels; x += nt) s_loff[x] = p.level_off[x];
    }
    int rung = p.rung_of_slot[slot];
    load_thr(p, s_thr, rung, tid, nt);
    if (p.acc_in_smem)
        for (int x = tid; x < p.R * kAccCount; x += nt) s_acc[x] = 0ull;
    long long E = p.E[slot], M = p.M[slot];  // meaningful in thread 0 only

    const PhiloxKey key = philox_schedule(p.key0, p.key1);
    const int G = P >> 3;  // 8-copy chunks per row = 4-copy units per parity
    int lg = 0;
    while ((1 << lg) < G) ++lg;
    const int gmask = (1 << lg) - 1;
    const uint32_t* thr_c = thr_row(p, s_thr, rung) + 3 * p.Lmax;
    const int n_items = 2 * N;
    const int lane = tid & 31;
    if (tid == 0) {
        s_ctl[4] = -1;  // partner rung of the pending swap pass
        s_ctl[5] = 0;   // a swap wait gave up
        int* s_sum = reinterpret_cast<int*>(s_red);
        s_sum[0] = s_sum[1] = s_sum[2] = 0;  // the sweep's dE, dM and flips
    }
    if (CSWAP)
        for (int x = tid; x < kClusterMailPasses * p.R * 2; x += nt) s_cmb[x] = 0ull;
    __syncthreads();
    if (CSWAP) cluster_barrier();  // every CTA's mailboxes are clear before anyone publishes
    if (PRE && !PEER && !consumer)
        produce_words(rbuf, (uint32_t)t0, s_items, n_items, G, lg, gmask, tid - NC, nt - NC, (uint32_t)slot, key);
    if (PEER) {
        // the peer CTA has written the first sweep's words (its arrival releases them); this
        // CTA's arrival orders nothing of its own, so it is relaxed
        cluster_arrive_relaxed();
        cluster_wait_acquire();
    } else if (PRE) {
        __syncthreads();
    }

    // Level 0 of the next sweep can be evaluated while the swap decision is still pending:
    // its inputs are the spins after this sweep and the next sweep's random words; only its
    // threshold row depends on the decision, and both candidate rows are in shared memory.
    // Up to two level-0 units per consumer thread are held in registers.
    // Warp 0 takes no level-0 unit, so that thread 0 can poll the partner's mailbox at once.
    const int units0 = (s_loff[1] - s_loff[0]) << lg;
    const bool spec_ok = SPEC && !BITS && p.tables_in_smem && NC > 32 && units0 <= 2 * (NC - 32);
    bool spec_done = false;  // level 0 of sweep s was applied at the end of sweep s - 1
    // units u = tid + k NC of a level have the same column g = u mod 2^lg when NC is a
    // multiple of 2^lg: the thread then walks items q = base + (tid >> lg) + k (NC >> lg)
    const bool g_fixed = (NC & gmask) == 0;
    const int g_own = tid & gmask, q_lane = tid >> lg, q_step = NC >> lg;
    int sumL = 0, sumC = 0, nf = 0;  // sumC and nf count twice (see unit_commit)
    SwapSide side;  // thread 0
    side.active = 0;
    const uint32_t qmod0 = (uint32_t)(q0 % kTagPeriod);
    int since_pass = 0, next_pass = 0, sweep_flips = 0;  // thread 0

    for (int s = 0; s < n_sweeps; ++s) {
        const uint32_t t = (uint32_t)(t0 + s);
        if (consumer && !s_ctl[5]) {
            const uint4* rb = rbuf + (size_t)(s & 1) * n_items * G;
            if (!spec_done) sumL = sumC = nf = 0;
            for (int lev = spec_done ? 1 : 0; lev < p.n_levels; ++lev) {
                const int base = s_loff[lev];
                if (g_fixed) {
                    // this thread's column g never changes: its row offsets are loop invariants
                    if (g_own < G) {
                        const int end = s_loff[lev + 1];
                        for (int q = base + q_lane; q < end; q += q_step) {
                            if (BITS)
                                packed_unit_bits<DC, PRE>(bp, s_desc, s_items[q], rb, q, g_own, G, s_lut, t,
                                                          (uint32_t)slot, key, thr_c, sumL, sumC, nf);
                            else
                                packed_unit<DC, PRE>(sp, s_desc, s_items[q], rb, q, g_own, G, P, t, (uint32_t)slot,
                                                     key, thr_c, sumL, sumC, nf);
                        }
                    }
                } else {
                    const int units = (s_loff[lev + 1] - base) << lg;
                    for (int u = tid; u < units; u += NC) {
                        const int g = u & gmask;
                        if (g >= G) continue;
                        const int q = base + (u >> lg);
                        if (BITS)
                            packed_unit_bits<DC, PRE>(bp, s_desc, s_items[q], rb, q, g, G, s_lut, t, (uint32_t)slot,
                                                      key, thr_c, sumL, sumC, nf);
                        else
                            packed_unit<DC, PRE>(sp, s_desc, s_items[q], rb, q, g, G, P, t, (uint32_t)slot, key,
                                                 thr_c, sumL, sumC, nf);
                    }
                }
                if (PRE) named_barrier(1, NC); else __syncthreads();
            }
            // a chain's per-sweep changes fit in 32 bits: each warp adds its sums to three
            // shared counters, which thread 0 reads and clears
            const int dE = __reduce_add_sync(0xFFFFFFFFu, -2 * sumL);
            const int dM = __reduce_add_sync(0xFFFFFFFFu, -2 * (sumC - nf));  // both counted twice
            const int dF = __reduce_add_sync(0xFFFFFFFFu, nf) >> 1;
            int* s_sum = reinterpret_cast<int*>(s_red);
            if (lane == 0) {
                atomicAdd(s_sum + 0, dE);
                atomicAdd(s_sum + 1, dM);
                atomicAdd(s_sum + 2, dF);
            }
            if (PRE) named_barrier(1, NC); else __syncthreads();
            if (tid == 0) {
                const int sE = s_sum[0], sM = s_sum[1];
                sweep_flips = s_sum[2];
                s_sum[0] = s_sum[1] = s_sum[2] = 0;
                // a swap pass follows every sweeps_per_swap-th sweep (counted, not divided)
                int pass = -1;
                if (sweeps_per_swap > 0 && ++since_pass == sweeps_per_swap) {
                    since_pass = 0;
                    pass = next_pass++;
                }
                side = eos_publish(p, rung, E, M, sE, sM, pass, q0, qmod0, !CSWAP);
                s_ctl[4] = side.active ? side.partner : -1;
                if (CSWAP && side.active && rung != p.withhold_rung) {
                    // the publication, into every CTA of the cluster (thread 0 alone: having
                    // warp 0's lanes share the stores would make them wait for this thread,
                    // which measured slower)
                    const int idx = ((side.pass & (kClusterMailPasses - 1)) * p.R + rung) * 2;
                    const unsigned long long wa = ((unsigned long long)E << 24) | side.tag;
                    const unsigned long long wb = ((unsigned long long)(uint32_t)(int32_t)M << 32) | side.tag;
                    for (int r = 0; r < p.R; ++r) st_cluster_u64x2(s_cmb + idx, (unsigned)r, wa, wb);
                }
            }
        } else if (PRE && !consumer && s + 1 < n_sweeps) {
            // producer warps only: a consumer whose swap wait gave up skips to the barrier below
            produce_words(rbuf + (size_t)((s + 1) & 1) * n_items * G, t + 1u, s_items, n_items, G, lg, gmask,
                          tid - NC, nt - NC, (uint32_t)slot, key);
        }
        // the next sweep's random words are complete and every consumer has finished sweep s;
        // a wait that gave up in the previous sweep ends the launch here, for every thread
        if constexpr (PEER) {
            // the peer CTA learns at the same barrier that this CTA leaves, and leaves too.
            // Otherwise the arrival is relaxed: a release would first wait for this sweep's
            // mailbox store to reach L2, on the way to the swap decision. The words this CTA
            // read are in registers by now, so the peer may overwrite their buffer.
            if (s_ctl[5]) {
                if (tid == 0) cg::this_cluster().map_shared_rank(s_ctl, 1)[6] = 1;
                cluster_arrive_release();
            } else {
                cluster_arrive_relaxed();
            }
            cluster_wait_acquire();
        } else {
            __syncthreads();
        }
        if (s_ctl[5]) {  // status holds PT_ETIMEDOUT
            if (CSWAP) break;  // to the cluster barrier that every CTA passes before leaving
            return;
        }
        if (!consumer) continue;

        // level 0 of sweep s + 1 under both candidate rungs
        const bool spec = spec_ok && s + 1 < n_sweeps;
        const int prung = s_ctl[4];
        UnitEval ev[2];
        uint32_t Fa[2] = {0u, 0u}, Fb[2] = {0u, 0u};
        bool valid[2] = {false, false};
        if (spec) {
            const uint4* rb1 = rbuf + (size_t)((s + 1) & 1) * n_items * G;
            const uint32_t* thr_b = prung >= 0 ? thr_row(p, s_thr, prung) + 3 * p.Lmax : thr_c;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int u = (tid - 32) + k * (NC - 32);
                const int g = u & gmask;
                valid[k] = tid >= 32 && u < units0 && g < G;
                if (valid[k]) {
                    const int q = s_loff[0] + (u >> lg);
                    ev[k] = packed_unit_eval<DC, PRE>(sp, s_desc, s_items[q], rb1, q, g, G, P, t + 1u, (uint32_t)slot,
                                                      key);
                    Fa[k] = unit_flips<PRE>(ev[k], thr_c);
                    Fb[k] = prung >= 0 ? unit_flips<PRE>(ev[k], thr_b) : Fa[k];
                }
            }
        }
        if (tid == 0) {
            // the statistics of sweep s (rung unchanged until the decision below), while
            // the partner's mailbox may still be on its way
            eos_stats(p, p.acc_in_smem ? s_acc : p.acc, rung, E, M, sweep_flips);
            int abort_flag = 0;
            s_ctl[2 * (s & 1)] = CSWAP ? eos_decide_cluster(p, s_cmb, side, rung, E, M, timeout_ns, key, &abort_flag)
                                       : eos_decide(p, side, rung, E, M, timeout_ns, key, &abort_flag);
            if (abort_flag) s_ctl[5] = 1;  // a partner never arrived
        }
        if (PRE) named_barrier(1, NC); else __syncthreads();
        if (s_ctl[5]) continue;  // skip to the next barrier with the producers, then leave
        const int nr = s_ctl[2 * (s & 1)];
        const bool moved = nr != rung;
        if (moved) {
            rung = nr;
            if (!p.tables_in_smem) load_thr(p, s_thr, rung, tid, NC);
            thr_c = thr_row(p, s_thr, rung) + 3 * p.Lmax;
        }
        spec_done = spec;
        if (spec) {
            sumL = sumC = nf = 0;
#pragma unroll
            for (int k = 0; k < 2; ++k)
                if (valid[k]) unit_commit(ev[k], moved ? Fb[k] : Fa[k], sumL, sumC, nf);
        }
        // the next sweep's reads of shared memory (level 1, or a reloaded threshold row) follow
        if (PRE) named_barrier(1, NC); else __syncthreads();
    }
    __syncthreads();
    // no CTA of a path-9 cluster leaves while another may still write its mailboxes (every
    // wait is bounded, so every CTA gets here)
    if (CSWAP) cluster_barrier();
    if (s_ctl[5]) return;  // the last sweep's wait gave up
    flush_acc(p, s_acc, tid, nt);

    if (BITS) {
        uint2* dst = reinterpret_cast<uint2*>(p.spins + (size_t)slot * p.slot_stride);
        for (int x = tid; x < N * (P / 8); x += nt) {
            const uint32_t b = bp[x];
            uint2 v = make_uint2(0u, 0u);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                v.x |= (((b >> k) & 1u) ? 0xFFu : 0x01u) << (8 * k);
                v.y |= (((b >> (k + 4)) & 1u) ? 0xFFu : 0x01u) << (8 * k);
            }
            dst[x] = v;
        }
    } else {
        store_split(p.spins + (size_t)slot * p.slot_stride, sp, N, P, P >> 3, chunk_ginv(P >> 3), tid, nt);
    }
    if (tid == 0) {
        p.E[slot] = E;
        p.M[slot] = M;
        p.rung_of_slot[slot] = rung;
        p.slot_of_rung[rung] = slot;
    }
}

// Path 8, rank 1 of each cluster: the random words of every sweep of chain `slot`, written
// one sweep ahead into rank 0's double buffer through distributed shared memory (the words
// are a function of the chain, the sweep and the update, never of the rung, so they need no
// swap decision). It passes the same cluster barriers as rank 0 (one before the first sweep,
// one per sweep) and leaves after the one at which rank 0 reports that it leaves.
template <int DC>
__device__ void peer_producer(const DevProblem& p, int slot, long long t0, int n_sweeps, unsigned char* smem) {
    cg::cluster_group cluster = cg::this_cluster();
    const int tid = threadIdx.x, nt = blockDim.x;
    const FastLayout L(p, DC, true, false);
    uint32_t* s_items = reinterpret_cast<uint32_t*>(smem + L.items);
    int* s_ctl = reinterpret_cast<int*>(smem + L.ctl);
    uint4* peer_rbuf = cluster.map_shared_rank(reinterpret_cast<uint4*>(smem + L.rbuf), 0);
    const int n_items = 2 * p.N, G = p.P >> 3;
    int lg = 0;
    while ((1 << lg) < G) ++lg;
    const int gmask = (1 << lg) - 1;
    for (int x = tid; x < n_items; x += nt) s_items[x] = p.items[x];
    if (tid == 0) s_ctl[6] = 0;
    const PhiloxKey key = philox_schedule(p.key0, p.key1);
    __syncthreads();
    produce_words(peer_rbuf, (uint32_t)t0, s_items, n_items, G, lg, gmask, tid, nt, (uint32_t)slot, key);
    cluster_barrier();  // release: the words are visible to rank 0 after its wait
    for (int s = 0; s < n_sweeps; ++s) {
        if (s + 1 < n_sweeps)
            produce_words(peer_rbuf + (size_t)((s + 1) & 1) * n_items * G, (uint32_t)(t0 + s + 1), s_items, n_items, G,
                          lg, gmask, tid, nt, (uint32_t)slot, key);
        cluster_barrier();
        if (s_ctl[6]) return;  // rank 0's swap wait gave up; it leaves after this barrier too
    }
}

// Path 8: R clusters of two CTAs; rank 0 sweeps chain (cluster index) with every thread,
// rank 1 produces its random words. The cluster shape is compiled in, and checked on entry
// (both CTAs return before any barrier or remote access if it is not 2).
template <int DC>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(512, 1)
    sweep_peer_kernel(DevProblem p, long long t0, long long q0, int n_sweeps, int sweeps_per_swap,
                      long long timeout_ns, int n_consumer) {
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cluster = cg::this_cluster();
    if (cluster.num_blocks() != 2) {
        if (threadIdx.x == 0) atomicCAS(p.status, 0, PT_ECUDA);
        return;
    }
    const int slot = (int)(blockIdx.x >> 1);
    if (cluster.block_rank() == 0)
        sweep_packed_body<DC, true, false, true, true>(p, slot, t0, q0, n_sweeps, sweeps_per_swap, timeout_ns,
                                                       blockDim.x, smem);
    else
        peer_producer<DC>(p, slot, t0, n_sweeps, smem);
}

template <int DC, bool PRE, int MAXT, bool BITS = false>
__global__ void __launch_bounds__(MAXT, 1)
sweep_packed_kernel(DevProblem p, long long t0, long long q0, int n_sweeps, int sweeps_per_swap,
                    long long timeout_ns, int n_consumer) {
    extern __shared__ __align__(16) unsigned char smem[];
    // the held level-0 units do not fit the 64 registers of a 1024-thread block
    sweep_packed_body<DC, PRE, BITS, (MAXT <= 512)>(p, blockIdx.x, t0, q0, n_sweeps, sweeps_per_swap, timeout_ns,
                                                    n_consumer, smem);
}

// Path 9: one cluster of R CTAs, CTA r sweeping chain r as paths 2 (PRE = false) and 3 do,
// with the swap mailboxes in shared memory. The cluster shape is set at launch and checked
// on entry: if the cluster is not the whole grid, every CTA returns before any cluster
// barrier or remote access.
template <int DC, bool PRE>
__global__ void __launch_bounds__(384, 1)
    sweep_cluster_kernel(DevProblem p, long long t0, long long q0, int n_sweeps, int sweeps_per_swap,
                         long long timeout_ns, int n_consumer) {
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cluster = cg::this_cluster();
    if (cluster.num_blocks() != (unsigned)p.R || gridDim.x != (unsigned)p.R) {
        if (threadIdx.x == 0) atomicCAS(p.status, 0, PT_ECUDA);
        return;
    }
    sweep_packed_body<DC, PRE, false, true, false, true>(p, (int)cluster.block_rank(), t0, q0, n_sweeps,
                                                         sweeps_per_swap, timeout_ns, n_consumer, smem);
}

// Several problems in one cooperative launch (all chains resident at once): block b sweeps
// chain map[b].y of problem map[b].x with the random words computed inline. Swap passes use
// each problem's own mailboxes, so problems never wait for one another.
__global__ void __launch_bounds__(512, 1) sweep_packed_multi_kernel(const MultiProblem* probs, const int2* map) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int2 m = map[blockIdx.x];
    const MultiProblem mp = probs[m.x];
    if (mp.dc == 4)
        sweep_packed_body<4, false>(mp.p, m.y, mp.t0, mp.q0, mp.n_sweeps, mp.sweeps_per_swap, mp.timeout_ns,
                                    blockDim.x, smem);
    else
        sweep_packed_body<8, false>(mp.p, m.y, mp.t0, mp.q0, mp.n_sweeps, mp.sweeps_per_swap, mp.timeout_ns,
                                    blockDim.x, smem);
}

size_t multi_smem_bytes(const DevProblem& p, int dc) { return FastLayout(p, dc, false).total; }

cudaError_t multi_prepare(int threads, size_t smem, int* blocks_per_sm) {
    int dev = 0, max_smem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sweep_packed_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, sweep_packed_multi_kernel, threads, smem);
}

cudaError_t launch_multi(const MultiProblem* probs, const int2* map, int n_blocks, int threads, size_t smem,
                         cudaStream_t s) {
    void* args[] = {(void*)&probs, (void*)&map};
    return cudaLaunchCooperativeKernel((const void*)sweep_packed_multi_kernel, dim3(n_blocks), dim3(threads), args,
                                       smem, s);
}

// ------------------------------------------------------------------------- split sweep
// One chain on a cluster of two CTAs (P % 16 == 0), for ladders short enough that a CTA per
// chain would leave SMs idle. CTA h owns copies [h P/2, (h+1) P/2): W = P/16 four-copy words
// per parity. Updates couple a copy only to its Trotter neighbours k +- 1 (Eq. 3), so the
// only copies a CTA needs from its peer are
//   - the peer's first even word (copies h P/2 + P/2 .. +6): recomputed here every sweep,
//     with the same inputs, random words and order as the peer, so bit for bit the same;
//   - the peer's first odd word and its last odd copy as of the previous sweep, which the
//     recomputed word and the own first even word read; the peer writes them into this
//     CTA's shared memory once per sweep, into one of two buffers by sweep parity.
// Each CTA therefore runs the whole level schedule on 2W + 1 words per site, and the two meet
// once per sweep at a cluster barrier, where they also add their halves of dE, dM and the
// flip count. Both CTAs take the swap decision from the same mailbox values; the first CTA
// alone publishes, counts and writes the chain's statistics.
//
// Row layout (bytes) of site i, RB = 8W + 16 per row:
//   [0, 4W+4)         even words 0..W-1 (own), word W = the peer's first even word
//   [4W+4, 8W+4)      odd words 0..W-1 (own)
//   [8W+4, 8W+12)     the peer's first odd word, previous sweep, buffers 0 and 1
//   [8W+12, 8W+14)    the peer's last odd copy, previous sweep, buffers 0 and 1
// and one row of +1 copies after the last site (the field's h slot).
struct SplitLayout {
    size_t spins, desc, items, loff, thr, acc, red, ctl, xch, rbuf, total;
    int W, RB, Gc;
    __host__ __device__ SplitLayout(const DevProblem& p, int dc, bool pre) {
        const int N = p.N;
        W = p.P / 16;
        RB = 8 * W + 16;
        Gc = W + 1;  // word columns of an even item; odd items use W of them
        size_t o = 0;
        spins = o; o += up16((size_t)(N + 1) * RB);
        desc = o;  o += (size_t)N * (dc == 4 ? 32 : 48);
        items = o; o += up16((size_t)2 * N * 4);
        loff = o;  o += up16((size_t)(p.n_levels + 1) * 4);
        thr = o;   o += thr_bytes(p);
        acc = o;   o += acc_bytes(p);
        red = o;   o += 32 * 3 * 8;
        ctl = o;   o += 32;
        xch = o;   o += 64;  // written by the peer: [sweep parity][dE, dM, flips, abort], final abort
        rbuf = o;
        if (pre) o += (size_t)2 * (2 * N) * Gc * 16;
        total = o;
    }
};

size_t split_smem_bytes(const DevProblem& p, int dclass, bool pre) { return SplitLayout(p, dclass, pre).total; }

// Global copy held at byte c of a split row of CTA h, or -1 for padding.
__device__ __forceinline__ int split_copy(int c, int W, int h, int P) {
    const int hs = 4 * W + 4;
    if (c < hs) return 8 * ((h * W + (c >> 2)) % (2 * W)) + 2 * (c & 3);
    if (c < 8 * W + 4) return 8 * (h * W + ((c - hs) >> 2)) + 2 * (c & 3) + 1;
    if (c < 8 * W + 12) return 8 * (((h + 1) * W) % (2 * W)) + 2 * (c & 3) + 1;
    if (c < 8 * W + 14) return (8 * h * W - 1 + P) % P;
    return -1;
}

// Offsets of column g's reads (see UnitOffsets) while the peer's previous-sweep copies sit
// in buffer b.
__device__ __forceinline__ UnitOffsets split_offsets(int g, int W, int b) {
    const uint32_t hs = 4u * W + 4u, w4 = 4u * (uint32_t)g;
    UnitOffsets o;
    o.own[0] = w4;
    o.own[1] = hs + w4;
    o.opp[0] = g < W ? hs + w4 : 8u * W + 4u + 4u * (uint32_t)b;
    o.opp[1] = w4;
    o.edge[0] = g >= 1 ? hs + w4 - 1u : 8u * W + 12u + (uint32_t)b;
    o.edge[1] = w4 + 4u;
    return o;
}

template <int DC, bool PRE>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(512, 1)
sweep_split_kernel(DevProblem p, long long t0, long long q0, int n_sweeps, int sweeps_per_swap,
                   long long timeout_ns, int n_consumer) {
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cluster = cg::this_cluster();
    // the cluster shape is compiled in; should a launch ever run without it, no CTA touches
    // a peer's shared memory or waits at a cluster barrier
    if (cluster.num_blocks() != 2) {
        if (threadIdx.x == 0) atomicCAS(p.status, 0, PT_ECUDA);
        return;
    }
    const int h = (int)cluster.block_rank();
    const bool lead = h == 0;
    const int slot = blockIdx.x >> 1;
    const int N = p.N, P = p.P;
    const int tid = threadIdx.x, nt = blockDim.x;
    const SplitLayout L(p, DC, PRE);
    const int W = L.W, RB = L.RB, Gc = L.Gc;
    const int hs = 4 * W + 4;
    int8_t* sp = reinterpret_cast<int8_t*>(smem + L.spins);
    uint32_t* s_desc = reinterpret_cast<uint32_t*>(smem + L.desc);
    uint32_t* s_items = reinterpret_cast<uint32_t*>(smem + L.items);
    int32_t* s_loff = reinterpret_cast<int32_t*>(smem + L.loff);
    uint32_t* s_thr = reinterpret_cast<uint32_t*>(smem + L.thr);
    long long* s_red = reinterpret_cast<long long*>(smem + L.red);
    int* s_ctl = reinterpret_cast<int*>(smem + L.ctl);
    int* s_xch = reinterpret_cast<int*>(smem + L.xch);
    uint4* rbuf = reinterpret_cast<uint4*>(smem + L.rbuf);
    unsigned long long* s_acc = reinterpret_cast<unsigned long long*>(smem + L.acc);
    int8_t* peer_sp = cluster.map_shared_rank(sp, h ^ 1);
    int* peer_xch = cluster.map_shared_rank(s_xch, h ^ 1);
    const int NC = PRE ? n_consumer : nt;
    const bool consumer = tid < NC;
    const int DW = SiteDesc<DC>::DW;

    {
        const int8_t* src = p.spins + (size_t)slot * p.slot_stride;
        for (int x = tid; x < N * RB; x += nt) {
            const int i = x / RB, c = x - i * RB;
            const int k = split_copy(c, W, h, P);
            sp[x] = k >= 0 ? src[(size_t)i * P + k] : (int8_t)0;
        }
        for (int x = tid; x < RB; x += nt) sp[(size_t)N * RB + x] = 1;
        // descriptors with the row offsets rescaled from P to RB bytes per row
        const uint32_t NP = (uint32_t)N * (uint32_t)P;
        for (int x = tid; x < N * DW; x += nt) {
            const int f = x % DW;
            uint32_t v = p.desc[x];
            if (f == 0 || f >= 4) v = v >= NP ? (uint32_t)N * RB : (v / (uint32_t)P) * (uint32_t)RB;
            s_desc[x] = v;
        }
        for (int x = tid; x < 2 * N; x += nt) s_items[x] = p.items[x];
        for (int x = tid; x <= p.n_levels; x += nt) s_loff[x] = p.level_off[x];
        for (int x = tid; x < 16; x += nt) s_xch[x] = 0;
    }
    int rung = p.rung_of_slot[slot];
    load_thr(p, s_thr, rung, tid, nt);
    if (p.acc_in_smem)
        for (int x = tid; x < p.R * kAccCount; x += nt) s_acc[x] = 0ull;
    long long E = p.E[slot], M = p.M[slot];  // meaningful in thread 0 only

    const PhiloxKey key = philox_schedule(p.key0, p.key1);
    const uint32_t* thr_c = thr_row(p, s_thr, rung) + 3 * p.Lmax;
    const int n_items = 2 * N;
    const int lane = tid & 31;
    if (tid == 0) {
        s_ctl[4] = -1;  // partner rung of the pending swap pass
        s_ctl[5] = 0;   // this CTA's swap wait gave up
        s_ctl[6] = 0;   // either CTA's wait gave up (known at the last cluster barrier)
        int* s_sum = reinterpret_cast<int*>(s_red);
        s_sum[0] = s_sum[1] = s_sum[2] = 0;
    }
    // every CTA of the cluster is running and initialised before any shared-memory exchange
    cluster_barrier();

    // random words of sweep t for this CTA's columns (global chunk (hW + g) mod 2W)
    auto produce = [&](uint4* buf, uint32_t t) {
        const int ptid = tid - NC, np = nt - NC;
        const int pg = ptid % Gc, pstep = np / Gc;
        if (ptid / Gc >= pstep) return;
        const uint32_t gg = (uint32_t)((h * W + pg) % (2 * W));
        for (int q = ptid / Gc; q < n_items; q += pstep) {
            const uint32_t it = s_items[q];
            if ((it & 1u) && pg == W) continue;
            const uint4 r = philox(make_uint4(t, it >> 1, (uint32_t)slot, ((it & 1u) << 24) | gg), key);
            buf[q * Gc + pg] = make_uint4(min(r.x, 0xFFFFFFFEu), min(r.y, 0xFFFFFFFEu), min(r.z, 0xFFFFFFFEu),
                                          min(r.w, 0xFFFFFFFEu));
        }
    };
    if (PRE && !consumer) produce(rbuf, (uint32_t)t0);
    __syncthreads();

    // consumers: a fixed column g_own per thread, items q_lane, q_lane + q_step, ... of a level
    const int g_own = tid % Gc, q_lane = tid / Gc, q_step = NC / Gc;
    const bool lane_ok = consumer && q_lane < q_step;
    const bool ghost_col = g_own == W;  // the recomputed peer word: its flips are the peer's
    const uint32_t gg_own = (uint32_t)((h * W + g_own) % (2 * W));  // its chunk in the whole chain
    // level 0 of the next sweep during the swap wait: units v, v + (NC - 32) of the level
    // (v = tid - 32), so that warp 0 is free to poll the partner's mailbox
    const int units0 = (s_loff[1] - s_loff[0]) * Gc;
    const bool spec_ok = p.tables_in_smem && NC > 32 && units0 <= 2 * (NC - 32);
    int sq[2], sg[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int u = (tid - 32) + k * (NC - 32);
        sg[k] = u % Gc;
        sq[k] = (tid >= 32 && consumer && u < units0) ? s_loff[0] + u / Gc : -1;
    }
    bool spec_done = false;
    int lL = 0, lC = 0, lF = 0;  // this sweep's own units in the levels (counts twice, see unit_commit)
    int pL = 0, pC = 0, pF = 0;  // the level-0 units applied early
    SwapSide side;
    side.active = 0;
    const uint32_t qmod0 = (uint32_t)(q0 % kTagPeriod);
    int since_pass = 0, next_pass = 0;  // thread 0
    long long sE = 0, sM = 0, sF = 0;   // thread 0: this CTA's half of the sweep's changes

    for (int s = 0; s < n_sweeps; ++s) {
        const uint32_t t = (uint32_t)(t0 + s);
        const int b = s & 1;
        const bool dead = (s_ctl[5] | s_ctl[6]) != 0;
        if (consumer) {
            if (!dead) {
                const uint4* rb = rbuf + (size_t)b * n_items * Gc;
                const UnitOffsets off = split_offsets(g_own, W, b);
                if (!spec_done) pL = pC = pF = 0;
                lL = lC = lF = 0;
                for (int lev = spec_done ? 1 : 0; lev < p.n_levels; ++lev) {
                    if (lane_ok) {
                        const int end = s_loff[lev + 1];
                        for (int q = s_loff[lev] + q_lane; q < end; q += q_step) {
                            const uint32_t it = s_items[q];
                            if (ghost_col && (it & 1u)) continue;
                            const UnitEval e = split_unit_eval<DC, PRE>(sp, s_desc, it, rb + q * Gc + g_own, off, t,
                                                                        (uint32_t)slot, gg_own, key);
                            unit_decide_commit<PRE>(e, thr_c, lL, lC, lF);
                        }
                    }
                    named_barrier(1, NC);
                }
                if (ghost_col) lL = lC = lF = 0;
                const int mL = lL + pL, mC = lC + pC, mF = lF + pF;
                const int dE = __reduce_add_sync(0xFFFFFFFFu, -2 * mL);
                const int dM = __reduce_add_sync(0xFFFFFFFFu, -2 * (mC - mF));
                const int dF = __reduce_add_sync(0xFFFFFFFFu, mF) >> 1;
                int* s_sum = reinterpret_cast<int*>(s_red);
                if (lane == 0) {
                    atomicAdd(s_sum + 0, dE);
                    atomicAdd(s_sum + 1, dM);
                    atomicAdd(s_sum + 2, dF);
                }
                named_barrier(1, NC);
                // the peer's next sweep reads this sweep's first odd word and last odd copy
                const int bn = b ^ 1;
                for (int i = tid; i < N; i += NC) {
                    const int8_t* r = sp + (size_t)i * RB;
                    int8_t* pr = peer_sp + (size_t)i * RB;
                    *reinterpret_cast<uint32_t*>(pr + 8 * W + 4 + 4 * bn) = *reinterpret_cast<const uint32_t*>(r + hs);
                    pr[8 * W + 12 + bn] = r[hs + 4 * W - 1];
                }
            }
            if (tid == 0) {
                int* s_sum = reinterpret_cast<int*>(s_red);
                sE = s_sum[0];
                sM = s_sum[1];
                sF = s_sum[2];
                s_sum[0] = s_sum[1] = s_sum[2] = 0;
                int* x = peer_xch + 4 * b;
                x[0] = (int)sE;
                x[1] = (int)sM;
                x[2] = (int)sF;
                x[3] = s_ctl[5];
            }
        } else if (PRE && !dead && s + 1 < n_sweeps) {
            produce(rbuf + (size_t)(b ^ 1) * n_items * Gc, t + 1u);
        }
        // both halves of the sweep are done, the exchanged words and sums are visible and
        // the next sweep's random words are complete
        cluster_barrier();
        if (tid == 0) {
            const int* x = s_xch + 4 * b;
            if (x[3] || s_ctl[5]) s_ctl[6] = 1;
            if (!s_ctl[6]) {
                int pass = -1;
                if (sweeps_per_swap > 0 && ++since_pass == sweeps_per_swap) {
                    since_pass = 0;
                    pass = next_pass++;
                }
                side = eos_publish(p, rung, E, M, sE + x[0], sM + x[1], pass, q0, qmod0, lead);
                sF += x[2];
                s_ctl[4] = side.active ? side.partner : -1;
            }
        }
        __syncthreads();
        if (s_ctl[6] || !consumer) continue;

        // level 0 of sweep s + 1 under both candidate rungs
        const bool spec = spec_ok && s + 1 < n_sweeps;
        const int prung = s_ctl[4];
        UnitEval ev[2];
        uint32_t Fa[2] = {0u, 0u}, Fb[2] = {0u, 0u};
        bool valid[2] = {false, false};
        if (spec) {
            const uint4* rb1 = rbuf + (size_t)(b ^ 1) * n_items * Gc;
            const uint32_t* thr_b = prung >= 0 ? thr_row(p, s_thr, prung) + 3 * p.Lmax : thr_c;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (sq[k] < 0) continue;
                const uint32_t it = s_items[sq[k]];
                valid[k] = !((it & 1u) && sg[k] == W);
                if (valid[k]) {
                    ev[k] = split_unit_eval<DC, PRE>(sp, s_desc, it, rb1 + sq[k] * Gc + sg[k],
                                                     split_offsets(sg[k], W, b ^ 1), t + 1u, (uint32_t)slot,
                                                     (uint32_t)((h * W + sg[k]) % (2 * W)), key);
                    Fa[k] = unit_flips<PRE>(ev[k], thr_c);
                    Fb[k] = prung >= 0 ? unit_flips<PRE>(ev[k], thr_b) : Fa[k];
                }
            }
        }
        if (tid == 0) {
            if (lead) eos_stats(p, p.acc_in_smem ? s_acc : p.acc, rung, E, M, sF);
            int abort_flag = 0;
            s_ctl[2 * b] = eos_decide(p, side, rung, E, M, timeout_ns, key, &abort_flag, lead);
            if (abort_flag) s_ctl[5] = 1;
        }
        named_barrier(1, NC);
        if (s_ctl[5]) continue;  // the next sweep is skipped; the cluster barriers go on
        const int nr = s_ctl[2 * b];
        const bool moved = nr != rung;
        if (moved) {
            rung = nr;
            if (!p.tables_in_smem) load_thr(p, s_thr, rung, tid, NC);
            thr_c = thr_row(p, s_thr, rung) + 3 * p.Lmax;
        }
        spec_done = spec;
        if (spec) {
            pL = pC = pF = 0;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (!valid[k]) continue;
                int jL = 0, jC = 0, jF = 0;
                unit_commit(ev[k], moved ? Fb[k] : Fa[k], jL, jC, jF);
                if (sg[k] != W) {
                    pL += jL;
                    pC += jC;
                    pF += jF;
                }
            }
        }
        named_barrier(1, NC);
    }
    // both CTAs agree whether a swap wait gave up before either writes anything back
    if (tid == 0) peer_xch[8] = s_ctl[5] | s_ctl[6];
    cluster_barrier();
    if (tid == 0 && (s_xch[8] || s_ctl[5] || s_ctl[6])) s_ctl[6] = 1;
    __syncthreads();
    if (s_ctl[6]) return;
    if (lead) flush_acc(p, s_acc, tid, nt);
    {
        int8_t* dst = p.spins + (size_t)slot * p.slot_stride;
        for (int x = tid; x < N * RB; x += nt) {
            const int i = x / RB, c = x - i * RB;
            if (c < 4 * W || (c >= hs && c < hs + 4 * W)) dst[(size_t)i * P + split_copy(c, W, h, P)] = sp[x];
        }
    }
    if (tid == 0 && lead) {
        p.E[slot] = E;
        p.M[slot] = M;
        p.rung_of_slot[slot] = rung;
        p.slot_of_rung[rung] = slot;
    }
}

// ------------------------------------------------------------------------- init / energy
// Initial spins: copy k of site i of chain rho is -1 iff bit 31 of word k%4 of
// philox((0, i, rho, INIT<<28 | k/4)) is set.
__global__ void init_kernel(DevProblem p) {
    const int slot = blockIdx.x;
    const int P4 = (p.P + 3) >> 2;
    const PhiloxKey key = philox_schedule(p.key0, p.key1);
    int8_t* dst = p.spins + (size_t)slot * p.slot_stride;
    for (int x = threadIdx.x; x < p.N * P4; x += blockDim.x) {
        const int i = x / P4, g4 = x - i * P4;
        const uint4 u = philox(make_uint4(0u, (uint32_t)i, (uint32_t)slot, (kTagInit << 28) | (uint32_t)g4), key);
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int k = 4 * g4 + b;
            if (k < p.P) dst[(size_t)i * p.P + k] = (w[b] >> 31) ? (int8_t)-1 : (int8_t)1;
        }
    }
    if (threadIdx.x == 0) {
        p.rung_of_slot[slot] = slot;
        p.slot_of_rung[slot] = slot;
    }
}

// E = sum_k E(s^k) and M = sum_k sum_i s_i^k s_i^{k+1} of every chain from scratch.
__global__ void energy_kernel(DevProblem p) {
    __shared__ long long red[2][32];
    const int slot = blockIdx.x;
    const int8_t* sp = p.spins + (size_t)slot * p.slot_stride;
    long long e = 0, m = 0;
    for (int x = threadIdx.x; x < p.N * p.P; x += blockDim.x) {
        const int i = x / p.P, k = x - i * p.P;
        const int si = sp[x];
        int f = p.h[i];
        for (int d = 0; d < p.dmax; ++d) {
            const uint32_t e8 = p.nbr[(size_t)i * p.dmax + d];
            const int j = (int)(e8 >> 8);
            if (j > i) f += (int)(int8_t)(e8 & 0xFFu) * (int)sp[(size_t)j * p.P + k];
        }
        e += (long long)si * f;
        m += (long long)si * sp[(size_t)i * p.P + ((k + 1 == p.P) ? 0 : k + 1)];
    }
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_xor_sync(0xFFFFFFFFu, e, o);
        m += __shfl_xor_sync(0xFFFFFFFFu, m, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][warp] = e;
        red[1][warp] = m;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long se = 0, sm = 0;
        for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) {
            se += red[0][w];
            sm += red[1][w];
        }
        p.E[slot] = se;
        p.M[slot] = sm;
    }
}

// ------------------------------------------------------------------------- swap / copies
// One swap pass q with chains in place (state already in global memory).
__global__ void swap_kernel(DevProblem p, long long q) {
    const PhiloxKey key = philox_schedule(p.key0, p.key1);
    for (int rl = (int)(q & 1) + 2 * (int)threadIdx.x; rl + 1 < p.R; rl += 2 * (int)blockDim.x) {
        const int X = p.slot_of_rung[rl], Y = p.slot_of_rung[rl + 1];
        const bool acc = swap_accept_fast(p.E[X], p.E[Y], p.M[X], p.M[Y], p.coef[rl], p.coef[(p.R - 1) + rl],
                                          (uint32_t)q, (uint32_t)rl, key, p.exact_swaps != 0);
        p.swap_stats[2 * rl] += 1ull;
        if (acc) {
            p.swap_stats[2 * rl + 1] += 1ull;
            p.slot_of_rung[rl] = Y;
            p.slot_of_rung[rl + 1] = X;
            p.rung_of_slot[X] = rl + 1;
            p.rung_of_slot[Y] = rl;
        }
    }
}

__global__ void gather_kernel(DevProblem p, int8_t* out) {
    const int r = blockIdx.x;
    const int8_t* src = p.spins + (size_t)p.slot_of_rung[r] * p.slot_stride;
    int8_t* dst = out + (size_t)r * p.N * p.P;
    const int n = p.N * p.P;
    if ((n & 15) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
        // 16 bytes a thread: chains start on 16-byte boundaries (slot_stride), and so does
        // every rung's output row when a chain is a whole number of 16-byte words
        const uint4* s4 = reinterpret_cast<const uint4*>(src);
        uint4* d4 = reinterpret_cast<uint4*>(dst);
        for (int x = threadIdx.x; x < (n >> 4); x += blockDim.x) d4[x] = s4[x];
    } else {
        for (int x = threadIdx.x; x < n; x += blockDim.x) dst[x] = src[x];
    }
}

__global__ void scatter_kernel(DevProblem p, const int8_t* in) {
    const int r = blockIdx.x;
    int8_t* dst = p.spins + (size_t)p.slot_of_rung[r] * p.slot_stride;
    const int8_t* src = in + (size_t)r * p.N * p.P;
    for (int x = threadIdx.x; x < p.N * p.P; x += blockDim.x) dst[x] = src[x];
}

// ------------------------------------------------------------------------- launchers
static const void* sweep_fn(const LaunchPlan& plan) {
    if (plan.path == kPathClassical) {
        switch (plan.dclass) {
            case 4: return (const void*)sweep_classical_kernel<4>;
            case 8: return (const void*)sweep_classical_kernel<8>;
            default: return (const void*)sweep_classical_kernel<32>;
        }
    }
    if (plan.path == kPathGeneric) {
        switch (plan.dclass) {
            case 4: return (const void*)sweep_kernel<4>;
            case 8: return (const void*)sweep_kernel<8>;
            default: return (const void*)sweep_kernel<32>;
        }
    }
    if (plan.path == kPathPeer)
        return plan.dclass == 4 ? (const void*)sweep_peer_kernel<4> : (const void*)sweep_peer_kernel<8>;
    if (plan.path == kPathCluster) {
        const bool pre = plan.n_consumer < plan.threads;
        if (plan.dclass == 4)
            return pre ? (const void*)sweep_cluster_kernel<4, true> : (const void*)sweep_cluster_kernel<4, false>;
        return pre ? (const void*)sweep_cluster_kernel<8, true> : (const void*)sweep_cluster_kernel<8, false>;
    }
    if (plan.path == kPathSplit)
        return plan.dclass == 4 ? (const void*)sweep_split_kernel<4, true> : (const void*)sweep_split_kernel<8, true>;
    if (plan.path == kPathSplitInline)
        return plan.dclass == 4 ? (const void*)sweep_split_kernel<4, false> : (const void*)sweep_split_kernel<8, false>;
    if (plan.path == kPathBits) {
        if (plan.threads > 512)
            return plan.dclass == 4 ? (const void*)sweep_packed_kernel<4, false, 1024, true>
                                    : (const void*)sweep_packed_kernel<8, false, 1024, true>;
        return plan.dclass == 4 ? (const void*)sweep_packed_kernel<4, false, 512, true>
                                : (const void*)sweep_packed_kernel<8, false, 512, true>;
    }
    const bool pre = plan.path == kPathPacked;
    if (plan.threads > 512) {
        if (plan.dclass == 4)
            return pre ? (const void*)sweep_packed_kernel<4, true, 1024> : (const void*)sweep_packed_kernel<4, false, 1024>;
        return pre ? (const void*)sweep_packed_kernel<8, true, 1024> : (const void*)sweep_packed_kernel<8, false, 1024>;
    }
    if (!pre && plan.threads <= 384)
        // blocks of at most 384 threads may use up to 168 registers per thread
        return plan.dclass == 4 ? (const void*)sweep_packed_kernel<4, false, 384>
                                : (const void*)sweep_packed_kernel<8, false, 384>;
    if (plan.dclass == 4)
        return pre ? (const void*)sweep_packed_kernel<4, true, 512> : (const void*)sweep_packed_kernel<4, false, 512>;
    return pre ? (const void*)sweep_packed_kernel<8, true, 512> : (const void*)sweep_packed_kernel<8, false, 512>;
}

// The dynamic shared-memory limit is a per-function attribute shared by every context, so
// it is raised once to the device's opt-in maximum rather than to one context's size.
cudaError_t prepare_sweep_kernel(const LaunchPlan& plan) {
    int dev = 0, max_smem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (plan.path == kPathCluster || plan.path == kPathClassical) {
        // clusters of up to 16 CTAs (above 8 is a non-portable size)
        e = cudaFuncSetAttribute(sweep_fn(plan), cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    return cudaFuncSetAttribute(sweep_fn(plan), cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
}

cudaError_t sweep_kernel_occupancy(const DevProblem& p, const LaunchPlan& plan, int* blocks_per_sm) {
    (void)p;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, sweep_fn(plan), plan.threads,
                                                         plan.smem_bytes);
}

// The split kernel's launch: R clusters of two CTAs (the cluster shape is compiled into the
// kernel); cooperative when swap passes run inside.
static cudaLaunchConfig_t split_config(const DevProblem& p, const LaunchPlan& plan, bool cooperative,
                                       cudaStream_t s, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * p.R);
    cfg.blockDim = dim3(plan.threads);
    cfg.dynamicSmemBytes = plan.smem_bytes;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = cooperative ? 1 : 0;
    return cfg;
}

// Path 9's launch: one cluster of all R CTAs; path 10's: one cluster of ceil(R / C) CTAs.
static cudaLaunchConfig_t cluster_config(const DevProblem& p, const LaunchPlan& plan, cudaStream_t s,
                                         cudaLaunchAttribute* attr) {
    const int ctas = plan.path == kPathClassical ? (p.R + plan.chains_per_cta - 1) / plan.chains_per_cta : p.R;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(plan.threads);
    cfg.dynamicSmemBytes = plan.smem_bytes;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

cudaError_t sweep_resident_chains(const DevProblem& p, const LaunchPlan& plan, long long* chains) {
    *chains = 0;
    if (plan.path == kPathCluster || plan.path == kPathClassical) {
        const int ctas = plan.path == kPathClassical ? (p.R + plan.chains_per_cta - 1) / plan.chains_per_cta : p.R;
        if (ctas > 16) return cudaSuccess;
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = cluster_config(p, plan, 0, attr);
        int clusters = 0;
        cudaError_t e = cudaOccupancyMaxActiveClusters(&clusters, sweep_fn(plan), &cfg);
        if (e == cudaSuccess) *chains = (long long)clusters * p.R;
        return e;
    }
    if (plan.path == kPathSplit || plan.path == kPathSplitInline || plan.path == kPathPeer) {
        cudaLaunchAttribute attr[2];
        cudaLaunchConfig_t cfg = split_config(p, plan, false, 0, attr);
        int clusters = 0;
        cudaError_t e = cudaOccupancyMaxActiveClusters(&clusters, sweep_fn(plan), &cfg);
        if (e == cudaSuccess) *chains = clusters;
        return e;
    }
    int dev = 0, n_sm = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = sweep_kernel_occupancy(p, plan, &per_sm);
    if (e == cudaSuccess) *chains = (long long)per_sm * n_sm;
    return e;
}

cudaError_t launch_sweeps(const DevProblem& p, const LaunchPlan& plan, long long t0, long long q0,
                          int n_sweeps, int sweeps_per_swap, long long timeout_ns, bool cooperative,
                          cudaStream_t s) {
    DevProblem pp = p;
    // the last argument: consumer threads, or (path 10) chains per CTA
    int n_consumer = plan.path == kPathClassical ? plan.chains_per_cta : plan.n_consumer;
    void* args[] = {&pp, &t0, &q0, &n_sweeps, &sweeps_per_swap, &timeout_ns, &n_consumer};
    const void* fn = sweep_fn(plan);
    if (plan.path == kPathCluster || plan.path == kPathClassical) {
        // one cluster holds every chain, so the swap passes never need a cooperative launch
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = cluster_config(p, plan, s, attr);
        const cudaError_t e = cudaLaunchKernelExC(&cfg, fn, args);
        if (e != cudaSuccess) (void)cudaGetLastError();
        return e;
    }
    if (plan.path == kPathSplit || plan.path == kPathSplitInline || plan.path == kPathPeer) {
        cudaLaunchAttribute attr[2];
        cudaLaunchConfig_t cfg = split_config(p, plan, cooperative, s, attr);
        const cudaError_t e = cudaLaunchKernelExC(&cfg, fn, args);
        if (e != cudaSuccess) (void)cudaGetLastError();  // a rejected launch leaves no error for the next one
        return e;
    }
    if (cooperative)
        return cudaLaunchCooperativeKernel(fn, dim3(p.R), dim3(plan.threads), args, plan.smem_bytes, s);
    return cudaLaunchKernel(fn, dim3(p.R), dim3(plan.threads), args, plan.smem_bytes, s);
}

cudaError_t launch_init(const DevProblem& p, cudaStream_t s) {
    init_kernel<<<p.R, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_energy(const DevProblem& p, cudaStream_t s) {
    energy_kernel<<<p.R, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_swap(const DevProblem& p, long long q, cudaStream_t s) {
    swap_kernel<<<1, 256, 0, s>>>(p, q);
    return cudaGetLastError();
}

cudaError_t launch_gather_state(const DevProblem& p, int8_t* out, cudaStream_t s) {
    gather_kernel<<<p.R, 256, 0, s>>>(p, out);
    return cudaGetLastError();
}

cudaError_t launch_scatter_state(const DevProblem& p, const int8_t* in, cudaStream_t s) {
    scatter_kernel<<<p.R, 256, 0, s>>>(p, in);
    return cudaGetLastError();
}

}  // namespace ptq
