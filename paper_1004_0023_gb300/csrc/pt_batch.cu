// pt_batch.cu -- many independent PT-QMC problems in one persistent launch.
//
// Each thread-block cluster pulls a whole problem from a work counter (problems sorted by
// work, largest first) and owns it until every sweep is done: CTA r of the cluster sweeps
// chains [r*C, (r+1)*C), C = ceil(R / cluster). Within a CTA the chains are "packed" onto
// groups of threads (the paper's chain packing, Sec. 5): a group sweeps one chain at a time
// with the same level schedule, random-number counters and 4-copy update unit as the
// single-problem kernel, so every problem gets exactly the bits it would get alone. For a
// swap pass the CTAs publish (E, M) of their chains in shared memory, meet at one cluster
// barrier, and each CTA evaluates every pair's decision from the peers' shared memory
// (the same inputs everywhere give the same rung permutation everywhere). No CTA ever waits
// for another cluster, so the persistent launch needs no co-residency guarantee beyond
// the cluster's own.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "pt.h"
#include "pt_device.cuh"
#include "pt_internal.h"

namespace cg = cooperative_groups;

namespace ptq {

// Shared memory of one CTA while it owns problem I.
struct BatchLayout {
    size_t sdesc, items, loff, rung, slot, E, M, pub, thr, red, chains, total;
    int C, ngroups, chain_stride, nbufs, DW, thr_words;
    __host__ __device__ BatchLayout(const BatchInstance& I, int K, int threads) {
        DW = I.dc == 4 ? 8 : 12;
        C = (I.R + K - 1) / K;
        ngroups = threads / I.group_threads;
        chain_stride = (int)(up16((size_t)I.slot_stride) + up16((size_t)I.P));
        nbufs = I.resident ? C : ngroups;
        thr_words = (int)(up16((size_t)I.nL3 * 4) / 4);
        size_t o = 0;
        sdesc = o;  o += (size_t)I.N * DW * 4;
        items = o;  o += up16((size_t)2 * I.N * 4);
        loff = o;   o += up16((size_t)(I.n_levels + 1) * 4);
        rung = o;   o += up16((size_t)I.R * 4);
        slot = o;   o += up16((size_t)I.R * 4);
        E = o;      o += up16((size_t)C * 8);
        M = o;      o += up16((size_t)C * 8);
        pub = o;    o += (size_t)2 * C * 16;
        thr = o;    o += (size_t)(I.thr_resident ? I.R : ngroups) * thr_words * 4;
        red = o;    o += up16((size_t)ngroups * (I.group_threads / 32) * 3 * 8);
        chains = o; o += (size_t)nbufs * chain_stride;
        total = o;
    }
};

size_t batch_smem_bytes(const BatchInstance& I, int cluster, int threads) {
    return BatchLayout(I, cluster, threads).total;
}

// A chain group's barrier: a named barrier of its warps, or just the warp for one-warp groups.
__device__ __forceinline__ void group_sync(int bar, int gsize) {
    if (gsize == 32)
        __syncwarp();
    else
        named_barrier(bar, gsize);
}

template <int DC>
__device__ void run_problem(const BatchInstance& I, unsigned char* smem, uint4* s_keys, cg::cluster_group& cluster,
                            int rank, int K) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const BatchLayout L(I, K, nt);
    uint32_t* s_sdesc = reinterpret_cast<uint32_t*>(smem + L.sdesc);
    uint32_t* s_items = reinterpret_cast<uint32_t*>(smem + L.items);
    int32_t* s_loff = reinterpret_cast<int32_t*>(smem + L.loff);
    int32_t* s_rung = reinterpret_cast<int32_t*>(smem + L.rung);
    int32_t* s_slot = reinterpret_cast<int32_t*>(smem + L.slot);
    long long* s_E = reinterpret_cast<long long*>(smem + L.E);
    long long* s_M = reinterpret_cast<long long*>(smem + L.M);
    longlong2* s_pub = reinterpret_cast<longlong2*>(smem + L.pub);
    uint32_t* s_thr = reinterpret_cast<uint32_t*>(smem + L.thr);
    long long* s_red = reinterpret_cast<long long*>(smem + L.red);
    unsigned char* s_chains = smem + L.chains;

    const int N = I.N, P = I.P, R = I.R, C = L.C;
    const int c_begin = rank * C;
    const int c_count = max(0, min(C, R - c_begin));
    const int gsize = I.group_threads, ngroups = L.ngroups;
    const int grp = tid / gsize, gtid = tid - grp * gsize;

    // ---- the problem's schedule, descriptors, round keys and rung permutation; this CTA's chains
    {
        if (tid < 10)
            reinterpret_cast<uint2*>(s_keys)[tid] =
                make_uint2(I.key0 + (uint32_t)tid * 0x9E3779B9u, I.key1 + (uint32_t)tid * 0xBB67AE85u);
        const int4* src = reinterpret_cast<const int4*>(I.sdesc);
        int4* dst = reinterpret_cast<int4*>(s_sdesc);
        for (int x = tid; x < N * L.DW / 4; x += nt) dst[x] = src[x];
        for (int x = tid; x < 2 * N; x += nt) s_items[x] = I.items[x];
        for (int x = tid; x <= I.n_levels; x += nt) s_loff[x] = I.level_off[x];
        for (int x = tid; x < R; x += nt) {
            s_rung[x] = I.rung_of_slot[x];
            s_slot[x] = I.slot_of_rung[x];
        }
        for (int x = tid; x < c_count; x += nt) {
            s_E[x] = I.E[c_begin + x];
            s_M[x] = I.M[c_begin + x];
        }
        if (I.thr_resident)  // every rung's row, so a chain never reloads one after a swap
            for (int x = tid; x < I.R * L.thr_words; x += nt) {
                const int r = x / L.thr_words, c = x - r * L.thr_words;
                s_thr[x] = c < I.nL3 ? I.thr[(size_t)r * I.nL3 + c] : 0u;
            }
        for (int b = 0; b < L.nbufs; ++b) {
            int8_t* ones = reinterpret_cast<int8_t*>(s_chains + (size_t)b * L.chain_stride + I.slot_stride);
            for (int x = tid; x < P; x += nt) ones[x] = 1;
        }
        if (I.resident) {
            for (int lc = 0; lc < c_count; ++lc)
                load_split(reinterpret_cast<int8_t*>(s_chains + (size_t)lc * L.chain_stride),
                           I.spins + (size_t)(c_begin + lc) * I.slot_stride, N, P, P >> 3, chunk_ginv(P >> 3), tid,
                           nt);
        }
    }
    __syncthreads();

    const PhiloxKeyShared skey{s_keys};  // update units and swap decisions: round keys in shared memory
    const int G = P >> 3;
    const uint32_t ginv = chunk_ginv(G);
    const bool p16 = (P & 15) == 0;  // streamed chains move 16 copies per load and store
    const uint32_t hinv = chunk_ginv(P >> 4);
    int lg = 0;
    while ((1 << lg) < G) ++lg;
    const int gmask = (1 << lg) - 1;
    const int bar = 1 + grp;
    uint32_t* thr_g = s_thr + (size_t)grp * L.thr_words;
    long long* red_g = s_red + (size_t)grp * (gsize / 32) * 3;
    const int lane = tid & 31, gwarp = gtid >> 5;
    const bool g_fixed = (gsize & gmask) == 0;
    const int g_own = gtid & gmask, q_lane = gtid >> lg, q_step = gsize >> lg;

    for (int s = 0; s < I.n_sweeps; ++s) {
        const uint32_t t = (uint32_t)(I.t0 + s);
        for (int lc = grp < ngroups ? grp : c_count; lc < c_count; lc += ngroups) {  // threads past the last group idle
            const int rho = c_begin + lc;
            int8_t* buf = reinterpret_cast<int8_t*>(s_chains + (size_t)(I.resident ? lc : grp) * L.chain_stride);
            if (!I.resident) {
                if (p16)
                    load_split16(buf, I.spins + (size_t)rho * I.slot_stride, N, P, P >> 4, hinv, gtid, gsize);
                else
                    load_split(buf, I.spins + (size_t)rho * I.slot_stride, N, P, G, ginv, gtid, gsize);
            }
            const int rung = s_rung[rho];
            const uint32_t* thr_c;
            if (I.thr_resident) {
                thr_c = s_thr + (size_t)rung * L.thr_words + 3 * I.Lmax;
                if (!I.resident) group_sync(bar, gsize);  // the streamed chain is in place
            } else {
                for (int x = gtid; x < I.nL3; x += gsize) thr_g[x] = I.thr[(size_t)rung * I.nL3 + x];
                group_sync(bar, gsize);
                thr_c = thr_g + 3 * I.Lmax;
            }
            int sumL = 0, sumC = 0, nf = 0;  // sumC and nf count twice (see unit_commit)
            for (int lev = 0; lev < I.n_levels; ++lev) {
                const int base = s_loff[lev];
                if (g_fixed) {
                    // this thread's column g never changes (see the single-problem kernel)
                    if (g_own < G) {
                        const int end = s_loff[lev + 1];
                        for (int q = base + q_lane; q < end; q += q_step)
                            packed_unit<DC, false>(buf, s_sdesc, s_items[q], nullptr, q, g_own, G, P, t,
                                                   (uint32_t)rho, skey, thr_c, sumL, sumC, nf);
                    }
                } else {
                    const int units = (s_loff[lev + 1] - base) << lg;
                    for (int u = gtid; u < units; u += gsize) {
                        const int g = u & gmask;
                        if (g >= G) continue;
                        const int q = base + (u >> lg);
                        packed_unit<DC, false>(buf, s_sdesc, s_items[q], nullptr, q, g, G, P, t, (uint32_t)rho, skey,
                                               thr_c, sumL, sumC, nf);
                    }
                }
                group_sync(bar, gsize);
            }
            const int dE = __reduce_add_sync(0xFFFFFFFFu, -2 * sumL);
            const int dM = __reduce_add_sync(0xFFFFFFFFu, -2 * (sumC - nf));  // both counted twice
            nf = __reduce_add_sync(0xFFFFFFFFu, nf) >> 1;
            if (lane == 0) {
                red_g[gwarp * 3 + 0] = dE;
                red_g[gwarp * 3 + 1] = dM;
                red_g[gwarp * 3 + 2] = nf;
            }
            if (!I.resident) {
                if (p16)
                    store_split16(I.spins + (size_t)rho * I.slot_stride, buf, N, P, P >> 4, hinv, gtid, gsize);
                else
                    store_split(I.spins + (size_t)rho * I.slot_stride, buf, N, P, G, ginv, gtid, gsize);
            }
            group_sync(bar, gsize);
            if (gtid == 0) {
                long long sE = 0, sM = 0, sF = 0;
                for (int w = 0; w < gsize / 32; ++w) {
                    sE += red_g[w * 3 + 0];
                    sM += red_g[w * 3 + 1];
                    sF += red_g[w * 3 + 2];
                }
                const long long E = s_E[lc] + sE, M = s_M[lc] + sM;
                s_E[lc] = E;
                s_M[lc] = M;
                unsigned long long* a = I.acc + (size_t)rung * kAccCount;
                atomicAdd(a + kAccN, 1ull);
                atomicAdd(a + kAccE, (unsigned long long)E);
                atomicAdd(a + kAccE2, (unsigned long long)(E * E));
                atomicAdd(a + kAccM, (unsigned long long)M);
                atomicAdd(a + kAccM2, (unsigned long long)(M * M));
                atomicAdd(a + kAccFlip, (unsigned long long)sF);
            }
            group_sync(bar, gsize);
        }
        __syncthreads();
        if (I.sweeps_per_swap > 0 && (s + 1) % I.sweeps_per_swap == 0) {
            const int pass = (s + 1) / I.sweeps_per_swap - 1;
            const long long q = I.q0 + pass;
            const int pb = pass & 1;
            for (int lc = tid; lc < c_count; lc += nt) s_pub[pb * C + lc] = make_longlong2(s_E[lc], s_M[lc]);
            if (K == 1)
                __syncthreads();
            else
                cluster.sync();
            for (int rl = (int)(q & 1) + 2 * tid; rl + 1 < R; rl += 2 * nt) {
                const int X = s_slot[rl], Y = s_slot[rl + 1];
                const longlong2 px = K == 1 ? s_pub[pb * C + X] : cluster.map_shared_rank(s_pub, X / C)[pb * C + X % C];
                const longlong2 py = K == 1 ? s_pub[pb * C + Y] : cluster.map_shared_rank(s_pub, Y / C)[pb * C + Y % C];
                const bool acc = swap_accept_fast(px.x, py.x, px.y, py.y, I.coef[rl], I.coef[(R - 1) + rl],
                                                  (uint32_t)q, (uint32_t)rl, skey, false);
                if (rank == 0) {
                    atomicAdd(I.swap_stats + 2 * rl, 1ull);
                    if (acc) atomicAdd(I.swap_stats + 2 * rl + 1, 1ull);
                }
                if (acc) {
                    s_slot[rl] = Y;
                    s_slot[rl + 1] = X;
                    s_rung[X] = rl + 1;
                    s_rung[Y] = rl;
                }
            }
            __syncthreads();
        }
    }

    // ---- write the problem back
    for (int x = tid; x < c_count; x += nt) {
        I.E[c_begin + x] = s_E[x];
        I.M[c_begin + x] = s_M[x];
    }
    if (I.resident) {
        for (int lc = 0; lc < c_count; ++lc)
            store_split(I.spins + (size_t)(c_begin + lc) * I.slot_stride,
                        reinterpret_cast<const int8_t*>(s_chains + (size_t)lc * L.chain_stride), N, P, G, ginv, tid,
                        nt);
    }
    if (rank == 0) {
        for (int x = tid; x < R; x += nt) {
            I.rung_of_slot[x] = s_rung[x];
            I.slot_of_rung[x] = s_slot[x];
        }
    }
}

__global__ void __launch_bounds__(512, 1) batch_kernel(BatchParams bp) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_job;
    __shared__ uint4 s_keys[5];  // round keys, two rounds per word
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int K = (int)cluster.num_blocks();
    if (bp.single) {
        // one problem on this one cluster; the host keeps its counters
        if (bp.one.dc == 4)
            run_problem<4>(bp.one, smem, s_keys, cluster, rank, K);
        else
            run_problem<8>(bp.one, smem, s_keys, cluster, rank, K);
        if (K > 1) cluster.sync();  // peers are done reading this CTA's published (E, M)
        return;
    }
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) s_job = atomicAdd(bp.next_job, 1);
        cluster.sync();
        const int job = *cluster.map_shared_rank(&s_job, 0);
        cluster.sync();  // every CTA has read the job before rank 0 may reuse or release s_job
        if (job >= bp.count) break;
        const BatchInstance I = bp.inst[bp.order[job]];
        if (I.dc == 4)
            run_problem<4>(I, smem, s_keys, cluster, rank, K);
        else
            run_problem<8>(I, smem, s_keys, cluster, rank, K);
        cluster.sync();  // peers are done reading this CTA's published (E, M)
        if (rank == 0 && threadIdx.x == 0) {
            // a finished problem's counters advance on the device, so the same launch can be
            // replayed (a CUDA graph) without uploading the problem records again
            BatchInstance* W = bp.inst + bp.order[job];
            W->t0 = I.t0 + I.n_sweeps;
            if (I.sweeps_per_swap > 0) W->q0 = I.q0 + I.n_sweeps / I.sweeps_per_swap;
            if (bp.done) {
                // every CTA of the cluster wrote its chains back before the barrier above;
                // the fence makes those writes visible before the flag, to the host's copies
                __threadfence_system();
                atomicExch(bp.done + bp.order[job], bp.done_token);
            }
        }
    }
}

// Initial spins and (E, M) of every chain of every problem: block b handles chain map[b].
__global__ void batch_init_kernel(const BatchInstance* inst, const int2* map) {
    __shared__ long long red[2][32];
    const int2 m = map[blockIdx.x];
    const BatchInstance& I = inst[m.x];
    const int rho = m.y;
    const PhiloxKey key = philox_schedule(I.key0, I.key1);
    int8_t* sp = I.spins + (size_t)rho * I.slot_stride;
    const int P4 = (I.P + 3) >> 2;
    for (int x = threadIdx.x; x < I.N * P4; x += blockDim.x) {
        const int i = x / P4, g4 = x - i * P4;
        const uint4 u = philox(make_uint4(0u, (uint32_t)i, (uint32_t)rho, (kTagInit << 28) | (uint32_t)g4), key);
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int k = 4 * g4 + b;
            if (k < I.P) sp[(size_t)i * I.P + k] = (w[b] >> 31) ? (int8_t)-1 : (int8_t)1;
        }
    }
    if (threadIdx.x == 0) {
        I.rung_of_slot[rho] = rho;
        I.slot_of_rung[rho] = rho;
    }
    __syncthreads();
    // E from the site descriptors: each edge once (neighbour row > own row), h once (the
    // slot whose row is the constant +1 row)
    const int DW = I.dc == 4 ? 8 : 12;
    const uint32_t np = (uint32_t)I.N * (uint32_t)I.P;
    long long e = 0, mm = 0;
    for (int x = threadIdx.x; x < I.N * I.P; x += blockDim.x) {
        const int i = x / I.P, k = x - i * I.P;
        const uint32_t* d = I.sdesc + (size_t)i * DW;
        const int si = sp[x];
        int f = 0;
        for (int sl = 0; sl < I.dc; ++sl) {
            const uint32_t row = d[4 + sl];
            if (row <= d[0]) continue;
            const int J = (int)(int8_t)((d[2 + (sl >> 2)] >> (8 * (sl & 3))) & 0xFFu);
            f += J * (row >= np ? 1 : (int)sp[row + k]);
        }
        e += (long long)si * f;
        mm += (long long)si * sp[(size_t)i * I.P + ((k + 1 == I.P) ? 0 : k + 1)];
    }
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_xor_sync(0xFFFFFFFFu, e, o);
        mm += __shfl_xor_sync(0xFFFFFFFFu, mm, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = e;
        red[1][threadIdx.x >> 5] = mm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long se = 0, sm = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            se += red[0][w];
            sm += red[1][w];
        }
        I.E[rho] = se;
        I.M[rho] = sm;
    }
}

cudaError_t launch_batch(const BatchParams& bp, int cluster, int n_clusters, int threads, size_t smem,
                         cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster * n_clusters);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    BatchParams p = bp;
    return cudaLaunchKernelEx(&cfg, batch_kernel, p);
}

cudaError_t batch_max_clusters(int cluster, int threads, size_t smem, int* n_clusters) {
    // the limit is a per-function attribute shared by every batch, so it is raised once to
    // the device's opt-in maximum (less this kernel's static shared memory)
    int dev = 0, max_smem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem - 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(n_clusters, (void*)batch_kernel, &cfg);
}

size_t batch_smem_cap() {
    int dev = 0, max_smem = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return 0;
    return (size_t)max_smem - 1024;  // room for the kernel's static shared memory
}

cudaError_t launch_batch_single(const BatchInstance& I, int cluster, int threads, size_t smem, cudaStream_t s) {
    BatchParams bp;
    bp.inst = nullptr;
    bp.order = nullptr;
    bp.count = 1;
    bp.next_job = nullptr;
    bp.status = nullptr;
    bp.single = 1;
    bp.one = I;
    return launch_batch(bp, cluster, 1, threads, smem, s);
}

cudaError_t launch_batch_init(const BatchInstance* inst, const int2* map, int n_chains, cudaStream_t s) {
    batch_init_kernel<<<n_chains, 256, 0, s>>>(inst, map);
    return cudaGetLastError();
}

}  // namespace ptq

// ===================================================================================== host
using namespace ptq;

struct pt_batch {
    int count;
    cudaStream_t stream;
    bool own_stream;
    int cluster, threads, n_clusters;
    size_t smem;
    std::vector<void*> allocs;
    int64_t device_bytes, launches, h2d_bytes;
    BatchInstance* d_inst;
    int32_t* d_order;
    int* d_counter;
    int* d_status;
    int8_t* d_staging;
    std::vector<BatchInstance> h_inst;
    std::vector<long long> sweep_limit;
    unsigned char* arena;    // constants [0, const_bytes), then every request's state
    size_t const_bytes, arena_bytes, smem_cap;
    int2* d_map;             // (request, chain) of every chain, for the initial-state kernel
    int n_map;
    int widen;               // group widening of the chosen layout (choose_groups)
    int tuned;               // layouts timed by the autotuner (0 = layout given)
    cudaGraphExec_t exec;    // the captured run (memset of the work counter + persistent launch)
    int graph_failed;        // capture was not possible; runs launch directly
    unsigned char* h_obs;    // pinned staging for pt_batch_read_observables: the device record,
    size_t h_obs_bytes;      // then one request's (E, M, permutation, statistics) block; the
                             // status word follows at h_obs + h_obs_bytes
    int err;
    char msg[256];
};

static thread_local char g_batch_create_msg[256] = "";

// Layouts chosen by the autotuner, per batch shape (every request's sizes, level count and
// sweeps), for the process: a create of a batch of the same shapes reuses the choice and
// times nothing. The layout never changes a result, so reuse is always safe.
struct BatchLayoutChoice {
    int cluster, widen;
};
static std::mutex g_layout_mutex;
static std::map<std::vector<long long>, BatchLayoutChoice> g_layout_cache;

static std::vector<long long> batch_shape_key(const std::vector<BatchInstance>& insts, int threads) {
    std::vector<long long> key;
    key.reserve(insts.size() * 7 + 1);
    key.push_back(threads);
    for (const BatchInstance& I : insts) {
        key.push_back(I.N);
        key.push_back(I.P);
        key.push_back(I.R);
        key.push_back(I.dc);
        key.push_back(I.n_levels);
        key.push_back(I.n_sweeps);
        key.push_back(I.sweeps_per_swap);
    }
    return key;
}

static int bfail(pt_batch* b, int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b ? b->msg : g_batch_create_msg, 256, fmt, ap);
    va_end(ap);
    if (b && (code == PT_ECUDA || code == PT_ETIMEDOUT)) b->err = code;
    return code;
}

static void free_batch(pt_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->h_obs) cudaFreeHost(b->h_obs);
    for (void* p : b->allocs) cudaFree(p);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

template <typename T>
static cudaError_t balloc(pt_batch* b, T** ptr, size_t bytes) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) return e;
    b->allocs.push_back(p);
    b->device_bytes += (int64_t)std::max<size_t>(bytes, 16);
    *ptr = (T*)p;
    return cudaSuccess;
}

int ptq::prepare_request(const pt_request& r, Prepared& pr, char* why, size_t why_len, int per_round) {
    const pt_instance* inst = &r.inst;
    const int N = inst->n, nE = inst->n_edges, P = r.P, R = r.R;
    if (N < 1 || N > 65535 || nE < 0 || !inst->h || (nE > 0 && (!inst->ei || !inst->ej || !inst->J))) {
        snprintf(why, why_len, "bad instance arrays");
        return PT_EINVAL;
    }
    if (P < 8 || P % 8 || P > 4096) {
        snprintf(why, why_len, "batched problems need P %% 8 == 0 and 8 <= P <= 4096");
        return PT_EINVAL;
    }
    if (R < 1 || R > 1024 || !r.ladder) {
        snprintf(why, why_len, "batched problems need 1 <= R <= 1024 rungs");
        return PT_EINVAL;
    }
    if (r.n_sweeps < 0 || r.n_sweeps > (1ll << 30) || r.sweeps_per_swap < 0) {
        snprintf(why, why_len, "n_sweeps must be in [0, 2^30] and sweeps_per_swap >= 0");
        return PT_EINVAL;
    }
    for (int q = 0; q < R; ++q)
        if (!(r.ladder[q].T > 0.0) || !(r.ladder[q].gamma > 0.0) || !std::isfinite(r.ladder[q].T) ||
            !std::isfinite(r.ladder[q].gamma)) {
            snprintf(why, why_len, "rung %d: T and gamma must be finite and > 0", q);
            return PT_EINVAL;
        }
    std::vector<std::vector<int>> adj(N), adjJ(N);
    long long eb = 0;
    for (int b = 0; b < nE; ++b) {
        const int u = inst->ei[b], v = inst->ej[b], J = inst->J[b];
        if (u < 0 || u >= N || v < 0 || v >= N || u == v || J == 0 || J < -127 || J > 127) {
            snprintf(why, why_len, "edge %d invalid", b);
            return PT_EINVAL;
        }
        adj[u].push_back(v);
        adjJ[u].push_back(J);
        adj[v].push_back(u);
        adjJ[v].push_back(J);
        eb += abs(J);
    }
    int dmax = 0, Lmax = 0;
    for (int i = 0; i < N; ++i) {
        std::vector<int> sorted = adj[i];
        std::sort(sorted.begin(), sorted.end());
        if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) {
            snprintf(why, why_len, "duplicate edge at site %d", i);
            return PT_EINVAL;
        }
        dmax = std::max(dmax, (int)adj[i].size());
        if (inst->h[i] < -127 || inst->h[i] > 127) {
            snprintf(why, why_len, "site %d: h must be in [-127,127]", i);
            return PT_EINVAL;
        }
        int l = abs(inst->h[i]);
        for (int J : adjJ[i]) l += abs(J);
        if (l > 127) {
            snprintf(why, why_len, "site %d: |h| + sum |J| > 127", i);
            return PT_EINVAL;
        }
        Lmax = std::max(Lmax, l);
        eb += abs(inst->h[i]);
    }
    if (dmax + 1 > 8) {
        snprintf(why, why_len, "batched problems need degree <= 7");
        return PT_EINVAL;
    }
    eb *= P;
    const long long mb = (long long)N * P;
    if (eb >= (1ll << 39) || mb >= (1ll << 31)) {
        snprintf(why, why_len, "energy or Trotter sum too large");
        return PT_EINVAL;
    }
    const long long big = std::max(std::max(eb, mb), 1ll);
    pr.sweep_limit = std::min<long long>(big > 3037000499ll ? 0 : 9223372036854775807ll / (big * big), 0xFFFFFFFFll);
    pr.N = N;
    pr.P = P;
    pr.R = R;
    pr.Lmax = Lmax;
    pr.dc = (dmax + 1 <= 4) ? 4 : 8;
    pr.slot_stride = (int)(((size_t)N * P + 15) & ~(size_t)15);
    build_tables(R, P, Lmax, r.ladder, pr.thr, pr.coef);
    if (pr.coef.size() < 2) pr.coef.assign(2, 0.0);
    level_schedule(N, adj, pr.items, pr.level_off, per_round, P / 4);  // rows of P bytes (int8 packed)
    pr.n_levels = (int)pr.level_off.size() - 1;
    build_site_desc(N, P, pr.dc, adj, adjJ, inst->h, pr.sdesc);
    return PT_OK;
}

// Offsets of one request's data inside a block of its own (constants, then state).
size_t ptq::request_block_layout(Prepared& p, size_t mailbox_entries) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    p.off_sdesc = take(p.sdesc.size() * 4);
    p.off_items = take(p.items.size() * 4);
    p.off_loff = take(p.level_off.size() * 4);
    p.off_thr = take(p.thr.size() * 4);
    p.off_coef = take(p.coef.size() * 8);
    p.off_spins = take((size_t)p.R * p.slot_stride);
    p.off_E = take((size_t)p.R * 8);
    p.off_M = take((size_t)p.R * 8);
    p.off_rung = take((size_t)p.R * 4);
    p.off_slot = take((size_t)p.R * 4);
    p.off_acc = take((size_t)p.R * kAccCount * 8);
    p.off_sw = take((size_t)p.R * 16);
    p.off_mbox = take(mailbox_entries * sizeof(Mailbox));
    p.off_inst = take(sizeof(BatchInstance));
    p.off_map = take((size_t)p.R * sizeof(int2));
    p.off_status = take(16);
    return off;
}

void ptq::fill_instance(BatchInstance& I, const Prepared& p, unsigned char* base, const pt_request& r) {
    memset(&I, 0, sizeof(I));
    I.N = p.N;
    I.P = p.P;
    I.R = p.R;
    I.Lmax = p.Lmax;
    I.nL3 = (2 * p.Lmax + 1) * 3;
    I.n_levels = p.n_levels;
    I.dc = p.dc;
    I.slot_stride = p.slot_stride;
    I.key0 = (uint32_t)(r.seed & 0xFFFFFFFFu);
    I.key1 = (uint32_t)(r.seed >> 32);
    I.n_sweeps = (int)r.n_sweeps;
    I.sweeps_per_swap = r.sweeps_per_swap;
    I.sdesc = (const uint32_t*)(base + p.off_sdesc);
    I.items = (const uint32_t*)(base + p.off_items);
    I.level_off = (const int32_t*)(base + p.off_loff);
    I.thr = (const uint32_t*)(base + p.off_thr);
    I.coef = (const double*)(base + p.off_coef);
    I.spins = (int8_t*)(base + p.off_spins);
    I.E = (long long*)(base + p.off_E);
    I.M = (long long*)(base + p.off_M);
    I.rung_of_slot = (int32_t*)(base + p.off_rung);
    I.slot_of_rung = (int32_t*)(base + p.off_slot);
    I.acc = (unsigned long long*)(base + p.off_acc);
    I.swap_stats = (unsigned long long*)(base + p.off_sw);
}

void ptq::choose_groups(BatchInstance& I, int cluster, int threads, size_t smem_cap, int widen) {
    // threads per chain: about one 4-copy unit per thread in an average level, at least two
    // warps, and no more groups than a CTA has chains; chains stay resident when they fit.
    // widen > 0 doubles the group that many times (fewer chains at once, shorter levels);
    // widen < 0 halves it (more chains at once, each with more rounds per level), as long as
    // the CTA's chain buffers still fit.
    const long long units = 2ll * I.N * (I.P / 8);
    const long long avg = (units + I.n_levels - 1) / I.n_levels;
    const int C = (I.R + cluster - 1) / cluster;
    // widths are powers of two that divide the CTA, so every thread is in a group
    auto up_ok = [&](int x) {
        const int y = 2 * x;
        return y <= threads && threads % y == 0;
    };
    int g = 64;
    while (up_ok(g) && g < avg) g <<= 1;
    while (up_ok(g) && threads / g > C) g <<= 1;
    for (int w = 0; w < widen && up_ok(g); ++w) g <<= 1;
    for (int w = 0; w < -widen && g > 32; ++w) g >>= 1;  // down to one warp per chain
    while (up_ok(g) && threads / g > C) g <<= 1;         // still no more groups than chains
    while (g > 32 && up_ok(g) && threads / g > 15) g <<= 1;  // named barriers 1..15 (0: the CTA's)
    // every rung's threshold row in shared memory when the rows take at most 48 KB and the
    // chains still fit; resident chains come first
    const int thr_words = (int)(up16((size_t)I.nL3 * 4) / 4);
    const int thr_ok = (size_t)I.R * thr_words * 4 <= 49152 ? 1 : 0;
    for (;;) {
        I.group_threads = g;
        I.resident = 1;
        I.thr_resident = thr_ok;
        if (batch_smem_bytes(I, cluster, threads) <= smem_cap) break;
        I.thr_resident = 0;
        if (batch_smem_bytes(I, cluster, threads) <= smem_cap) break;
        I.resident = 0;
        I.thr_resident = thr_ok;
        if (batch_smem_bytes(I, cluster, threads) <= smem_cap) break;
        I.thr_resident = 0;
        if (batch_smem_bytes(I, cluster, threads) <= smem_cap || !up_ok(g)) break;
        g <<= 1;  // one streaming buffer per group: fewer, larger groups
        while (up_ok(g) && threads / g > 15) g <<= 1;
    }
}

// Groups per request, the CTA's shared memory and the persistent grid for one layout.
static int plan_layout(pt_batch* b, int cluster, int widen, char* why, size_t why_len) {
    size_t smem = 0;
    for (int k = 0; k < b->count; ++k) {
        BatchInstance& I = b->h_inst[k];
        choose_groups(I, cluster, b->threads, b->smem_cap, widen);
        const size_t need = batch_smem_bytes(I, cluster, b->threads);
        if (need > b->smem_cap) {
            snprintf(why, why_len, "request %d needs %zu bytes of shared memory per CTA (device: %zu)", k, need,
                     b->smem_cap);
            return PT_EINVAL;
        }
        smem = std::max(smem, need);
    }
    int ncl = 0;
    const cudaError_t e = batch_max_clusters(cluster, b->threads, smem, &ncl);
    if (e != cudaSuccess || ncl < 1) {
        cudaGetLastError();
        snprintf(why, why_len, "no cluster of %d CTAs with %zu bytes of shared memory fits (%s)", cluster, smem,
                 cudaGetErrorString(e));
        return PT_EINVAL;
    }
    b->cluster = cluster;
    b->widen = widen;
    b->smem = smem;
    b->n_clusters = std::min(ncl, b->count);
    return PT_OK;
}

// Every request back to its initial state: zero statistics, counters at 0, initial spins
// and (E, M) from the Philox init stream. Synchronous.
static cudaError_t reset_state(pt_batch* b) {
    for (BatchInstance& I : b->h_inst) I.t0 = I.q0 = 0;
    cudaStream_t s = b->stream;
    cudaError_t e;
    if ((e = cudaMemsetAsync(b->arena + b->const_bytes, 0, b->arena_bytes - b->const_bytes, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(b->d_inst, b->h_inst.data(), sizeof(BatchInstance) * b->count, cudaMemcpyHostToDevice,
                             s)) != cudaSuccess ||
        (e = cudaMemsetAsync(b->d_status, 0, 16, s)) != cudaSuccess ||
        (e = launch_batch_init(b->d_inst, b->d_map, b->n_map, s)) != cudaSuccess)
        return e;
    b->launches += 1;
    b->h2d_bytes += (int64_t)(sizeof(BatchInstance) * b->count);
    return cudaStreamSynchronize(s);
}

// One run of every request: reset the work counter, then the persistent launch.
static cudaError_t enqueue_run(pt_batch* b) {
    cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), b->stream);
    if (e != cudaSuccess) return e;
    BatchParams bp;
    bp.inst = b->d_inst;
    bp.order = b->d_order;
    bp.count = b->count;
    bp.next_job = b->d_counter;
    bp.status = b->d_status;
    return launch_batch(bp, b->cluster, b->n_clusters, b->threads, b->smem, b->stream);
}

// Layout autotuner: times a short run (1 % of every request's sweeps, at least one) for
// each cluster size and group width that fits and keeps the fastest. The layout changes
// which CTA sweeps which chain and when, never the arithmetic or the random counters, so
// the choice cannot change any result; the state is reset afterwards.
static int autotune(pt_batch* b) {
    static const int kClusters[] = {1, 2, 4, 8};
    std::vector<int> full(b->count);
    for (int k = 0; k < b->count; ++k) {
        full[k] = b->h_inst[k].n_sweeps;
        b->h_inst[k].n_sweeps = std::max(1, full[k] / 100);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best_ms = 0.f;
    int best_c = 0, best_w = 0, timed = 0;
    char why[200];
    for (int ci = 0; ci < 4 && e == cudaSuccess; ++ci) {
        for (int w = -4; w < 2 && e == cudaSuccess; ++w) {
            if (plan_layout(b, kClusters[ci], w, why, sizeof(why)) != PT_OK) continue;
            for (int rep = 0; rep < (timed == 0 ? 2 : 1) && e == cudaSuccess; ++rep) {  // first: one warm-up
                for (BatchInstance& I : b->h_inst) I.t0 = I.q0 = 0;
                if ((e = cudaMemcpyAsync(b->d_inst, b->h_inst.data(), sizeof(BatchInstance) * b->count,
                                         cudaMemcpyHostToDevice, b->stream)) != cudaSuccess ||
                    (e = cudaEventRecord(e0, b->stream)) != cudaSuccess || (e = enqueue_run(b)) != cudaSuccess ||
                    (e = cudaEventRecord(e1, b->stream)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess)
                    break;
                b->launches += 1;
            }
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) break;
            if (timed == 0 || ms < best_ms) {
                best_ms = ms;
                best_c = kClusters[ci];
                best_w = w;
            }
            ++timed;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (int k = 0; k < b->count; ++k) b->h_inst[k].n_sweeps = full[k];
    if (e != cudaSuccess) return bfail(b, PT_ECUDA, "autotuner: %s", cudaGetErrorString(e));
    int st = 0;
    if ((e = cudaMemcpy(&st, b->d_status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess || st)
        return bfail(b, PT_ECUDA, "autotuner: device status %d (%s)", st, cudaGetErrorString(e));
    if (timed == 0) return bfail(b, PT_EINVAL, "no batched layout fits: %s", why);
    b->tuned = timed;
    const int rc = plan_layout(b, best_c, best_w, why, sizeof(why));
    if (rc) return bfail(b, rc, "%s", why);
    if ((e = reset_state(b)) != cudaSuccess) return bfail(b, PT_ECUDA, "autotuner reset: %s", cudaGetErrorString(e));
    return PT_OK;
}

extern "C" int pt_batch_create(const pt_request* reqs, int32_t count, const pt_options* opt, void* cuda_stream,
                               pt_batch** out) {
    if (!reqs || !out || count < 1) return bfail(nullptr, PT_EINVAL, "need at least one request");
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1) return bfail(nullptr, PT_ENODEV, "no CUDA device");
    std::vector<Prepared> pr(count);
    char why[200];
    {
        // Requests are prepared independently (checks, tables, level schedule, descriptors),
        // on up to 16 host threads; the first failing request in index order is reported.
        // Levels are balanced for one-warp chain groups (the default and the usual autotuned
        // width): 32 threads over the power-of-two word columns of an item.
        std::vector<int> rcs(count, PT_OK);
        std::vector<std::string> whys(count);
        auto work = [&](int first, int step) {
            char w[200];
            for (int k = first; k < count; k += step) {
                int cols = 1;
                while (cols < reqs[k].P / 8) cols <<= 1;
                rcs[k] = prepare_request(reqs[k], pr[k], w, sizeof(w), reqs[k].P >= 8 ? std::max(1, 32 / cols) : 0);
                if (rcs[k]) whys[k] = w;
            }
        };
        const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
        const int n_threads = (int)std::min<unsigned>(std::min(hw, 16u), (unsigned)((count + 7) / 8));
        if (n_threads <= 1) {
            work(0, 1);
        } else {
            std::vector<std::thread> pool;
            pool.reserve(n_threads - 1);
            for (int t = 1; t < n_threads; ++t) pool.emplace_back(work, t, n_threads);
            work(0, n_threads);
            for (std::thread& th : pool) th.join();
        }
        for (int k = 0; k < count; ++k)
            if (rcs[k]) return bfail(nullptr, rcs[k], "request %d: %s", k, whys[k].c_str());
    }
    if (opt && (opt->cluster_size < 0 || opt->cluster_size > 16))
        return bfail(nullptr, PT_EINVAL, "cluster_size must be 0 (autotune) or 1..16");
    pt_batch* b = new pt_batch();
    b->count = count;
    b->stream = (cudaStream_t)cuda_stream;
    b->own_stream = false;
    b->device_bytes = b->launches = b->h2d_bytes = 0;
    b->arena = nullptr;
    b->d_map = nullptr;
    b->exec = nullptr;
    b->graph_failed = 0;
    b->h_obs = nullptr;
    b->h_obs_bytes = 0;
    b->tuned = 0;
    b->widen = 0;
    b->err = 0;
    b->msg[0] = 0;
    if (!b->stream) {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return bfail(nullptr, PT_ECUDA, "cudaStreamCreate failed");
        }
        b->own_stream = true;
    }
    int dev = 0, max_smem = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    b->smem_cap = (size_t)max_smem - 1024;  // room for the kernel's static shared memory
    b->threads = 512;

    // device layout of every request in one arena: constants first, then state
    b->h_inst.resize(count);
    b->sweep_limit.resize(count);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    size_t max_state = 0;
    for (int k = 0; k < count; ++k) {
        Prepared& p = pr[k];
        p.off_sdesc = take(p.sdesc.size() * 4);
        p.off_items = take(p.items.size() * 4);
        p.off_loff = take(p.level_off.size() * 4);
        p.off_thr = take(p.thr.size() * 4);
        p.off_coef = take(p.coef.size() * 8);
    }
    const size_t const_bytes = off;
    for (int k = 0; k < count; ++k) {
        Prepared& p = pr[k];
        p.off_spins = take((size_t)p.R * p.slot_stride);
        p.off_E = take((size_t)p.R * 8);
        p.off_M = take((size_t)p.R * 8);
        p.off_rung = take((size_t)p.R * 4);
        p.off_slot = take((size_t)p.R * 4);
        p.off_acc = take((size_t)p.R * kAccCount * 8);
        p.off_sw = take((size_t)p.R * 16);
        max_state = std::max(max_state, (size_t)p.R * p.N * p.P);
        BatchInstance& I = b->h_inst[k];
        memset(&I, 0, sizeof(I));
        I.N = p.N;
        I.P = p.P;
        I.R = p.R;
        I.Lmax = p.Lmax;
        I.nL3 = (2 * p.Lmax + 1) * 3;
        I.n_levels = p.n_levels;
        I.dc = p.dc;
        I.slot_stride = p.slot_stride;
        I.key0 = (uint32_t)(reqs[k].seed & 0xFFFFFFFFu);
        I.key1 = (uint32_t)(reqs[k].seed >> 32);
        I.n_sweeps = (int)reqs[k].n_sweeps;
        I.sweeps_per_swap = reqs[k].sweeps_per_swap;
        b->sweep_limit[k] = p.sweep_limit;
    }
    b->const_bytes = const_bytes;
    b->arena_bytes = off;
    const int fixed_cluster = (opt && opt->cluster_size > 0) ? opt->cluster_size : 0;
    {
        // the given layout, or (autotuning) the smallest cluster, which needs the most
        // shared memory per CTA: a request that fits nowhere is rejected before allocating
        const int rc = plan_layout(b, fixed_cluster ? fixed_cluster : 1, kGroupWidenDefault, why, sizeof(why));
        if (rc != PT_OK &&
            (fixed_cluster || plan_layout(b, 8, kGroupWidenDefault, why, sizeof(why)) != PT_OK)) {
            free_batch(b);
            return bfail(nullptr, PT_EINVAL, "%s", why);
        }
    }

    unsigned char* arena = nullptr;
    cudaError_t e;
    if ((e = balloc(b, &arena, off)) != cudaSuccess || (e = balloc(b, &b->d_inst, sizeof(BatchInstance) * count)) ||
        (e = balloc(b, &b->d_order, sizeof(int32_t) * count)) || (e = balloc(b, &b->d_counter, 16)) ||
        (e = balloc(b, &b->d_status, 16)) || (e = balloc(b, &b->d_staging, max_state))) {
        free_batch(b);
        return bfail(nullptr, e == cudaErrorMemoryAllocation ? PT_ENOMEM : PT_ECUDA, "cudaMalloc: %s",
                     cudaGetErrorString(e));
    }
    b->arena = arena;
    {
        size_t most = 0;
        for (int k = 0; k < count; ++k) most = std::max(most, pr[k].off_sw + (size_t)pr[k].R * 16 - pr[k].off_E);
        b->h_obs_bytes = (sizeof(BatchInstance) + most + 15) & ~(size_t)15;
        if ((e = cudaMallocHost(&b->h_obs, b->h_obs_bytes + 16)) != cudaSuccess) {  // + the status word
            b->h_obs = nullptr;
            free_batch(b);
            return bfail(nullptr, PT_ENOMEM, "cudaMallocHost: %s", cudaGetErrorString(e));
        }
    }
    std::vector<unsigned char> host_const(const_bytes, 0);
    std::vector<int2> map;
    for (int k = 0; k < count; ++k) {
        Prepared& p = pr[k];
        memcpy(&host_const[p.off_sdesc], p.sdesc.data(), p.sdesc.size() * 4);
        memcpy(&host_const[p.off_items], p.items.data(), p.items.size() * 4);
        memcpy(&host_const[p.off_loff], p.level_off.data(), p.level_off.size() * 4);
        memcpy(&host_const[p.off_thr], p.thr.data(), p.thr.size() * 4);
        memcpy(&host_const[p.off_coef], p.coef.data(), p.coef.size() * 8);
        BatchInstance& I = b->h_inst[k];
        I.sdesc = (const uint32_t*)(arena + p.off_sdesc);
        I.items = (const uint32_t*)(arena + p.off_items);
        I.level_off = (const int32_t*)(arena + p.off_loff);
        I.thr = (const uint32_t*)(arena + p.off_thr);
        I.coef = (const double*)(arena + p.off_coef);
        I.spins = (int8_t*)(arena + p.off_spins);
        I.E = (long long*)(arena + p.off_E);
        I.M = (long long*)(arena + p.off_M);
        I.rung_of_slot = (int32_t*)(arena + p.off_rung);
        I.slot_of_rung = (int32_t*)(arena + p.off_slot);
        I.acc = (unsigned long long*)(arena + p.off_acc);
        I.swap_stats = (unsigned long long*)(arena + p.off_sw);
        for (int rho = 0; rho < p.R; ++rho) map.push_back(make_int2(k, rho));
    }
    // requests with the most work first, so the last ones to finish are small
    std::vector<int32_t> order(count);
    for (int k = 0; k < count; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        const double wa = (double)pr[a].N * pr[a].P * pr[a].R * (double)reqs[a].n_sweeps;
        const double wc = (double)pr[c].N * pr[c].P * pr[c].R * (double)reqs[c].n_sweeps;
        return wa > wc;
    });
    cudaStream_t s = b->stream;
    b->n_map = (int)map.size();
    if ((e = balloc(b, &b->d_map, map.size() * sizeof(int2))) != cudaSuccess ||
        (e = cudaMemcpyAsync(arena, host_const.data(), const_bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(b->d_order, order.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(b->d_map, map.data(), map.size() * sizeof(int2), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (e = reset_state(b)) != cudaSuccess) {
        cudaStreamSynchronize(s);
        free_batch(b);
        return bfail(nullptr, PT_ECUDA, "batch setup: %s", cudaGetErrorString(e));
    }
    b->h2d_bytes += (int64_t)(const_bytes + sizeof(int32_t) * count + map.size() * sizeof(int2));
    if (!fixed_cluster) {
        const std::vector<long long> key = batch_shape_key(b->h_inst, b->threads);
        BatchLayoutChoice cached{0, 0};
        {
            std::lock_guard<std::mutex> lock(g_layout_mutex);
            auto it = g_layout_cache.find(key);
            if (it != g_layout_cache.end()) cached = it->second;
        }
        if (cached.cluster > 0 && plan_layout(b, cached.cluster, cached.widen, why, sizeof(why)) == PT_OK) {
            *out = b;
            return PT_OK;
        }
        const int rc = autotune(b);
        if (rc == PT_OK) {
            std::lock_guard<std::mutex> lock(g_layout_mutex);
            g_layout_cache[key] = BatchLayoutChoice{b->cluster, b->widen};
        }
        if (rc != PT_OK) {
            snprintf(g_batch_create_msg, sizeof(g_batch_create_msg), "%s", b->msg);
            free_batch(b);
            return rc;
        }
    }
    *out = b;
    return PT_OK;
}

static int bguard(pt_batch* b) {
    if (!b) return PT_EINVAL;
    return b->err;
}

static int bcheck(pt_batch* b) {
    // the status word through the pinned staging once it exists (a copy into pageable memory
    // is staged by the driver and costs more than the synchronisation itself)
    int local = 0;
    int* st = b->h_obs ? reinterpret_cast<int*>(b->h_obs + b->h_obs_bytes) : &local;
    *st = 0;
    cudaError_t e = cudaMemcpyAsync(st, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, PT_ECUDA, "CUDA error: %s", cudaGetErrorString(e));
    if (*st) return bfail(b, PT_ECUDA, "device status %d", *st);
    return PT_OK;
}

extern "C" int pt_batch_run(pt_batch* b) {
    int g = bguard(b);
    if (g) return g;
    for (int k = 0; k < b->count; ++k) {
        const BatchInstance& I = b->h_inst[k];
        const long long passes = I.sweeps_per_swap > 0 ? I.n_sweeps / I.sweeps_per_swap : 0;
        if (I.t0 + I.n_sweeps > b->sweep_limit[k] || I.q0 + passes > 0xFFFFFFFFll)
            return bfail(b, PT_EOVERFLOW, "request %d: sweep or pass counter would overflow", k);
    }
    cudaError_t e = cudaSuccess;
    if (!b->exec && !b->graph_failed) {
        // the first run is captured into a CUDA graph and every run replays it (the problem
        // records on the device carry the counters forward). A stream that is already
        // capturing gets the plain launch, recorded into the caller's own graph.
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(b->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
            cudaGetLastError();
        } else if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            cudaGraph_t graph = nullptr;
            const cudaError_t le = enqueue_run(b);
            const cudaError_t ce = cudaStreamEndCapture(b->stream, &graph);
            if (le == cudaSuccess && ce == cudaSuccess && graph &&
                cudaGraphInstantiate(&b->exec, graph, 0) != cudaSuccess)
                b->exec = nullptr;
            if (graph) cudaGraphDestroy(graph);
            if (!b->exec) {
                b->graph_failed = 1;
                cudaGetLastError();
            }
        } else {
            b->graph_failed = 1;
            cudaGetLastError();
        }
    }
    if (b->exec)
        e = cudaGraphLaunch(b->exec, b->stream);
    else
        e = enqueue_run(b);
    if (e != cudaSuccess) return bfail(b, PT_ECUDA, "batch launch: %s", cudaGetErrorString(e));
    b->launches += 1;
    for (int k = 0; k < b->count; ++k) {
        BatchInstance& I = b->h_inst[k];
        I.t0 += I.n_sweeps;
        if (I.sweeps_per_swap > 0) I.q0 += I.n_sweeps / I.sweeps_per_swap;
    }
    return PT_OK;
}

extern "C" int pt_batch_sync(pt_batch* b) {
    int g = bguard(b);
    if (g) return g;
    return bcheck(b);
}

extern "C" int pt_batch_read_state(pt_batch* b, int32_t index, int8_t* out, size_t bytes) {
    int g = bguard(b);
    if (g) return g;
    if (index < 0 || index >= b->count) return bfail(b, PT_EINVAL, "index out of range");
    const BatchInstance& I = b->h_inst[index];
    const size_t need = (size_t)I.R * I.N * I.P;
    if (!out || bytes < need) return bfail(b, PT_EINVAL, "state buffer needs %zu bytes", need);
    DevProblem p;
    memset(&p, 0, sizeof(p));
    p.spins = I.spins;
    p.slot_of_rung = I.slot_of_rung;
    p.N = I.N;
    p.P = I.P;
    p.R = I.R;
    p.slot_stride = I.slot_stride;
    cudaError_t e;
    if ((e = launch_gather_state(p, b->d_staging, b->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(out, b->d_staging, need, cudaMemcpyDeviceToHost, b->stream)) != cudaSuccess)
        return bfail(b, PT_ECUDA, "%s", cudaGetErrorString(e));
    b->launches += 1;
    return bcheck(b);
}

extern "C" int pt_batch_read_observables(pt_batch* b, int32_t index, pt_observables* o) {
    int g = bguard(b);
    if (g) return g;
    if (index < 0 || index >= b->count || !o) return bfail(b, PT_EINVAL, "bad index or null observables");
    const BatchInstance& I = b->h_inst[index];
    const int R = I.R;
    // the device record (its counters also count replays of a caller's graph), then the
    // request's state block from E to the swap counts (contiguous in the arena), in two copies
    // into pinned staging
    const unsigned char* blk = reinterpret_cast<const unsigned char*>(I.E);
    const size_t blk_bytes =
        (size_t)(reinterpret_cast<const unsigned char*>(I.swap_stats) - blk) + (size_t)R * 16;
    unsigned char* h_blk = b->h_obs + sizeof(BatchInstance);
    cudaStream_t s = b->stream;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(b->h_obs, b->d_inst + index, sizeof(BatchInstance), cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(h_blk, blk, blk_bytes, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return bfail(b, PT_ECUDA, "%s", cudaGetErrorString(e));
    int rc = bcheck(b);
    if (rc) return rc;
    BatchInstance dev_rec;
    memcpy(&dev_rec, b->h_obs, sizeof(BatchInstance));
    auto at = [&](const void* dev) { return h_blk + (reinterpret_cast<const unsigned char*>(dev) - blk); };
    const long long* E = reinterpret_cast<const long long*>(at(I.E));
    const long long* M = reinterpret_cast<const long long*>(at(I.M));
    const int32_t* slot_of = reinterpret_cast<const int32_t*>(at(I.slot_of_rung));
    const unsigned long long* acc = reinterpret_cast<const unsigned long long*>(at(I.acc));
    const unsigned long long* sw = reinterpret_cast<const unsigned long long*>(at(I.swap_stats));
    o->t = dev_rec.t0;
    o->q = dev_rec.q0;
    for (int r = 0; r < R; ++r) {
        const int slot = slot_of[r];
        if (o->E) o->E[r] = E[slot];
        if (o->M) o->M[r] = M[slot];
        const unsigned long long* a = &acc[(size_t)r * kAccCount];
        if (o->n_meas) o->n_meas[r] = (int64_t)a[kAccN];
        if (o->sum_E) o->sum_E[r] = (int64_t)a[kAccE];
        if (o->sum_E2) o->sum_E2[r] = (int64_t)a[kAccE2];
        if (o->sum_M) o->sum_M[r] = (int64_t)a[kAccM];
        if (o->sum_M2) o->sum_M2[r] = (int64_t)a[kAccM2];
        if (o->flip_acc) o->flip_acc[r] = (int64_t)a[kAccFlip];
        if (o->replica_at) o->replica_at[r] = slot;
    }
    for (int r = 0; r + 1 < R; ++r) {
        if (o->swap_att) o->swap_att[r] = (int64_t)sw[2 * r];
        if (o->swap_acc) o->swap_acc[r] = (int64_t)sw[2 * r + 1];
    }
    return PT_OK;
}

extern "C" int pt_batch_get_info(const pt_batch* b, pt_batch_info* o) {
    if (!b || !o) return PT_EINVAL;
    o->count = b->count;
    o->cluster = b->cluster;
    o->n_clusters = b->n_clusters;
    o->threads_per_block = b->threads;
    o->smem_bytes = (int64_t)b->smem;
    o->device_bytes = b->device_bytes;
    o->kernel_launches = b->launches;
    o->h2d_bytes = b->h2d_bytes;
    o->tuned_layouts = b->tuned;
    o->group_widen = b->widen;
    o->graph = b->exec ? 1 : 0;
    o->reserved = 0;
    return PT_OK;
}

extern "C" int pt_batch_destroy(pt_batch* b) {
    if (!b) return PT_OK;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    return PT_OK;
}

extern "C" const char* pt_batch_last_error(const pt_batch* b) { return b ? b->msg : g_batch_create_msg; }
