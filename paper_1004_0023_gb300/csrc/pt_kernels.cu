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
#include <cuda_runtime.h>
#include <stdint.h>

#include "pt.h"
#include "pt_internal.h"

namespace ptq {

// ------------------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, SC'11: round (c0,c1,c2,c3) -> (hi(M1 c2)^c1^k0, lo(M1 c2),
// hi(M0 c0)^c3^k1, lo(M0 c0)); the round-r key is (k0 + r W0, k1 + r W1).
struct PhiloxKey {
    uint32_t k0[10];
    uint32_t k1[10];
};

__device__ __forceinline__ PhiloxKey philox_schedule(uint32_t key0, uint32_t key1) {
    PhiloxKey k;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        k.k0[r] = key0 + (uint32_t)r * 0x9E3779B9u;
        k.k1[r] = key1 + (uint32_t)r * 0xBB67AE85u;
    }
    return k;
}

__device__ __forceinline__ uint4 philox(uint4 c, const PhiloxKey& k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k.k0[r], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ k.k1[r], (uint32_t)p0);
    }
    return c;
}

// ------------------------------------------------------------------------- det_exp
// exp(x) for x in (-23, 0] from IEEE round-to-nearest basic operations only (Cody & Waite
// argument reduction with a two-part ln 2, then the degree-13 Taylor series of exp by
// Horner's rule, then an exact scaling by 2^n). Each operation is an explicit _rn
// intrinsic so no multiply-add is fused; the host computes the same sequence.
__device__ __forceinline__ double det_exp(double x) {
    const double LN2_HI = 0x1.62e42ff000000p-1;
    const double LN2_LO = -0x1.718432a1b0e26p-35;
    const double INV_LN2 = 0x1.71547652b82fep+0;
    double inv_fact[14];
    double fact = 1.0;
#pragma unroll
    for (int k = 0; k < 14; ++k) {
        if (k > 0) fact = __dmul_rn(fact, (double)k);
        inv_fact[k] = __ddiv_rn(1.0, fact);
    }
    const double nd = rint(__dmul_rn(x, INV_LN2));
    const double r = __dsub_rn(__dsub_rn(x, __dmul_rn(nd, LN2_HI)), __dmul_rn(nd, LN2_LO));
    double poly = inv_fact[13];
#pragma unroll
    for (int k = 12; k >= 0; --k) poly = __dadd_rn(__dmul_rn(poly, r), inv_fact[k]);
    const int n = (int)nd;  // in [-34, 0]
    const double scale = __hiloint2double((1023 + n) << 20, 0);
    return __dmul_rn(poly, scale);
}

// Swap decision for X on rung rl and Y on rung rl + 1 at pass q.
__device__ __forceinline__ bool swap_accept(long long EX, long long EY, long long MX, long long MY,
                                            double a, double c, uint32_t q, uint32_t rl,
                                            const PhiloxKey& key) {
    const double dE = __ll2double_rn(EX - EY);
    const double dM = __ll2double_rn(MX - MY);
    const double delta = __dadd_rn(__dmul_rn(a, dE), __dmul_rn(c, dM));
    if (delta >= 0.0) return true;
    if (!(delta > -23.0)) return false;
    const uint4 u = philox(make_uint4(q, rl, 0u, kTagSwap << 28), key);
    const double v = floor(__dmul_rn(det_exp(delta), 4294967296.0));
    const uint32_t ts = (v >= 4294967295.0) ? 0xFFFFFFFFu : (uint32_t)v;
    return u.x < ts;
}

// ------------------------------------------------------------------------- PTX helpers
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ long long ld_relaxed_s64(const long long* p) {
    long long v;
    asm volatile("ld.relaxed.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_s64(long long* p, long long v) {
    asm volatile("st.relaxed.gpu.global.s64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ------------------------------------------------------------------------- smem layout
struct SmemLayout {
    size_t spins, nbr, h, items, loff, thr, red, ctl, total;
    __host__ __device__ static size_t up16(size_t x) { return (x + 15) & ~(size_t)15; }
    __host__ __device__ SmemLayout(int N, int P, int dmax, int n_levels, int nL3) {
        size_t o = 0;
        spins = o; o += up16((size_t)N * P);
        nbr = o;   o += up16((size_t)N * dmax * 4);
        h = o;     o += up16((size_t)N);
        items = o; o += up16((size_t)2 * N * 4);
        loff = o;  o += up16((size_t)(n_levels + 1) * 4);
        thr = o;   o += up16((size_t)nL3 * 4);
        red = o;   o += 32 * 3 * 8;
        ctl = o;   o += 16;
        total = o;
    }
};

size_t sweep_smem_bytes(const DevProblem& p) {
    return SmemLayout(p.N, p.P, p.dmax, p.n_levels, p.nL3).total;
}

// ------------------------------------------------------------------------- sweep kernel
// One CTA per chain (slot). n_sweeps sweeps; when sweeps_per_swap > 0, a swap pass after
// every sweeps_per_swap-th sweep (cooperative launch only).
template <int DCLASS>
__global__ void __launch_bounds__(512, 1)
sweep_kernel(DevProblem p, long long t0, long long q0, int n_sweeps, int sweeps_per_swap,
             int n_passes, long long timeout_ns) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = p.N, P = p.P, R = p.R;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int slot = blockIdx.x;
    const SmemLayout L(N, P, DCLASS, p.n_levels, p.nL3);
    int8_t* sp = reinterpret_cast<int8_t*>(smem + L.spins);
    uint32_t* s_nbr = reinterpret_cast<uint32_t*>(smem + L.nbr);
    int8_t* s_h = reinterpret_cast<int8_t*>(smem + L.h);
    uint32_t* s_items = reinterpret_cast<uint32_t*>(smem + L.items);
    int32_t* s_loff = reinterpret_cast<int32_t*>(smem + L.loff);
    uint32_t* s_thr = reinterpret_cast<uint32_t*>(smem + L.thr);
    long long* s_red = reinterpret_cast<long long*>(smem + L.red);
    int* s_ctl = reinterpret_cast<int*>(smem + L.ctl);

    // ---- load the chain and the instance into shared memory
    {
        const int4* src = reinterpret_cast<const int4*>(p.spins + (size_t)slot * p.slot_stride);
        int4* dst = reinterpret_cast<int4*>(sp);
        const int n16 = (int)(SmemLayout::up16((size_t)N * P) / 16);
        for (int x = tid; x < n16; x += nt) dst[x] = src[x];
        for (int x = tid; x < N * DCLASS; x += nt) s_nbr[x] = p.nbr[x];
        for (int x = tid; x < N; x += nt) s_h[x] = p.h[x];
        for (int x = tid; x < 2 * N; x += nt) s_items[x] = p.items[x];
        for (int x = tid; x <= p.n_levels; x += nt) s_loff[x] = p.level_off[x];
    }
    int rung = p.rung_of_slot[slot];
    for (int x = tid; x < p.nL3; x += nt) s_thr[x] = p.thr[(size_t)rung * p.nL3 + x];
    long long E = p.E[slot], M = p.M[slot];  // meaningful in thread 0 only
    __syncthreads();

    const PhiloxKey key = philox_schedule(p.key0, p.key1);
    const int half = P >> 1;
    const int G = (half + 3) >> 2;  // 4-copy groups per parity
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
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    const int hh = 4 * g + w;
                    if (hh < half) {
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
                        const int m = sk * ((int)row[km1] + (int)row[kp1]);
                        const uint32_t th = s_thr[(Lf + Lmax) * 3 + (m >> 1) + 1];
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
        // ---- per-chain reduction of the sweep's energy / Trotter-term changes and flips
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
            E += sE;
            M += sM;
            // statistics after every sweep, attributed to the rung the chain sits on
            unsigned long long* a = p.acc + (size_t)rung * kAccCount;
            atomicAdd(a + kAccN, 1ull);
            atomicAdd(a + kAccE, (unsigned long long)E);
            atomicAdd(a + kAccE2, (unsigned long long)(E * E));
            atomicAdd(a + kAccM, (unsigned long long)M);
            atomicAdd(a + kAccM2, (unsigned long long)(M * M));
            atomicAdd(a + kAccFlip, (unsigned long long)sF);

            int abort_flag = 0;
            const int new_rung_base = rung;
            int new_rung = new_rung_base;
            if (sweeps_per_swap > 0 && (s + 1) % sweeps_per_swap == 0) {
                const int pass = (s + 1) / sweeps_per_swap - 1;
                const long long q = q0 + pass;
                Mailbox* mb = p.mbox + (size_t)pass * R;
                if (rung != p.withhold_rung) {
                    st_relaxed_s64(&mb[rung].E, E);
                    st_relaxed_s64(&mb[rung].M, M);
                    __threadfence();
                    st_release_u64(&mb[rung].tag, (unsigned long long)(q + 1));
                }
                int rl, partner;
                if ((rung & 1) == (int)(q & 1)) {
                    rl = rung;
                    partner = rung + 1;
                } else {
                    rl = rung - 1;
                    partner = rung - 1;
                }
                if (rl >= 0 && rl + 1 < R) {
                    const unsigned long long start = globaltimer_ns();
                    while (ld_acquire_u64(&mb[partner].tag) != (unsigned long long)(q + 1)) {
                        if ((long long)(globaltimer_ns() - start) > timeout_ns) {
                            abort_flag = 1;
                            atomicCAS(p.status, 0, PT_ETIMEDOUT);
                            break;
                        }
                    }
                    if (!abort_flag) {
                        const long long pE = ld_relaxed_s64(&mb[partner].E);
                        const long long pM = ld_relaxed_s64(&mb[partner].M);
                        const bool lower = (rung == rl);
                        const bool acc = swap_accept(lower ? E : pE, lower ? pE : E, lower ? M : pM,
                                                     lower ? pM : M, p.coef[rl], p.coef[(R - 1) + rl],
                                                     (uint32_t)q, (uint32_t)rl, key);
                        if (lower) {
                            atomicAdd(p.swap_stats + 2 * rl, 1ull);
                            if (acc) atomicAdd(p.swap_stats + 2 * rl + 1, 1ull);
                        }
                        if (acc) new_rung = partner;
                    }
                }
            }
            s_ctl[0] = new_rung;
            s_ctl[1] = abort_flag;
        }
        __syncthreads();
        if (s_ctl[1]) return;  // a partner never arrived; status holds PT_ETIMEDOUT
        const int nr = s_ctl[0];
        if (nr != rung) {
            rung = nr;
            for (int x = tid; x < p.nL3; x += nt) s_thr[x] = p.thr[(size_t)rung * p.nL3 + x];
        }
        __syncthreads();
    }
    (void)n_passes;

    // ---- write the chain back
    {
        int4* dst = reinterpret_cast<int4*>(p.spins + (size_t)slot * p.slot_stride);
        const int4* src = reinterpret_cast<const int4*>(sp);
        const int n16 = (int)(SmemLayout::up16((size_t)N * P) / 16);
        for (int x = tid; x < n16; x += nt) dst[x] = src[x];
    }
    if (tid == 0) {
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
        const bool acc = swap_accept(p.E[X], p.E[Y], p.M[X], p.M[Y], p.coef[rl], p.coef[(p.R - 1) + rl],
                                     (uint32_t)q, (uint32_t)rl, key);
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
    for (int x = threadIdx.x; x < p.N * p.P; x += blockDim.x) dst[x] = src[x];
}

__global__ void scatter_kernel(DevProblem p, const int8_t* in) {
    const int r = blockIdx.x;
    int8_t* dst = p.spins + (size_t)p.slot_of_rung[r] * p.slot_stride;
    const int8_t* src = in + (size_t)r * p.N * p.P;
    for (int x = threadIdx.x; x < p.N * p.P; x += blockDim.x) dst[x] = src[x];
}

// ------------------------------------------------------------------------- launchers
static const void* sweep_fn(int dclass) {
    switch (dclass) {
        case 4: return (const void*)sweep_kernel<4>;
        case 8: return (const void*)sweep_kernel<8>;
        default: return (const void*)sweep_kernel<32>;
    }
}

// The dynamic shared-memory limit is a per-function attribute shared by every context, so
// it is raised once to the device's opt-in maximum rather than to one context's size.
cudaError_t prepare_sweep_kernel(const LaunchPlan& plan) {
    int dev = 0, max_smem = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(sweep_fn(plan.dclass), cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
}

cudaError_t sweep_kernel_occupancy(const DevProblem& p, const LaunchPlan& plan, int* blocks_per_sm) {
    (void)p;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, sweep_fn(plan.dclass), plan.threads,
                                                         plan.smem_bytes);
}

cudaError_t launch_sweeps(const DevProblem& p, const LaunchPlan& plan, long long t0, long long q0,
                          int n_sweeps, int sweeps_per_swap, int n_passes, long long timeout_ns,
                          bool cooperative, cudaStream_t s) {
    DevProblem pp = p;
    void* args[] = {&pp, &t0, &q0, &n_sweeps, &sweeps_per_swap, &n_passes, &timeout_ns};
    const void* fn = sweep_fn(plan.dclass);
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
