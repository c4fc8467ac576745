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
    // 1/k! rounded to nearest (k! is exact in double for k <= 13); folded at compile time
    const double inv_fact[14] = {1.0, 1.0, 1.0 / 2.0, 1.0 / 6.0, 1.0 / 24.0, 1.0 / 120.0, 1.0 / 720.0,
                                 1.0 / 5040.0, 1.0 / 40320.0, 1.0 / 362880.0, 1.0 / 3628800.0,
                                 1.0 / 39916800.0, 1.0 / 479001600.0, 1.0 / 6227020800.0};
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

// The same decision without FP64 in the common case. GB300's FP64 pipe makes the ~40
// dependent FP64 operations of swap_accept cost over a microsecond, so Delta and exp(Delta)
// are first estimated in FP32 with an error bound:
//   |D - Delta| <= err = 5*2^-24 * (|a dE| + |c dM|)   (conversions of a, c, dE, dM, two
//   products, one sum, and the FP64 roundings of Delta itself, with room to spare), and
//   2^32 exp(D) within a relative 1e-5 + 1.01 err of 2^32 exp(Delta) (expf is within 2 ulp).
// The estimate decides only when u is farther than that margin (plus float rounding of u)
// from the threshold, or Delta's sign and the -23 cut are certain; otherwise swap_accept
// decides. Either way the result equals swap_accept's.
__device__ __forceinline__ bool swap_accept_fast(long long EX, long long EY, long long MX, long long MY,
                                                 double a, double c, uint32_t q, uint32_t rl,
                                                 const PhiloxKey& key, bool exact_only) {
    if (!exact_only) {
        const float pa = (float)a * (float)(EX - EY);
        const float pc = (float)c * (float)(MX - MY);
        const float D = pa + pc;
        const float err = (fabsf(pa) + fabsf(pc)) * 2.99e-7f + 1e-30f;
        if (D >= 2.0f * err) return true;                       // Delta >= 0
        if (err < 0.25f) {
            if (D < -23.5f) return false;                         // Delta <= -23
            if (D + 2.0f * err < 0.0f && D > -22.5f) {
                const uint4 r4 = philox(make_uint4(q, rl, 0u, kTagSwap << 28), key);
                const float v = 4294967296.0f * expf(D);
                const float margin = v * (1.0e-5f + 1.01f * err) + 512.0f;
                const float uf = (float)r4.x;
                if (uf + margin < v) return true;
                if (uf - margin > v) return false;
            }
        }
    }
    return swap_accept(EX, EY, MX, MY, a, c, q, rl, key);
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
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_s64(long long* p, long long v) {
    asm volatile("st.relaxed.gpu.global.s64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// prmt.b32 in its generic mode: a selector nibble with its top bit set replicates the
// sign of the selected byte (used to sign-extend packed int8 spins).
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ------------------------------------------------------------------------- smem layouts
__host__ __device__ inline size_t up16(size_t x) { return (x + 15) & ~(size_t)15; }

// Byte-wise path (any even P, any degree up to 32).
// Threshold rows and per-rung statistics in shared memory (when they fit).
__host__ __device__ inline size_t thr_bytes(const DevProblem& p) {
    return up16((size_t)(p.tables_in_smem ? p.R : 1) * p.nL3 * 4);
}
__host__ __device__ inline size_t acc_bytes(const DevProblem& p) {
    return p.acc_in_smem ? (size_t)p.R * kAccCount * 8 : 0;
}

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
// slot points at it), per-position unit descriptors, the schedule (read by the random-word
// producer), level offsets, the threshold row, reduction scratch, control words and, when
// the random words are produced ahead, two buffers of one sweep's words each.
struct FastLayout {
    size_t spins, ones, desc, items, loff, thr, acc, red, ctl, rbuf, total;
    __host__ __device__ FastLayout(const DevProblem& p, int dc, bool pre) {
        const int N = p.N, P = p.P;
        size_t o = 0;
        spins = o; o += up16((size_t)N * P);
        ones = o;  o += up16((size_t)P);
        desc = o;  o += (size_t)2 * N * (dc == 4 ? 32 : 64);
        items = o; o += up16((size_t)2 * N * 4);
        loff = o;  o += up16((size_t)(p.n_levels + 1) * 4);
        thr = o;   o += thr_bytes(p);
        acc = o;   o += acc_bytes(p);
        red = o;   o += 32 * 3 * 8;
        ctl = o;   o += 16;
        rbuf = o;
        if (pre) o += (size_t)2 * (2 * N) * (P / 8) * 16;
        total = o;
    }
};

size_t sweep_smem_bytes(const DevProblem& p, int path, int dclass) {
    if (path == kPathGeneric) return GenericLayout(p).total;
    return FastLayout(p, dclass, path == kPathPacked).total;
}

__device__ __forceinline__ void named_barrier(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// ------------------------------------------------------------------------- end of a sweep
__device__ __forceinline__ unsigned long long mbox_tag(long long q) {
    return (unsigned long long)(q % kTagPeriod) + 1ull;
}

// Thread 0 of a chain's CTA, after the sweep's changes are reduced: update E and M, add the
// statistics of the rung the chain sits on (to `acc`, shared or global), and run the chain's
// side of swap pass q when one follows this sweep. Returns the chain's rung for the next
// sweep; sets *abort when the partner's mailbox never arrived within the time limit.
__device__ int end_of_sweep(const DevProblem& p, unsigned long long* acc, int rung, long long& E, long long& M,
                            long long dE, long long dM, long long nflip, int s, long long q0, int sweeps_per_swap,
                            long long timeout_ns, const PhiloxKey& key, int* abort) {
    E += dE;
    M += dM;
    unsigned long long* a = acc + (size_t)rung * kAccCount;
    if (p.acc_in_smem) {
        a[kAccN] += 1ull;
        a[kAccE] += (unsigned long long)E;
        a[kAccE2] += (unsigned long long)(E * E);
        a[kAccM] += (unsigned long long)M;
        a[kAccM2] += (unsigned long long)(M * M);
        a[kAccFlip] += (unsigned long long)nflip;
    } else {
        atomicAdd(a + kAccN, 1ull);
        atomicAdd(a + kAccE, (unsigned long long)E);
        atomicAdd(a + kAccE2, (unsigned long long)(E * E));
        atomicAdd(a + kAccM, (unsigned long long)M);
        atomicAdd(a + kAccM2, (unsigned long long)(M * M));
        atomicAdd(a + kAccFlip, (unsigned long long)nflip);
    }
    *abort = 0;
    if (sweeps_per_swap <= 0 || (s + 1) % sweeps_per_swap != 0) return rung;
    const int R = p.R;
    const int pass = (s + 1) / sweeps_per_swap - 1;
    const long long q = q0 + pass;
    const unsigned long long tag = mbox_tag(q);
    Mailbox* mb = p.mbox + (size_t)pass * R;
    if (rung != p.withhold_rung) {
        st_relaxed_u64(&mb[rung].a, ((unsigned long long)E << 24) | tag);
        st_relaxed_u64(&mb[rung].b, ((unsigned long long)(uint32_t)(int32_t)M << 32) | tag);
    }
    int rl, partner;
    if ((rung & 1) == (int)(q & 1)) {
        rl = rung;
        partner = rung + 1;
    } else {
        rl = rung - 1;
        partner = rung - 1;
    }
    if (rl < 0 || rl + 1 >= R) return rung;
    long long pE, pM;
    const unsigned long long start = globaltimer_ns();
    for (;;) {
        const unsigned long long wa = ld_relaxed_u64(&mb[partner].a);
        const unsigned long long wb = ld_relaxed_u64(&mb[partner].b);
        if ((wa & 0xFFFFFFull) == tag && (wb & 0xFFFFFFull) == tag) {
            pE = (long long)wa >> 24;
            pM = (long long)(int32_t)(uint32_t)(wb >> 32);
            break;
        }
        if ((long long)(globaltimer_ns() - start) > timeout_ns) {
            atomicCAS(p.status, 0, PT_ETIMEDOUT);
            *abort = 1;
            return rung;
        }
    }
    const bool lower = (rung == rl);
    const bool acc_swap = swap_accept_fast(lower ? E : pE, lower ? pE : E, lower ? M : pM, lower ? pM : M,
                                           p.coef[rl], p.coef[(R - 1) + rl], (uint32_t)q, (uint32_t)rl, key,
                                           p.exact_swaps != 0);
    if (lower) {
        atomicAdd(p.swap_stats + 2 * rl, 1ull);
        if (acc_swap) atomicAdd(p.swap_stats + 2 * rl + 1, 1ull);
    }
    return acc_swap ? partner : rung;
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

// ------------------------------------------------------------------------- packed sweep
// Random words of one sweep for the producer warps: word w of philox((t, i, slot,
// p<<24 | g)) goes with copy 8g + p + 2w of site i (the same counter the update would use).
__device__ __forceinline__ void produce_words(uint4* buf, uint32_t t, const uint32_t* s_items, int n_items, int G,
                                              int lg, int gmask, int ptid, int np, uint32_t slot,
                                              const PhiloxKey& key) {
    const int total = n_items << lg;
    for (int x = ptid; x < total; x += np) {
        const int g = x & gmask;
        if (g >= G) continue;
        const int q = x >> lg;
        const uint32_t it = s_items[q];
        buf[q * G + g] = philox(make_uint4(t, it >> 1, slot, ((it & 1u) << 24) | (uint32_t)g), key);
    }
}

// One 4-copy unit of the packed path: copies k = 8g + par + 2w (w = 0..3) of site i.
// Each neighbour row contributes one 8-byte load; the field of the four copies comes from
// a 4x4 byte transpose and dp4a (the site's h rides in a spare neighbour slot whose spins
// are the constant +1 row); the Trotter column m/2+1 = 2 - [left differs] - [right differs]
// is formed for all four copies at once from byte XORs.
template <int DC, bool PRE>
__device__ __forceinline__ void packed_unit(int8_t* sp, const uint32_t* desc, const uint4* rb, int q, int g, int G,
                                            int P, uint32_t t, uint32_t slot, const PhiloxKey& key,
                                            const uint32_t* thr_c, int& sumL, int& sumC, int& nflip) {
    const uint4 d0 = *reinterpret_cast<const uint4*>(desc);
    const uint32_t row = d0.x;
    const uint32_t par = d0.y >> 31;
    const uint32_t c = 8u * (uint32_t)g;
    uint32_t nrow[DC];
    uint32_t jpack[DC / 4];
    {
        const uint4 d1 = *reinterpret_cast<const uint4*>(desc + 4);
        nrow[0] = d1.x;
        nrow[1] = d1.y;
        nrow[2] = d1.z;
        nrow[3] = d1.w;
        jpack[0] = d0.z;
        if (DC == 8) {
            const uint4 d2 = *reinterpret_cast<const uint4*>(desc + 8);
            nrow[DC > 4 ? 4 : 0] = d2.x;
            nrow[DC > 5 ? 5 : 0] = d2.y;
            nrow[DC > 6 ? 6 : 0] = d2.z;
            nrow[DC > 7 ? 7 : 0] = d2.w;
            jpack[DC > 4 ? 1 : 0] = d0.w;
        }
    }
    const uint2 own = *reinterpret_cast<const uint2*>(sp + row + c);
    // the one Trotter neighbour outside the chunk: copy c-1 for even copies, c+8 for odd
    const uint32_t eoff = par ? (c + 8 == (uint32_t)P ? 0u : c + 8) : (c == 0 ? (uint32_t)P - 1 : c - 1);
    const uint32_t edge = (uint8_t)sp[row + eoff];
    uint2 nb[DC];
#pragma unroll
    for (int d = 0; d < DC; ++d) nb[d] = *reinterpret_cast<const uint2*>(sp + nrow[d] + c);
    uint4 r4;
    if (PRE) {
        r4 = rb[q * G + g];
    } else {
        r4 = philox(make_uint4(t, d0.y & 0x7FFFFFFFu, slot, (par << 24) | (uint32_t)g), key);
    }
    const uint32_t u[4] = {r4.x, r4.y, r4.z, r4.w};

    const uint32_t selS = par ? 0x7531u : 0x6420u;
    const uint32_t S = __byte_perm(own.x, own.y, selS);
    uint32_t Rn = __byte_perm(own.x, own.y, par ? 0x0642u : 0x7531u);
    Rn = par ? __byte_perm(Rn, edge, 0x4210u) : Rn;
    uint32_t Ln = __byte_perm(own.x, own.y, par ? 0x6420u : 0x5310u);
    Ln = par ? Ln : __byte_perm(Ln, edge, 0x3214u);
    const uint32_t X = (S ^ Ln) & 0x02020202u;
    const uint32_t Y = (S ^ Rn) & 0x02020202u;
    const uint32_t Z = 0x02020202u - ((X + Y) >> 1);

    int f[4] = {0, 0, 0, 0};
#pragma unroll
    for (int b = 0; b < DC / 4; ++b) {
        const uint32_t a0 = __byte_perm(nb[4 * b + 0].x, nb[4 * b + 0].y, selS);
        const uint32_t a1 = __byte_perm(nb[4 * b + 1].x, nb[4 * b + 1].y, selS);
        const uint32_t a2 = __byte_perm(nb[4 * b + 2].x, nb[4 * b + 2].y, selS);
        const uint32_t a3 = __byte_perm(nb[4 * b + 3].x, nb[4 * b + 3].y, selS);
        const uint32_t t0 = __byte_perm(a0, a1, 0x5140u), t1 = __byte_perm(a0, a1, 0x7362u);
        const uint32_t t2 = __byte_perm(a2, a3, 0x5140u), t3 = __byte_perm(a2, a3, 0x7362u);
        f[0] = __dp4a((int)__byte_perm(t0, t2, 0x5410u), (int)jpack[b], f[0]);
        f[1] = __dp4a((int)__byte_perm(t0, t2, 0x7632u), (int)jpack[b], f[1]);
        f[2] = __dp4a((int)__byte_perm(t1, t3, 0x5410u), (int)jpack[b], f[2]);
        f[3] = __dp4a((int)__byte_perm(t1, t3, 0x7632u), (int)jpack[b], f[3]);
    }
    uint32_t F = 0;  // 0xFE in byte w when copy w flips (XOR turns +1 <-> -1)
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const int sw = (int)prmt(S, 0u, 0x8880u | (0x1110u * (uint32_t)w) | (uint32_t)w);
        const int Lw = sw * f[w];
        const int col = (int)__byte_perm(Z, 0u, 0x4440u | (uint32_t)w);
        const uint32_t th = thr_c[3 * Lw + col];
        const bool acc = (u[w] < th) | (th == 0xFFFFFFFFu);
        F |= acc ? (0xFEu << (8 * w)) : 0u;
        sumL += acc ? Lw : 0;
    }
    // flips and their Trotter columns from the packed flip mask
    nflip += __popc(F & 0x02020202u);
    sumC = __dp4a((int)(Z & (F >> 1)), 0x01010101, sumC);
    if (F) {
        const uint32_t lo = __byte_perm(F, 0u, par ? 0x1404u : 0x4140u);
        const uint32_t hi = __byte_perm(F, 0u, par ? 0x3424u : 0x4342u);
        *reinterpret_cast<uint2*>(sp + row + c) = make_uint2(own.x ^ lo, own.y ^ hi);
    }
}

// One CTA per chain with the chain, the unit descriptors and the threshold row in shared
// memory. PRE: the last (blockDim - n_consumer) threads are producer warps that write the
// random words of sweep s+1 into one shared buffer while the consumer warps run the levels
// of sweep s out of the other; consumers synchronise levels on named barrier 1 and both
// groups meet once per sweep.
template <int DC, bool PRE, int MAXT>
__global__ void __launch_bounds__(MAXT, 1)
sweep_packed_kernel(DevProblem p, long long t0, long long q0, int n_sweeps, int sweeps_per_swap,
                    long long timeout_ns, int n_consumer) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = p.N, P = p.P;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int slot = blockIdx.x;
    const FastLayout L(p, DC, PRE);
    int8_t* sp = reinterpret_cast<int8_t*>(smem + L.spins);
    uint32_t* s_desc = reinterpret_cast<uint32_t*>(smem + L.desc);
    uint32_t* s_items = reinterpret_cast<uint32_t*>(smem + L.items);
    int32_t* s_loff = reinterpret_cast<int32_t*>(smem + L.loff);
    uint32_t* s_thr = reinterpret_cast<uint32_t*>(smem + L.thr);
    long long* s_red = reinterpret_cast<long long*>(smem + L.red);
    int* s_ctl = reinterpret_cast<int*>(smem + L.ctl);
    uint4* rbuf = reinterpret_cast<uint4*>(smem + L.rbuf);
    unsigned long long* s_acc = reinterpret_cast<unsigned long long*>(smem + L.acc);
    const int NC = PRE ? n_consumer : nt;
    const bool consumer = tid < NC;
    const int DW = (DC == 4) ? 8 : 16;

    {
        const int4* src = reinterpret_cast<const int4*>(p.spins + (size_t)slot * p.slot_stride);
        int4* dst = reinterpret_cast<int4*>(sp);
        const int n16 = (int)(up16((size_t)N * P) / 16);
        for (int x = tid; x < n16; x += nt) dst[x] = src[x];
        int8_t* ones = reinterpret_cast<int8_t*>(smem + L.ones);
        for (int x = tid; x < P; x += nt) ones[x] = 1;
        const int4* dsrc = reinterpret_cast<const int4*>(p.desc);
        int4* ddst = reinterpret_cast<int4*>(s_desc);
        for (int x = tid; x < 2 * N * DW / 4; x += nt) ddst[x] = dsrc[x];
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
    const int lane = tid & 31, warp = tid >> 5;
    __syncthreads();
    if (PRE && !consumer)
        produce_words(rbuf, (uint32_t)t0, s_items, n_items, G, lg, gmask, tid - NC, nt - NC, (uint32_t)slot, key);
    if (PRE) __syncthreads();

    for (int s = 0; s < n_sweeps; ++s) {
        const uint32_t t = (uint32_t)(t0 + s);
        if (consumer) {
            const uint4* rb = rbuf + (size_t)(s & 1) * n_items * G;
            int sumL = 0, sumC = 0, nf = 0;
            for (int lev = 0; lev < p.n_levels; ++lev) {
                const int base = s_loff[lev];
                const int units = (s_loff[lev + 1] - base) << lg;
                for (int u = tid; u < units; u += NC) {
                    const int g = u & gmask;
                    if (g >= G) continue;
                    const int q = base + (u >> lg);
                    packed_unit<DC, PRE>(sp, s_desc + (size_t)q * DW, rb, q, g, G, P, t, (uint32_t)slot, key, thr_c,
                                         sumL, sumC, nf);
                }
                if (PRE) named_barrier(1, NC); else __syncthreads();
            }
            int dE = -2 * sumL, dM = -4 * (sumC - nf);
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
            if (PRE) named_barrier(1, NC); else __syncthreads();
            if (tid == 0) {
                long long sE = 0, sM = 0, sF = 0;
                for (int w = 0; w < NC / 32; ++w) {
                    sE += s_red[w * 3 + 0];
                    sM += s_red[w * 3 + 1];
                    sF += s_red[w * 3 + 2];
                }
                int abort_flag = 0;
                s_ctl[2 * (s & 1)] = end_of_sweep(p, p.acc_in_smem ? s_acc : p.acc, rung, E, M, sE, sM, sF, s,
                                                  q0, sweeps_per_swap, timeout_ns, key, &abort_flag);
                s_ctl[2 * (s & 1) + 1] = abort_flag;
            }
            if (PRE) named_barrier(1, NC); else __syncthreads();
            const int nr = s_ctl[2 * (s & 1)];
            if (!s_ctl[2 * (s & 1) + 1] && nr != rung) {
                rung = nr;
                if (!p.tables_in_smem) load_thr(p, s_thr, rung, tid, NC);
                thr_c = thr_row(p, s_thr, rung) + 3 * p.Lmax;
            }
        } else if (s + 1 < n_sweeps) {
            produce_words(rbuf + (size_t)((s + 1) & 1) * n_items * G, t + 1u, s_items, n_items, G, lg, gmask,
                          tid - NC, nt - NC, (uint32_t)slot, key);
        }
        __syncthreads();
        if (s_ctl[2 * (s & 1) + 1]) return;  // a partner never arrived; status holds PT_ETIMEDOUT
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
    for (int x = threadIdx.x; x < p.N * p.P; x += blockDim.x) dst[x] = src[x];
}

__global__ void scatter_kernel(DevProblem p, const int8_t* in) {
    const int r = blockIdx.x;
    int8_t* dst = p.spins + (size_t)p.slot_of_rung[r] * p.slot_stride;
    const int8_t* src = in + (size_t)r * p.N * p.P;
    for (int x = threadIdx.x; x < p.N * p.P; x += blockDim.x) dst[x] = src[x];
}

// ------------------------------------------------------------------------- launchers
static const void* sweep_fn(const LaunchPlan& plan) {
    if (plan.path == kPathGeneric) {
        switch (plan.dclass) {
            case 4: return (const void*)sweep_kernel<4>;
            case 8: return (const void*)sweep_kernel<8>;
            default: return (const void*)sweep_kernel<32>;
        }
    }
    const bool pre = plan.path == kPathPacked;
    if (plan.threads > 512) {
        if (plan.dclass == 4)
            return pre ? (const void*)sweep_packed_kernel<4, true, 1024> : (const void*)sweep_packed_kernel<4, false, 1024>;
        return pre ? (const void*)sweep_packed_kernel<8, true, 1024> : (const void*)sweep_packed_kernel<8, false, 1024>;
    }
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
    return cudaFuncSetAttribute(sweep_fn(plan), cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
}

cudaError_t sweep_kernel_occupancy(const DevProblem& p, const LaunchPlan& plan, int* blocks_per_sm) {
    (void)p;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, sweep_fn(plan), plan.threads,
                                                         plan.smem_bytes);
}

cudaError_t launch_sweeps(const DevProblem& p, const LaunchPlan& plan, long long t0, long long q0,
                          int n_sweeps, int sweeps_per_swap, long long timeout_ns, bool cooperative,
                          cudaStream_t s) {
    DevProblem pp = p;
    int n_consumer = plan.n_consumer;
    void* args[] = {&pp, &t0, &q0, &n_sweeps, &sweeps_per_swap, &timeout_ns, &n_consumer};
    const void* fn = sweep_fn(plan);
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
