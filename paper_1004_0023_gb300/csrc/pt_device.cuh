// pt_device.cuh -- device building blocks shared by the PT-QMC kernels: Philox4x32-10,
// the deterministic exp and swap rule, PTX helpers and the packed 4-copy update unit.
#pragma once

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
    __device__ __forceinline__ uint32_t a(int r) const { return k0[r]; }
    __device__ __forceinline__ uint32_t b(int r) const { return k1[r]; }
};

// The same round keys read from shared memory, for kernels that cannot spare 20 registers
// per thread for them: rounds 2j and 2j+1 in one 16-byte word k[j] = (k0, k1, k0', k1'), so a
// pair of rounds costs one shared load.
struct PhiloxKeyShared {
    const uint4* k;
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

__device__ __forceinline__ uint4 philox_round(uint4 c, uint32_t ka, uint32_t kb) {
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
    return make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ ka, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ kb, (uint32_t)p0);
}

__device__ __forceinline__ uint4 philox(uint4 c, const PhiloxKey& k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) c = philox_round(c, k.a(r), k.b(r));
    return c;
}

__device__ __forceinline__ uint4 philox(uint4 c, const PhiloxKeyShared& k) {
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const uint4 kk = k.k[j];
        c = philox_round(c, kk.x, kk.y);
        c = philox_round(c, kk.z, kk.w);
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

// The uniform word of swap pass q for the pair (rl, rl + 1).
template <typename Key = PhiloxKey>
__device__ __forceinline__ uint32_t swap_word(uint32_t q, uint32_t rl, const Key& key) {
    return philox(make_uint4(q, rl, 0u, kTagSwap << 28), key).x;
}

// Swap decision for X on rung rl and Y on rung rl + 1, with the pass's uniform word from
// word() (called only when Delta falls in the band where it matters).
template <typename WordFn>
__device__ __forceinline__ bool swap_accept_by(long long EX, long long EY, long long MX, long long MY, double a,
                                               double c, WordFn word) {
    const double dE = __ll2double_rn(EX - EY);
    const double dM = __ll2double_rn(MX - MY);
    const double delta = __dadd_rn(__dmul_rn(a, dE), __dmul_rn(c, dM));
    if (delta >= 0.0) return true;
    if (!(delta > -23.0)) return false;
    const double v = floor(__dmul_rn(det_exp(delta), 4294967296.0));
    const uint32_t ts = (v >= 4294967295.0) ? 0xFFFFFFFFu : (uint32_t)v;
    return word() < ts;
}

// The same decision without FP64 in the common case. GB300's FP64 pipe makes the ~40
// dependent FP64 operations of swap_accept_by cost over a microsecond, so Delta and exp(Delta)
// are first estimated in FP32 with an error bound:
//   |D - Delta| <= err = 5*2^-24 * (|a dE| + |c dM|)   (conversions of a, c, dE, dM, two
//   products, one sum, and the FP64 roundings of Delta itself, with room to spare), and
//   2^32 exp(D) within a relative 1e-5 + 1.01 err of 2^32 exp(Delta) (expf is within 2 ulp).
// The estimate decides only when u is farther than that margin (plus float rounding of u)
// from the threshold, or Delta's sign and the -23 cut are certain; otherwise swap_accept_by
// decides. Either way the result equals swap_accept_by's.
template <typename WordFn>
__device__ __forceinline__ bool swap_accept_fast_by(long long EX, long long EY, long long MX, long long MY,
                                                    double a, double c, WordFn word, bool exact_only) {
    if (!exact_only) {
        const float pa = (float)a * (float)(EX - EY);
        const float pc = (float)c * (float)(MX - MY);
        const float D = pa + pc;
        const float err = (fabsf(pa) + fabsf(pc)) * 2.99e-7f + 1e-30f;
        if (D >= 2.0f * err) return true;                       // Delta >= 0
        if (err < 0.25f) {
            if (D < -23.5f) return false;                         // Delta <= -23
            if (D + 2.0f * err < 0.0f && D > -22.5f) {
                const float v = 4294967296.0f * expf(D);
                const float margin = v * (1.0e-5f + 1.01f * err) + 512.0f;
                const float uf = (float)word();
                if (uf + margin < v) return true;
                if (uf - margin > v) return false;
            }
        }
    }
    return swap_accept_by(EX, EY, MX, MY, a, c, word);
}

// The two rules with the word drawn from (q, rl) under `key` when needed.
template <typename Key = PhiloxKey>
__device__ __forceinline__ bool swap_accept(long long EX, long long EY, long long MX, long long MY,
                                            double a, double c, uint32_t q, uint32_t rl,
                                            const Key& key) {
    return swap_accept_by(EX, EY, MX, MY, a, c, [&] { return swap_word(q, rl, key); });
}
template <typename Key = PhiloxKey>
__device__ __forceinline__ bool swap_accept_fast(long long EX, long long EY, long long MX, long long MY,
                                                 double a, double c, uint32_t q, uint32_t rl,
                                                 const Key& key, bool exact_only) {
    return swap_accept_fast_by(EX, EY, MX, MY, a, c, [&] { return swap_word(q, rl, key); }, exact_only);
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
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ------------------------------------------------------------------------- misc
__host__ __device__ inline size_t up16(size_t x) { return (x + 15) & ~(size_t)15; }

// Every thread of every CTA of the cluster: release this CTA's shared-memory writes (own and
// remote) and acquire the others'. The non-.aligned form, so threads of a warp may arrive
// from different branches.
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// The two halves of a cluster barrier, for CTAs whose arrival orders none of their own
// earlier writes for the peers (relaxed) or does (release), and whose wait must see the
// peers' writes (acquire). A release arrival also waits for the thread's earlier global
// stores, which a relaxed one does not.
__device__ __forceinline__ void cluster_arrive_relaxed() { asm volatile("barrier.cluster.arrive.relaxed;" ::: "memory"); }
__device__ __forceinline__ void cluster_arrive_release() { asm volatile("barrier.cluster.arrive.release;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait_acquire() { asm volatile("barrier.cluster.wait.acquire;" ::: "memory"); }

// Two adjacent 64-bit words (16-byte aligned) into CTA `rank`'s copy of a shared-memory
// location (distributed shared memory), in one store, relaxed at cluster scope: each word
// carries its own tag and the readers poll the words themselves, so no other ordering is
// needed.
__device__ __forceinline__ void st_cluster_u64x2(const void* local, unsigned rank, unsigned long long a,
                                                 unsigned long long b) {
    const unsigned l = (unsigned)__cvta_generic_to_shared(local);
    unsigned ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(l), "r"(rank));
    asm volatile("st.relaxed.cluster.shared::cluster.v2.u64 [%0], {%1, %2};" ::"r"(ra), "l"(a), "l"(b) : "memory");
}

// This CTA's shared-memory word, as the other CTAs of the cluster last wrote it.
__device__ __forceinline__ unsigned long long ld_cluster_local_u64(const void* local) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(local);
    unsigned long long v;
    asm volatile("ld.relaxed.cluster.shared::cta.u64 %0, [%1];" : "=l"(v) : "r"(a) : "memory");
    return v;
}

__device__ __forceinline__ void named_barrier(int id, int count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Shared-memory rows of the int8 packed path are split by parity: row i holds the P/2 even
// copies of site i, then its P/2 odd copies, so the 4 copies of one parity in an update
// unit are one aligned word. Global rows interleave the copies (k fastest); these convert
// one 8-copy chunk (copies 8g..8g+7) between the two layouts.
__device__ __forceinline__ void split_chunk(uint2 v, uint32_t& even, uint32_t& odd) {
    even = __byte_perm(v.x, v.y, 0x6420u);
    odd = __byte_perm(v.x, v.y, 0x7531u);
}
__device__ __forceinline__ uint2 join_chunk(uint32_t even, uint32_t odd) {
    return make_uint2(__byte_perm(even, odd, 0x5140u), __byte_perm(even, odd, 0x7362u));
}

// ceil(2^32 / G) for G > 1: with it, __umulhi(x, ginv) = x / G exactly while x * G < 2^32,
// which holds for every chunk index of a chain that fits in shared memory. 0 for G = 1.
__host__ __device__ inline uint32_t chunk_ginv(int G) {
    return G > 1 ? (uint32_t)((0x100000000ull + (unsigned long long)G - 1ull) / (unsigned long long)G) : 0u;
}
__device__ __forceinline__ int chunk_of_row(int x, int G, uint32_t ginv) {
    return ginv ? x - G * (int)__umulhi((uint32_t)x, ginv) : 0;
}

// Copy an interleaved chain (N sites x P copies, global) into the split layout (shared),
// threads [tid0, tid0 + nthr) taking 8-copy chunks; and back. G = P / 8, ginv = chunk_ginv(G).
__device__ __forceinline__ void load_split(int8_t* dst, const int8_t* src, int N, int P, int G, uint32_t ginv,
                                           int tid0, int nthr) {
    const uint2* s2 = reinterpret_cast<const uint2*>(src);
    const int half = P >> 1;
    const int n = N * G;
    // eight loads in flight per thread before any shared store (the stores could alias the
    // loads as far as the compiler knows, which would otherwise serialise every load)
    for (int x0 = tid0; x0 < n; x0 += 8 * nthr) {
        uint2 v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int x = x0 + k * nthr;
            v[k] = x < n ? s2[x] : make_uint2(0u, 0u);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int x = x0 + k * nthr;
            if (x < n) {
                const int g = chunk_of_row(x, G, ginv);
                const int row = 8 * x - 8 * g;  // i * P
                uint32_t ev, od;
                split_chunk(v[k], ev, od);
                *reinterpret_cast<uint32_t*>(dst + row + 4 * g) = ev;
                *reinterpret_cast<uint32_t*>(dst + row + half + 4 * g) = od;
            }
        }
    }
}
__device__ __forceinline__ void store_split(int8_t* dst, const int8_t* src, int N, int P, int G, uint32_t ginv,
                                            int tid0, int nthr) {
    uint2* d2 = reinterpret_cast<uint2*>(dst);
    const int half = P >> 1;
    for (int x = tid0; x < N * G; x += nthr) {
        const int g = chunk_of_row(x, G, ginv);
        const int row = 8 * x - 8 * g;
        d2[x] = join_chunk(*reinterpret_cast<const uint32_t*>(src + row + 4 * g),
                           *reinterpret_cast<const uint32_t*>(src + row + half + 4 * g));
    }
}

// The same copies for rows of a multiple of 16 copies, 16 copies (one 16-byte word) at a
// time: half the loads, stores and index arithmetic of the 8-copy form per byte. H = P / 16,
// hinv = chunk_ginv(H).
__device__ __forceinline__ void load_split16(int8_t* dst, const int8_t* src, int N, int P, int H, uint32_t hinv,
                                             int tid0, int nthr) {
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    const int half = P >> 1;
    const int n = N * H;
    for (int x0 = tid0; x0 < n; x0 += 4 * nthr) {
        uint4 v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int x = x0 + k * nthr;
            v[k] = x < n ? s4[x] : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int x = x0 + k * nthr;
            if (x < n) {
                const int h = chunk_of_row(x, H, hinv);
                const int row = 16 * x - 16 * h;  // i * P
                uint2 ev, od;
                split_chunk(make_uint2(v[k].x, v[k].y), ev.x, od.x);  // copies 16h .. 16h+7
                split_chunk(make_uint2(v[k].z, v[k].w), ev.y, od.y);  // copies 16h+8 .. 16h+15
                *reinterpret_cast<uint2*>(dst + row + 8 * h) = ev;
                *reinterpret_cast<uint2*>(dst + row + half + 8 * h) = od;
            }
        }
    }
}
__device__ __forceinline__ void store_split16(int8_t* dst, const int8_t* src, int N, int P, int H, uint32_t hinv,
                                              int tid0, int nthr) {
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    const int half = P >> 1;
    const int n = N * H;
    for (int x0 = tid0; x0 < n; x0 += 4 * nthr) {
        uint2 ev[4], od[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int x = min(x0 + k * nthr, n - 1);
            const int h = chunk_of_row(x, H, hinv);
            const int row = 16 * x - 16 * h;
            ev[k] = *reinterpret_cast<const uint2*>(src + row + 8 * h);
            od[k] = *reinterpret_cast<const uint2*>(src + row + half + 8 * h);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int x = x0 + k * nthr;
            if (x < n) {
                const uint2 lo = join_chunk(ev[k].x, od[k].x), hi = join_chunk(ev[k].y, od[k].y);
                d4[x] = make_uint4(lo.x, lo.y, hi.x, hi.y);
            }
        }
    }
}

// One 4-copy unit of the packed path: copies k = 8g + par + 2w (w = 0..3) of site i, which
// are bytes 4g..4g+3 of the row's parity-par half.
// Site descriptor (DW words): row offset i*P, i, packed J bytes (two words), then the row
// offsets of the DC neighbour slots (the slot after the last neighbour holds h against the
// constant +1 row; the remaining slots have J = 0).
// Each neighbour slot contributes one word (its 4 copies) to field_times_spin, which forms
// L = s (h + sum_j J_ij s_j) of the four copies. The Trotter column
// m/2+1 = 2 - [left differs] - [right differs] comes from the opposite-parity word and one
// edge byte with byte XORs.
template <int DC>
struct SiteDesc {
    static constexpr int DW = (DC == 4) ? 8 : 12;
};

// L_w = s_w (h + sum_j J_j s_j,w) for the four copies w of a unit, from the DC neighbour
// words a[d] (4 copies of slot d as +-1 bytes), the own word S and the J bytes. A 4x4 byte
// transpose per four slots feeds dp4a. With four slots the neighbour bytes are first
// multiplied by the own spins ((a ^ s) | 1 is the product of two +-1 bytes), so dp4a gives
// L directly; with eight the field is formed first and multiplied by the spin after, which
// takes fewer ALU operations.
template <int DC>
__device__ __forceinline__ void field_times_spin(const uint32_t* a, uint32_t S, const uint32_t* jpack, int* L) {
    int f[4] = {0, 0, 0, 0};
#pragma unroll
    for (int b = 0; b < DC / 4; ++b) {
        uint32_t a0 = a[4 * b + 0], a1 = a[4 * b + 1], a2 = a[4 * b + 2], a3 = a[4 * b + 3];
        if (DC == 4) {
            a0 = (a0 ^ S) | 0x01010101u;
            a1 = (a1 ^ S) | 0x01010101u;
            a2 = (a2 ^ S) | 0x01010101u;
            a3 = (a3 ^ S) | 0x01010101u;
        }
        const uint32_t t0 = __byte_perm(a0, a1, 0x5140u), t1 = __byte_perm(a0, a1, 0x7362u);
        const uint32_t t2 = __byte_perm(a2, a3, 0x5140u), t3 = __byte_perm(a2, a3, 0x7362u);
        f[0] = __dp4a((int)__byte_perm(t0, t2, 0x5410u), (int)jpack[b], f[0]);
        f[1] = __dp4a((int)__byte_perm(t0, t2, 0x7632u), (int)jpack[b], f[1]);
        f[2] = __dp4a((int)__byte_perm(t1, t3, 0x5410u), (int)jpack[b], f[2]);
        f[3] = __dp4a((int)__byte_perm(t1, t3, 0x7632u), (int)jpack[b], f[3]);
    }
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        if (DC == 4) {
            L[w] = f[w];
        } else {
            const int sw = (int)(int8_t)((S >> (8 * w)) & 0xFFu);  // +1 or -1
            L[w] = sw * f[w];
        }
    }
}

// All ones when the attempt with random word u is accepted against threshold th, else zero:
// u < th, read off the borrow of u - th (one subtract with carry out, one subtract of the
// carry), so that the flip mask and the sums below are formed by multiply-adds on the FMA
// pipe instead of compares and selects on the ALU pipe. Inline words (PRE = false) are first
// capped at 2^32 - 2, which folds in the "accept always" entry 0xFFFFFFFF exactly.
template <bool PRE>
__device__ __forceinline__ uint32_t accept_mask(uint32_t u, uint32_t th) {
    if (!PRE) u = min(u, 0xFFFFFFFEu);
    uint32_t d, m;
    asm("sub.cc.u32 %0, %2, %3;\n\tsubc.u32 %1, 0, 0;" : "=r"(d), "=r"(m) : "r"(u), "r"(th));
    return m;
}

// Threshold entry thr_c[3 L + col] of copy w, col = byte w of Z: the byte offset
// 4 (3 L + col) comes out of one dp4a (Z's byte w times 4, plus 12 L), keeping the byte
// extraction and the index arithmetic off the ALU pipe.
__device__ __forceinline__ uint32_t thr_entry(const uint32_t* thr_c, uint32_t Z, int L, int w) {
    const int off = __dp4a((int)Z, 4 << (8 * w), 12 * L);
    return *reinterpret_cast<const uint32_t*>(reinterpret_cast<const char*>(thr_c) + off);
}

// The packed unit in three steps, so that a unit can be evaluated before the threshold row
// it needs is known: evaluate (loads, fields, Trotter columns, random words), decide the
// flips against one threshold row, commit (flip store and the sweep's sums).
struct UnitEval {
    uint32_t* own;  // the unit's word in shared memory
    uint32_t S;     // its 4 copies as +-1 bytes
    uint32_t Z;     // Trotter column m/2+1 per copy
    int L[4];       // L = s (h + sum_j J s_j) per copy
    uint32_t u[4];  // random words
};

template <int DC, bool PRE, typename Key = PhiloxKey>
__device__ __forceinline__ UnitEval packed_unit_eval(int8_t* sp, const uint32_t* s_sdesc, uint32_t item,
                                                     const uint4* rb, int q, int g, int G, int P, uint32_t t,
                                                     uint32_t slot, const Key& key) {
    UnitEval e;
    const uint32_t par = item & 1u;
    const uint32_t* desc = s_sdesc + (item >> 1) * SiteDesc<DC>::DW;
    const uint4 d0 = *reinterpret_cast<const uint4*>(desc);
    const uint32_t half = (uint32_t)P >> 1;
    const uint32_t w4 = 4u * (uint32_t)g;
    const uint32_t own_off = par * half + w4;  // this parity's word in every row
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
    const uint32_t row = d0.x;
    e.own = reinterpret_cast<uint32_t*>(sp + row + own_off);
    const uint32_t S = *e.own;
    const uint32_t O = *reinterpret_cast<const uint32_t*>(sp + row + (half - par * half) + w4);
    // the one Trotter neighbour outside the word: odd copy 8g-1 for even copies, even copy
    // 8g+8 for odd ones (periodic); parity selects by multiply-add, not by select
    const uint32_t e_even = half + (g == 0 ? half - 1u : w4 - 1u);
    const uint32_t e_odd = (w4 + 4u == half) ? 0u : w4 + 4u;
    const uint32_t edge = (uint8_t)sp[row + e_even + par * (e_odd - e_even)];
    uint32_t a[DC];
#pragma unroll
    for (int d = 0; d < DC; ++d) a[d] = *reinterpret_cast<const uint32_t*>(sp + nrow[d] + own_off);
    uint4 r4;
    if (PRE) {
        r4 = rb[q * G + g];
    } else {
        r4 = philox(make_uint4(t, d0.y, slot, (par << 24) | (uint32_t)g), key);
    }
    e.u[0] = r4.x;
    e.u[1] = r4.y;
    e.u[2] = r4.z;
    e.u[3] = r4.w;

    // left / right Trotter neighbours: the opposite-parity word itself or shifted by one byte
    // with the edge copy (selectors 0x3210 = itself, 0x2104 = up, 0x4321 = down)
    const uint32_t Ln = __byte_perm(O, edge, 0x2104u + par * (0x3210u - 0x2104u));
    const uint32_t Rn = __byte_perm(O, edge, 0x3210u + par * (0x4321u - 0x3210u));
    const uint32_t X = (S ^ Ln) & 0x02020202u;
    const uint32_t Y = (S ^ Rn) & 0x02020202u;
    e.Z = 0x02020202u - ((X + Y) >> 1);
    e.S = S;
    field_times_spin<DC>(a, S, jpack, e.L);
    return e;
}

// 0xFE in byte w when copy w flips under the threshold row thr_c (offset to L = 0, m = -2).
// Produced words (PRE) are already min(u, 2^32 - 2), which folds in the "always" entry.
template <bool PRE>
__device__ __forceinline__ uint32_t unit_flips(const UnitEval& e, const uint32_t* thr_c) {
    uint32_t F = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        F -= accept_mask<PRE>(e.u[w], thr_entry(thr_c, e.Z, e.L[w], w)) * (0xFEu << (8 * w));
    }
    return F;
}

// sumC2 and nflip2 count twice the Trotter columns and the flips: the flip mask bytes
// (F & 0x02020202 = 2 per flip) feed dp4a directly.
__device__ __forceinline__ void unit_commit(const UnitEval& e, uint32_t F, int& sumL, int& sumC2, int& nflip2) {
#pragma unroll
    for (int w = 0; w < 4; ++w) sumL += ((F >> (8 * w)) & 0x2u) ? e.L[w] : 0;
    const uint32_t Fm = F & 0x02020202u;
    nflip2 = __dp4a((int)Fm, 0x01010101, nflip2);
    sumC2 = __dp4a((int)e.Z, (int)Fm, sumC2);
    if (F) *e.own = e.S ^ F;
}

template <int DC, bool PRE, typename Key = PhiloxKey>
__device__ __forceinline__ void packed_unit(int8_t* sp, const uint32_t* s_sdesc, uint32_t item, const uint4* rb,
                                            int q, int g, int G, int P, uint32_t t, uint32_t slot,
                                            const Key& key, const uint32_t* thr_c, int& sumL, int& sumC2,
                                            int& nflip2) {
    const UnitEval e = packed_unit_eval<DC, PRE, Key>(sp, s_sdesc, item, rb, q, g, G, P, t, slot, key);
    // flips and sums in one pass (the acceptance predicate feeds both)
    uint32_t F = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const uint32_t m = accept_mask<PRE>(e.u[w], thr_entry(thr_c, e.Z, e.L[w], w));
        F -= m * (0xFEu << (8 * w));
        sumL -= (int)m * e.L[w];
    }
    const uint32_t Fm = F & 0x02020202u;
    nflip2 = __dp4a((int)Fm, 0x01010101, nflip2);
    sumC2 = __dp4a((int)e.Z, (int)Fm, sumC2);
    if (F) *e.own = e.S ^ F;
}

// Byte offsets, within a shared-memory row, of what a unit of one fixed column reads: its
// own word, the opposite-parity word at the same copies, and the one Trotter neighbour
// outside that word. [0] for an even-copy unit, [1] for an odd one. Used by the split
// kernel, whose rows also hold copies of the neighbouring CTA.
struct UnitOffsets {
    uint32_t own[2], opp[2], edge[2];
};

// The packed unit evaluated from precomputed row offsets (the split kernel's rows). PRE: the
// random words are read from *rbq; else word w of philox((t, i, slot, p<<24 | gg)), gg the
// unit's 8-copy chunk in the whole chain.
template <int DC, bool PRE>
__device__ __forceinline__ UnitEval split_unit_eval(int8_t* sp, const uint32_t* s_sdesc, uint32_t item,
                                                    const uint4* rbq, const UnitOffsets& o, uint32_t t,
                                                    uint32_t slot, uint32_t gg, const PhiloxKey& key) {
    UnitEval e;
    const uint32_t par = item & 1u;
    const uint32_t* desc = s_sdesc + (item >> 1) * SiteDesc<DC>::DW;
    const uint4 d0 = *reinterpret_cast<const uint4*>(desc);
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
    const uint32_t row = d0.x;
    const uint32_t own_off = o.own[0] + par * (o.own[1] - o.own[0]);
    e.own = reinterpret_cast<uint32_t*>(sp + row + own_off);
    const uint32_t S = *e.own;
    const uint32_t O = *reinterpret_cast<const uint32_t*>(sp + row + o.opp[0] + par * (o.opp[1] - o.opp[0]));
    const uint32_t edge = (uint8_t)sp[row + o.edge[0] + par * (o.edge[1] - o.edge[0])];
    uint32_t a[DC];
#pragma unroll
    for (int d = 0; d < DC; ++d) a[d] = *reinterpret_cast<const uint32_t*>(sp + nrow[d] + own_off);
    const uint4 r4 = PRE ? *rbq : philox(make_uint4(t, d0.y, slot, (par << 24) | gg), key);
    e.u[0] = r4.x;
    e.u[1] = r4.y;
    e.u[2] = r4.z;
    e.u[3] = r4.w;
    const uint32_t Ln = __byte_perm(O, edge, 0x2104u + par * (0x3210u - 0x2104u));
    const uint32_t Rn = __byte_perm(O, edge, 0x3210u + par * (0x4321u - 0x3210u));
    const uint32_t X = (S ^ Ln) & 0x02020202u;
    const uint32_t Y = (S ^ Rn) & 0x02020202u;
    e.Z = 0x02020202u - ((X + Y) >> 1);
    e.S = S;
    field_times_spin<DC>(a, S, jpack, e.L);
    return e;
}

// Decide and commit in one pass (PRE: produced words, u < thr alone is the rule).
template <bool PRE>
__device__ __forceinline__ void unit_decide_commit(const UnitEval& e, const uint32_t* thr_c, int& sumL, int& sumC2,
                                                   int& nflip2) {
    uint32_t F = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const uint32_t m = accept_mask<PRE>(e.u[w], thr_entry(thr_c, e.Z, e.L[w], w));
        F -= m * (0xFEu << (8 * w));
        sumL -= (int)m * e.L[w];
    }
    const uint32_t Fm = F & 0x02020202u;
    nflip2 = __dp4a((int)Fm, 0x01010101, nflip2);
    sumC2 = __dp4a((int)e.Z, (int)Fm, sumC2);
    if (F) *e.own = e.S ^ F;
}

}  // namespace ptq

namespace ptq {

// Bit-packed chains (shared memory only): row i is P/8 bytes, bit k of byte g is copy 8g+k,
// set = spin -1. lut[p*256 + b] spreads the four parity-p bits (p, p+2, p+4, p+6) of byte b
// into four +1/-1 bytes, so each neighbour contributes one byte load and one table load and
// the field / Trotter logic of packed_unit is reused unchanged.
template <int DC, bool PRE>
__device__ __forceinline__ void packed_unit_bits(uint8_t* bp, const uint32_t* s_sdesc, uint32_t item,
                                                 const uint4* rb, int q, int g, int G, const uint32_t* lut,
                                                 uint32_t t, uint32_t slot, const PhiloxKey& key,
                                                 const uint32_t* thr_c, int& sumL, int& sumC2, int& nflip2) {
    const uint32_t par = item & 1u;
    const uint32_t* desc = s_sdesc + (item >> 1) * SiteDesc<DC>::DW;
    const uint4 d0 = *reinterpret_cast<const uint4*>(desc);
    const uint32_t row = d0.x;
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
    const uint32_t ug = (uint32_t)g, last = (uint32_t)G - 1u;
    const uint32_t own = bp[row + ug];
    // the one Trotter neighbour outside the byte: copy 8g-1 (bit 7 of byte g-1) for even
    // copies, copy 8g+8 (bit 0 of byte g+1) for odd ones, periodic in the row
    const uint32_t eb = par ? (bp[row + (ug == last ? 0u : ug + 1u)] & 1u)
                            : ((uint32_t)bp[row + (ug == 0 ? last : ug - 1u)] >> 7);
    const uint32_t* lut_p = lut + (par << 8);
    uint32_t nbyte[DC];
#pragma unroll
    for (int d = 0; d < DC; ++d) nbyte[d] = bp[nrow[d] + ug];
    uint4 r4;
    if (PRE) {
        r4 = rb[q * G + g];
    } else {
        r4 = philox(make_uint4(t, d0.y, slot, (par << 24) | (uint32_t)g), key);
    }
    const uint32_t u[4] = {r4.x, r4.y, r4.z, r4.w};
    const uint32_t S = lut_p[own];
    const uint32_t Rn = par ? lut[256 + (((own >> 1) | (eb << 7)) & 0xFFu)] : lut[256 + own];
    const uint32_t Ln = par ? lut[own] : lut[((own << 1) | eb) & 0xFFu];
    const uint32_t X = (S ^ Ln) & 0x02020202u;
    const uint32_t Y = (S ^ Rn) & 0x02020202u;
    const uint32_t Z = 0x02020202u - ((X + Y) >> 1);

    uint32_t a[DC];
#pragma unroll
    for (int d = 0; d < DC; ++d) a[d] = lut_p[nbyte[d]];
    int L[4];
    field_times_spin<DC>(a, S, jpack, L);
    uint32_t F = 0, flipbits = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
        const uint32_t m = accept_mask<PRE>(u[w], thr_entry(thr_c, Z, L[w], w));
        F -= m * (0xFEu << (8 * w));
        flipbits -= m * (1u << (2 * w));
        sumL -= (int)m * L[w];
    }
    const uint32_t Fm = F & 0x02020202u;
    nflip2 = __dp4a((int)Fm, 0x01010101, nflip2);
    sumC2 = __dp4a((int)Z, (int)Fm, sumC2);
    if (flipbits) bp[row + ug] = (uint8_t)(own ^ (flipbits << par));
}

}  // namespace ptq
