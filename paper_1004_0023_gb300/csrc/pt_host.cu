// pt_host.cu -- host side of the PT-QMC C ABI (include/pt.h): validation, the FP64
// Metropolis and swap tables, the neighbour table, the sweep's level schedule, device
// memory, and the launch sequence. Every step of the method itself runs in the kernels
// of pt_kernels.cu; this file only prepares inputs and orders launches.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "pt.h"
#include "pt_internal.h"

using namespace ptq;

struct pt_ctx {
    DevProblem dp;
    LaunchPlan plan;
    cudaStream_t stream;
    bool own_stream;
    int device;
    int n_edges;
    int max_degree;
    long long t, q;
    long long sweep_limit;   // t never exceeds this (int64 statistics, 32-bit Philox counter)
    int max_passes;          // mailbox capacity of one launch
    long long mbox_clear_q;  // pass index at which the mailboxes were last cleared
    bool cooperative;
    long long timeout_ns;
    int err;
    char msg[256];
    std::vector<uint32_t> thr;   // host copy of the tables
    std::vector<double> coef;
    std::vector<void*> allocs;
    int8_t* staging;             // [R*N*P] rung-ordered state for reads and writes
    int64_t device_bytes;
    int64_t launches;            // kernels launched by this context
    int64_t h2d_bytes;           // bytes copied host -> device
    int tuned_plans;             // candidate plans timed at create
};

// Plans chosen by the create-time autotuner, per problem shape, for the process.
struct PlanKey {
    int N, P, R, dc, n_levels, n_edges;
    bool operator<(const PlanKey& o) const {
        return std::tie(N, P, R, dc, n_levels, n_edges) < std::tie(o.N, o.P, o.R, o.dc, o.n_levels, o.n_edges);
    }
};
struct PlanChoice {
    int path, threads, producers;
    int cluster, group_threads, thr_resident;  // path 7
};
static std::mutex g_plan_mutex;
static std::map<PlanKey, PlanChoice> g_plan_cache;

static thread_local char g_create_msg[256] = "";

static int ctx_fail(pt_ctx* c, int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->msg, sizeof(c->msg), fmt, ap);
    va_end(ap);
    if (code == PT_ECUDA || code == PT_ETIMEDOUT) c->err = code;  // sticky
    return code;
}

static int create_fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_create_msg, sizeof(g_create_msg), fmt, ap);
    va_end(ap);
    return code;
}

// ---------------------------------------------------------------------------------
// Metropolis thresholds and swap coefficients in FP64 (host libm), in this order of
// operations: beta = 1/T; a = (beta*Gamma)/P; K = -0.5*log(tanh(a)); for copy flips
// x = ((2*beta)/P)*L - (2*K)*m and thr = 0xFFFFFFFF if x >= 0, else
// min(floor(exp(x)*2^32), 0xFFFFFFFF); for swaps a_r = beta_r/P - beta_{r+1}/P and
// c_r = K_{r+1} - K_r. Flipping copy k of site i changes the action S by
// -(2 beta/P) L + 2 K m, with L = s(h + sum J s_j) and m = s(s^{k-1} + s^{k+1}).
// P = 1 is classical parallel tempering over T (Gamma = 0): K = 0 and m = 0.
void ptq::build_tables(int R, int P, int Lmax, const pt_rung* ladder, std::vector<uint32_t>& thr,
                         std::vector<double>& coef) {
    const int nL = 2 * Lmax + 1;
    thr.assign((size_t)R * nL * 3, 0u);
    coef.assign(2 * (size_t)(R > 1 ? R - 1 : 0), 0.0);
    std::vector<double> K(R), b(R);
    for (int r = 0; r < R; ++r) {
        const double beta = 1.0 / ladder[r].T;
        const double a = beta * ladder[r].gamma / (double)P;
        K[r] = P == 1 ? 0.0 : -0.5 * log(tanh(a));  // classical chains (P = 1): no Trotter coupling
        b[r] = beta / (double)P;
        const double c_flip = 2.0 * beta / (double)P;
        const double c_trot = 2.0 * K[r];
        for (int L = -Lmax; L <= Lmax; ++L) {
            for (int mi = 0; mi < 3; ++mi) {
                const int m = 2 * mi - 2;
                const double x = c_flip * (double)L - c_trot * (double)m;
                uint32_t v;
                if (x >= 0.0) {
                    v = 0xFFFFFFFFu;
                } else {
                    const double f = floor(ldexp(exp(x), 32));
                    v = (f >= 4294967295.0) ? 0xFFFFFFFFu : (uint32_t)f;
                }
                thr[((size_t)r * nL + (size_t)(L + Lmax)) * 3 + (size_t)mi] = v;
            }
        }
    }
    for (int r = 0; r + 1 < R; ++r) {
        coef[r] = b[r] - b[r + 1];
        coef[(size_t)(R - 1) + r] = K[r + 1] - K[r];
    }
}

// ---------------------------------------------------------------------------------
// Level schedule of one sweep. The sequential order is (0,0), (0,1), (1,0), (1,1), ...
// where (i, p) updates every copy of parity p of site i. Two updates conflict only if
// they are (i,0) and (i,1), or (i,p) and (j,p) with i, j adjacent; the level of an update
// is one more than the largest level of the earlier updates it conflicts with.
void ptq::level_schedule(int N, const std::vector<std::vector<int>>& adj, std::vector<uint32_t>& items,
                           std::vector<int32_t>& level_off, int per_round, int row_words) {
    // as early as possible: l0 / l1 = the longest chain of predecessors of (i, 0) / (i, 1)
    std::vector<int> l0(N), l1(N);
    int nlev = 0;
    for (int i = 0; i < N; ++i) {
        int a = 0, b = 0;
        for (int j : adj[i])
            if (j < i) {
                a = std::max(a, l0[j] + 1);
                b = std::max(b, l1[j] + 1);
            }
        l0[i] = a;
        l1[i] = std::max(b, a + 1);
        nlev = std::max(nlev, l1[i] + 1);
    }
    if (per_round > 0) {
        // Balanced: the same number of levels, each update between its earliest level and
        // the latest one its successors allow (b0 / b1), the levels filled in whole rounds
        // of per_round items, most urgent first. Items (i, p) are numbered 2i + p; the
        // successors of (i, p) are (j, p) for neighbours j > i, and (i, 1) when p = 0.
        std::vector<int> b0(N), b1(N);
        for (int i = N - 1; i >= 0; --i) {
            int a = nlev - 1, b = nlev - 1;
            for (int j : adj[i])
                if (j > i) {
                    a = std::min(a, b0[j] - 1);
                    b = std::min(b, b1[j] - 1);
                }
            b1[i] = b;
            b0[i] = std::min(a, b - 1);
        }
        auto latest = [&](int x) { return (x & 1) ? b1[x >> 1] : b0[x >> 1]; };
        std::vector<int> waiting(2 * (size_t)N, 0), level(2 * (size_t)N, -1);
        for (int i = 0; i < N; ++i) {
            for (int j : adj[i])
                if (j < i) {
                    waiting[2 * i]++;
                    waiting[2 * i + 1]++;
                }
            waiting[2 * i + 1]++;
        }
        std::vector<int> ready, next;
        for (int x = 0; x < 2 * N; ++x)
            if (waiting[x] == 0) ready.push_back(x);
        int left = 2 * N;
        for (int l = 0; l < nlev; ++l) {
            std::sort(ready.begin(), ready.end(), [&](int x, int y) {
                const int bx = latest(x), by = latest(y);
                return bx != by ? bx < by : x < y;
            });
            int must = 0;
            while (must < (int)ready.size() && latest(ready[must]) == l) ++must;
            const int even_share = (left + (nlev - l) - 1) / (nlev - l);
            const int cap = std::max(must, (even_share + per_round - 1) / per_round * per_round);
            const int take = std::min(cap, (int)ready.size());
            next.clear();
            for (int k = 0; k < take; ++k) {
                const int x = ready[k], i = x >> 1;
                level[x] = l;
                auto release = [&](int y) {
                    if (--waiting[y] == 0) next.push_back(y);
                };
                for (int j : adj[i])
                    if (j > i) release(2 * j + (x & 1));
                if (!(x & 1)) release(x + 1);
            }
            left -= take;
            ready.erase(ready.begin(), ready.begin() + take);
            ready.insert(ready.end(), next.begin(), next.end());
        }
        // keep the as-early-as-possible levels where the fill takes more rounds than they do
        // (it can, by one, on long chains with small rounds)
        std::vector<int> ca(nlev, 0), cb(nlev, 0);
        for (int i = 0; i < N; ++i) {
            ca[l0[i]]++;
            ca[l1[i]]++;
            cb[level[2 * i]]++;
            cb[level[2 * i + 1]]++;
        }
        long long ra = 0, rb = 0;
        for (int l = 0; l < nlev; ++l) {
            ra += (ca[l] + per_round - 1) / per_round;
            rb += (cb[l] + per_round - 1) / per_round;
        }
        if (rb <= ra)
            for (int i = 0; i < N; ++i) {
                l0[i] = level[2 * i];
                l1[i] = level[2 * i + 1];
            }
    }
    std::vector<int> count(nlev + 1, 0);
    for (int i = 0; i < N; ++i) {
        count[l0[i] + 1]++;
        count[l1[i] + 1]++;
    }
    level_off.assign(nlev + 1, 0);
    for (int l = 0; l < nlev; ++l) level_off[l + 1] = level_off[l] + count[l + 1];
    items.assign(2 * (size_t)N, 0u);
    std::vector<int> fill(level_off.begin(), level_off.end() - 1);
    for (int i = 0; i < N; ++i) {
        items[fill[l0[i]]++] = ((uint32_t)i << 1) | 0u;
        items[fill[l1[i]]++] = ((uint32_t)i << 1) | 1u;
    }
    if (row_words > 0) {
        // Within a level the order is free. The packed kernels give consecutive items of a
        // level to neighbouring lanes of a warp, each lane a 4-byte word at column g of the
        // item's row half, so an item's words start at shared-memory bank
        // (i * row_words + parity * row_words / 2) mod 32. Dealing the level's items round
        // robin over those start banks puts items with different starts side by side, so a
        // warp's loads of its items' own words (and, for rows of 32 words, of every
        // neighbour word) fall in different banks.
        std::vector<uint32_t> lev_items;
        std::vector<std::vector<uint32_t>> by_bank(32);
        for (int l = 0; l < nlev; ++l) {
            for (auto& b : by_bank) b.clear();
            for (int x = level_off[l]; x < level_off[l + 1]; ++x) {
                const uint32_t it = items[x], i = it >> 1, par = it & 1u;
                by_bank[(i * (uint32_t)row_words + par * (uint32_t)(row_words / 2)) & 31u].push_back(it);
            }
            lev_items.clear();
            for (size_t k = 0;; ++k) {
                bool any = false;
                for (auto& b : by_bank)
                    if (k < b.size()) {
                        lev_items.push_back(b[k]);
                        any = true;
                    }
                if (!any) break;
            }
            std::copy(lev_items.begin(), lev_items.end(), items.begin() + level_off[l]);
        }
    }
}

// A classical chain (P = 1) has no odd-parity copy: its updates (i, 1) change nothing, so
// they are dropped with the levels they leave empty. Each remaining level is a subset of a
// valid one, in the same order, so the result is the same; the sweep has fewer levels.
static void drop_odd_updates(std::vector<uint32_t>& items, std::vector<int32_t>& level_off) {
    std::vector<uint32_t> it;
    std::vector<int32_t> off(1, 0);
    for (size_t l = 0; l + 1 < level_off.size(); ++l) {
        for (int x = level_off[l]; x < level_off[l + 1]; ++x)
            if (!(items[x] & 1u)) it.push_back(items[x]);
        if ((int32_t)it.size() > off.back()) off.push_back((int32_t)it.size());
    }
    items.swap(it);
    level_off.swap(off);
}

// ---------------------------------------------------------------------------------
// Packed-path site descriptors (see SiteDesc in pt_kernels.cu).
// P = bytes per chain row: the copy count for int8 chains, copies / 8 for bit-packed ones.
void ptq::build_site_desc(int N, int P, int dclass, const std::vector<std::vector<int>>& adj,
                            const std::vector<std::vector<int>>& adjJ, const int32_t* h, std::vector<uint32_t>& desc) {
    const int DW = dclass == 4 ? 8 : 12;
    const uint32_t ones_row = (uint32_t)(((size_t)N * P + 15) & ~(size_t)15);
    desc.assign((size_t)N * DW, 0u);
    for (int i = 0; i < N; ++i) {
        uint32_t* d = &desc[(size_t)i * DW];
        d[0] = (uint32_t)i * (uint32_t)P;
        d[1] = (uint32_t)i;
        uint32_t jp[2] = {0u, 0u};
        for (int s8 = 0; s8 < dclass; ++s8) {
            int J = 0;
            uint32_t r = ones_row;
            if (s8 < (int)adj[i].size()) {
                J = adjJ[i][s8];
                r = (uint32_t)adj[i][s8] * (uint32_t)P;
            } else if (s8 == (int)adj[i].size()) {
                J = h[i];
            }
            d[4 + s8] = r;
            jp[s8 / 4] |= (uint32_t)(uint8_t)(int8_t)J << (8 * (s8 % 4));
        }
        d[2] = jp[0];
        d[3] = jp[1];
    }
}

// All of a context's device buffers are carved out of one allocation, so a create costs one
// cudaMalloc: first every buffer is placed (256-byte aligned), then the pointers are set.
struct DevCarve {
    size_t total = 0;
    std::vector<std::pair<void**, size_t>> slots;  // where to store each buffer's address
    template <typename T>
    void add(T** ptr, size_t count) {
        slots.push_back({reinterpret_cast<void**>(ptr), total});
        total += (std::max<size_t>(count * sizeof(T), 16) + 255) & ~(size_t)255;
    }
    cudaError_t allocate(pt_ctx* c) {
        void* base = nullptr;
        const cudaError_t e = cudaMalloc(&base, total);
        if (e != cudaSuccess) return e;
        c->allocs.push_back(base);
        c->device_bytes += (int64_t)total;
        for (auto& sl : slots) *sl.first = static_cast<unsigned char*>(base) + sl.second;
        return cudaSuccess;
    }
};

static void free_ctx(pt_ctx* c) {
    for (void* p : c->allocs) cudaFree(p);
    c->allocs.clear();
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

static int check_status(pt_ctx* c) {
    int st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, c->dp.status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return ctx_fail(c, PT_ECUDA, "CUDA error: %s", cudaGetErrorString(e));
    if (st == PT_ETIMEDOUT) return ctx_fail(c, PT_ETIMEDOUT, "a device-side wait for a swap partner timed out");
    if (st != 0) return ctx_fail(c, PT_ECUDA, "device status %d", st);
    return PT_OK;
}

#define CUDA_OR_FAIL(c, call)                                                                   \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return ctx_fail((c), PT_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// Path 7: the context's problem as the batched kernel's one request, for one launch of
// n sweeps starting at counters (t0, q0).
static BatchInstance chains_instance(const DevProblem& p, const LaunchPlan& plan, long long t0, long long q0, int n,
                                     int sps) {
    BatchInstance I;
    memset(&I, 0, sizeof(I));
    I.sdesc = p.desc;
    I.items = p.items;
    I.level_off = p.level_off;
    I.thr = p.thr;
    I.coef = p.coef;
    I.spins = p.spins;
    I.E = p.E;
    I.M = p.M;
    I.rung_of_slot = p.rung_of_slot;
    I.slot_of_rung = p.slot_of_rung;
    I.acc = p.acc;
    I.swap_stats = p.swap_stats;
    I.N = p.N;
    I.P = p.P;
    I.R = p.R;
    I.Lmax = p.Lmax;
    I.nL3 = p.nL3;
    I.n_levels = p.n_levels;
    I.dc = plan.dclass;
    I.slot_stride = p.slot_stride;
    I.group_threads = plan.group_threads;
    I.resident = 1;
    I.thr_resident = plan.thr_resident;
    I.key0 = p.key0;
    I.key1 = p.key1;
    I.t0 = t0;
    I.q0 = q0;
    I.n_sweeps = n;
    I.sweeps_per_swap = sps;
    return I;
}

// n sweeps (a swap pass after every sps-th) of any plan, starting at counters (t0, q0).
static cudaError_t launch_plan_sweeps(const DevProblem& p, const LaunchPlan& plan, long long t0, long long q0, int n,
                                      int sps, long long timeout_ns, bool cooperative, cudaStream_t s) {
    if (plan.path == kPathPackedChains)
        return launch_batch_single(chains_instance(p, plan, t0, q0, n, sps), plan.cluster, plan.threads,
                                   plan.smem_bytes, s);
    return launch_sweeps(p, plan, t0, q0, n, sps, timeout_ns, cooperative, s);
}

// Path 7 for a problem: the narrowest chain groups (widen < 0 halves the size-based width,
// down to one warp) with every chain resident on one cluster of `cluster` CTAs. Returns
// false when the chains do not all fit or no such cluster can run.
static bool chains_plan(const DevProblem& p, int dclass, int cluster, int widen, LaunchPlan& pl,
                        int force_group = 0) {
    BatchInstance I = chains_instance(p, pl, 0, 0, 0, 0);
    I.dc = dclass;
    const size_t cap = batch_smem_cap();
    choose_groups(I, cluster, 512, cap, widen);
    if (force_group > 0) {
        // the given width, with every rung's threshold row resident if that still fits
        I.group_threads = force_group;
        I.resident = 1;
        I.thr_resident = 1;
        if (batch_smem_bytes(I, cluster, 512) > cap || (size_t)I.R * ((I.nL3 * 4 + 15) / 16 * 16) > 49152)
            I.thr_resident = 0;
    }
    if (!I.resident) return false;
    const size_t smem = batch_smem_bytes(I, cluster, 512);
    if (smem > cap) return false;
    int ncl = 0;
    if (batch_max_clusters(cluster, 512, smem, &ncl) != cudaSuccess || ncl < 1) {
        (void)cudaGetLastError();
        return false;
    }
    pl.path = kPathPackedChains;
    pl.dclass = dclass;
    pl.threads = 512;
    pl.n_consumer = 512;
    pl.smem_bytes = smem;
    pl.cluster = cluster;
    pl.group_threads = I.group_threads;
    pl.thr_resident = I.thr_resident;
    return true;
}

extern "C" int pt_create(const pt_instance* inst, int32_t P, const pt_rung* ladder, int32_t R,
                         const uint32_t* flip_thr, const double* swap_coef, uint64_t seed,
                         const pt_options* opt, void* cuda_stream, pt_ctx** out) {
    if (!inst || !ladder || !out) return create_fail(PT_EINVAL, "null argument");
    const int N = inst->n, nE = inst->n_edges;
    if (N < 1 || N > 65535) return create_fail(PT_EINVAL, "n must be in [1, 65535]");
    if (nE < 0 || (nE > 0 && (!inst->ei || !inst->ej || !inst->J)) || !inst->h)
        return create_fail(PT_EINVAL, "bad edge arrays");
    if (P != 1 && (P < 2 || (P & 1) || P > 4096))
        return create_fail(PT_EINVAL, "P must be 1 (classical) or even and in [2, 4096]");
    if (R < 1 || R > 65535) return create_fail(PT_EINVAL, "R must be in [1, 65535]");
    const bool need_ladder = !flip_thr || !swap_coef;
    if (need_ladder)
        for (int r = 0; r < R; ++r) {
            const bool gamma_ok = P == 1 ? ladder[r].gamma == 0.0 : ladder[r].gamma > 0.0;
            if (!(ladder[r].T > 0.0) || !gamma_ok || !isfinite(ladder[r].T) || !isfinite(ladder[r].gamma))
                return create_fail(PT_EINVAL, "rung %d: T must be finite and > 0; gamma > 0 for P >= 2, 0 for P = 1",
                                   r);
        }

    // adjacency, duplicate / self-loop checks
    std::vector<std::vector<int>> adj(N);
    std::vector<std::vector<int>> adjJ(N);
    for (int b = 0; b < nE; ++b) {
        const int u = inst->ei[b], v = inst->ej[b], J = inst->J[b];
        if (u < 0 || u >= N || v < 0 || v >= N || u == v)
            return create_fail(PT_EINVAL, "edge %d: endpoints must be distinct sites in range", b);
        if (J == 0 || J < -127 || J > 127) return create_fail(PT_EINVAL, "edge %d: J must be in [-127,127]\\{0}", b);
        adj[u].push_back(v);
        adjJ[u].push_back(J);
        adj[v].push_back(u);
        adjJ[v].push_back(J);
    }
    int dmax = 0, Lmax = 0;
    for (int i = 0; i < N; ++i) {
        std::vector<int> sorted = adj[i];
        std::sort(sorted.begin(), sorted.end());
        if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end())
            return create_fail(PT_EINVAL, "duplicate edge at site %d", i);
        dmax = std::max(dmax, (int)adj[i].size());
        if (inst->h[i] < -127 || inst->h[i] > 127) return create_fail(PT_EINVAL, "site %d: h must be in [-127,127]", i);
        int l = abs(inst->h[i]);
        for (int J : adjJ[i]) l += abs(J);
        if (l > 127) return create_fail(PT_EINVAL, "site %d: |h| + sum |J| must be <= 127", i);
        Lmax = std::max(Lmax, l);
    }
    if (dmax > 32) return create_fail(PT_EINVAL, "maximum degree 32 supported");
    const int dclass = dmax <= 4 ? 4 : (dmax <= 8 ? 8 : 32);

    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1)
        return create_fail(PT_ENODEV, "no CUDA device");

    pt_ctx* c = new pt_ctx();
    c->own_stream = false;
    c->stream = (cudaStream_t)cuda_stream;
    c->t = c->q = 0;
    c->mbox_clear_q = 0;
    c->err = 0;
    c->msg[0] = 0;
    c->staging = nullptr;
    c->device_bytes = 0;
    c->launches = 0;
    c->h2d_bytes = 0;
    c->n_edges = nE;
    c->max_degree = dmax;
    cudaGetDevice(&c->device);
    if (!c->stream) {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return create_fail(PT_ECUDA, "cudaStreamCreate failed");
        }
        c->own_stream = true;
    }
    const int timeout_ms = (opt && opt->wait_timeout_ms > 0) ? opt->wait_timeout_ms : 5000;
    c->timeout_ns = (long long)timeout_ms * 1000000ll;

    // tables
    if (!flip_thr || !swap_coef) build_tables(R, P, Lmax, ladder, c->thr, c->coef);
    const size_t nthr = (size_t)R * (2 * Lmax + 1) * 3;
    if (flip_thr) c->thr.assign(flip_thr, flip_thr + nthr);
    if (swap_coef) c->coef.assign(swap_coef, swap_coef + 2 * (size_t)(R - 1));
    if (c->coef.empty()) c->coef.assign(2, 0.0);

    // neighbour table (j << 8) | (uint8)J, rows padded to the kernel's degree class with (i, 0)
    std::vector<uint32_t> nbr((size_t)N * dclass);
    std::vector<int8_t> h8(N);
    for (int i = 0; i < N; ++i) {
        h8[i] = (int8_t)inst->h[i];
        for (int d = 0; d < dclass; ++d) {
            if (d < (int)adj[i].size())
                nbr[(size_t)i * dclass + d] = ((uint32_t)adj[i][d] << 8) | (uint32_t)(uint8_t)(int8_t)adjJ[i][d];
            else
                nbr[(size_t)i * dclass + d] = (uint32_t)i << 8;
        }
    }
    std::vector<uint32_t> items;
    std::vector<int32_t> level_off;
    level_schedule(N, adj, items, level_off);
    if (P == 1) drop_odd_updates(items, level_off);

    DevProblem& p = c->dp;
    memset(&p, 0, sizeof(p));
    p.N = N;
    p.P = P;
    p.R = R;
    p.Lmax = Lmax;
    p.nL3 = (2 * Lmax + 1) * 3;
    p.dmax = dclass;
    p.n_levels = (int)level_off.size() - 1;
    p.slot_stride = (int)(((size_t)N * P + 15) & ~(size_t)15);
    p.withhold_rung = (opt && opt->test_withhold_rung > 0) ? opt->test_withhold_rung - 1 : -1;
    p.exact_swaps = (opt && opt->test_exact_swaps) ? 1 : 0;
    p.key0 = (uint32_t)(seed & 0xFFFFFFFFu);
    p.key1 = (uint32_t)(seed >> 32);

    // launch plan: the packed path needs P % 8 == 0 and a spare neighbour slot for h
    int max_smem = 0, n_sm = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, c->device);
    const int packed_dc = (dmax + 1 <= 4) ? 4 : ((dmax + 1 <= 8) ? 8 : 0);
    const bool packed_ok = (P % 8 == 0) && packed_dc > 0;
    const int want_path = opt ? opt->kernel_path : 0;
    if (want_path < 0 || want_path > 10) {
        free_ctx(c);
        return create_fail(PT_EINVAL, "kernel_path must be 0..10");
    }
    if (want_path == kPathClassical &&
        (P != 1 || opt->cluster_size < 0 || opt->cluster_size > 16 ||
         (opt->threads_per_block != 0 &&
          (opt->threads_per_block < 32 || opt->threads_per_block > 512 || opt->threads_per_block % 32)))) {
        free_ctx(c);
        return create_fail(PT_EINVAL,
                           "kernel_path 10 needs P = 1, cluster_size 0..16 and threads_per_block 0 or a multiple "
                           "of 32 up to 512");
    }
    if ((want_path == kPathPacked || want_path == kPathPackedInline || want_path == kPathBits ||
         want_path == kPathSplit || want_path == kPathSplitInline || want_path == kPathPackedChains ||
         want_path == kPathPeer || want_path == kPathCluster) && !packed_ok) {
        free_ctx(c);
        return create_fail(PT_EINVAL, "the packed kernel needs P %% 8 == 0 and degree <= 7");
    }
    if ((want_path == kPathSplit || want_path == kPathSplitInline) && P % 16 != 0) {
        free_ctx(c);
        return create_fail(PT_EINVAL, "the split kernel needs P %% 16 == 0");
    }
    // statistics in shared memory for ladders up to 341 rungs (16 KB); all threshold rows in
    // shared memory when they take at most 48 KB and the chosen layout still fits
    p.acc_in_smem = (size_t)R * kAccCount * 8 <= 16384 ? 1 : 0;
    p.tables_in_smem = (size_t)R * p.nL3 * 4 <= 49152 ? 1 : 0;
    // path 7 is set up on the inline-word plan's data (int8 rows, site descriptors) and
    // switched to the packed-chains launch once the device state exists
    const bool want_chains = want_path == kPathPackedChains;
    if (want_chains && ((opt->threads_per_block != 0) || p.withhold_rung >= 0 || p.exact_swaps ||
                        opt->cluster_size < 0 || opt->cluster_size > 16 ||
                        (opt->group_threads != 0 && (opt->group_threads < 32 || opt->group_threads > 512 ||
                                                     (opt->group_threads & (opt->group_threads - 1)))))) {
        free_ctx(c);
        return create_fail(PT_EINVAL,
                           "kernel_path 7 takes cluster_size (0..16) and group_threads (0 or 32..512, a power of "
                           "two), no threads_per_block and no test hooks");
    }
    if (want_path == kPathCluster &&
        (R > 16 || (opt->threads_per_block != 0 && (opt->threads_per_block < 64 || opt->threads_per_block > 384)) ||
         opt->producer_threads < 0 || opt->producer_threads % 32 ||
         opt->producer_threads >= (opt->threads_per_block ? opt->threads_per_block : 128))) {
        free_ctx(c);
        return create_fail(PT_EINVAL,
                           "kernel_path 9 needs R <= 16, threads_per_block 0 or 64..384 and producer_threads a "
                           "multiple of 32 below it (0 = random words inline)");
    }
    int path = want_chains ? kPathPackedInline : want_path;
    const int want_threads = opt ? opt->threads_per_block : 0;
    // path 10's shape for a cluster of about K CTAs: C = the power of two at or above R / K
    // chains per CTA, ceil(R / C) CTAs; and its block: a multiple of 32 and of C holding one
    // update of every chain of the CTA for the average level, at most 512 threads
    // the int8 packed kernels' rows are P bytes, P/4 words: their levels are ordered for the
    // shared-memory banks (see level_schedule); the other layouts keep site order
    auto row_words_for = [&](int pth) {
        return (pth == kPathPacked || pth == kPathPackedInline || pth == kPathPeer || pth == kPathCluster ||
                pth == kPathPackedChains)
                   ? P / 4
                   : 0;
    };
    auto classical_chains = [&](int K) {
        int C = 1;
        while ((long long)C * K < R) C <<= 1;
        return C;
    };
    auto classical_threads = [&](int C) {
        const int unit = std::max(32, C);
        const long long per_level = ((long long)items.size() + p.n_levels - 1) / p.n_levels;
        long long t = (per_level * C + unit - 1) / unit * unit;
        t = std::max<long long>(t, std::max(64, unit));
        return (int)std::min<long long>(t, 512 / unit * unit);
    };
    // a layout fits if it does with the threshold rows and / or the statistics moved out
    auto fits = [&](int pth) {
        DevProblem q = p;
        if (sweep_smem_bytes(q, pth, packed_dc) <= (size_t)max_smem) return true;
        q.tables_in_smem = 0;
        if (sweep_smem_bytes(q, pth, packed_dc) <= (size_t)max_smem) return true;
        q.acc_in_smem = 0;
        return sweep_smem_bytes(q, pth, packed_dc) <= (size_t)max_smem;
    };
    // the split kernel when a chain and its produced random words do not fit one CTA but do
    // fit two, and every chain's cluster can be resident at once
    auto split_fits = [&](int spath = kPathSplit) {
        if (P % 16 != 0 || !(want_threads == 0 || (want_threads >= 64 && want_threads <= 512)) || !fits(spath))
            return false;
        // every one of the P/16 + 1 word columns needs a consumer (and, with producer warps,
        // a producer) thread
        const int th = want_threads > 0 ? want_threads : 512;
        const int cols = P / 16 + 1;
        if (spath == kPathSplit ? (th / 4 < cols || th - th / 4 < cols) : th < cols) return false;
        DevProblem q = p;
        if (sweep_smem_bytes(q, spath, packed_dc) > (size_t)max_smem) q.tables_in_smem = 0;
        if (sweep_smem_bytes(q, spath, packed_dc) > (size_t)max_smem) q.acc_in_smem = 0;
        LaunchPlan probe;
        probe.path = spath;
        probe.dclass = packed_dc;
        probe.threads = want_threads > 0 ? want_threads : 512;
        probe.n_consumer = spath == kPathSplit ? probe.threads - probe.threads / 4 : probe.threads;
        probe.smem_bytes = sweep_smem_bytes(q, spath, packed_dc);
        long long resident = 0;
        if (prepare_sweep_kernel(probe) != cudaSuccess || sweep_resident_chains(q, probe, &resident) != cudaSuccess) {
            (void)cudaGetLastError();
            return false;
        }
        return resident >= R;
    };
    // path 8 when the produced-words layout fits and all R two-CTA clusters can be resident
    auto peer_fits = [&](int th) {
        if (!fits(kPathPacked) || th < 64) return false;
        DevProblem q = p;
        if (sweep_smem_bytes(q, kPathPeer, packed_dc) > (size_t)max_smem) q.tables_in_smem = 0;
        if (sweep_smem_bytes(q, kPathPeer, packed_dc) > (size_t)max_smem) q.acc_in_smem = 0;
        LaunchPlan probe;
        probe.path = kPathPeer;
        probe.dclass = packed_dc;
        probe.threads = th;
        probe.n_consumer = th;
        probe.smem_bytes = sweep_smem_bytes(q, kPathPeer, packed_dc);
        long long resident = 0;
        if (prepare_sweep_kernel(probe) != cudaSuccess || sweep_resident_chains(q, probe, &resident) != cudaSuccess) {
            (void)cudaGetLastError();
            return false;
        }
        return resident >= R;
    };
    if (path == 0) {
        path = kPathGeneric;
        if (packed_ok) {
            // producer warps need a block of at least two warps; int8 chains before bit-packed ones
            if ((want_threads == 0 || want_threads >= 64) && fits(kPathPacked))
                path = kPathPacked;
            else if (split_fits())
                path = kPathSplit;
            else if (fits(kPathPackedInline))
                path = kPathPackedInline;
            else if (fits(kPathBits))
                path = kPathBits;
        }
    }
    c->plan.path = path;
    c->plan.dclass = (path == kPathGeneric || path == kPathClassical) ? dclass : packed_dc;
    if (path == kPathClassical) {
        // every rung's row and this launch's statistics live in each CTA's shared memory
        const int C = classical_chains(opt->cluster_size > 0 ? opt->cluster_size : std::max(1, (R + 15) / 16));
        c->plan.chains_per_cta = C;
        c->plan.cluster = (R + C - 1) / C;
        p.acc_in_smem = 1;
        p.tables_in_smem = 1;
        if (C > 512 || c->plan.cluster > 16 || (want_threads > 0 && want_threads % C)) {
            free_ctx(c);
            return create_fail(PT_EINVAL, "kernel_path 10: %d chains per CTA on %d CTAs does not fit (threads %d)", C,
                               c->plan.cluster, want_threads);
        }
    }
    const bool cl_pre = path == kPathCluster && opt->producer_threads > 0;
    if (p.tables_in_smem && sweep_smem_bytes(p, path, c->plan.dclass, cl_pre) > (size_t)max_smem)
        p.tables_in_smem = 0;
    if (p.acc_in_smem && sweep_smem_bytes(p, path, c->plan.dclass, cl_pre) > (size_t)max_smem) p.acc_in_smem = 0;
    c->plan.smem_bytes = path == kPathClassical ? classical_smem_bytes(p, c->plan.chains_per_cta)
                                                : sweep_smem_bytes(p, path, c->plan.dclass, cl_pre);
    if ((long long)c->plan.smem_bytes > (long long)max_smem) {
        free_ctx(c);
        return create_fail(PT_EINVAL, "one chain needs %zu bytes of shared memory; the device allows %d",
                           c->plan.smem_bytes, max_smem);
    }
    if (opt && opt->threads_per_block > 0) {
        const int tmax =
            (path == kPathGeneric || path == kPathSplit || path == kPathSplitInline || path == kPathPeer) ? 512 : 1024;
        if (opt->threads_per_block % 32 || opt->threads_per_block > tmax) {
            free_ctx(c);
            return create_fail(PT_EINVAL, "threads_per_block must be a multiple of 32 <= %d for this kernel", tmax);
        }
        c->plan.threads = opt->threads_per_block;
    } else if (path == kPathPacked || path == kPathSplit || path == kPathSplitInline || path == kPathPeer) {
        c->plan.threads = 512;
    } else if (path == kPathCluster) {
        c->plan.threads = 128;
    } else if (path == kPathClassical) {
        c->plan.threads = classical_threads(c->plan.chains_per_cta);
    } else {
        // enough threads for the average level (units = items * padded groups per parity)
        int G = ((P / 2) + 3) / 4, Gp = 1;
        while (Gp < G) Gp <<= 1;
        const long long units = (long long)items.size() * Gp;
        long long avg = (units + p.n_levels - 1) / p.n_levels;
        avg = ((avg + 31) / 32) * 32;
        c->plan.threads = (int)std::min<long long>(512, std::max<long long>(128, avg));
    }
    c->plan.n_consumer = c->plan.threads;
    if (path == kPathCluster) c->plan.n_consumer = c->plan.threads - opt->producer_threads;
    if (path == kPathPacked || path == kPathSplit) {
        int prod = (opt && opt->producer_threads > 0) ? opt->producer_threads
                                                      : std::max(32, (c->plan.threads / 4) / 32 * 32);
        if (prod % 32 || prod >= c->plan.threads) {
            free_ctx(c);
            return create_fail(PT_EINVAL, "producer_threads must be a multiple of 32 below threads_per_block");
        }
        c->plan.n_consumer = c->plan.threads - prod;
        // the split kernel gives each of its P/16 + 1 word columns at least one thread
        if (path == kPathSplit && (c->plan.n_consumer < P / 16 + 1 || prod < P / 16 + 1)) {
            free_ctx(c);
            return create_fail(PT_EINVAL, "the split kernel needs at least P/16 + 1 = %d consumer and producer threads",
                               P / 16 + 1);
        }
    }
    if (path == kPathSplitInline && c->plan.threads < P / 16 + 1) {
        free_ctx(c);
        return create_fail(PT_EINVAL, "the split kernel needs at least P/16 + 1 = %d threads", P / 16 + 1);
    }

    // the levels, rebalanced for the items this plan's kernel takes per round: consumer
    // threads over word columns per item (a power of two for the one-CTA kernels, W + 1 for
    // the split one); the level count and the dependencies stay the same
    {
        int cols = 1;
        if (path == kPathSplit || path == kPathSplitInline) {
            cols = P / 16 + 1;
        } else {
            const int G = (path == kPathGeneric) ? ((P / 2) + 3) / 4 : P / 8;
            while (cols < G) cols <<= 1;
        }
        const int per_round = path == kPathClassical ? c->plan.threads / c->plan.chains_per_cta
                                                     : c->plan.n_consumer / cols;
        level_schedule(N, adj, items, level_off, std::max(1, per_round), row_words_for(path));
        if (P == 1) drop_odd_updates(items, level_off);
        p.n_levels = (int)level_off.size() - 1;
        // the level offsets live in shared memory: size it for this schedule's level count
        c->plan.smem_bytes = path == kPathClassical ? classical_smem_bytes(p, c->plan.chains_per_cta)
                                                    : sweep_smem_bytes(p, path, c->plan.dclass, cl_pre);
        if ((long long)c->plan.smem_bytes > (long long)max_smem) {
            free_ctx(c);
            return create_fail(PT_EINVAL, "one chain needs %zu bytes of shared memory; the device allows %d",
                               c->plan.smem_bytes, max_smem);
        }
    }

    // packed-path site descriptors: row offset i*P, i, packed J bytes (two words), then the
    // row offsets of the neighbour slots; the slot after the last neighbour carries h
    // against a constant row of +1 copies, the remaining slots have J = 0.
    std::vector<uint32_t> desc;
    if (path != kPathGeneric)
        build_site_desc(N, path == kPathBits ? P / 8 : P, c->plan.dclass, adj, adjJ, inst->h, desc);

    // overflow guard: |E| <= P * (sum|J| + sum|h|), |M| <= N*P; sum of squares stays in int64
    {
        long long eb = 0;
        for (int b = 0; b < nE; ++b) eb += abs(inst->J[b]);
        for (int i = 0; i < N; ++i) eb += abs(inst->h[i]);
        eb *= P;
        const long long mb = (long long)N * P;
        const long long big = std::max(std::max(eb, mb), 1ll);
        const long long lim_sq = big > 3037000499ll ? 0 : (long long)(9223372036854775807ll / (big * big));
        c->sweep_limit = std::min<long long>(lim_sq, 0xFFFFFFFFll);
        // the swap mailbox packs E into 40 bits and M into 32 bits
        if (eb >= (1ll << 39) || mb >= (1ll << 31)) {
            free_ctx(c);
            return create_fail(PT_EINVAL, "energy or Trotter sum too large for this library");
        }
    }

    // device memory
    cudaError_t e = cudaSuccess;
    uint32_t *d_nbr, *d_items, *d_thr, *d_desc;
    int8_t* d_h;
    int32_t* d_loff;
    double* d_coef;
    const int max_passes = 1024;
    c->max_passes = max_passes;
    DevCarve carve;
    carve.add(&d_nbr, nbr.size());
    carve.add(&d_h, (size_t)N);
    carve.add(&d_items, 2 * (size_t)N);  // room for both parities' updates (P = 1 uses half)
    carve.add(&d_loff, level_off.size());
    carve.add(&d_thr, c->thr.size());
    carve.add(&d_desc, desc.size());
    carve.add(&d_coef, c->coef.size());
    carve.add(&p.spins, (size_t)R * p.slot_stride);
    carve.add(&p.E, (size_t)R);
    carve.add(&p.M, (size_t)R);
    carve.add(&p.rung_of_slot, (size_t)R);
    carve.add(&p.slot_of_rung, (size_t)R);
    carve.add(&p.acc, (size_t)R * kAccCount);
    carve.add(&p.swap_stats, 2 * (size_t)R);
    carve.add(&p.mbox, (size_t)max_passes * R);
    carve.add(&p.status, (size_t)4);
    carve.add(&c->staging, (size_t)R * N * P);
    if ((e = carve.allocate(c)) != cudaSuccess) {
        free_ctx(c);
        return create_fail(e == cudaErrorMemoryAllocation ? PT_ENOMEM : PT_ECUDA, "cudaMalloc: %s",
                           cudaGetErrorString(e));
    }
    p.nbr = d_nbr;
    p.h = d_h;
    p.items = d_items;
    p.level_off = d_loff;
    p.thr = d_thr;
    p.desc = d_desc;
    p.coef = d_coef;

    cudaStream_t s = c->stream;
#define CREATE_CUDA(call)                                                              \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            cudaStreamSynchronize(s);                                                  \
            free_ctx(c);                                                               \
            return create_fail(PT_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));     \
        }                                                                              \
    } while (0)
    CREATE_CUDA(cudaMemcpyAsync(d_nbr, nbr.data(), nbr.size() * 4, cudaMemcpyHostToDevice, s));
    CREATE_CUDA(cudaMemcpyAsync(d_h, h8.data(), (size_t)N, cudaMemcpyHostToDevice, s));
    CREATE_CUDA(cudaMemcpyAsync(d_items, items.data(), items.size() * 4, cudaMemcpyHostToDevice, s));
    CREATE_CUDA(cudaMemcpyAsync(d_loff, level_off.data(), level_off.size() * 4, cudaMemcpyHostToDevice, s));
    CREATE_CUDA(cudaMemcpyAsync(d_thr, c->thr.data(), c->thr.size() * 4, cudaMemcpyHostToDevice, s));
    if (!desc.empty())
        CREATE_CUDA(cudaMemcpyAsync(d_desc, desc.data(), desc.size() * 4, cudaMemcpyHostToDevice, s));
    CREATE_CUDA(cudaMemcpyAsync(d_coef, c->coef.data(), c->coef.size() * 8, cudaMemcpyHostToDevice, s));
    CREATE_CUDA(cudaMemsetAsync(p.spins, 0, (size_t)R * p.slot_stride, s));
    CREATE_CUDA(cudaMemsetAsync(p.acc, 0, (size_t)R * kAccCount * 8, s));
    CREATE_CUDA(cudaMemsetAsync(p.swap_stats, 0, 2 * (size_t)R * 8, s));
    CREATE_CUDA(cudaMemsetAsync(p.mbox, 0, (size_t)max_passes * R * sizeof(Mailbox), s));
    CREATE_CUDA(cudaMemsetAsync(p.status, 0, 16, s));
    CREATE_CUDA(launch_init(p, s));
    CREATE_CUDA(launch_energy(p, s));
    c->launches += 2;
    c->h2d_bytes += (int64_t)(nbr.size() * 4 + (size_t)N + items.size() * 4 + level_off.size() * 4 +
                              c->thr.size() * 4 + c->coef.size() * 8 + desc.size() * 4);
    CREATE_CUDA(prepare_sweep_kernel(c->plan));
    CREATE_CUDA(cudaStreamSynchronize(s));
#undef CREATE_CUDA

    // cooperative launch (swaps inside one launch) needs every chain resident at once
    long long resident = 0;
    int coop_ok = 0;
    cudaDeviceGetAttribute(&coop_ok, cudaDevAttrCooperativeLaunch, c->device);
    if (sweep_resident_chains(p, c->plan, &resident) != cudaSuccess) resident = 0;
    const int mode = opt ? opt->swap_mode : 0;
    c->cooperative = coop_ok && resident >= R && mode != 2;
    if (mode == 1 && !c->cooperative) {
        free_ctx(c);
        return create_fail(PT_EINVAL, "swap_mode 1 needs all %d chains resident at once (%lld fit on %d SMs)", R,
                           resident, n_sm);
    }
    if ((path == kPathSplit || path == kPathSplitInline || path == kPathPeer || path == kPathCluster ||
         path == kPathClassical) &&
        resident < R) {
        // the two CTAs of a chain always run together, but the swap passes need every chain
        free_ctx(c);
        return create_fail(PT_EINVAL, "the split kernel needs all %d chains resident at once (%lld fit)", R,
                           resident);
    }

    if (want_chains) {
        // the packed-chains plan: the given cluster size, or the smallest that holds every
        // chain; the given chain-group width, or the narrowest that fits
        LaunchPlan pl;
        bool ok = false;
        for (int K = opt->cluster_size > 0 ? opt->cluster_size : 1; K <= 16 && !ok; K *= 2) {
            ok = chains_plan(p, packed_dc, K, kGroupWidenDefault, pl, opt->group_threads);
            if (opt->cluster_size > 0) break;
        }
        if (!ok) {
            free_ctx(c);
            return create_fail(PT_EINVAL, "kernel_path 7: the chains do not all fit the cluster's shared memory");
        }
        int cols = 1;
        while (cols < P / 8) cols <<= 1;
        level_schedule(N, adj, items, level_off, std::max(1, pl.group_threads / cols), P / 4);
        cudaStream_t s = c->stream;
        if ((e = cudaMemcpyAsync(d_items, items.data(), items.size() * 4, cudaMemcpyHostToDevice, s)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(d_loff, level_off.data(), level_off.size() * 4, cudaMemcpyHostToDevice, s)) !=
                cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess) {
            free_ctx(c);
            return create_fail(PT_ECUDA, "schedule upload: %s", cudaGetErrorString(e));
        }
        p.n_levels = (int)level_off.size() - 1;
        c->plan = pl;
        c->cooperative = true;
    }

    // Plan autotuning. When the path and the block size are automatic and the chains are
    // int8 in shared memory, each candidate plan (producer-warp kernel, inline-word kernel
    // with 256, 384 or 512 threads, split kernels, peer-produced words, chains packed on one
    // cluster, one cluster of one-chain CTAs) sweeps a short stretch of one continuous run,
    // twice, and the fastest is kept. Results do not depend on the plan; the context is then
    // reset to its initial state. The choice is cached per problem shape for the process.
    // (also when the fixed plan cannot hold every chain at once: a candidate that can runs the
    // swap passes inside its launch; every candidate timed is one whose chains are all resident)
    const bool tune = want_path == 0 && want_threads == 0 && !(opt && opt->no_autotune) && coop_ok && mode != 2 &&
                      R > 1 && p.withhold_rung < 0 && !p.exact_swaps &&
                      (path == kPathPacked || path == kPathPackedInline || path == kPathSplit ||
                       (path == kPathGeneric && P == 1));
    if (tune) {
        struct Cand {
            int path, threads, producers;
            int cluster = 1, group_threads = 0;  // path 7; path 10: CTAs and chains per CTA
        };
        const PlanKey key{N, P, R, packed_dc, p.n_levels, nE};
        std::vector<Cand> cands;
        {
            std::lock_guard<std::mutex> lock(g_plan_mutex);
            auto it = g_plan_cache.find(key);
            if (it != g_plan_cache.end())
                cands.push_back({it->second.path, it->second.threads, it->second.producers, it->second.cluster,
                                 it->second.group_threads});
        }
        const bool cached = !cands.empty();
        if (!cached && P == 1) {
            // classical chains: one chain a CTA (byte-wise kernel), or several chains a CTA on
            // one cluster (path 10) for clusters of about 1 to 16 CTAs
            cands.push_back({kPathGeneric, 128, 0});
            cands.push_back({kPathGeneric, 64, 0});
            for (int K : {1, 2, 4, 8, 16}) {
                const int C = classical_chains(K), ctas = (R + C - 1) / C;
                bool dup = C > 512 || ctas > 16;
                for (const Cand& cd : cands) dup = dup || (cd.path == kPathClassical && cd.group_threads == C);
                if (!dup) cands.push_back({kPathClassical, classical_threads(C), 0, ctas, C});
            }
        } else if (!cached) {
            if (fits(kPathPacked)) cands.push_back({kPathPacked, 512, 128});
            if (split_fits()) cands.push_back({kPathSplit, 512, 128});
            if (split_fits(kPathSplitInline))
                for (int th : {384, 512})
                    if (th >= P / 16 + 1) cands.push_back({kPathSplitInline, th, 0});
            if (fits(kPathPackedInline))
                for (int th : {256, 384, 512}) cands.push_back({kPathPackedInline, th, 0});
            for (int th : {384, 512})
                if (peer_fits(th)) cands.push_back({kPathPeer, th, 0});
            // every chain's CTA in one cluster, swap mailboxes in shared memory (R <= 16), with
            // the random words inline or from producer warps
            if (R <= 16)
                for (int th : {128, 256}) {
                    cands.push_back({kPathCluster, th, 0});
                    cands.push_back({kPathCluster, th, th / 4});
                }
            // every chain resident on one cluster (small problems: swaps never leave the
            // cluster), at the narrowest chain groups that fit and two wider ones
            for (int K : {1, 2, 4, 8})
                for (int widen : {kGroupWidenDefault, -2, 0}) {
                    LaunchPlan pl;
                    if (!chains_plan(p, packed_dc, K, widen, pl)) continue;
                    bool dup = false;
                    for (const Cand& cd : cands)
                        dup = dup || (cd.path == kPathPackedChains && cd.cluster == K && cd.group_threads == pl.group_threads);
                    if (!dup) cands.push_back({kPathPackedChains, 512, 0, K, pl.group_threads});
                }
        }
        // a candidate's plan, shared-memory flags and level schedule
        auto make = [&](const Cand& cd, LaunchPlan& pl, DevProblem& pc, std::vector<uint32_t>& it_c,
                        std::vector<int32_t>& off_c) {
            pc = p;
            if (cd.path == kPathClassical) {
                pc.acc_in_smem = 1;
                pc.tables_in_smem = 1;
                pl.path = kPathClassical;
                pl.dclass = dclass;
                pl.threads = cd.threads;
                pl.n_consumer = cd.threads;
                pl.chains_per_cta = cd.group_threads;
                pl.cluster = cd.cluster;
                level_schedule(N, adj, it_c, off_c, std::max(1, cd.threads / cd.group_threads));
                drop_odd_updates(it_c, off_c);
                pc.n_levels = (int)off_c.size() - 1;
                pl.smem_bytes = classical_smem_bytes(pc, cd.group_threads);  // sized for this schedule
                return pl.smem_bytes <= (size_t)max_smem;
            }
            if (cd.path == kPathPackedChains) {
                if (!chains_plan(pc, packed_dc, cd.cluster, kGroupWidenDefault, pl, cd.group_threads)) return false;
                int cols = 1;
                while (cols < P / 8) cols <<= 1;
                level_schedule(N, adj, it_c, off_c, std::max(1, pl.group_threads / cols), P / 4);
                pc.n_levels = (int)off_c.size() - 1;
                return true;
            }
            pc.acc_in_smem = (size_t)R * kAccCount * 8 <= 16384 ? 1 : 0;
            pc.tables_in_smem = (size_t)R * p.nL3 * 4 <= 49152 ? 1 : 0;
            const bool cpre = cd.path == kPathCluster && cd.producers > 0;
            if (pc.tables_in_smem && sweep_smem_bytes(pc, cd.path, packed_dc, cpre) > (size_t)max_smem)
                pc.tables_in_smem = 0;
            if (pc.acc_in_smem && sweep_smem_bytes(pc, cd.path, packed_dc, cpre) > (size_t)max_smem) pc.acc_in_smem = 0;
            pl.path = cd.path;
            pl.dclass = cd.path == kPathGeneric ? dclass : packed_dc;
            pl.threads = cd.threads;
            pl.n_consumer = cd.threads - cd.producers;
            pl.smem_bytes = sweep_smem_bytes(pc, cd.path, packed_dc, cpre);
            int cols = 1;
            if (cd.path == kPathSplit || cd.path == kPathSplitInline) {
                cols = P / 16 + 1;
            } else {
                while (cols < P / 8) cols <<= 1;
            }
            level_schedule(N, adj, it_c, off_c, std::max(1, pl.n_consumer / cols), row_words_for(cd.path));
            if (P == 1) drop_odd_updates(it_c, off_c);
            pc.n_levels = (int)off_c.size() - 1;
            pl.smem_bytes = sweep_smem_bytes(pc, cd.path, pl.dclass, cpre);  // sized for this schedule
            return pl.smem_bytes <= (size_t)max_smem;
        };
        cudaStream_t s = c->stream;
        int best = -1, timed_plans = 0;
        if (cands.size() == 1) {
            best = 0;
        } else if (cands.size() > 1) {
            // per-sweep cost = (time of a long launch - time of a short one) / the sweep
            // difference, so that a kernel's per-launch setup does not count
            cudaEvent_t ev[3];
            cudaEventCreate(&ev[0]);
            cudaEventCreate(&ev[1]);
            cudaEventCreate(&ev[2]);
            long long t = 0, q = 0;
            const int warm = 4, shortn = 4, longn = std::min(36, c->max_passes);
            // two passes, the second in reverse order, keeping each candidate's faster time:
            // a clock still rising at the start of the timing then favours no candidate
            std::vector<float> cand_ms(cands.size(), 1e30f);
            bool stop = false;
            for (int pass = 0; pass < 2 && !stop; ++pass)
            for (size_t i = 0; i < cands.size() && !stop; ++i) {
                const size_t k = pass == 0 ? i : cands.size() - 1 - i;
                LaunchPlan pl;
                DevProblem pc;
                std::vector<uint32_t> it_c;
                std::vector<int32_t> off_c;
                if (!make(cands[k], pl, pc, it_c, off_c)) continue;
                long long res = 0;
                if (pl.path != kPathPackedChains &&
                    (prepare_sweep_kernel(pl) != cudaSuccess || sweep_resident_chains(pc, pl, &res) != cudaSuccess ||
                     res < R)) {
                    (void)cudaGetLastError();
                    continue;
                }
                cudaError_t e1 = cudaMemcpyAsync(d_items, it_c.data(), it_c.size() * 4, cudaMemcpyHostToDevice, s);
                if (e1 == cudaSuccess)
                    e1 = cudaMemcpyAsync(d_loff, off_c.data(), off_c.size() * 4, cudaMemcpyHostToDevice, s);
                if (e1 == cudaSuccess) e1 = launch_plan_sweeps(pc, pl, t, q, warm, 1, c->timeout_ns, true, s);
                if (e1 == cudaSuccess) e1 = cudaEventRecord(ev[0], s);
                if (e1 == cudaSuccess)
                    e1 = launch_plan_sweeps(pc, pl, t + warm, q + warm, shortn, 1, c->timeout_ns, true, s);
                if (e1 == cudaSuccess) e1 = cudaEventRecord(ev[1], s);
                if (e1 == cudaSuccess)
                    e1 = launch_plan_sweeps(pc, pl, t + warm + shortn, q + warm + shortn, longn, 1, c->timeout_ns,
                                            true, s);
                if (e1 == cudaSuccess) e1 = cudaEventRecord(ev[2], s);
                if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(s);
                int status = 0;
                if (e1 == cudaSuccess) e1 = cudaMemcpy(&status, p.status, sizeof(int), cudaMemcpyDeviceToHost);
                c->launches += 3;
                t += warm + shortn + longn;
                q += warm + shortn + longn;
                if (e1 != cudaSuccess || status != 0) {
                    // a candidate that reports an error ends the tuning (the best plan timed so
                    // far, or the fixed one, is kept; every sweep is undone below); an error that
                    // outlives the launch ends the create
                    (void)cudaGetLastError();
                    if (cudaStreamSynchronize(s) != cudaSuccess ||
                        cudaMemsetAsync(p.status, 0, sizeof(int), s) != cudaSuccess ||
                        cudaStreamSynchronize(s) != cudaSuccess) {
                        for (cudaEvent_t x : ev) cudaEventDestroy(x);
                        free_ctx(c);
                        return create_fail(PT_ECUDA, "plan autotuning: %s", cudaGetErrorString(cudaGetLastError()));
                    }
                    if (pass == 0) ++timed_plans;
                    stop = true;
                    break;
                }
                float ms_short = 0.f, ms_long = 0.f;
                cudaEventElapsedTime(&ms_short, ev[0], ev[1]);
                cudaEventElapsedTime(&ms_long, ev[1], ev[2]);
                const float ms = (ms_long - ms_short) / (float)(longn - shortn);
                if (pass == 0) ++timed_plans;
                cand_ms[k] = std::min(cand_ms[k], ms);
            }
            float best_ms = 1e30f;
            for (size_t k = 0; k < cands.size(); ++k)
                if (cand_ms[k] < best_ms) {
                    best_ms = cand_ms[k];
                    best = (int)k;
                }
            for (cudaEvent_t x : ev) cudaEventDestroy(x);
        }
        if (best >= 0) {
            LaunchPlan pl;
            DevProblem pc;
            std::vector<uint32_t> it_b;
            std::vector<int32_t> off_b;
            if (make(cands[best], pl, pc, it_b, off_b)) {
                long long res = 0;
                if (pl.path == kPathPackedChains ||
                    (prepare_sweep_kernel(pl) == cudaSuccess && sweep_resident_chains(pc, pl, &res) == cudaSuccess &&
                     res >= R)) {
                    // the plan with the schedule its shared memory was sized for
                    items.swap(it_b);
                    level_off.swap(off_b);
                    p.n_levels = pc.n_levels;
                    c->plan = pl;
                    c->cooperative = true;  // resident (checked above), cooperative launch available
                    p.acc_in_smem = pc.acc_in_smem;
                    p.tables_in_smem = pc.tables_in_smem;
                    if (!cached) {
                        std::lock_guard<std::mutex> lock(g_plan_mutex);
                        const Cand& cb = cands[best];
                        g_plan_cache[key] = PlanChoice{cb.path, cb.threads, cb.producers, cb.cluster, cb.group_threads,
                                                       pl.thr_resident};
                    }
                }
                (void)cudaGetLastError();
            }
            c->tuned_plans = timed_plans;
        }
        // the chosen plan's schedule, and the initial state again
#define TUNE_CUDA(call)                                                              \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            cudaStreamSynchronize(s);                                                \
            free_ctx(c);                                                             \
            return create_fail(PT_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
        }                                                                            \
    } while (0)
        if (c->plan.path != kPathPackedChains) TUNE_CUDA(prepare_sweep_kernel(c->plan));
        TUNE_CUDA(cudaMemcpyAsync(d_items, items.data(), items.size() * 4, cudaMemcpyHostToDevice, s));
        TUNE_CUDA(cudaMemcpyAsync(d_loff, level_off.data(), level_off.size() * 4, cudaMemcpyHostToDevice, s));
        if (timed_plans > 0) {
            TUNE_CUDA(cudaMemsetAsync(p.acc, 0, (size_t)R * kAccCount * 8, s));
            TUNE_CUDA(cudaMemsetAsync(p.swap_stats, 0, 2 * (size_t)R * 8, s));
            TUNE_CUDA(cudaMemsetAsync(p.mbox, 0, (size_t)max_passes * R * sizeof(Mailbox), s));
            TUNE_CUDA(launch_init(p, s));
            TUNE_CUDA(launch_energy(p, s));
            c->launches += 2;
        }
        TUNE_CUDA(cudaStreamSynchronize(s));
#undef TUNE_CUDA
    }
    *out = c;
    return PT_OK;
}

static int guard(pt_ctx* c) {
    if (!c) return PT_EINVAL;
    if (c->err) return c->err;
    return PT_OK;
}

static int enqueue_sweeps(pt_ctx* c, long long n, int sps) {
    if (c->plan.path == kPathCluster) {
        // mailboxes in shared memory, cleared by every launch: only the sweep counter bounds one
        long long done = 0;
        while (done < n) {
            long long chunk = n - done;
            chunk = std::min<long long>(chunk, sps > 0 ? ((1ll << 30) / sps) * sps : (1ll << 30));
            CUDA_OR_FAIL(c, launch_sweeps(c->dp, c->plan, c->t, c->q, (int)chunk, sps, c->timeout_ns, sps > 0,
                                          c->stream));
            c->launches += 1;
            c->t += chunk;
            if (sps > 0) c->q += chunk / sps;
            done += chunk;
        }
        return PT_OK;
    }
    if (c->plan.path == kPathPackedChains) {
        // swaps in shared memory: no mailboxes, so only the sweep counter bounds a launch
        long long done = 0;
        while (done < n) {
            long long chunk = n - done;
            chunk = std::min<long long>(chunk, sps > 0 ? ((1ll << 30) / sps) * sps : (1ll << 30));
            CUDA_OR_FAIL(c, launch_batch_single(chains_instance(c->dp, c->plan, c->t, c->q, (int)chunk, sps),
                                                c->plan.cluster, c->plan.threads, c->plan.smem_bytes, c->stream));
            c->launches += 1;
            c->t += chunk;
            if (sps > 0) c->q += chunk / sps;
            done += chunk;
        }
        return PT_OK;
    }
    // chunks of at most max_passes swap passes (mailbox capacity), aligned to the swap interval
    long long done = 0;
    while (done < n) {
        // with swaps, whole intervals only (n is a multiple of sps), so every launch starts on
        // an interval boundary
        long long chunk = n - done;
        if (sps > 0) {
            chunk = std::min<long long>(chunk, (long long)c->max_passes * sps);
            chunk = std::min<long long>(chunk, ((1ll << 30) / sps) * sps);
        } else {
            chunk = std::min<long long>(chunk, 1ll << 30);
        }
        const int passes = sps > 0 ? (int)(chunk / sps) : 0;
        if (passes > 0 && c->q + passes - c->mbox_clear_q >= kTagPeriod - 1) {
            // a mailbox tag is q mod (2^24 - 1) + 1: clear before any tag value could repeat
            CUDA_OR_FAIL(c, cudaMemsetAsync(c->dp.mbox, 0, (size_t)c->max_passes * c->dp.R * sizeof(Mailbox),
                                            c->stream));
            c->mbox_clear_q = c->q;
        }
        CUDA_OR_FAIL(c, launch_sweeps(c->dp, c->plan, c->t, c->q, (int)chunk, sps, c->timeout_ns, sps > 0,
                                      c->stream));
        c->launches += 1;
        c->t += chunk;
        c->q += passes;
        done += chunk;
    }
    return PT_OK;
}

extern "C" int pt_sweep(pt_ctx* c, int64_t n) {
    int g = guard(c);
    if (g) return g;
    if (n < 0) return ctx_fail(c, PT_EINVAL, "n must be >= 0");
    if (c->t + n > c->sweep_limit) return ctx_fail(c, PT_EOVERFLOW, "sweep count would exceed %lld", c->sweep_limit);
    return enqueue_sweeps(c, n, 0);
}

extern "C" int pt_swap(pt_ctx* c) {
    int g = guard(c);
    if (g) return g;
    if (c->q + 1 > 0xFFFFFFFFll) return ctx_fail(c, PT_EOVERFLOW, "swap pass counter exhausted");
    CUDA_OR_FAIL(c, launch_swap(c->dp, c->q, c->stream));
    c->launches += 1;
    c->q += 1;
    return PT_OK;
}

extern "C" int pt_run(pt_ctx* c, int64_t n_sweeps, int32_t sps) {
    int g = guard(c);
    if (g) return g;
    if (n_sweeps < 0 || sps < 0 || sps > (1 << 30))
        return ctx_fail(c, PT_EINVAL, "need n_sweeps >= 0 and 0 <= sweeps_per_swap <= 2^30");
    if (c->t + n_sweeps > c->sweep_limit)
        return ctx_fail(c, PT_EOVERFLOW, "sweep count would exceed %lld", c->sweep_limit);
    if (sps == 0 || c->dp.R == 1) {
        int rc = enqueue_sweeps(c, n_sweeps, 0);
        if (rc) return rc;
        if (sps > 0) c->q += n_sweeps / sps;  // R == 1: passes have no pairs
        return PT_OK;
    }
    if (c->q + n_sweeps / sps > 0xFFFFFFFFll) return ctx_fail(c, PT_EOVERFLOW, "swap pass counter exhausted");
    if (c->cooperative) {
        const long long full = (n_sweeps / sps) * sps;
        int rc = enqueue_sweeps(c, full, sps);
        if (rc) return rc;
        return enqueue_sweeps(c, n_sweeps - full, 0);
    }
    for (long long s = 0; s + sps <= n_sweeps; s += sps) {
        int rc = enqueue_sweeps(c, sps, 0);
        if (rc) return rc;
        CUDA_OR_FAIL(c, launch_swap(c->dp, c->q, c->stream));
        c->launches += 1;
        c->q += 1;
    }
    return enqueue_sweeps(c, n_sweeps % sps, 0);
}

extern "C" int pt_sync(pt_ctx* c) {
    int g = guard(c);
    if (g) return g;
    return check_status(c);
}

extern "C" int pt_read_state(pt_ctx* c, int8_t* out, size_t bytes) {
    int g = guard(c);
    if (g) return g;
    const size_t need = (size_t)c->dp.R * c->dp.N * c->dp.P;
    if (!out || bytes < need) return ctx_fail(c, PT_EINVAL, "state buffer needs %zu bytes", need);
    CUDA_OR_FAIL(c, launch_gather_state(c->dp, c->staging, c->stream));
    c->launches += 1;
    CUDA_OR_FAIL(c, cudaMemcpyAsync(out, c->staging, need, cudaMemcpyDeviceToHost, c->stream));
    return check_status(c);
}

extern "C" int pt_write_state(pt_ctx* c, const int8_t* in, size_t bytes) {
    int g = guard(c);
    if (g) return g;
    const size_t need = (size_t)c->dp.R * c->dp.N * c->dp.P;
    if (!in || bytes != need) return ctx_fail(c, PT_EINVAL, "state buffer must be %zu bytes", need);
    for (size_t x = 0; x < need; ++x)
        if (in[x] != 1 && in[x] != -1) return ctx_fail(c, PT_EINVAL, "spins must be +1 or -1");
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->staging, in, need, cudaMemcpyHostToDevice, c->stream));
    CUDA_OR_FAIL(c, launch_scatter_state(c->dp, c->staging, c->stream));
    CUDA_OR_FAIL(c, launch_energy(c->dp, c->stream));
    c->launches += 2;
    c->h2d_bytes += (int64_t)need;
    return check_status(c);
}

extern "C" int pt_restore(pt_ctx* c, const int8_t* in, size_t bytes, const pt_observables* snap) {
    int g = guard(c);
    if (g) return g;
    const int R = c->dp.R;
    const size_t need = (size_t)R * c->dp.N * c->dp.P;
    if (!in || bytes != need) return ctx_fail(c, PT_EINVAL, "state buffer must be %zu bytes", need);
    if (!snap || !snap->replica_at || !snap->n_meas || !snap->sum_E || !snap->sum_E2 || !snap->sum_M ||
        !snap->sum_M2 || !snap->flip_acc || (R > 1 && (!snap->swap_att || !snap->swap_acc)))
        return ctx_fail(c, PT_EINVAL, "the snapshot needs the permutation, every statistic and both counters");
    for (size_t x = 0; x < need; ++x)
        if (in[x] != 1 && in[x] != -1) return ctx_fail(c, PT_EINVAL, "spins must be +1 or -1");
    if (snap->t < 0 || snap->t > c->sweep_limit || snap->q < 0 || snap->q > 0xFFFFFFFFll)
        return ctx_fail(c, PT_EOVERFLOW, "snapshot counters out of range");
    std::vector<int32_t> slot_of(R), rung_of(R, -1);
    for (int r = 0; r < R; ++r) {
        const int slot = snap->replica_at[r];
        if (slot < 0 || slot >= R || rung_of[slot] >= 0) return ctx_fail(c, PT_EINVAL, "replica_at is not a permutation");
        slot_of[r] = slot;
        rung_of[slot] = r;
    }
    std::vector<unsigned long long> acc((size_t)R * kAccCount, 0ull), sw(2 * (size_t)R, 0ull);
    for (int r = 0; r < R; ++r) {
        unsigned long long* a = &acc[(size_t)r * kAccCount];
        a[kAccN] = (unsigned long long)snap->n_meas[r];
        a[kAccE] = (unsigned long long)snap->sum_E[r];
        a[kAccE2] = (unsigned long long)snap->sum_E2[r];
        a[kAccM] = (unsigned long long)snap->sum_M[r];
        a[kAccM2] = (unsigned long long)snap->sum_M2[r];
        a[kAccFlip] = (unsigned long long)snap->flip_acc[r];
    }
    for (int r = 0; r + 1 < R; ++r) {
        sw[2 * r] = (unsigned long long)snap->swap_att[r];
        sw[2 * r + 1] = (unsigned long long)snap->swap_acc[r];
    }
    cudaStream_t s = c->stream;
    // the random streams belong to the chains, so each chain returns to its own slot; stale
    // mailboxes could carry the tags of the restored passes and are cleared
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->dp.slot_of_rung, slot_of.data(), R * 4, cudaMemcpyHostToDevice, s));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->dp.rung_of_slot, rung_of.data(), R * 4, cudaMemcpyHostToDevice, s));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->dp.acc, acc.data(), acc.size() * 8, cudaMemcpyHostToDevice, s));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->dp.swap_stats, sw.data(), sw.size() * 8, cudaMemcpyHostToDevice, s));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(c->staging, in, need, cudaMemcpyHostToDevice, s));
    CUDA_OR_FAIL(c, cudaMemsetAsync(c->dp.mbox, 0, (size_t)c->max_passes * R * sizeof(Mailbox), s));
    CUDA_OR_FAIL(c, launch_scatter_state(c->dp, c->staging, s));
    CUDA_OR_FAIL(c, launch_energy(c->dp, s));
    c->launches += 2;
    c->h2d_bytes += (int64_t)(need + R * 8 + acc.size() * 8 + sw.size() * 8);
    c->t = snap->t;
    c->q = snap->q;
    c->mbox_clear_q = snap->q;
    return check_status(c);
}

extern "C" int pt_read_observables(pt_ctx* c, pt_observables* o) {
    int g = guard(c);
    if (g) return g;
    if (!o) return ctx_fail(c, PT_EINVAL, "null observables");
    const int R = c->dp.R;
    std::vector<long long> E(R), M(R);
    std::vector<int32_t> rung_of(R), slot_of(R);
    std::vector<unsigned long long> acc((size_t)R * kAccCount), sw(2 * (size_t)R);
    cudaStream_t s = c->stream;
    CUDA_OR_FAIL(c, cudaMemcpyAsync(E.data(), c->dp.E, R * 8, cudaMemcpyDeviceToHost, s));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(M.data(), c->dp.M, R * 8, cudaMemcpyDeviceToHost, s));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(slot_of.data(), c->dp.slot_of_rung, R * 4, cudaMemcpyDeviceToHost, s));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(acc.data(), c->dp.acc, acc.size() * 8, cudaMemcpyDeviceToHost, s));
    CUDA_OR_FAIL(c, cudaMemcpyAsync(sw.data(), c->dp.swap_stats, sw.size() * 8, cudaMemcpyDeviceToHost, s));
    int rc = check_status(c);
    if (rc) return rc;
    o->t = c->t;
    o->q = c->q;
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

extern "C" int pt_read_tables(const pt_ctx* c, uint32_t* thr, size_t thr_count, double* coef, size_t coef_count) {
    if (!c) return PT_EINVAL;
    if (thr) {
        if (thr_count < c->thr.size()) return PT_EINVAL;
        memcpy(thr, c->thr.data(), c->thr.size() * 4);
    }
    if (coef) {
        const size_t n = 2 * (size_t)(c->dp.R - 1);
        if (coef_count < n) return PT_EINVAL;
        memcpy(coef, c->coef.data(), n * 8);
    }
    return PT_OK;
}

extern "C" int pt_get_info(const pt_ctx* c, pt_info* o) {
    if (!c || !o) return PT_EINVAL;
    o->n = c->dp.N;
    o->P = c->dp.P;
    o->R = c->dp.R;
    o->lmax = c->dp.Lmax;
    o->max_degree = c->max_degree;
    o->n_levels = c->dp.n_levels;
    o->threads_per_block = c->plan.threads;
    o->cooperative = c->cooperative ? 1 : 0;
    o->kernel_path = c->plan.path;
    o->producer_threads = c->plan.threads - c->plan.n_consumer;
    o->device_bytes = c->device_bytes;
    o->kernel_launches = c->launches;
    o->h2d_bytes = c->h2d_bytes;
    o->tuned_plans = c->tuned_plans;
    o->reserved = 0;
    return PT_OK;
}

extern "C" int pt_make_tables(int32_t P, const pt_rung* ladder, int32_t R, int32_t lmax, uint32_t* thr,
                              double* coef) {
    if (!ladder || (P != 1 && (P < 2 || (P & 1))) || R < 1 || lmax < 0 || lmax > 127) return PT_EINVAL;
    for (int r = 0; r < R; ++r)
        if (!(ladder[r].T > 0.0) || (P == 1 ? !(ladder[r].gamma == 0.0) : !(ladder[r].gamma > 0.0)))
            return PT_EINVAL;
    std::vector<uint32_t> t;
    std::vector<double> c;
    build_tables(R, P, lmax, ladder, t, c);
    if (thr) memcpy(thr, t.data(), t.size() * 4);
    if (coef && R > 1) memcpy(coef, c.data(), 2 * (size_t)(R - 1) * 8);
    return PT_OK;
}

extern "C" int pt_make_schedule(const pt_instance* inst, uint32_t* items, int32_t* level_off, int32_t* n_levels) {
    return pt_make_schedule_balanced(inst, 0, items, level_off, n_levels);
}

extern "C" int pt_make_schedule_balanced(const pt_instance* inst, int32_t items_per_round, uint32_t* items,
                                         int32_t* level_off, int32_t* n_levels) {
    if (!inst || !items || !level_off || !n_levels || inst->n < 1 || items_per_round < 0) return PT_EINVAL;
    std::vector<std::vector<int>> adj(inst->n);
    for (int b = 0; b < inst->n_edges; ++b) {
        const int u = inst->ei[b], v = inst->ej[b];
        if (u < 0 || u >= inst->n || v < 0 || v >= inst->n || u == v) return PT_EINVAL;
        adj[u].push_back(v);
        adj[v].push_back(u);
    }
    std::vector<uint32_t> it;
    std::vector<int32_t> off;
    level_schedule(inst->n, adj, it, off, items_per_round);
    memcpy(items, it.data(), it.size() * 4);
    memcpy(level_off, off.data(), off.size() * 4);
    *n_levels = (int32_t)off.size() - 1;
    return PT_OK;
}

extern "C" int pt_destroy(pt_ctx* c) {
    if (!c) return PT_OK;
    cudaStreamSynchronize(c->stream);
    free_ctx(c);
    return PT_OK;
}

extern "C" const char* pt_last_error(const pt_ctx* c) { return c ? c->msg : g_create_msg; }
